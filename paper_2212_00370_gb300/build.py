"""Build librrmhd.so (the C-ABI library of include/rrmhd.h) for sm_103a.

Each translation unit is compiled in parallel with nvcc, then linked as a
shared library next to this file (in-tree, git-ignored).  The FP64 kernels are
compiled with --fmad=false: their arithmetic order is part of the
specification of the FP64 path (bit-reproducible results).  The FP32-bulk unit
takes FP32 division and square root in their fast forms (-prec-div=false,
-prec-sqrt=false: ~2 ulp instead of correctly rounded); its FP64 arithmetic is
unaffected.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librrmhd.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]

# translation unit -> extra flags
UNITS = {
    "rrmhd_f64.cu": ["--fmad=false"],
    "rrmhd_api.cu": [],
    "rrmhd_noalloc.cu": ["--fmad=false"],
    "rrmhd_f32.cu": ["-prec-div=false", "-prec-sqrt=false"],
    "rrmhd_server.cu": ["--fmad=false"],
    "rrmhd_probe.cu": [],
}
HEADERS = ["physics_f64.cuh", "scheme_f64.cuh", "physics_tangent.cuh", "batch.h", "batch_index.cuh",
           "engine.h"]


def _deps():
    deps = [os.path.join(CSRC, u) for u in UNITS] + [os.path.join(CSRC, h) for h in HEADERS]
    deps += [os.path.join(INCLUDE, "rrmhd.h"), os.path.abspath(__file__)]
    return deps


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps() if os.path.exists(p))


def _compile(unit, flags, verbose):
    obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
    extra = os.environ.get("RRMHD_NVCC_FLAGS", "").split()   # tuning knobs, e.g. -DRR_F64_CELL_WARPS=12
    cmd = [NVCC, *ARCH, *COMMON, *flags, *extra, "-c", os.path.join(CSRC, unit), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{r.stderr}")
    return obj, r.stderr


def build(force=False, verbose=False):
    """Compile librrmhd.so in-tree (no-op when up to date); returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        futs = [ex.submit(_compile, u, f, verbose) for u, f in UNITS.items()]
        objs = []
        for fu in futs:
            obj, log = fu.result()
            objs.append(obj)
            if verbose and log:
                print(log, file=sys.stderr)
    tmp = LIB + ".tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))

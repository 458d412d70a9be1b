"""Build the FP64 CPU oracle (``liboracle.so``).

Test infrastructure only: the oracle is the reference the CUDA path is checked
against, never part of it.  Compiled with ``-ffp-contract=off`` so that no
multiply-add is contracted (aarch64 gcc contracts by default), and without
``-march=native`` so the result is the same bit pattern on x86-64 and aarch64.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["physics.c", "scheme.c", "implicit.c", "grid.c", "ct.c"]
LIB = os.path.join(HERE, "liboracle.so")
CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-Wall", "-Wno-unused-function"]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["oracle.h", "build.py"]
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in deps)


def build(force=False, verbose=False):
    """Compile liboracle.so next to this file (no-op when up to date)."""
    if not force and not _stale():
        return LIB
    cmd = ["gcc", *CFLAGS, "-o", LIB + ".tmp", *[os.path.join(HERE, s) for s in SOURCES], "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))

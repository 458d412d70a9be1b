"""The C-ABI library builds, loads and exports every entry point that
include/rrmhd.h declares (no GPU needed: nothing is called that touches CUDA)."""
import ctypes
import os
import re

import pytest

from paper_2212_00370_gb300 import build as B
from paper_2212_00370_gb300 import rrmhd

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rrmhd.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rrmhd_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def test_header_declares_the_boundary():
    names = declared()
    for must in ("rrmhd_create", "rrmhd_prim2con", "rrmhd_con2prim", "rrmhd_flux_sweep",
                 "rrmhd_implicit_source", "rrmhd_imex_step", "rrmhd_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib_path):
    assert sorted(rrmhd.exported_names()) == declared()
    rrmhd.lib()  # loads and sets every signature


def test_default_opts_without_gpu(lib_path):
    o = rrmhd.make_opts()
    assert o.gamma == pytest.approx(5 / 3) and o.pvm_eps == 1e-8 and o.recon == 3
    assert o.beta_mode == 1 and o.cfl == pytest.approx(0.4)


def test_struct_layouts_match_the_header(tmp_path):
    """ctypes mirrors of the header's structs have the C sizes and field offsets."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"rrmhd_grid": rrmhd.rrmhd_grid, "rrmhd_opts": rrmhd.rrmhd_opts,
               "rrmhd_tuning": rrmhd.rrmhd_tuning,
               "rrmhd_server_config": rrmhd.rrmhd_server_config,
               "rrmhd_result": rrmhd.rrmhd_result, "rrmhd_server_stats": rrmhd.rrmhd_server_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rrmhd.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[name + "." + f]) == getattr(cls, f).offset, (name, f)


def test_create_rejects_a_closure_other_than_m1(lib_path):
    """Argument checks run before any CUDA call: no GPU needed."""
    import ctypes as C
    grid = rrmhd.make_grid(1, (8,), (0.125,))
    opts = rrmhd.make_opts()
    assert opts.closure == 0
    opts.closure = 1
    out = C.c_void_p()
    rc = rrmhd.lib().rrmhd_create(1, C.byref(grid), C.byref(opts), None, C.byref(out))
    assert rrmhd.STATUS[rc] == "EINVAL" and not out.value

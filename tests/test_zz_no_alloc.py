"""The alloc-free CFL entry point (rrmhd_cfl_dt_noalloc), called through the C ABI.

It serves callers that cannot allocate device memory themselves (their GPU
memory is owned by their own pool or fixed arena): its scratch is a fixed array
inside the library.  Its time step must equal, bit for bit, the one the
context path (rrmhd_imex_step) takes from the same state, on consecutive calls
that share that scratch.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2212_00370_gb300 import rrmhd
from paper_2212_00370_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_00370_gb300 import build
    build.build()


def _context_dt(w):
    """dt of the first step the existing entry point (rrmhd_imex_step) takes."""
    g = w.grids[0]
    ctx = rrmhd.Context([rrmhd.make_grid(g["ndim"], g["n"], g["dx"], g["bc"])], gamma=w.gamma,
                        a_rad=w.a_rad, cfl=w.cfl)
    ctx.set_opacity(torch.tensor(w.kappa, device="cuda"), torch.tensor(w.sigma, device="cuda"))
    ctx.set_state(torch.tensor(w.V, device="cuda"))
    ctx.set_times([0.0], [np.inf])
    ctx.imex_step(1)
    t, dt = ctx.get_times()
    ctx.close()
    return dt[0]


def _noalloc_dt(w, out):
    g = w.grids[0]
    grid = rrmhd.make_grid(g["ndim"], g["n"], g["dx"], g["bc"])
    opts = rrmhd.make_opts(gamma=w.gamma, a_rad=w.a_rad, cfl=w.cfl)
    V = torch.tensor(w.V, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = rrmhd.lib().rrmhd_cfl_dt_noalloc(C.byref(grid), C.byref(opts), C.c_void_p(V.data_ptr()),
                                          C.c_void_p(out.data_ptr()), stream)
    assert rc == 0, rrmhd.STATUS.get(rc, rc)
    torch.cuda.synchronize()
    return out.item()


def test_noalloc_cfl_matches_context_path_on_consecutive_calls():
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cases = [W.shock_tube(400), W.turbulent_3d(40), W.blast_2d(96), W.shock_tube(1000)]
    for w in cases:
        ref = _context_dt(w)
        a = _noalloc_dt(w, out)
        b = _noalloc_dt(w, out)          # second call in a row reuses the scratch
        assert a == ref and b == ref, (w.name, a, b, ref)


def test_noalloc_cfl_rejects_oversized_grids():
    grid = rrmhd.make_grid(3, (512, 512, 129), (1.0, 1.0, 1.0))   # > RRMHD_NOALLOC_MAX_CELLS
    opts = rrmhd.make_opts()
    dummy = torch.zeros(2, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    rc = rrmhd.lib().rrmhd_cfl_dt_noalloc(C.byref(grid), C.byref(opts), p, p, None)
    assert rrmhd.STATUS[rc] == "ECAPACITY"
    rc = rrmhd.lib().rrmhd_cfl_dt_noalloc(C.byref(grid), C.byref(opts), None, p, None)
    assert rrmhd.STATUS[rc] == "EINVAL"


def test_noalloc_cfl_nan_cell_gives_nan_dt():
    """A NaN radiation energy makes both radiation speeds of its cell NaN, and so its
    signal speed, which wins the maximum: dt = NaN on two calls in a row, and the
    next admissible grid gets its own dt again (nothing of the NaN stays in the
    shared scratch)."""
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    w = W.shock_tube(400)
    bad = W.shock_tube(400)
    bad.V = bad.V.copy()
    bad.V[8, 123] = np.nan
    assert np.isnan(_noalloc_dt(bad, out)) and np.isnan(_noalloc_dt(bad, out))
    assert _noalloc_dt(w, out) == _context_dt(w)

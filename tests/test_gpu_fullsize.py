"""C2 (2D 1024^2 periodic blast) and C3 (3D 256^3 periodic box) at full size.

One IMEX step of the whole grid on the GPU; then sampled cells are recomputed
one by one by the oracle.  One step of a cell depends only on the cells within
distance 5 per stage (the +-2 PLM stencil of its faces, plus one cell for each
of the 3 passes of the admissibility fallback), so 15 over the three stages.  A
periodic patch of half-width 16 around the cell, stepped by the oracle with the
GPU's time step, therefore reproduces that cell exactly.  FP64: bit for bit (time step
included).  FP32-bulk: per-variable relative L1 <= 1e-5 against FP64.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import compare_bitwise, gpu_context, oracle_grid, oracle_params
from paper_2212_00370_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HALF = 16


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_00370_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def c2():
    return W.blast_2d()


@pytest.fixture(scope="module")
def c3():
    return W.turbulent_3d()


def patch_index(g, center, h=HALF):
    """Flat indices (x fastest) of the periodic box of half-width h around center."""
    nd = g["ndim"]
    n = g["n"][:nd]
    ax = [(np.arange(-h, h + 1) + center[d]) % n[d] for d in range(nd)]
    if nd == 2:
        J, I = np.meshgrid(ax[1], ax[0], indexing="ij")
        return (J * n[0] + I).reshape(-1)
    K, J, I = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return ((K * n[1] + J) * n[0] + I).reshape(-1)


def oracle_cell(w, center, dt, P):
    g = w.grids[0]
    nd = g["ndim"]
    flat = patch_index(g, center)
    pg = O.Grid(nd, (2 * HALF + 1,) * nd, tuple(g["dx"][:nd]), ("outflow",) * nd)
    V = np.ascontiguousarray(w.V[:, flat])
    U = O.prim2con(V, P)
    jc = np.zeros(17 * len(flat))   # the implicit solve's per-cell cache starts empty, as on the GPU
    nfail = O.step(pg, dt, U, V, w.kappa[flat], w.sigma[flat], P, jcache=jc)
    m = len(flat) // 2
    return U[:, m].copy(), V[:, m].copy(), nfail


def flat_of(g, c):
    n = g["n"]
    return (c[2] * n[1] + c[1]) * n[0] + c[0] if g["ndim"] == 3 else c[1] * n[0] + c[0]


def samples(w, k, seed, extra=()):
    g = w.grids[0]
    nd = g["ndim"]
    rng = np.random.default_rng(seed)
    pts = [list(e) for e in extra]
    pts += [[int(rng.integers(0, g["n"][d])) for d in range(nd)] for _ in range(k)]
    return [p + [0] * (3 - nd) for p in pts]


def gpu_one_step(w, precision):
    ctx = gpu_context(w, precision=precision)
    ctx.imex_step(1)
    U, V = ctx.get_state()
    t, dt = ctx.get_times()
    st = ctx.inst_status()
    out = (U.cpu().numpy(), V.cpu().numpy(), dt[0], st[0])
    ctx.close()
    torch.cuda.empty_cache()
    return out


VARS = ["D", "Sx", "Sy", "Sz", "tau", "Bx", "By", "Bz", "E", "Fx", "Fy", "Fz"]


def check_fp64(w, pts):
    """Time step and sampled cells bit for bit."""
    P = oracle_params(w)
    dt_o = O.grid_dt(oracle_grid(w.grids[0]), np.ascontiguousarray(w.V), P)
    U, V, dt, st = gpu_one_step(w, "fp64")
    assert st == 0
    assert dt == dt_o, (dt, dt_o)
    g = w.grids[0]
    for c in pts:
        Uo, Vo, nfail = oracle_cell(w, c[:g["ndim"]], dt, P)
        assert nfail == 0
        j = flat_of(g, c)
        compare_bitwise(U[:, j], Uo, f"U at {c}")
        compare_bitwise(V[:, j], Vo, f"V at {c}")


def check_fp32_bulk(w, pts):
    """Per-variable relative L1 of the whole grid against the FP64 path (which the
    FP64 tests pin to the oracle bit for bit) <= 1e-5; sampled cells against the
    oracle directly, per-variable relative L1 over the samples <= 1e-5."""
    U32, _, dt32, st32 = gpu_one_step(w, "fp32_bulk")
    U64, _, dt64, st64 = gpu_one_step(w, "fp64")
    assert st32 == 0 and st64 == 0 and dt32 == dt64
    l1 = {}
    for k in range(12):
        den = np.abs(U64[k]).sum()
        if den > 0:
            l1[VARS[k]] = float(np.abs(U32[k] - U64[k]).sum() / den)
    P = oracle_params(w)
    g = w.grids[0]
    num = np.zeros(12)
    den = np.zeros(12)
    for c in pts:
        Uo, _, nfail = oracle_cell(w, c[:g["ndim"]], dt64, P)
        assert nfail == 0
        j = flat_of(g, c)
        num += np.abs(U32[:, j] - Uo)
        den += np.abs(Uo)
    samp = {VARS[k]: float(num[k] / den[k]) for k in range(12) if den[k] > 0}
    print(f"{w.name} FP32-bulk one step, rel L1 vs FP64 (whole grid):",
          {k: "%.2e" % v for k, v in l1.items()})
    print(f"{w.name} FP32-bulk one step, rel L1 vs oracle (samples):",
          {k: "%.2e" % v for k, v in samp.items()})
    for k, v in l1.items():
        assert v <= 1e-5, (k, v)
    for k, v in samp.items():
        assert v <= 1e-5, (k, v)


# blast edge (r = 0.1 around the centre) and random cells
C2_EDGE = [(614, 512), (512, 410), (584, 584), (512, 512)]


def test_c2_full_size_fp64_sampled_bitwise(c2):
    check_fp64(c2, samples(c2, 8, 21, C2_EDGE))


def test_c2_full_size_fp32_bulk(c2):
    check_fp32_bulk(c2, samples(c2, 8, 22, C2_EDGE))


def test_c3_full_size_fp64_sampled_bitwise(c3):
    check_fp64(c3, samples(c3, 5, 31))


def test_c3_full_size_fp32_bulk(c3):
    check_fp32_bulk(c3, samples(c3, 5, 32))

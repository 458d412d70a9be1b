"""FP32-bulk form against the FP64 oracle.

Faces (PLM, fluxes, PVM-int-8 with tangent products) and the flux difference in
FP32; cell con2prim, implicit solve and U accumulation in FP64.  The bounds:
per-variable relative L1 <= 1e-5 against the FP64 oracle, and below the oracle's
own N-vs-2N truncation difference on the C0 shock tube.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import gpu_context, oracle_grid, oracle_params, oracle_run_instance
from paper_2212_00370_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARS = ["D", "Sx", "Sy", "Sz", "tau", "Bx", "By", "Bz", "E", "Fx", "Fy", "Fz"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_00370_gb300 import build
    build.build()


def rel_l1(a, b):
    """Per-variable relative L1 sum|a-b| / sum|b| (variables with sum|b| = 0 skipped)."""
    out = {}
    for k in range(12):
        den = np.abs(b[k]).sum()
        if den > 0:
            out[VARS[k]] = float(np.abs(a[k] - b[k]).sum() / den)
    return out


def _oracle_faces(w, d, P):
    out = []
    for i in range(w.n_inst):
        g, V, kappa, sigma = w.instance(i)
        V = np.ascontiguousarray(V)
        F = O.face_flux(oracle_grid(g), d, O.prim2con(V, P), V, kappa, sigma, P)
        out.append(F.reshape(12, -1))
    return np.concatenate(out, axis=1)


def test_fp32_faces_track_fp64_faces():
    w = W.riemann_batch(24, seed=11, nmin=16, nmax=140)
    F64 = _oracle_faces(w, 0, oracle_params(w))
    ctx = gpu_context(w, precision="fp32_bulk")
    F32 = ctx.flux_sweep(0).cpu().numpy()
    err = np.abs(F32 - F64).max(0) / np.maximum(np.abs(F64).max(0), 1e-30)
    print("face relative error: median %.2e  p99 %.2e  max %.2e" % (
        np.median(err), np.percentile(err, 99), err.max()))
    assert np.median(err) < 1e-5
    assert np.percentile(err, 99) < 1e-3


def test_fp32_bulk_c0_to_t_end_within_bounds():
    w = W.shock_tube(400)
    ctx = gpu_context(w, precision="fp32_bulk")
    ctx.imex_step(10000)
    U32 = ctx.get_state()[0].cpu().numpy()
    assert ctx.inst_status()[0] == 0 and ctx.get_times()[0][0] == 0.4
    U64 = oracle_run_instance(w, 0, 10000)[0]
    # the oracle's own N-vs-2N truncation difference (2N averaged onto N)
    w2 = W.shock_tube(800)
    U2 = oracle_run_instance(w2, 0, 10000)[0]
    U2c = 0.5 * (U2[:, 0::2] + U2[:, 1::2])
    e32 = rel_l1(U32, U64)
    trunc = rel_l1(U2c, U64)
    print("FP32-bulk rel L1:", {k: "%.2e" % v for k, v in e32.items()})
    print("N vs 2N   rel L1:", {k: "%.2e" % v for k, v in trunc.items()})
    for k, v in e32.items():
        assert v <= 1e-5, (k, v)
        assert v < trunc[k], (k, v, trunc[k])


def test_fp32_bulk_c1_steps():
    w = W.riemann_batch(40, seed=23, nmin=20, nmax=200)
    ctx = gpu_context(w, precision="fp32_bulk")
    ctx.imex_step(5)
    U32 = ctx.get_state()[0].cpu().numpy()
    st = ctx.inst_status()
    off = w.cell_offsets()
    worst = {}
    for i in range(w.n_inst):
        Ur, Vr, tr, steps, nfail = oracle_run_instance(w, i, 5)
        if nfail or st[i]:
            continue
        for k, v in rel_l1(U32[:, off[i]:off[i + 1]], Ur).items():
            worst[k] = max(worst.get(k, 0.0), v)
    print("C1 5 steps, worst per-variable rel L1:", {k: "%.2e" % v for k, v in worst.items()})
    assert max(worst.values()) < 1e-3

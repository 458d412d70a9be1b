"""FP64 form with exact tangent products (pvm_products = 1) against the oracle.

The paper forms A w by nested flux differences with eps = 1e-8 (Eq. utilde); the
tangent variant differentiates F(c2p(U)) exactly, with the same reconstruction,
central fluxes and beta.  The two differ by the finite-difference error,
O(eps |w|) relative plus O(eps_mach / eps) of rounding in the products, about
1e-8 of the viscous term.  The bounds below are that error with margin.  The
viscous term must still differ from the finite-difference one (a real switch).
"""
import numpy as np
import pytest

from gpu_helpers import gpu_context, oracle_params, oracle_run_instance
from paper_2212_00370_gb300 import workloads as W
from test_gpu_parity import _oracle_faces

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
    out = {}
    for k in range(12):
        den = np.abs(b[k]).sum()
        if den > 0:
            out[VARS[k]] = float(np.abs(a[k] - b[k]).sum() / den)
    return out


@pytest.mark.parametrize("pvm_k", [3, 4])
def test_tangent_faces_match_finite_differences(pvm_k):
    w = W.riemann_batch(24, seed=11, nmin=16, nmax=140)
    Ffd = _oracle_faces(w, 0, oracle_params(w, pvm_k=pvm_k))
    Ft = gpu_context(w, pvm_products="tangent", pvm_k=pvm_k).flux_sweep(0).cpu().numpy()
    err = np.abs(Ft - Ffd).max(0) / np.maximum(np.abs(Ffd).max(0), 1e-30)
    print("FP64 tangent vs FD faces (k=%d): median %.2e p99 %.2e max %.2e" % (
        pvm_k, np.median(err), np.percentile(err, 99), err.max()))
    assert not np.array_equal(Ft, Ffd)
    assert np.median(err) < 1e-8
    assert np.percentile(err, 99) < 1e-6


def test_tangent_c0_to_t_end():
    w = W.shock_tube(400)
    ctx = gpu_context(w, pvm_products="tangent")
    ctx.imex_step(10000)
    assert ctx.inst_status()[0] == 0 and ctx.get_times()[0][0] == 0.4
    Ut = ctx.get_state()[0].cpu().numpy()
    Ur = oracle_run_instance(w, 0, 10000)[0]
    e = rel_l1(Ut, Ur)
    print("FP64 tangent C0 t_end rel L1:", {k: "%.2e" % v for k, v in e.items()})
    assert max(e.values()) < 1e-7


def test_tangent_c1_steps():
    w = W.riemann_batch(40, seed=23, nmin=20, nmax=200)
    ctx = gpu_context(w, pvm_products="tangent")
    ctx.imex_step(5)
    U = ctx.get_state()[0].cpu().numpy()
    st = ctx.inst_status()
    off = w.cell_offsets()
    worst = {}
    for i in range(w.n_inst):
        Ur, Vr, tr, steps, nfail = oracle_run_instance(w, i, 5)
        if nfail or st[i]:
            continue
        for k, v in rel_l1(U[:, off[i]:off[i + 1]], Ur).items():
            worst[k] = max(worst.get(k, 0.0), v)
    print("FP64 tangent C1 5 steps, worst rel L1:", {k: "%.2e" % v for k, v in worst.items()})
    assert max(worst.values()) < 1e-6

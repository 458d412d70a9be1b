"""beta_mode 2 on the GPU against the oracle: Eq. beta damps the PVM viscosity of the
radiation block (E_r, F_r) only, beta = 1 on the magnetofluid (a variant; the paper
leaves other choices of beta open, Sec. 5).

FP64: faces bit for bit (1D, 2D, 3D), whole C1 steps, and the optically thick
radiative pulse run to t = 600.  FP32-bulk and FP64 tangent faces: within their
forms' error of the FP64 oracle.
"""
import numpy as np
import pytest

from gpu_helpers import compare_bitwise, gpu_context, oracle_params
from paper_2212_00370_gb300 import workloads as W
from test_gpu_parity import _check_instances, _gpu_steps, _oracle_faces

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

B = "radiation"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_00370_gb300 import build
    build.build()


def test_faces_bitwise():
    w = W.riemann_batch(24, seed=11, nmin=16, nmax=140)
    P = oracle_params(w, beta=B)
    F = gpu_context(w, beta=B).flux_sweep(0).cpu().numpy()
    compare_bitwise(F, _oracle_faces(w, 0, P), "beta_mode 2 faces")
    # a real switch: the magnetofluid rows differ from beta_mode 1 where beta < 1
    F1 = gpu_context(w, beta=True).flux_sweep(0).cpu().numpy()
    F0 = gpu_context(w, beta=False).flux_sweep(0).cpu().numpy()
    compare_bitwise(F[:8], F0[:8], "magnetofluid rows = beta 1")
    compare_bitwise(F[8:], F1[8:], "radiation rows = Eq. beta")
    assert not np.array_equal(F[:8], F1[:8])
    for w in (W.blast_2d(20), W.turbulent_3d(8)):
        P = oracle_params(w, beta=B)
        ctx = gpu_context(w, beta=B)
        for d in range(w.grids[0]["ndim"]):
            compare_bitwise(ctx.flux_sweep(d).cpu().numpy(), _oracle_faces(w, d, P),
                            f"{w.name} dir {d}")


def test_c1_steps_bitwise():
    w = W.riemann_batch(40, seed=23, nmin=20, nmax=200)
    U, V, t, st = _gpu_steps(w, 3, beta=B)
    _check_instances(w, U, V, t, st, 3, P=oracle_params(w, beta=B))


def test_pulse_bitwise():
    from test_oracle_radhll import A_R, pulse_exact
    N = 100
    x = -50 + (np.arange(N) + 0.5)
    V = np.zeros((12, N))
    V[0], V[4] = 1.0, 1.0
    V[8] = pulse_exact(x, 0.0, 1.0)
    w = W.Workload("pulse", [W.grid1d(N, length=100.0)], V, np.zeros(N), np.full(N, 100.0),
                   np.array([600.0]), 5 / 3, A_R, 0.4)
    U, Vg, t, st = _gpu_steps(w, 3000, beta=B)
    assert st[0] == 0 and t[0] == 600.0
    _check_instances(w, U, Vg, t, st, 3000, P=oracle_params(w, beta=B))


@pytest.mark.parametrize("opts", [dict(precision="fp32_bulk"), dict(pvm_products="tangent")])
def test_fp32_and_tangent_faces(opts):
    w = W.riemann_batch(24, seed=11, nmin=16, nmax=140)
    F64 = _oracle_faces(w, 0, oracle_params(w, beta=B))
    F = gpu_context(w, beta=B, **opts).flux_sweep(0).cpu().numpy()
    err = np.abs(F - F64).max(0) / np.maximum(np.abs(F64).max(0), 1e-30)
    print("%s beta_mode 2 face relative error: median %.2e  p99 %.2e" % (
        opts, np.median(err), np.percentile(err, 99)))
    assert np.median(err) < 1e-6
    assert np.percentile(err, 99) < 1e-4

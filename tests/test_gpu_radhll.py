"""Radiative HLL (Sec. 3.2.1) on the GPU against the oracle.

FP64: faces bit for bit (1D, 2D, 3D; Eq. limits on and off), whole C1 steps, and
the optically thick radiative pulse run to t = 600 (implicit scattering solve in
every cell).  FP32-bulk: faces within FP32 rounding of the FP64 oracle.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import compare_bitwise, gpu_context, oracle_params
from paper_2212_00370_gb300 import workloads as W
from test_gpu_parity import _check_instances, _gpu_steps, _oracle_faces

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_00370_gb300 import build
    build.build()


@pytest.mark.parametrize("beta", [True, False])
def test_radhll_faces_bitwise(beta):
    w = W.riemann_batch(24, seed=11, nmin=16, nmax=140)
    P = oracle_params(w, solver="radhll", beta=beta)
    F = gpu_context(w, solver="radhll", beta=beta).flux_sweep(0).cpu().numpy()
    compare_bitwise(F, _oracle_faces(w, 0, P), "Rad-HLL faces")
    for w in (W.blast_2d(20), W.turbulent_3d(8)):
        P = oracle_params(w, solver="radhll", beta=beta)
        ctx = gpu_context(w, solver="radhll", beta=beta)
        for d in range(w.grids[0]["ndim"]):
            compare_bitwise(ctx.flux_sweep(d).cpu().numpy(), _oracle_faces(w, d, P),
                            f"{w.name} dir {d}")


def test_radhll_c1_steps_bitwise():
    w = W.riemann_batch(40, seed=23, nmin=20, nmax=200)
    U, V, t, st = _gpu_steps(w, 3, solver="radhll")
    _check_instances(w, U, V, t, st, 3, P=oracle_params(w, solver="radhll"))


def test_radhll_pulse_bitwise():
    from test_oracle_radhll import A_R, pulse_exact
    N = 100
    x = -50 + (np.arange(N) + 0.5)
    V = np.zeros((12, N))
    V[0], V[4] = 1.0, 1.0
    V[8] = pulse_exact(x, 0.0, 1.0)
    w = W.Workload("pulse", [W.grid1d(N, length=100.0)], V, np.zeros(N), np.full(N, 100.0),
                   np.array([600.0]), 5 / 3, A_R, 0.4)
    for solver in ("radhll", "pvm"):
        U, Vg, t, st = _gpu_steps(w, 3000, solver=solver)   # about 1040 steps to t = 600
        assert st[0] == 0 and t[0] == 600.0
        _check_instances(w, U, Vg, t, st, 3000, P=oracle_params(w, solver=solver))


def test_radhll_fp32_bulk_faces():
    w = W.riemann_batch(24, seed=11, nmin=16, nmax=140)
    F64 = _oracle_faces(w, 0, oracle_params(w, solver="radhll"))
    F32 = gpu_context(w, precision="fp32_bulk", solver="radhll").flux_sweep(0).cpu().numpy()
    err = np.abs(F32 - F64).max(0) / np.maximum(np.abs(F64).max(0), 1e-30)
    print("Rad-HLL FP32 face relative error: median %.2e  p99 %.2e" % (
        np.median(err), np.percentile(err, 99)))
    assert np.median(err) < 1e-6
    assert np.percentile(err, 99) < 1e-4

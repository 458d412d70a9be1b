"""PVM-int-16 (Eq. iterat with k = 4: eight A^2 products per face) on the GPU.

The paper reports testing this variant; its coefficients are the recurrence's,
pinned in the oracle tests.  FP64: bit for bit against the oracle (faces in 1D,
2D and 3D, and whole steps of a C1 batch).  FP32-bulk: against the FP64 oracle
within the FP32 bounds.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import compare_bitwise, gpu_context, oracle_grid, oracle_params
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


def test_pvm16_faces_bitwise():
    w = W.riemann_batch(24, seed=11, nmin=16, nmax=140)
    P = oracle_params(w, pvm_k=4)
    ctx = gpu_context(w, pvm_k=4)
    F16 = ctx.flux_sweep(0).cpu().numpy()
    compare_bitwise(F16, _oracle_faces(w, 0, P), "PVM-int-16 faces")
    F8 = gpu_context(w).flux_sweep(0).cpu().numpy()
    assert not np.array_equal(F16, F8)   # a different solver, not a silent PVM-int-8
    for w in (W.blast_2d(20), W.turbulent_3d(8)):
        P = oracle_params(w, pvm_k=4)
        ctx = gpu_context(w, pvm_k=4)
        for d in range(w.grids[0]["ndim"]):
            compare_bitwise(ctx.flux_sweep(d).cpu().numpy(), _oracle_faces(w, d, P),
                            f"{w.name} dir {d}")


def test_pvm16_c1_steps_bitwise():
    w = W.riemann_batch(40, seed=23, nmin=20, nmax=200)
    U, V, t, st = _gpu_steps(w, 3, pvm_k=4)
    _check_instances(w, U, V, t, st, 3, P=oracle_params(w, pvm_k=4))


def test_pvm16_fp32_bulk_faces_track_the_oracle():
    w = W.riemann_batch(24, seed=11, nmin=16, nmax=140)
    F64 = _oracle_faces(w, 0, oracle_params(w, pvm_k=4))
    F32 = gpu_context(w, precision="fp32_bulk", pvm_k=4).flux_sweep(0).cpu().numpy()
    err = np.abs(F32 - F64).max(0) / np.maximum(np.abs(F64).max(0), 1e-30)
    print("PVM-int-16 FP32 face relative error: median %.2e  p99 %.2e" % (
        np.median(err), np.percentile(err, 99)))
    assert np.median(err) < 1e-5
    assert np.percentile(err, 99) < 1e-3


def test_invalid_pvm_order_is_rejected():
    from paper_2212_00370_gb300 import rrmhd
    w = W.riemann_batch(2, seed=1, nmin=10, nmax=12)
    with pytest.raises(rrmhd.RRMHDError) as e:
        gpu_context(w, pvm_k=5)
    assert e.value.code == 10

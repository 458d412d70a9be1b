"""Checkpoints: a run restored from a checkpoint continues bit for bit as the run
that wrote it (state, Jacobian cache of the implicit solve, times, statuses, the
staggered face field under constrained transport), in the same context or in a
new one with other launch shapes, from a device or a host buffer."""
import numpy as np
import pytest

from gpu_helpers import compare_bitwise, gpu_context
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


def _snap(ctx):
    U, V = ctx.get_state()
    t, dt = ctx.get_times()
    return U.cpu().numpy(), V.cpu().numpy(), t, dt, ctx.inst_status(), ctx.first_bad_cell()


def _same(a, b, what):
    compare_bitwise(a[0], b[0], what + " U")
    compare_bitwise(a[1], b[1], what + " V")
    for k in range(2, 6):
        assert np.array_equal(a[k], b[k]), (what, k)


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_restore_continues_bit_for_bit(precision):
    w = W.riemann_batch(40, seed=23, nmin=20, nmax=300)
    ctx = gpu_context(w, precision=precision, lanes=3)
    ctx.set_times(np.zeros(w.n_inst), np.where(np.arange(w.n_inst) % 4 == 0, 5e-3, np.inf))
    ctx.imex_step(3)
    dev = ctx.checkpoint()
    host = ctx.checkpoint(device=False)
    ctx.imex_step(4)
    ref = _snap(ctx)
    # the same context, from the device buffer
    ctx.checkpoint_restore(dev)
    ctx.imex_step(4)
    _same(_snap(ctx), ref, "same context")
    # a new context with other launch shapes, from the host buffer
    ctx2 = gpu_context(w, precision=precision, lanes=5)
    ctx2.set_tuning(cell_block=32, face_block=256, lanes=5)
    torch.cuda.synchronize()
    ctx2.checkpoint_restore(host)
    ctx2.imex_step(2)
    ctx2.imex_step(2)
    _same(_snap(ctx2), ref, "new context")
    # a restart from the state alone empties the Jacobian cache: not the same run
    ctx3 = gpu_context(w, precision=precision)
    ctx3.checkpoint_restore(dev)
    U, V = ctx3.get_state()
    ctx3.set_state(V.clone())
    ctx3.imex_step(4)
    assert not np.array_equal(_snap(ctx3)[0], ref[0])
    for c in (ctx, ctx2, ctx3):
        c.close()


def test_restore_under_constrained_transport():
    w = W.blast_2d(48)
    ctx = gpu_context(w, ct=1)
    ctx.imex_step(3)
    buf = ctx.checkpoint()
    ctx.imex_step(3)
    ref = _snap(ctx)
    bref = ctx.get_face_field().cpu().numpy()
    ctx2 = gpu_context(w, ct=1)
    ctx2.checkpoint_restore(buf)
    ctx2.imex_step(3)
    _same(_snap(ctx2), ref, "ct")
    compare_bitwise(ctx2.get_face_field().cpu().numpy(), bref, "ct face field")
    ctx.close()
    ctx2.close()


def test_checkpoint_of_another_layout_is_rejected():
    w = W.riemann_batch(6, seed=3, nmin=20, nmax=40)
    ctx = gpu_context(w)
    buf = ctx.checkpoint()
    other = gpu_context(W.riemann_batch(7, seed=4, nmin=20, nmax=40))
    with pytest.raises(rrmhd.RRMHDError) as e:
        other.checkpoint_restore(buf)
    assert e.value.code == 10
    bulk = gpu_context(w, precision="fp32_bulk")
    with pytest.raises(rrmhd.RRMHDError):
        bulk.checkpoint_restore(buf)
    for c in (ctx, other, bulk):
        c.close()

"""Launch shapes and the autotuner.

Shapes (block size, items per thread, grid or persistent schedule, lanes) only
change how faces and cells are spread over threads; every item is computed once
by the same arithmetic, so results must be bit-identical under every shape.  The
autotuner times real steps from the context's state and must leave that state
exactly as it found it.
"""
import numpy as np
import pytest

from gpu_helpers import compare_bitwise, gpu_context
from paper_2212_00370_gb300 import rrmhd
from paper_2212_00370_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [
    dict(face_block=32, face_per_thread=1, face_persistent=0, cell_block=32, cell_per_thread=2,
         cell_persistent=0, lanes=1),
    dict(face_block=256, face_per_thread=2, face_persistent=0, cell_block=64, cell_per_thread=1,
         cell_persistent=1, lanes=3),
    dict(face_block=64, face_per_thread=1, face_persistent=1, cell_block=256, cell_per_thread=1,
         cell_persistent=1, lanes=16),
    dict(face_block=128, face_per_thread=2, face_persistent=0, cell_block=128, cell_per_thread=2,
         cell_persistent=0, lanes=5),
    dict(face_block=8, face_per_thread=1, face_persistent=0, cell_block=16, cell_per_thread=1,
         cell_persistent=0, lanes=2),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_00370_gb300 import build
    build.build()


def run(w, precision, steps, shape=None):
    ctx = gpu_context(w, precision=precision)
    if shape:
        ctx.set_tuning(**shape)
        assert ctx.get_tuning() == shape
    ctx.imex_step(steps)
    U, V = ctx.get_state()
    t, _ = ctx.get_times()
    out = U.cpu().numpy(), V.cpu().numpy(), t, ctx.inst_status()
    ctx.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_results_do_not_depend_on_the_launch_shape(precision):
    w = W.riemann_batch(40, seed=23, nmin=20, nmax=300)
    ref = run(w, precision, 3)
    for shape in SHAPES:
        got = run(w, precision, 3, shape)
        compare_bitwise(got[0], ref[0], f"U under {shape}")
        compare_bitwise(got[1], ref[1], f"V under {shape}")
        assert np.array_equal(got[2], ref[2]) and np.array_equal(got[3], ref[3])


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_one_call_of_n_steps_equals_n_calls(precision):
    """Lanes run the steps of one call back to back without joining in between;
    the result must be that of single steps, also where instances reach t_end at
    different steps and a lane runs out of live instances."""
    w = W.riemann_batch(40, seed=23, nmin=20, nmax=300)
    out = []
    for calls in ([5], [1] * 5, [2, 3]):
        ctx = gpu_context(w, precision=precision, lanes=5)
        ctx.set_times(np.zeros(w.n_inst), np.where(np.arange(w.n_inst) % 3 == 0, 2e-3, np.inf))
        for n in calls:
            ctx.imex_step(n)
        U, V = ctx.get_state()
        t, dt = ctx.get_times()
        out.append((U.cpu().numpy(), V.cpu().numpy(), t, dt, ctx.inst_status()))
        ctx.close()
    for got in out[1:]:
        compare_bitwise(got[0], out[0][0], "U")
        compare_bitwise(got[1], out[0][1], "V")
        for k in (2, 3, 4):
            assert np.array_equal(got[k], out[0][k])
    assert (out[0][2] == 2e-3).sum() > 0          # some instances stopped at t_end


def test_shapes_in_2d_and_3d():
    from test_gpu_parity import _periodic_smooth
    for shape_nd in [(24, 20), (10, 8, 6)]:
        w = _periodic_smooth(shape_nd, 5)
        ref = run(w, "fp64", 2)
        got = run(w, "fp64", 2, SHAPES[2])
        compare_bitwise(got[0], ref[0], f"U {shape_nd}")


def test_unsupported_shape_is_rejected():
    w = W.riemann_batch(4, seed=1, nmin=20, nmax=30)
    ctx = gpu_context(w)
    with pytest.raises(rrmhd.RRMHDError) as e:
        ctx.set_tuning(cell_block=96)
    assert e.value.code == 10
    with pytest.raises(rrmhd.RRMHDError):
        ctx.set_tuning(cell_persistent=1, cell_per_thread=2)
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_autotune_leaves_the_state_and_results_unchanged(precision):
    w = W.riemann_batch(64, seed=29, nmin=50, nmax=400)
    ref = run(w, precision, 2)
    ctx = gpu_context(w, precision=precision)
    ctx.imex_step(1)
    U1, V1 = [x.cpu().numpy() for x in ctx.get_state()]
    t1, _ = ctx.get_times()
    best, ms = ctx.autotune(repeats=1)
    assert ms > 0 and ctx.get_tuning() == best
    U1b, V1b = [x.cpu().numpy() for x in ctx.get_state()]
    compare_bitwise(U1b, U1, "U after autotune")
    compare_bitwise(V1b, V1, "V after autotune")
    assert np.array_equal(ctx.get_times()[0], t1)
    ctx.imex_step(1)
    U2, V2 = ctx.get_state()
    compare_bitwise(U2.cpu().numpy(), ref[0], "U, step after autotune")
    compare_bitwise(V2.cpu().numpy(), ref[1], "V, step after autotune")
    ctx.close()


def test_server_with_a_tuning_matches_the_default():
    from test_gpu_serving import GAMMA, grid_of, small_requests
    reqs = small_requests(6, seed=17)
    outs = []
    for tuning in (None, SHAPES[1]):
        srv = rrmhd.Server(gamma=GAMMA, precision="fp64", mem_bytes=1 << 28, tuning=tuning)
        ids = {srv.submit(grid_of(r[0]), *r[1:]): j for j, r in enumerate(reqs)}
        srv.wait_idle(120)
        got = {ids[res["id"]]: out for res, out in srv.poll()}
        srv.close()
        outs.append(got)
    for j in outs[0]:
        compare_bitwise(outs[1][j], outs[0][j], f"request {j}")

"""Entry points of the boundary beyond the step: the flux sweep accumulated into a
state (Eq. explicit, one direction), a step with its dt capped, and the first cell
whose failure froze an instance.  FP64 results are compared with the oracle bit
for bit."""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import compare_bitwise, gpu_context, oracle_grid, oracle_params
from paper_2212_00370_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_00370_gb300 import build
    build.build()


def _mixed_workload():
    """Three ragged 1D Riemann problems and one 2D blast (periodic), packed."""
    a = W.riemann_batch(3, seed=41, nmin=17, nmax=90)
    b = W.blast_2d(24)
    return W.Workload("mixed", a.grids + b.grids, np.concatenate([a.V, b.V], 1),
                      np.concatenate([a.kappa, b.kappa]), np.concatenate([a.sigma, b.sigma]),
                      np.concatenate([a.t_end, b.t_end]), 4.0 / 3.0)


def test_flux_accumulate_equals_the_oracle_difference():
    w = _mixed_workload()
    P = oracle_params(w)
    ctx = gpu_context(w)
    off = w.cell_offsets()
    for d, dtw in ((0, 1.7e-3), (1, 2.3e-3)):
        U = ctx.get_state()[0].clone()
        ctx.flux_accumulate(d, dtw, U)
        got = U.cpu().numpy()
        for i in range(w.n_inst):
            g, V, kappa, sigma = w.instance(i)
            V = np.ascontiguousarray(V)
            Ui = O.prim2con(V, P)
            if d < g["ndim"]:
                og = oracle_grid(g)
                F = O.face_flux(og, d, Ui, V, kappa, sigma, P)
                n = list(g["n"])
                Fd = F.reshape(12, n[2], n[1] + (d == 1), n[0] + (d == 0))
                lo = [slice(None)] * 4
                hi = [slice(None)] * 4
                axis = 3 - d
                lo[axis] = slice(0, -1)
                hi[axis] = slice(1, None)
                dF = (Fd[tuple(hi)] - Fd[tuple(lo)]).reshape(12, -1)
                ref = Ui - dF * (dtw / g["dx"][d])
            else:
                ref = Ui
            compare_bitwise(got[:, off[i]:off[i + 1]], ref, "instance %d dir %d" % (i, d))
    ctx.close()


def test_flux_accumulate_fp32_bulk_tracks_fp64():
    w = _mixed_workload()
    ctx64 = gpu_context(w)
    ctx32 = gpu_context(w, precision="fp32_bulk")
    U64 = ctx64.get_state()[0].clone()
    U32 = ctx32.get_state()[0].clone()
    ctx64.flux_accumulate(0, 2e-3, U64)
    ctx32.flux_accumulate(0, 2e-3, U32)
    U0 = ctx64.get_state()[0]
    d64, d32 = (U64 - U0).cpu().numpy(), (U32 - U0).cpu().numpy()
    err = np.abs(d32 - d64).sum(1) / np.maximum(np.abs(d64).sum(1), 1e-300)
    assert err.max() < 1e-4, err
    ctx64.close()
    ctx32.close()


def test_step_with_capped_dt_equals_the_oracle():
    w = W.riemann_batch(6, seed=43, nmin=20, nmax=120)
    P = oracle_params(w)
    ctx = gpu_context(w)
    ctx.set_times(np.zeros(w.n_inst), np.full(w.n_inst, np.inf))
    # the CFL dt of each instance, then a cap below the smallest of them
    dts = [O.grid_dt(oracle_grid(g), np.ascontiguousarray(V), P)
           for g, V, _, _ in (w.instance(i) for i in range(w.n_inst))]
    cap = 0.5 * min(dts)
    taken = ctx.imex_step_dt(cap)
    assert np.all(taken == cap)
    got = ctx.get_state()[0].cpu().numpy()
    off = w.cell_offsets()
    for i in range(w.n_inst):
        g, V, kappa, sigma = w.instance(i)
        og = oracle_grid(g)
        V = np.ascontiguousarray(V).copy()
        U = O.prim2con(V, P)
        assert O.step(og, cap, U, V, kappa, sigma, P, jcache=np.zeros(17 * og.ncells)) == 0
        compare_bitwise(got[:, off[i]:off[i + 1]], U, "capped step, instance %d" % i)
    # the next plain step is not capped
    ctx.imex_step(1)
    assert np.all(ctx.get_times()[1] > cap)
    ctx.close()


def test_first_bad_cell_of_a_failing_instance():
    """C1 instance 3934 fails at its 29th step (no con2prim root even with first-order
    faces, a magnetisation of ~500); instance 3933 does not."""
    full = W.riemann_batch(4096, seed=W.SEED_BASE + 1)
    w = full.subset([3933, 3934])
    ctx = gpu_context(w)
    ctx.set_times(np.zeros(2), np.full(2, np.inf))
    assert list(ctx.first_bad_cell()) == [-1, -1]
    ctx.imex_step(40)
    st = ctx.inst_status()
    bad = ctx.first_bad_cell()
    off = w.cell_offsets()
    assert st[0] == 0 and bad[0] == -1
    assert st[1] != 0 and off[1] <= bad[1] < off[2]
    # set_state starts over
    ctx.set_state(torch.tensor(w.V, device="cuda"))
    assert list(ctx.first_bad_cell()) == [-1, -1]
    ctx.close()

"""Parity of the CUDA path with the FP64 oracle, element by element.

The FP64 path promises bit-for-bit the oracle's arithmetic (same IEEE
operation order, no contraction), so every comparison here is exact equality;
that is stricter than the relative-L1 bounds of 1e-12 after one step and
1e-9 at t_end that the benchmark configurations require.  All inputs are the
seeded synthetic workloads; sizes span many tiles and ragged tails.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import (compare_bitwise, gpu_context, oracle_grid, oracle_params,
                         oracle_run_instance)
from paper_2212_00370_gb300 import rrmhd
from paper_2212_00370_gb300 import workloads as W
from test_oracle_physics import random_states

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_00370_gb300 import build
    build.build()


def test_pointwise_prim2con_con2prim_bitwise():
    P = O.Params(gamma=4 / 3)
    V = random_states(20000, 3)
    U_ref = O.prim2con(V, P)
    w = W.shock_tube(8)
    w.gamma = 4 / 3
    ctx = gpu_context(w)
    Vt = torch.tensor(V, device="cuda")
    U = ctx.prim2con(Vt).cpu().numpy()
    compare_bitwise(U, U_ref, "prim2con")
    Z_ref = O.prim_Z(V, P)
    compare_bitwise(ctx.prim_z(Vt).cpu().numpy(), Z_ref, "rho h W^2")
    for Zg in (None, Z_ref * (1 + 1e-3)):
        V_ref, _, st_ref = O.con2prim(U_ref, P, Zguess=Zg)
        Vg, st = ctx.con2prim(torch.tensor(U_ref, device="cuda"),
                              None if Zg is None else torch.tensor(Zg, device="cuda"))
        compare_bitwise(st.cpu().numpy(), st_ref, "con2prim status")
        compare_bitwise(Vg.cpu().numpy(), V_ref, "con2prim")


def _oracle_faces(w, d, P):
    out = []
    for i in range(w.n_inst):
        g, V, kappa, sigma = w.instance(i)
        if g["ndim"] <= d:
            continue
        V = np.ascontiguousarray(V)
        U = O.prim2con(V, P)
        F = O.face_flux(oracle_grid(g), d, U, V, kappa, sigma, P)
        out.append(F.reshape(12, -1))
    return np.concatenate(out, axis=1)


@pytest.mark.parametrize("recon", ["vanleer", "minmod", "mc", "godunov"])
def test_flux_sweep_bitwise_c1_batch(recon):
    w = W.riemann_batch(24, seed=11, nmin=16, nmax=140)
    P = oracle_params(w, recon=recon)
    ctx = gpu_context(w, recon=recon)
    F = ctx.flux_sweep(0).cpu().numpy()
    compare_bitwise(F, _oracle_faces(w, 0, P), f"faces {recon}")


def test_flux_sweep_bitwise_2d_3d():
    w2 = W.blast_2d(20)
    w3 = W.turbulent_3d(8)
    for w in (w2, w3):
        P = oracle_params(w)
        ctx = gpu_context(w)
        for d in range(w.grids[0]["ndim"]):
            compare_bitwise(ctx.flux_sweep(d).cpu().numpy(), _oracle_faces(w, d, P),
                            f"{w.name} dir {d}")


@pytest.mark.parametrize("hdt", [1e-4, 1e-3, 1e-2])
def test_implicit_source_bitwise(hdt):
    rng = np.random.default_rng(17)
    n = 3000
    V = random_states(n, 17)
    w = W.Workload("cells", [W.grid1d(n)], V, 10 ** rng.uniform(-3, 3, n),
                   10 ** rng.uniform(-3, 2, n), np.array([1.0]), 4 / 3)
    P = oracle_params(w)
    Us = O.prim2con(V, P)
    Zg = O.prim_Z(V, P)
    U_ref, V_ref, st_ref = O.implicit(Us, w.kappa, w.sigma, hdt, P, Zguess=Zg)
    ctx = gpu_context(w)
    U, Vg, st = ctx.implicit_source(hdt, torch.tensor(Us, device="cuda"),
                                    torch.tensor(Zg, device="cuda"))
    compare_bitwise(st.cpu().numpy(), st_ref, "implicit status")
    ok = st_ref == 0
    compare_bitwise(U.cpu().numpy()[:, ok], U_ref[:, ok], "implicit U")
    compare_bitwise(Vg.cpu().numpy()[:, ok], V_ref[:, ok], "implicit V")


def _gpu_steps(w, nsteps, **opts):
    ctx = gpu_context(w, **opts)
    ctx.imex_step(nsteps)
    U, V = ctx.get_state()
    t, dt = ctx.get_times()
    return U.cpu().numpy(), V.cpu().numpy(), t, ctx.inst_status()


def _check_instances(w, U, V, t, st, nsteps, idx=None, P=None):
    """Status, state and time of each instance equal the oracle's; a failed
    instance is compared at its last good state (both sides freeze it there)."""
    off = w.cell_offsets()
    for i in (range(w.n_inst) if idx is None else idx):
        Ur, Vr, tr, steps, nfail = oracle_run_instance(w, i, nsteps, P)
        assert (st[i] != 0) == (nfail != 0), (i, st[i], nfail)
        s = slice(off[i], off[i + 1])
        compare_bitwise(U[:, s], Ur, f"instance {i} U")
        compare_bitwise(V[:, s], Vr, f"instance {i} V")
        assert t[i] == tr


def test_c0_one_step_bitwise():
    w = W.shock_tube(400)
    U, V, t, st = _gpu_steps(w, 1)
    _check_instances(w, U, V, t, st, 1)


@pytest.mark.parametrize("kappa", [1.0, 0.0])
def test_c0_to_t_end(kappa):
    """C0 to t_end = 0.4 (about 320 steps): relative L1 <= 1e-9 is required; the
    path is bit-identical."""
    w = W.shock_tube(400, kappa=kappa)
    U, V, t, st = _gpu_steps(w, 10000)
    assert st[0] == 0 and t[0] == 0.4
    _check_instances(w, U, V, t, st, 10000)


def test_c1_batch_several_steps_bitwise():
    w = W.riemann_batch(40, seed=23, nmin=20, nmax=200)
    U, V, t, st = _gpu_steps(w, 3)
    _check_instances(w, U, V, t, st, 3)


# The launch shapes the autotuner picks for the timed C1 batch (FP64 form)
BENCH_FP64_TUNING = dict(face_block=64, cell_block=32, lanes=32)


def test_c1_full_size_sampled():
    """The benchmark workload (4096 instances, 128..2048 cells) in the launch
    configuration it is timed in: one step on the GPU, sampled instances (the
    smallest, the largest, four at random) recomputed one by one by the oracle."""
    w = W.riemann_batch()
    ctx = gpu_context(w, lanes=BENCH_FP64_TUNING["lanes"])
    ctx.set_tuning(**BENCH_FP64_TUNING)
    ctx.imex_step(1)
    U, V = (x.cpu().numpy() for x in ctx.get_state())
    t, st = ctx.get_times()[0], ctx.inst_status()
    n = np.array([g["n"][0] for g in w.grids])
    idx = [int(np.argmin(n)), int(np.argmax(n))] + list(np.random.default_rng(0).choice(w.n_inst, 4, replace=False))
    _check_instances(w, U, V, t, st, 1, idx=idx)
    assert (st != 0).mean() < 0.03


def _periodic_smooth(shape, seed):
    rng = np.random.default_rng(seed)
    nd = len(shape)
    N = int(np.prod(shape))
    X = np.meshgrid(*[(np.arange(n) + 0.5) / n for n in shape], indexing="ij")
    ph = sum(2 * np.pi * X[k] * (k + 1) for k in range(nd))
    flat = lambda a: np.ascontiguousarray(a.T).reshape(-1)
    V = np.zeros((12, N))
    V[0] = flat(1 + 0.5 * np.sin(ph))
    V[1] = flat(0.3 * np.cos(ph))
    V[2] = flat(0.2 * np.sin(2 * ph))
    V[3] = 0.1
    V[4] = flat(0.5 + 0.3 * np.cos(ph))
    V[5], V[6], V[7] = 0.3, 0.2, flat(0.1 * np.cos(ph))
    V[8] = flat(0.8 + 0.5 * np.sin(ph))
    V[9] = V[8] * flat(0.3 * np.cos(ph))
    V[10] = 0.2 * V[8]
    g = {"ndim": nd, "n": tuple(shape) + (1,) * (3 - nd),
         "dx": tuple(1.0 / n for n in shape) + (1.0,) * (3 - nd),
         "bc": ("periodic",) * nd + ("outflow",) * (3 - nd)}
    return W.Workload("periodic-%dd" % nd, [g], V, 10 ** rng.uniform(-1, 1, N),
                      10 ** rng.uniform(-1, 1, N), np.array([np.inf]), 4 / 3)


@pytest.mark.parametrize("shape,steps", [((24, 20), 2), ((10, 8, 6), 1)])
def test_multid_periodic_bitwise(shape, steps):
    w = _periodic_smooth(shape, 5)
    U, V, t, st = _gpu_steps(w, steps)
    _check_instances(w, U, V, t, st, steps)


def test_ragged_and_degenerate_sizes():
    """Instances of 1, 2, 3, 5, 127, 128, 129 cells, outflow and periodic, in one batch."""
    base = W.riemann_batch(14, seed=31, nmin=8, nmax=12)
    grids, Vs, ks, ss = [], [], [], []
    sizes = [1, 2, 3, 5, 127, 128, 129]
    for j, n in enumerate(sizes * 2):
        g, V, k, s = base.instance(j)
        bc = "periodic" if j >= len(sizes) else "outflow"
        idx = np.arange(n) * V.shape[1] // n
        grids.append(W.grid1d(n, bc=bc))
        Vs.append(V[:, idx])
        ks.append(k[idx])
        ss.append(s[idx])
    w = W.Workload("ragged", grids, np.ascontiguousarray(np.concatenate(Vs, 1)), np.concatenate(ks),
                   np.concatenate(ss), np.full(len(grids), 0.2), 4 / 3)
    U, V, t, st = _gpu_steps(w, 2)
    _check_instances(w, U, V, t, st, 2)


def test_failure_is_isolated_to_its_instance():
    w = W.riemann_batch(3, seed=41, nmin=32, nmax=40)
    off = w.cell_offsets()
    w.V[8, off[1] + 5] = 0.0          # E_r = 0: inadmissible cell in instance 1
    U, V, t, st = _gpu_steps(w, 2)
    assert st[1] != 0
    _check_instances(w, U, V, t, st, 2, idx=[0, 2])   # the others follow the oracle, failures included


def test_invalid_arguments():
    with pytest.raises(rrmhd.RRMHDError) as e:
        rrmhd.Context([rrmhd.make_grid(1, (0,), (0.1,))])
    assert e.value.code == 10
    with pytest.raises(rrmhd.RRMHDError):
        rrmhd.Context([rrmhd.make_grid(1, (8,), (0.1,))], gamma=1.0)


def test_host_buffer_entry_continues_and_restarts_bitwise():
    """rrmhd_imex_step_host: a run fed its own previous output continues exactly as
    the device path; any other input restarts from it like set_state."""
    w = W.riemann_batch(30, seed=19, nmin=20, nmax=200)
    ref = gpu_context(w)
    ref.imex_step(4)
    Vref = ref.get_state()[1].cpu().numpy()
    ctx = gpu_context(w)
    h_in = np.ascontiguousarray(w.V.copy())
    h_out = np.empty_like(h_in)
    for _ in range(4):
        ctx.imex_step_host(h_in, h_out, 1)
        h_in, h_out = h_out.copy(), h_in
    compare_bitwise(h_in, Vref, "continuing host-buffer run")
    # another state on the same grids restarts from it, as a fresh context would
    V2 = np.ascontiguousarray(w.V.copy())
    V2[0] *= 1.01
    ctx.imex_step_host(V2, h_out, 2)
    w2 = W.Workload("restart", w.grids, V2, w.kappa, w.sigma, w.t_end, w.gamma)
    fresh = gpu_context(w2)
    fresh.imex_step(2)
    compare_bitwise(h_out, fresh.get_state()[1].cpu().numpy(), "restarted host-buffer run")

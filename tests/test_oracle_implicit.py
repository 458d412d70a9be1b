"""Pins of the oracle's implicit radiation-matter step (Sec. 3.3).

  * static gas (v = 0, B = 0, F_r = 0): the step reduces to the scalar equation
    E (1 + k) = E* + k a_R T^4 with T = (gamma-1)(tau_t - E)/rho, k = h rho kappa,
    solved here by bisection to machine precision, from weakly coupled to the
    stiff limit where E -> a_R T^4 at fixed total energy;
  * the matrix C^(m) of Sec. 3.3 step 2 reproduces the residual built from
    Eqs. g0/gi when matter and Eddington tensor are frozen (sign of C_{i+1,j+1});
  * for general states the result conserves D, B, tau_e + E_r, S + F_r exactly,
    is consistent with con2prim, and zeroes X - X* + h G(X, V(X)) with the
    four-force pinned by Lorentz covariance in test_oracle_physics;
  * Picard (paper) and Newton agree where Picard converges;
  * the matter-primitive form solves the same equations: it agrees with the
    iteration on X where both converge, and where the radiation carries nearly
    all the energy (the iteration on X fails) its result conserves the totals
    and zeroes the residual;
  * the result is a function of the cell's state, not of the solver's path: on
    C1 cell states at the three stage weights the solve with the cell's
    Jacobian cache, the solve without it and a plain damped Newton iteration
    written here from Sec. 3.3 agree to 1e-12 per component;
  * a run restarted with an empty cache: one step later it equals the
    continuing run to 1e-12 (Rad-HLL); with the paper's PVM-int-8, whose
    epsilon = 1e-8 differences turn any one-ulp change into ~1e-8, a restart
    moves the run no more than a one-ulp perturbation of its state does.
"""
import numpy as np
import pytest

import oracle as O
from test_oracle_physics import random_states


def _static_reference(rho, p, E0, k, a, g):
    taut = p / (g - 1) + E0

    def res(E):
        T = (g - 1) * (taut - E) / rho
        return E * (1 + k) - E0 - k * a * T ** 4

    lo, hi = 0.0, taut
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if res(mid) > 0:
            hi = mid
        else:
            lo = mid
    E = 0.5 * (lo + hi)
    return E, (g - 1) * (taut - E)


@pytest.mark.parametrize("k", [1e-4, 1e-1, 10.0, 1e3, 1e6])
@pytest.mark.parametrize("case", ["cold_gas_hot_radiation", "hot_gas_cold_radiation"])
def test_static_closed_form(k, case):
    g = 5 / 3
    a = 1.0
    rho, p, E0 = (2.0, 0.01, 3.0) if case == "cold_gas_hot_radiation" else (0.5, 2.0, 1e-3)
    P = O.Params(gamma=g, a_rad=a)
    V = np.array([rho, 0, 0, 0, p, 0, 0, 0, E0, 0, 0, 0])
    Us = O.prim2con(V, P)
    kappa, hdt = 1.0, k / rho
    U, Vn, st = O.implicit(Us, kappa, 0.7, hdt, P, Zguess=O.prim_Z(V, P))
    assert st == 0
    E, pe = _static_reference(rho, p, E0, k, a, g)
    assert U[8] == pytest.approx(E, rel=1e-12)
    assert Vn[4] == pytest.approx(pe, rel=1e-10, abs=1e-14 * (p / (g - 1) + E0))
    np.testing.assert_array_equal(U[9:], 0.0)
    np.testing.assert_array_equal(Vn[1:4], 0.0)
    # approach to equilibrium: E - a_R T^4 = (E* - a_R T^4)/(1 + k)
    aT4 = a * (Vn[4] / Vn[0]) ** 4
    assert abs(U[8] - aT4) <= 1.000001 * abs(E0 - aT4) / (1 + k) + 1e-12 * (E0 + aT4)


@pytest.mark.parametrize("seed", range(3))
def test_picard_matrix_reproduces_four_force(seed):
    rng = np.random.default_rng(seed)
    for _ in range(20):
        kappa, sigma = 10 ** rng.uniform(-2, 2), 10 ** rng.uniform(-2, 2)
        hdt, rho = 10 ** rng.uniform(-3, 0), 10 ** rng.uniform(-2, 1)
        u = rng.normal(size=3) * rng.uniform(0, 2)
        W = np.sqrt(1 + u @ u)
        BP = 10 ** rng.uniform(-2, 1)
        El = 10 ** rng.uniform(-1, 1)
        n = rng.normal(size=3)
        Fl = rng.uniform(0, 0.9) * El * n / np.linalg.norm(n)
        Dr = O.m1_pressure(El, Fl) / El
        Xs = np.array([1.3, 0.2, -0.1, 0.3])
        X = np.array([0.9, -0.3, 0.2, 0.1])
        Cm, rhs = O.picard_matrix(kappa, sigma, hdt, rho, u, W, BP, Dr, Xs)
        G = O.four_force(kappa, sigma, rho, u, W, BP, X[0], X[1:], Dr * X[0])
        R = X - Xs + hdt * G
        scale = 1 + hdt * rho * (kappa + sigma) * (W ** 3) * (1 + BP)
        np.testing.assert_allclose(Cm @ X - rhs, R, rtol=0, atol=1e-13 * scale)


def _c1_cells(n, seed):
    rng = np.random.default_rng(seed)
    V = random_states(n, seed)
    kappa = 10 ** rng.uniform(-3, 3, n)
    sigma = 10 ** rng.uniform(-3, 2, n)
    return V, kappa, sigma


@pytest.mark.parametrize("hdt", [1e-4, 1e-3, 1e-2])
def test_general_solution_conserves_and_solves(hdt):
    g = 4 / 3
    P = O.Params(gamma=g, a_rad=1.0)
    V, kappa, sigma = _c1_cells(400, 7)
    Us = O.prim2con(V, P)
    U, Vn, st = O.implicit(Us, kappa, sigma, hdt, P, Zguess=O.prim_Z(V, P))
    assert (st == 0).all(), np.where(st != 0)
    np.testing.assert_array_equal(U[0], Us[0])
    np.testing.assert_array_equal(U[5:8], Us[5:8])
    tot = np.abs(Us[4]) + Us[8]
    assert np.all(np.abs((U[4] + U[8]) - (Us[4] + Us[8])) <= 4e-16 * tot)
    assert np.all(np.abs((U[1:4] + U[9:12]) - (Us[1:4] + Us[9:12])) <= 4e-16 * (tot + Us[0]))
    Up = O.prim2con(Vn, P)
    assert np.max(np.abs(Up - U)[:5] / (np.abs(U[4]) + U[0] + U[8])) < 1e-12
    for i in range(U.shape[1]):
        v = Vn[1:4, i]
        W = 1 / np.sqrt(1 - v @ v)
        u = W * v
        T = Vn[4, i] / Vn[0, i]
        X = U[8:12, i]
        G = O.four_force(kappa[i], sigma[i], Vn[0, i], u, W, T ** 4, X[0], X[1:],
                         O.m1_pressure(X[0], X[1:]))
        R = X - Us[8:12, i] + hdt * G
        scale = Us[8, i] + X[0] + hdt * np.abs(G).max()
        assert np.abs(R).max() <= 1e-10 * scale, (i, R, scale)
    assert np.all(np.sqrt((U[9:12] ** 2).sum(0)) <= U[8] * (1 + 1e-12))


def test_picard_agrees_with_newton_when_it_converges():
    g = 4 / 3
    Pn = O.Params(gamma=g, a_rad=1e-4)
    Pp = O.Params(gamma=g, a_rad=1e-4, implicit="picard", imp_maxit=400)
    rng = np.random.default_rng(11)
    V = random_states(100, 11, wmax=2.0)
    kappa = 10 ** rng.uniform(-2, 0, 100)
    sigma = 10 ** rng.uniform(-2, 0, 100)
    Us = O.prim2con(V, Pn)
    Un, _, sn = O.implicit(Us, kappa, sigma, 1e-3, Pn, Zguess=O.prim_Z(V, Pn))
    Up, _, sp = O.implicit(Us, kappa, sigma, 1e-3, Pp, Zguess=O.prim_Z(V, Pn))
    assert (sn == 0).all() and (sp == 0).all()
    scale = np.abs(Us[4]) + Us[0] + Us[8]
    assert np.max(np.abs(Un - Up) / scale) < 1e-11


def test_picard_diverges_where_newton_converges():
    """The paper's lagged iteration fails once 4 a_R T^3 h kappa (gamma-1)/rho >> 1
    (hot gas, cold radiation, strong absorption); the Newton reading converges."""
    g = 4 / 3
    V = np.array([0.01, 0, 0, 0, 10.0, 0, 0, 0, 1e-3, 0, 0, 0])
    for mode, ok in (("newton", True), ("picard", False)):
        P = O.Params(gamma=g, a_rad=1.0, implicit=mode)
        Us = O.prim2con(V, P)
        _, _, st = O.implicit(Us, 1e3, 0.0, 1e-3, P, Zguess=O.prim_Z(V, P))
        assert (st == 0) == ok


# a radiation-dominated cell from the 2D blast (E_r ~ 1e6 x the gas energy, W ~ 2.6)
RAD_DOMINATED = np.array([0.285, 0.266, 0.873, 0.0, 9.17, 0.335, 0.0405, 0.0,
                          8.33e6, 2.30e6, 7.63e6, 0.0])


def _check_solution(Us, U, Vn, kappa, sigma, hdt, P):
    """Totals conserved, V consistent with U, and R(X) = 0 with the four-force."""
    tot = abs(Us[4]) + Us[8]
    assert U[0] == Us[0] and np.array_equal(U[5:8], Us[5:8])
    assert abs((U[4] + U[8]) - (Us[4] + Us[8])) <= 4e-16 * tot
    assert np.all(np.abs((U[1:4] + U[9:12]) - (Us[1:4] + Us[9:12])) <= 4e-16 * (tot + Us[0]))
    Um = O.prim2con(Vn, P)
    # the matter part of U is the totals minus X: compare on the scale of the totals
    assert np.max(np.abs(Um[:5] - U[:5])) <= 1e-14 * tot
    v = Vn[1:4]
    W = 1 / np.sqrt(1 - v @ v)
    T = Vn[4] / Vn[0]
    X = U[8:12]
    G = O.four_force(kappa, sigma, Vn[0], W * v, W, P.a_rad * T ** 4, X[0], X[1:],
                     O.m1_pressure(X[0], X[1:]))
    R = X - Us[8:12] + hdt * G
    assert np.abs(R).max() <= 1e-10 * (tot + Us[0] + hdt * np.abs(G).max())


@pytest.mark.parametrize("hdt", [3e-3, 5e-3])
def test_matter_form_rescues_radiation_dominated_cell(hdt):
    P = O.Params(gamma=4 / 3, a_rad=1.0)
    Us = O.prim2con(RAD_DOMINATED, P)
    st = O.Stats()
    U, Vn, rc = O.implicit(Us, 2.7, 0.0, hdt, P, Zguess=O.prim_Z(RAD_DOMINATED, P), stats=st)
    assert rc == 0 and st.imp_matter == 1      # the iteration on X failed, the matter form did not
    _check_solution(Us, U, Vn, 2.7, 0.0, hdt, P)
    # the matter was accelerated towards the radiation's frame and cooled
    assert np.linalg.norm(Vn[1:4]) > np.linalg.norm(RAD_DOMINATED[1:4]) and Vn[4] < RAD_DOMINATED[4]


def test_matter_form_agrees_with_the_iteration_on_x():
    g = 4 / 3
    Pn = O.Params(gamma=g, a_rad=1.0)
    Pm = O.Params(gamma=g, a_rad=1.0, implicit="matter")
    V, kappa, sigma = _c1_cells(400, 7)
    Us = O.prim2con(V, Pn)
    Un, Vx, sn = O.implicit(Us, kappa, sigma, 1e-3, Pn, Zguess=O.prim_Z(V, Pn))
    Um, Vm, sm = O.implicit(Us, kappa, sigma, 1e-3, Pm, Zguess=O.prim_Z(V, Pn))
    ok = (sn == 0) & (sm == 0)
    assert ok.mean() > 0.95
    scale = np.abs(Us[4]) + Us[0] + Us[8]
    assert np.max(np.abs(Un - Um)[:, ok] / scale[ok]) < 1e-9
    for i in np.where(sm == 0)[0][:50]:
        _check_solution(Us[:, i], Um[:, i], Vm[:, i], kappa[i], sigma[i], 1e-3, Pm)
    # and on the radiation-dominated cell at a weight where both forms converge
    Us = O.prim2con(RAD_DOMINATED, Pn)
    Zg = O.prim_Z(RAD_DOMINATED, Pn)
    st = O.Stats()
    Ux, _, rx = O.implicit(Us, 2.7, 0.0, 1e-3, Pn, Zguess=Zg, stats=st)
    Uy, _, ry = O.implicit(Us, 2.7, 0.0, 1e-3, Pm, Zguess=Zg)
    assert rx == 0 and ry == 0 and st.imp_matter == 0
    # the polished root of the iteration on X is the matter form's root; its
    # matter part (tau_e = tau_t - E_r, E_r ~ 1e6 x the gas energy) is only good
    # to ~1e-7 of itself here, which is the reason for the matter form
    assert np.max(np.abs(Ux - Uy)) <= 1e-11 * Us[8]


def test_matter_form_takes_over_where_the_iteration_on_x_stops():
    """At h = 1.9e-3 on the radiation-dominated cell, the iteration on X (at most ten
    backtracking halvings per step) and its continuation in h do not converge: the
    matter form takes over, and the result is the matter form's own."""
    g = 4 / 3
    Pn = O.Params(gamma=g, a_rad=1.0)
    Pm = O.Params(gamma=g, a_rad=1.0, implicit="matter")
    Us = O.prim2con(RAD_DOMINATED, Pn)
    Zg = O.prim_Z(RAD_DOMINATED, Pn)
    st = O.Stats()
    Ux, Vx, rx = O.implicit(Us, 2.7, 0.0, 1.9e-3, Pn, Zguess=Zg, stats=st)
    Uy, _, ry = O.implicit(Us, 2.7, 0.0, 1.9e-3, Pm, Zguess=Zg)
    assert rx == 0 and ry == 0 and st.imp_matter == 1
    np.testing.assert_array_equal(Ux, Uy)
    _check_solution(Us, Ux, Vx, 2.7, 0.0, 1.9e-3, Pn)


# ---------------------------------------------------------------- path independence
def _plain_residual(X, Xs, h, kappa, sigma, D, St, taut, B, Zg, P):
    """R(X) = X - X* + h G(X, V(X)) of Sec. 3.3 (Eqs. timeadv, totale, totalm): the
    matter is the conserved totals minus X, V(X) its con2prim; None if inadmissible."""
    if not X[0] > 0:
        return None
    Um = np.array([D, St[0] - X[1], St[1] - X[2], St[2] - X[3], taut - X[0], *B, *X])
    V, _, st = O.con2prim(Um, P, Zguess=Zg)
    if st != 0:
        return None
    v = V[1:4]
    W = 1 / np.sqrt(1 - v @ v)
    T = V[4] / V[0]
    G = O.four_force(kappa, sigma, V[0], W * v, W, P.a_rad * T ** 4, X[0], X[1:],
                     O.m1_pressure(X[0], X[1:]))
    return (X - Xs) + h * G


def _plain_newton(Us, h, kappa, sigma, Zg, P):
    """Damped Newton from X* with a forward-difference Jacobian at every iterate and
    no cache, run to the rounding floor of R.  Returns the full state U or None."""
    D, B = Us[0], Us[5:8]
    St, taut, Xs = Us[1:4] + Us[9:12], Us[4] + Us[8], Us[8:12].copy()
    args = (Xs, h, kappa, sigma, D, St, taut, B, Zg, P)
    X = Xs.copy()
    R = _plain_residual(X, *args)
    prev, flat = np.inf, 0
    for _ in range(200):
        J = np.empty((4, 4))
        for j in range(4):
            e = np.zeros(4)
            e[j] = 1e-7 * X[0]
            Rp = _plain_residual(X + e, *args)
            if Rp is None:
                e = -e
                Rp = _plain_residual(X + e, *args)
            J[:, j] = (Rp - R) / e[j]
        dX = np.linalg.solve(J, -R)
        step = np.abs(dX).max()
        if step <= 1e-16 * X[0]:
            break
        lam = 1.0
        while True:
            Rn = _plain_residual(X + lam * dX, *args)
            if Rn is not None and (Rn @ Rn <= (1 - 1e-4 * lam) * (R @ R) or step < 1e-12 * X[0]):
                break
            lam *= 0.5
            if lam < 1e-12:
                return None
        X, R = X + lam * dX, Rn
        if step < 1e-12 * X[0] and lam * step >= 0.5 * prev:
            flat += 1
            if flat == 3:      # three corrections at the rounding floor
                break
        prev = lam * step
    else:
        return None
    return np.array([D, St[0] - X[1], St[1] - X[2], St[2] - X[3], taut - X[0], *B, *X])


def _c1_stage_inputs(n_inst=6, steps=3, seed=31):
    """Explicit stage-1 states U* of C1 instances after a few steps, with each
    cell's Jacobian cache from those steps."""
    from paper_2212_00370_gb300 import workloads as W
    w = W.riemann_batch(n_inst, seed=seed, nmin=64, nmax=120)
    P = O.Params(gamma=w.gamma, a_rad=w.a_rad, cfl=w.cfl)
    out = []
    for i in range(w.n_inst):
        g, V, kappa, sigma = w.instance(i)
        og = O.Grid(1, (g["n"][0],), (g["dx"][0],))
        V = np.ascontiguousarray(V).copy()
        U = O.prim2con(V, P)
        jc = np.zeros(17 * og.ncells)
        for _ in range(steps):
            assert O.step(og, O.grid_dt(og, V, P), U, V, kappa, sigma, P, jcache=jc) == 0
        dt = O.grid_dt(og, V, P)
        F = O.face_flux(og, 0, U, V, kappa, sigma, P).reshape(12, -1)
        Ust = U - (dt / g["dx"][0]) * (F[:, 1:] - F[:, :-1])
        out.append((Ust, O.prim_Z(V, P), kappa, sigma, dt, jc.reshape(17, -1)))
    return P, out


def test_polished_result_is_path_independent():
    """The cell's cache (and whether the solve took Broyden updates, the cached
    matrix or C^(m) first) must not show in the result: cached path, cache-free
    path and the plain Newton above agree to 1e-12 per component, on the scale of
    the component with the radiation energy as its floor."""
    P, cells = _c1_stage_inputs()
    n, worst = 0, 0.0
    for Ust, Zg, kappa, sigma, dt, jc in cells:
        assert (jc[16] > 0).all()              # every cell has a cache entry
        for wgt in (1.0, 0.25, 2.0 / 3.0):     # the three stage weights
            Uc, _, sc = O.implicit_cached(Ust, kappa, sigma, wgt * dt, P, jc.copy(), Zguess=Zg)
            Un, _, sn = O.implicit(Ust, kappa, sigma, wgt * dt, P, Zguess=Zg)
            assert (sc == 0).all() and (sn == 0).all()
            for c in range(Ust.shape[1]):
                Ur = _plain_newton(Ust[:, c], wgt * dt, kappa[c], sigma[c], Zg[c], P)
                assert Ur is not None, c
                scale = Ur[8] + np.abs(Ur)
                for other in (Uc[:, c], Un[:, c]):
                    worst = max(worst, float((np.abs(other - Ur) / scale).max()))
                worst = max(worst, float((np.abs(Uc[:, c] - Un[:, c]) / scale).max()))
                n += 1
    print("cell solves %d, worst per-component difference %.2e" % (n, worst))
    assert n >= 600
    assert worst <= 1e-12


def _rel_l1(a, b):
    return max(np.abs(a[k] - b[k]).sum() / np.abs(b[k]).sum() for k in range(12)
               if np.abs(b[k]).sum() > 0)


def _steps(og, U, V, kappa, sigma, P, n, jc):
    for _ in range(n):
        assert O.step(og, O.grid_dt(og, V, P), U, V, kappa, sigma, P, jcache=jc) == 0


def _c1_runs(solver, n_inst, seed):
    from paper_2212_00370_gb300 import workloads as W
    w = W.riemann_batch(n_inst, seed=seed, nmin=64, nmax=200)
    P = O.Params(gamma=w.gamma, a_rad=w.a_rad, cfl=w.cfl, solver=solver)
    for i in range(w.n_inst):
        g, V, kappa, sigma = w.instance(i)
        og = O.Grid(1, (g["n"][0],), (g["dx"][0],))
        V = np.ascontiguousarray(V).copy()
        U = O.prim2con(V, P)
        jc = np.zeros(17 * og.ncells)
        _steps(og, U, V, kappa, sigma, P, 5, jc)
        yield P, og, U, V, kappa, sigma, jc


def test_restart_one_step_later_equals_continuing_run():
    """Rad-HLL (no 1/epsilon amplification of rounding): 5 steps, then one step with
    the cache carried and one from an emptied cache, as a restart from the state
    alone does; per-variable relative L1 <= 1e-12 on every instance."""
    worst = 0.0
    for P, og, U, V, kappa, sigma, jc in _c1_runs("radhll", 16, 5):
        Ua, Va, Ub, Vb = U.copy(), V.copy(), U.copy(), V.copy()
        _steps(og, Ua, Va, kappa, sigma, P, 1, jc.copy())
        _steps(og, Ub, Vb, kappa, sigma, P, 1, np.zeros_like(jc))
        worst = max(worst, _rel_l1(Ub, Ua))
    print("one step after restart: worst per-variable rel L1 %.2e" % worst)
    assert worst <= 1e-12


def test_restart_moves_the_run_no_more_than_rounding():
    """PVM-int-8 with the paper's epsilon = 1e-8 (Eq. utilde): the nested flux
    differences divide rounding by epsilon, so any one-ulp change of a state moves
    the next steps by ~1e-8.  Five steps after a restart (emptied cache) the run
    differs from the continuing one by no more than it differs after a one-ulp
    perturbation of U (cache kept): the cache changes only the rounding."""
    dr, du = [], []
    for P, og, U, V, kappa, sigma, jc in _c1_runs("pvm", 8, 5):
        Ua, Va, Ub, Vb = U.copy(), V.copy(), U.copy(), V.copy()
        Uc = np.nextafter(U, np.inf)
        Vc = O.con2prim(Uc, P, O.prim_Z(V, P))[0]
        _steps(og, Ua, Va, kappa, sigma, P, 5, jc.copy())
        _steps(og, Ub, Vb, kappa, sigma, P, 5, np.zeros_like(jc))
        _steps(og, Uc, Vc, kappa, sigma, P, 5, jc.copy())
        dr.append(_rel_l1(Ub, Ua))
        du.append(_rel_l1(Uc, Ua))
    dr, du = np.array(dr), np.array(du)
    print("restart: max %.2e median %.2e; one-ulp perturbation: max %.2e median %.2e"
          % (dr.max(), np.median(dr), du.max(), np.median(du)))
    assert dr.max() <= 4 * du.max() and np.median(dr) <= 4 * np.median(du)

"""Pins of the oracle's point functions against what the paper and physics fix.

Each test checks the oracle against an independent formulation or a closed
form, never against a retyped copy of the same expression:
  * prim2con and the fluxes against the covariant stress-energy tensor and the
    dual Faraday tensor assembled with 4x4 algebra (Sec. 2.1);
  * con2prim by round trips over the C1 state distribution and the v = 0 closed form;
  * the M1 closure by its limits and by the eigenvalues of the radiation block
    of the flux Jacobian, Eqs. lam1-lam3 (Sec. 3.2.1);
  * signal speeds by their textbook special cases;
  * the four-force by Lorentz covariance: boosted to the fluid frame it must be
    G~0 = rho kappa (E~ - 4 pi B), G~i = rho (kappa + sigma) F~i (Eqs. g0, gi at v = 0).
"""
import numpy as np
import pytest

import oracle as O

ETA = np.diag([-1.0, 1.0, 1.0, 1.0])


def random_states(n, seed, gamma=4.0 / 3.0, wmax=10.0, bmax=1.0):
    """States spanning the C1 distribution (log-uniform rho, p, E_r; W up to 10)."""
    rng = np.random.default_rng(seed)
    rho = 10 ** rng.uniform(-2, 1, n)
    p = 10 ** rng.uniform(-3, 1, n)
    W = rng.uniform(1, wmax, n)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    v = np.sqrt(1 - 1 / W ** 2) * d
    B = rng.uniform(-bmax, bmax, (3, n))
    E = 10 ** rng.uniform(-3, 1, n)
    f = rng.uniform(0, 0.99, n)
    dd = rng.normal(size=(3, n))
    dd /= np.linalg.norm(dd, axis=0)
    return np.vstack([rho, v, p, B, E, f * E * dd])


def covariant(V, gamma):
    """U and the three flux vectors of one state from T^{mu nu} and *F^{mu nu}."""
    rho, v, p, B = V[0], V[1:4], V[4], V[5:8]
    W = 1 / np.sqrt(1 - v @ v)
    u = np.concatenate([[W], W * v])
    b0 = W * (v @ B)
    b = np.concatenate([[b0], B / W + v * b0])
    bsq = b @ ETA @ b
    rhoh = rho + gamma / (gamma - 1) * p
    T = (rhoh + bsq) * np.outer(u, u) + (p + bsq / 2) * ETA - np.outer(b, b)
    Fd = np.outer(b, u) - np.outer(u, b)  # dual Faraday *F^{mu nu} = b^mu u^nu - b^nu u^mu
    D = rho * W
    U = np.concatenate([[D], T[0, 1:], [T[0, 0] - D], -Fd[0, 1:]])
    fl = []
    for i in range(3):
        # induction: d_t B^j + d_i(-*F^{ij}) = 0 since *F^{0j} = -B^j
        fi = np.concatenate([[rho * u[1 + i]], T[1 + i, 1:], [T[1 + i, 0] - rho * u[1 + i]],
                             -Fd[1 + i, 1:]])
        fl.append(fi)
    return U, fl


@pytest.mark.parametrize("seed", [0, 1])
def test_prim2con_and_flux_match_covariant_form(seed):
    g = 4.0 / 3.0
    P = O.Params(gamma=g)
    V = random_states(64, seed, wmax=4.0)
    U = O.prim2con(V, P)
    for i in range(V.shape[1]):
        Uc, fl = covariant(V[:, i], g)
        scale = np.abs(Uc[:5]).max()
        assert np.abs(U[:8, i] - Uc).max() <= 1e-13 * scale
        np.testing.assert_array_equal(U[8:, i], V[8:, i])
        for d in range(3):
            F = O.flux(V[:, i], U[:, i], d, P)
            fs = np.abs(fl[d]).max() + scale
            assert np.abs(F[:8] - fl[d]).max() <= 1e-13 * fs, (i, d)
            # radiation: energy flux is F_r^d, momentum flux row d of P_r
            assert F[8] == V[9 + d, i]


def test_prim2con_static_closed_form():
    """v = 0, B = 0: D = rho, S = 0, tau = p/(gamma-1), momentum flux = p."""
    g = 5.0 / 3.0
    P = O.Params(gamma=g)
    V = np.array([2.0, 0, 0, 0, 3.0, 0, 0, 0, 1.5, 0, 0, 0])
    U = O.prim2con(V, P)
    assert U[0] == 2.0 and U[1] == 0 and U[4] == pytest.approx(3.0 / (g - 1), rel=1e-15)
    F = O.flux(V, U, 0, P)
    assert F[1] == 3.0 and F[0] == 0.0 and F[4] == 0.0
    assert F[9] == pytest.approx(0.5, rel=1e-15)  # P_r = E/3 at F_r = 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_con2prim_round_trip(seed):
    """prim2con then con2prim over the C1 state distribution (W up to 10,
    |B| up to 1.7, rho down to 1e-2, p down to 1e-3)."""
    g = 4.0 / 3.0
    P = O.Params(gamma=g)
    V = random_states(4000, seed)
    U = O.prim2con(V, P)
    V2, Z, st = O.con2prim(U, P)
    assert (st == 0).all()
    # rho and v to 1e-12 relative; p relative to the energy scale it is recovered from
    assert np.max(np.abs(V2[0] - V[0]) / V[0]) < 1e-12
    vmag = np.sqrt((V[1:4] ** 2).sum(0))
    assert np.max(np.abs(V2[1:4] - V[1:4]).max(0) / vmag) < 1e-12
    scale = U[4] + U[0]
    assert np.max(np.abs(V2[4] - V[4]) / np.maximum(V[4], scale)) < 1e-13
    assert np.max(np.abs(V2[4] - V[4]) / V[4]) < 1e-9
    np.testing.assert_array_equal(V2[5:], V[5:])
    # the recovered Z is rho h W^2 of the state
    assert np.max(np.abs(Z - O.prim_Z(V, P)) / Z) < 1e-12


def test_con2prim_static_exact():
    """v = 0, B = 0: the root is found exactly to rounding from a cold start."""
    P = O.Params(gamma=5.0 / 3.0)
    V = np.array([1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0, 0, 0, 0])
    U = O.prim2con(V, P)
    V2, Z, st = O.con2prim(U, P)
    assert st == 0
    np.testing.assert_allclose(V2, V, rtol=1e-15, atol=1e-300)
    assert Z == pytest.approx(1.0 + 2.5, rel=1e-15)


def test_con2prim_rejects_inadmissible():
    P = O.Params(gamma=4.0 / 3.0)
    U = np.array([1.0, 5.0, 0, 0, 0.1, 0, 0, 0, 1.0, 0, 0, 0])  # |S| >> tau + D: no admissible root
    _, _, st = O.con2prim(U, P)
    assert st != 0
    U = np.array([-1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0, 0, 0, 0])
    assert O.con2prim(U, P)[2] == 3


def test_m1_closure_limits():
    """xi(0) = 1/3 (Eddington), xi(1) = 1 (free streaming), monotone in between;
    tr P = E; free streaming gives P = E n n."""
    assert O.eddington_factor(0.0) == pytest.approx(1 / 3, rel=1e-15)
    assert O.eddington_factor(1.0) == 1.0
    fs = np.linspace(0, 1, 101)
    xi = np.array([O.eddington_factor(f) for f in fs])
    assert np.all(np.diff(xi) > 0)
    rng = np.random.default_rng(3)
    for _ in range(50):
        E = 10 ** rng.uniform(-3, 2)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        f = rng.uniform(0, 1)
        Pr = O.m1_pressure(E, f * E * n)
        assert np.trace(Pr) == pytest.approx(E, rel=1e-14)
        np.testing.assert_allclose(Pr, Pr.T, rtol=0, atol=1e-15 * E)
    n = np.array([0.6, 0.8, 0.0])
    np.testing.assert_allclose(O.m1_pressure(2.0, 2.0 * n), 2.0 * np.outer(n, n), atol=1e-15)
    np.testing.assert_allclose(O.m1_pressure(2.0, np.zeros(3)), 2.0 / 3 * np.eye(3), rtol=1e-15)


def _paper_lams(f, ct):
    s = np.sqrt(4 - 3 * f * f)
    zeta = np.sqrt(2 / 3 * (4 - 3 * f * f - s) + 2 * ct * ct * (2 - f * f - s))
    xi = (3 + 4 * f * f) / (5 + 2 * s)
    l2 = ct * (3 * xi - 1) / (2 * f) if f > 0 else 0.0
    return (f * ct - zeta) / s, l2, (f * ct + zeta) / s


@pytest.mark.parametrize("f", [0.0, 0.2, 0.5, 0.8, 0.97])
def test_radiation_jacobian_eigenvalues(f):
    """Eigenvalues of the radiation block J_rad (Eq. jacobian), assembled by central
    differences of the oracle's flux, equal lambda_r1, lambda_r2 (twice), lambda_r3."""
    P = O.Params(gamma=4.0 / 3.0)
    rng = np.random.default_rng(int(f * 100))
    for d in range(3):
        E = 1.3
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        V = np.array([1.0, 0.1, 0.2, -0.1, 0.5, 0.3, 0.1, 0.2, E, *(f * E * n)])

        def rf(x):
            v = V.copy()
            v[8:12] = x
            return O.flux(v, O.prim2con(v, P), d, P)[8:12]

        J = np.zeros((4, 4))
        h = 1e-6 * E
        for j in range(4):
            e = np.zeros(4)
            e[j] = h
            J[:, j] = (rf(V[8:12] + e) - rf(V[8:12] - e)) / (2 * h)
        ev = np.sort(np.linalg.eigvals(J).real)
        l1, l2, l3 = _paper_lams(f, n[d] if f > 0 else 0.0)
        np.testing.assert_allclose(ev, np.sort([l1, l2, l2, l3]), atol=2e-7)
        # the radiation flux ignores the magnetofluid (block structure, Eq. jacobian)
        v = V.copy()
        v[0:8] = [2.0, -0.3, 0.1, 0.0, 0.2, -0.5, 0.4, 0.1]
        np.testing.assert_array_equal(O.flux(v, O.prim2con(v, P), d, P)[8:], rf(V[8:12]))


def test_signal_speed_special_cases():
    g = 5.0 / 3.0
    P = O.Params(gamma=g)
    # static unmagnetised gas, no radiation flux: max(c_s, 1/sqrt(3))
    rho, p = 1.0, 0.01
    cs = np.sqrt(g * p / (rho + g / (g - 1) * p))
    V = np.array([rho, 0, 0, 0, p, 0, 0, 0, 1.0, 0, 0, 0])
    assert O.signal_speed(V, 0, P) == pytest.approx(max(cs, 1 / np.sqrt(3)), rel=1e-14)
    # hot gas beats the radiation speed: relativistic velocity addition (v + c_s)/(1 + v c_s)
    p = 10.0
    cs = np.sqrt(g * p / (rho + g / (g - 1) * p))
    for v in (0.3, -0.6):
        V = np.array([rho, v, 0, 0, p, 0, 0, 0, 1.0, 0, 0, 0])
        expect = (abs(v) + cs) / (1 + abs(v) * cs)
        assert O.signal_speed(V, 0, P) == pytest.approx(expect, rel=1e-13)
    # free-streaming radiation along x: speed of light along x, none across
    V = np.array([1.0, 0, 0, 0, 1e-6, 0, 0, 0, 1.0, 1.0, 0, 0])
    assert O.signal_speed(V, 0, P) == pytest.approx(1.0, rel=1e-14)
    assert O.signal_speed(V, 1, P) < 0.01


def boost(u):
    """Lorentz matrix to the frame moving with four-velocity u (contravariant)."""
    W = np.sqrt(1 + u @ u)
    L = np.eye(4)
    L[0, 0] = W
    L[0, 1:] = -u
    L[1:, 0] = -u
    L[1:, 1:] += np.outer(u, u) / (W + 1)
    return L


@pytest.mark.parametrize("seed", range(4))
def test_four_force_lorentz_covariance(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(20):
        rho = 10 ** rng.uniform(-2, 1)
        kappa = 10 ** rng.uniform(-3, 3)
        sigma = 10 ** rng.uniform(-3, 2) * rng.integers(0, 2)
        u = rng.normal(size=3) * rng.uniform(0, 3)
        W = np.sqrt(1 + u @ u)
        BP = 10 ** rng.uniform(-3, 1)
        E = 10 ** rng.uniform(-3, 1)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        F = rng.uniform(0, 0.99) * E * n
        Pr = O.m1_pressure(E, F)
        G = O.four_force(kappa, sigma, rho, u, W, BP, E, F, Pr)
        T = np.zeros((4, 4))
        T[0, 0] = E
        T[0, 1:] = F
        T[1:, 0] = F
        T[1:, 1:] = Pr
        L = boost(u)
        Tc = L @ T @ L.T
        Gc = np.concatenate([[rho * kappa * (Tc[0, 0] - BP)], rho * (kappa + sigma) * Tc[0, 1:]])
        Gl = np.linalg.solve(L, Gc)
        scale = np.abs(Gl).max() + rho * (kappa + sigma) * (E + BP) * W ** 3
        np.testing.assert_allclose(G, Gl, rtol=0, atol=1e-12 * scale)

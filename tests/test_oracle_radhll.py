"""Pins of the oracle's Rad-HLL solver (Sec. 3.2.1) and of the diffusion limit.

  * consistency: equal states give the physical flux; supersonic states upwind;
  * the radiation eigenvalues of Eqs. lam1-lam3 reach the limits the paper states
    (f -> 0: +-1/sqrt 3; f -> 1: cos theta);
  * Eq. limits bounds the radiation speeds by 4/(3 tau);
  * conservation on periodic grids and first-order convergence to the exact
    relativistic Riemann solution with the radiation decoupled;
  * Table 1 of the paper (the Alfven wave with HLL, radiation passive): every error
    at or above the printed one (the fast-speed estimate bounds the exact speed from
    above) and within 10 % of it, with the printed order;
  * the optically thin radiation Riemann problem Test 1 (Sec. 4): PVM-int-8 is
    sharper than Rad-HLL at first order, as the paper reports;
  * the optically thick radiative pulse (Sec. 4, Eq. gaus_init): both solvers
    follow the exact solution of the diffusion equation with D = 1/(3 rho sigma)
    (the initial (1 + 100 g)^4 profile is a sum of five Gaussians, each spreading
    in closed form); without beta (PVM) or without Eq. limits (Rad-HLL) the
    solution is far too diffusive, as the paper reports.
"""
import numpy as np
import pytest

import oracle as O
import rhd_exact


def hll(sL, sR, UL, UR, FL, FR):
    if sL > 0:
        return FL
    if sR < 0:
        return FR
    return (sR * FL - sL * FR + sR * sL * (UR - UL)) / (sR - sL)


def state(rho, v, p, B, E, F):
    return np.array([rho, *v, p, *B, E, *F], dtype=float)


def test_equal_states_give_the_physical_flux():
    P = O.Params(gamma=4 / 3, solver="radhll")
    rng = np.random.default_rng(1)
    for d in range(3):
        V = state(1.3, rng.uniform(-0.3, 0.3, 3), 0.7, rng.uniform(-0.5, 0.5, 3), 2.0,
                  rng.uniform(-0.5, 0.5, 3))
        U = O.prim2con(V, P)
        np.testing.assert_allclose(O.radhll_flux(V, V, 0.0, 0.0, d, P), O.flux(V, U, d, P),
                                   rtol=1e-13, atol=1e-14)


def test_supersonic_states_upwind():
    P = O.Params(gamma=4 / 3, solver="radhll")
    VL = state(1.0, (0.995, 0, 0), 0.01, (0, 0, 0), 1.0, (0.999, 0, 0))
    VR = state(0.8, (0.99, 0, 0), 0.012, (0, 0, 0), 0.9, (0.899, 0, 0))
    UL = O.prim2con(VL, P)
    F = O.radhll_flux(VL, VR, 0.0, 0.0, 0, P)
    np.testing.assert_array_equal(F, O.flux(VL, UL, 0, P))
    VL[1], VR[1], VL[9], VR[9] = -0.995, -0.99, -0.999, -0.899
    UR = O.prim2con(VR, P)
    np.testing.assert_array_equal(O.radhll_flux(VL, VR, 0.0, 0.0, 0, P), O.flux(VR, UR, 0, P))


def test_radiation_eigenvalue_limits():
    V = state(1, (0, 0, 0), 1, (0, 0, 0), 1.0, (0, 0, 0))
    l1, l3 = O.rad_speeds(V, 0)
    assert l1 == pytest.approx(-1 / np.sqrt(3), abs=1e-15) and l3 == pytest.approx(1 / np.sqrt(3), abs=1e-15)
    for cth, d in ((1.0, 0), (0.0, 1)):
        V = state(1, (0, 0, 0), 1, (0, 0, 0), 1.0, (1.0, 0, 0))   # free streaming along x
        l1, l3 = O.rad_speeds(V, d)
        assert l1 == pytest.approx(cth, abs=1e-7) and l3 == pytest.approx(cth, abs=1e-7)
    # the MHD speeds bracket the flow velocity and stay below c
    P = O.Params(gamma=4 / 3)
    V = state(1, (0.5, 0.2, 0), 1, (0.3, 0.1, 0), 1, (0, 0, 0))
    lm, lp = O.mhd_speeds(V, 0, P)
    assert -1 < lm < 0.5 < lp < 1


def test_optically_thick_speeds_are_limited():
    P = O.Params(gamma=4 / 3, solver="radhll")
    VL = state(1, (0.1, 0, 0), 1, (0, 0, 0), 1.0, (0.2, 0, 0))
    VR = state(1.2, (0.05, 0, 0), 0.9, (0, 0, 0), 0.7, (0.05, 0.1, 0))
    UL, UR = O.prim2con(VL, P), O.prim2con(VR, P)
    FL, FR = O.flux(VL, UL, 0, P), O.flux(VR, UR, 0, P)
    for tau in (0.5, 10.0, 1e4):
        F = O.radhll_flux(VL, VR, tau, 0.3 * tau, 0, P)
        lim = 4 / (3 * tau)
        rL = max(min(O.rad_speeds(VL, 0)[0], O.rad_speeds(VR, 0)[0]), -lim)
        rR = min(max(O.rad_speeds(VL, 0)[1], O.rad_speeds(VR, 0)[1]), lim)
        np.testing.assert_allclose(F[8:], hll(rL, rR, UL[8:], UR[8:], FL[8:], FR[8:]), rtol=1e-13)
        lm = min(O.mhd_speeds(VL, 0, P)[0], O.mhd_speeds(VR, 0, P)[0])
        lp = max(O.mhd_speeds(VL, 0, P)[1], O.mhd_speeds(VR, 0, P)[1])
        np.testing.assert_allclose(F[:8], hll(lm, lp, UL[:8], UR[:8], FL[:8], FR[:8]), rtol=1e-13,
                                   atol=1e-15)
    # beta_mode = 0 switches the limiting off
    Pn = O.Params(gamma=4 / 3, solver="radhll", beta=False)
    np.testing.assert_array_equal(O.radhll_flux(VL, VR, 1e4, 1e4, 0, Pn),
                                  O.radhll_flux(VL, VR, 0.0, 0.0, 0, P))


def test_conservation_periodic_radhll():
    from test_oracle_scheme import _periodic_conservation
    _periodic_conservation(1, 64, 0, solver="radhll")
    _periodic_conservation(2, 12, 1, steps=2, solver="radhll")


def test_relativistic_riemann_problem_radhll():
    g = 5 / 3
    errs = []
    for N in (200, 400):
        P = O.Params(gamma=g, cfl=0.4, solver="radhll")
        dx = 1.0 / N
        x = (np.arange(N) + 0.5) * dx
        V = np.zeros((12, N))
        V[0] = np.where(x < 0.5, 1.0, 0.125)
        V[4] = np.where(x < 0.5, 1.0, 0.1)
        V[8] = 1.0
        U = O.prim2con(V, P)
        t, ns, nf = O.run(O.Grid(1, (N,), (dx,)), 0.0, 0.4, U, V, np.zeros(N), np.zeros(N), P)
        assert nf == 0
        ex = np.array(rhd_exact.sample((1.0, 1.0, 0.0), (0.125, 0.1, 0.0), g, (x - 0.5) / 0.4))
        errs.append([np.mean(np.abs(V[0] - ex[:, 0])), np.mean(np.abs(V[4] - ex[:, 1]))])
    errs = np.array(errs)
    assert np.all(errs[1] < [4e-3, 3e-3])
    assert np.all(errs[0] / errs[1] > 1.5)


def _thin_test(N, solver, recon, test):
    """Optically thin radiation Riemann problem on [-20, 20] to t = 20 (Sec. 4):
    Test 1 (E, Fx, Fy)_L = (1, 0, 1/2), _R = (1, 0, 0); Test 2 (1/10, 1/10, 0), (1, 0, 1).
    Matter uniform at rest (rho = p = 1, no field) and decoupled (kappa = sigma = 0)."""
    P = O.Params(gamma=4 / 3, cfl=0.4, recon=recon, solver=solver)
    dx = 40.0 / N
    x = -20 + (np.arange(N) + 0.5) * dx
    L = {1: (1.0, 0.0, 0.5), 2: (0.1, 0.1, 0.0)}[test]
    R = {1: (1.0, 0.0, 0.0), 2: (1.0, 0.0, 1.0)}[test]
    V = np.zeros((12, N))
    V[0], V[4] = 1.0, 1.0
    for k in range(3):
        V[8 + k] = np.where(x < 0, L[k], R[k])
    U = O.prim2con(V, P)
    t, ns, nf = O.run(O.Grid(1, (N,), (dx,)), 0.0, 20.0, U, V, np.zeros(N), np.zeros(N), P)
    assert nf == 0 and t == 20.0
    return x, V


def _cell_average(Vfine, factor):
    return Vfine.reshape(Vfine.shape[0], -1, factor).mean(axis=2)


def test_thin_test1_pvm_sharper_than_radhll():
    """At first order (256 zones) PVM-int-8 is closer than Rad-HLL to a resolved
    reference (1024 zones, VanLeer), above all around the contact wave."""
    _, Vref = _thin_test(1024, "pvm", "vanleer", 1)
    ref = _cell_average(Vref, 4)
    err = {}
    for solver in ("pvm", "radhll"):
        _, V = _thin_test(256, solver, "godunov", 1)
        err[solver] = np.abs(V[8:11] - ref[8:11]).mean(axis=1)
    print("Test 1 L1 (E, Fx, Fy): PVM", err["pvm"], " Rad-HLL", err["radhll"])
    assert err["pvm"].sum() < err["radhll"].sum()


def test_thin_test2_both_solvers_converge():
    _, Vref = _thin_test(1024, "pvm", "vanleer", 2)
    ref = _cell_average(Vref, 4)
    for solver in ("pvm", "radhll"):
        _, V = _thin_test(256, solver, "vanleer", 2)
        e = np.abs(V[8:11] - ref[8:11]).mean(axis=1)
        assert np.all(e < 0.02), (solver, e)


# ------------------------------------------------------------------ diffusion limit
T0, OMEGA, A_R = 1e6, 5.0, 6.24e-64


def pulse_exact(x, t, D):
    """E_r(x, t) of the diffusion equation from Eq. gaus_init: a T0^4 (1 + 100 g)^4,
    g = exp(-x^2/w^2), expands into C(4,k) 100^k g^k, and g^k = exp(-x^2/s_k),
    s_k = w^2/k, spreads as sqrt(s_k/(s_k + 4 D t)) exp(-x^2/(s_k + 4 D t))."""
    from math import comb
    E = np.full_like(x, 1.0)
    for k in range(1, 5):
        s = OMEGA ** 2 / k
        E += comb(4, k) * 100.0 ** k * np.sqrt(s / (s + 4 * D * t)) * np.exp(-x ** 2 / (s + 4 * D * t))
    return A_R * T0 ** 4 * E


def _pulse(solver, beta, sigma, t_end, recon="vanleer"):
    """Radiative pulse on [-50, 50], 100 zones, rho = 1, kappa = 0 (Sec. 4).  The gas
    is held uniform (p = 1): with kappa = 0 it exchanges no energy with the
    radiation, and the radiation (1e-32 of its energy) cannot move it, so E_r
    obeys the M1 equations with scattering only, which diffuse with
    D = 1/(3 rho sigma) in the thick limit."""
    N = 100
    P = O.Params(gamma=5 / 3, cfl=0.4, recon=recon, solver=solver, beta=beta, a_rad=A_R)
    dx = 1.0
    x = -50 + (np.arange(N) + 0.5) * dx
    V = np.zeros((12, N))
    V[0], V[4] = 1.0, 1.0
    V[8] = pulse_exact(x, 0.0, 1.0)
    U = O.prim2con(V, P)
    t, ns, nf = O.run(O.Grid(1, (N,), (dx,)), 0.0, t_end, U, V, np.zeros(N), np.full(N, sigma), P)
    assert nf == 0
    ex = pulse_exact(x, t_end, 1 / (3 * sigma))
    bg = A_R * T0 ** 4
    return np.abs(V[8] - ex).sum() / np.abs(ex - bg).sum()


@pytest.mark.parametrize("sigma", [100.0, 1000.0])
def test_pulse_follows_the_diffusion_solution(sigma):
    t_end = 600.0 if sigma == 100.0 else 6000.0     # 4 D t = 8 = w^2 / 3
    e = {s: _pulse(s, True, sigma, t_end) for s in ("pvm", "radhll")}
    print("pulse sigma=%g rel L1: PVM-int-8 %.3e  Rad-HLL %.3e" % (sigma, e["pvm"], e["radhll"]))
    # 100 zones resolve the narrowest Gaussian of the profile with 2.5 cells: a few
    # per cent of discretisation error; PVM-int-8 is the more accurate (Sec. 4)
    assert e["pvm"] < 0.05 and e["radhll"] < 0.10
    assert e["pvm"] < e["radhll"]


def test_pulse_with_radiation_only_beta():
    """beta on the radiation block alone (beta_mode 2) keeps the diffusion limit: the
    pulse is radiation diffusing through uniform gas, which the magnetofluid block's
    viscosity does not touch."""
    sigma, t_end = 100.0, 600.0
    full = _pulse("pvm", True, sigma, t_end)
    rad = _pulse("pvm", "radiation", sigma, t_end)
    print("pulse sigma=100 rel L1: beta on every component %.4e, on the radiation block %.4e" % (full, rad))
    assert rad < 0.05 and abs(rad - full) <= 0.02 * full


def test_pulse_without_damping_is_too_diffusive():
    sigma, t_end = 100.0, 600.0
    good = _pulse("pvm", True, sigma, t_end)
    for solver in ("pvm", "radhll"):
        bad = _pulse(solver, False, sigma, t_end, recon="godunov")
        print("pulse without beta / limits, first order, %s: %.3e (PVM with beta %.3e)" % (solver, bad, good))
        assert bad > 10 * good


def _table1():
    import os
    rows = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_hll_alfven.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        w = line.split()
        rows[w[0]] = [float(a) for a in w[1:]]
    return rows


@pytest.mark.parametrize("recon", ["godunov", "minmod", "mc", "vanleer"])
def test_table1_alfven_wave_hll(recon):
    """With the radiation passive (uniform E_r, F_r = 0, kappa = sigma = 0) Rad-HLL is
    the HLL solver of the magnetofluid, and the Alfven wave must reproduce Table 1.
    The fast-magnetosonic speed used here (the Del Zanna et al. 2007 estimate) bounds
    the exact one from above, so the scheme can only be as diffusive as the paper's
    HLL or more: every error is at or above the printed value and within 10 % of it,
    and the order between the last two resolutions matches."""
    from test_oracle_scheme import _alfven_solver
    ref = _table1()[recon]
    Ns = [8, 16, 32, 64]
    l1 = [_alfven_solver(N, recon, "radhll") for N in Ns]
    for N, a, b in zip(Ns, l1, ref):
        assert 0.995 <= a / b <= 1.10, (recon, N, a, b)
    order = np.log2(l1[-2] / l1[-1])
    assert abs(order - np.log2(ref[2] / ref[3])) < 0.1

"""Exact solution of the 1D special-relativistic hydrodynamics Riemann problem
with zero tangential velocity and an ideal gas (Marti & Mueller 1994, J. Fluid
Mech. 258, 317; see also their Living Reviews in Relativity 2003).

Independent test helper for the oracle: it knows nothing of the finite-volume
scheme.  Waves:
  * rarefaction: isentropic (p / rho^gamma const) with the Riemann invariant
    atanh(v) +- (2/sqrt(gamma-1)) atanh(c_s/sqrt(gamma-1)) constant;
  * shock: Taub adiabat [h^2] = (h_b/rho_b + h_a/rho_a)[p] with mass flux
    j^2 = -[p]/[h/rho]; the post-shock velocity and shock speed are checked
    against the lab-frame Rankine-Hugoniot conditions in ``check_shock``.
"""
import math

from scipy.optimize import brentq


def enthalpy(rho, p, g):
    return 1.0 + g / (g - 1.0) * p / rho


def sound(rho, p, g):
    return math.sqrt(g * p / (rho * enthalpy(rho, p, g)))


def _phi(c, g):
    s = math.sqrt(g - 1.0)
    return 2.0 / s * math.atanh(c / s)


def rarefaction(p, a, side, g):
    """State behind a rarefaction attached to state a=(rho, p, v); side -1 left, +1 right."""
    rho = a[0] * (p / a[1]) ** (1.0 / g)
    c = sound(rho, p, g)
    ca = sound(a[0], a[1], g)
    if side < 0:
        y = math.atanh(a[2]) + _phi(ca, g) - _phi(c, g)
    else:
        y = math.atanh(a[2]) - _phi(ca, g) + _phi(c, g)
    return math.tanh(y), rho


def shock(p, a, side, g):
    """(v_b, rho_b, V_s) behind a shock of pressure p moving into state a."""
    rho_a, p_a, v_a = a
    ha = enthalpy(rho_a, p_a, g)
    q = (g - 1.0) * (p_a - p) / (g * p)
    A, B = 1.0 + q, -q
    Cc = ha * (p_a - p) / rho_a - ha * ha
    hb = (-B + math.sqrt(B * B - 4.0 * A * Cc)) / (2.0 * A)
    rho_b = g * p / ((g - 1.0) * (hb - 1.0))
    j2 = (p - p_a) / (ha / rho_a - hb / rho_b)   # j^2 = -[p]/[h/rho]
    j = math.sqrt(j2)
    Wa2 = 1.0 / (1.0 - v_a * v_a)
    Wa = math.sqrt(Wa2)
    num = rho_a * rho_a * Wa2 * v_a + side * j * math.sqrt(j2 + rho_a * rho_a * Wa2 * (1.0 - v_a * v_a))
    Vs = num / (rho_a * rho_a * Wa2 + j2)
    Ws = 1.0 / math.sqrt(1.0 - Vs * Vs)
    js = side * j
    vb = (ha * Wa * v_a + Ws * (p - p_a) / js) / (ha * Wa + (p - p_a) * (Ws * v_a / js + 1.0 / (rho_a * Wa)))
    return vb, rho_b, Vs


def conserved(rho, p, v, g):
    W = 1.0 / math.sqrt(1.0 - v * v)
    h = enthalpy(rho, p, g)
    D = rho * W
    S = rho * h * W * W * v
    tau = rho * h * W * W - p - D
    return (D, S, tau), (D * v, S * v + p, S - D * v)


def check_shock(p, a, side, g):
    """Largest relative violation of V_s [U] = [F] across the computed shock."""
    vb, rho_b, Vs = shock(p, a, side, g)
    Ua, Fa = conserved(a[0], a[1], a[2], g)
    Ub, Fb = conserved(rho_b, p, vb, g)
    err = 0.0
    for k in range(3):
        lhs = Vs * (Ub[k] - Ua[k])
        rhs = Fb[k] - Fa[k]
        err = max(err, abs(lhs - rhs) / max(abs(rhs), abs(lhs), 1e-300))
    return err


def _vstar(p, a, side, g):
    if p <= a[1]:
        return rarefaction(p, a, side, g)[0]
    return shock(p, a, side, g)[0]


def solve(L, R, g):
    """Star pressure and velocity for left/right states (rho, p, v)."""
    f = lambda p: _vstar(p, L, -1, g) - _vstar(p, R, +1, g)
    lo = 1e-14 * min(L[1], R[1])
    hi = 1e4 * max(L[1], R[1])
    ps = brentq(f, lo, hi, xtol=1e-15, rtol=1e-14, maxiter=500)
    return ps, _vstar(ps, L, -1, g)


def sample(L, R, g, xi_list):
    """(rho, p, v) at each similarity coordinate xi = (x - x0)/t."""
    ps, vs = solve(L, R, g)
    out = []
    # left wave
    if ps > L[1]:
        _, rhoL, VsL = shock(ps, L, -1, g)
        left = ("shock", VsL, rhoL)
    else:
        _, rhoL = rarefaction(ps, L, -1, g)
        cL, cs_ = sound(*L[:2], g), sound(rhoL, ps, g)
        left = ("fan", (L[2] - cL) / (1 - L[2] * cL), (vs - cs_) / (1 - vs * cs_), rhoL)
    if ps > R[1]:
        _, rhoR, VsR = shock(ps, R, +1, g)
        right = ("shock", VsR, rhoR)
    else:
        _, rhoR = rarefaction(ps, R, +1, g)
        cR, cs_ = sound(*R[:2], g), sound(rhoR, ps, g)
        right = ("fan", (R[2] + cR) / (1 + R[2] * cR), (vs + cs_) / (1 + vs * cs_), rhoR)

    def in_fan(xi, a, side):
        def speed(p):
            v, rho = rarefaction(p, a, side, g)
            c = sound(rho, p, g)
            return (v + side * c) / (1 + side * v * c)
        p = brentq(lambda p: speed(p) - xi, min(ps, a[1]), max(ps, a[1]), xtol=1e-15, rtol=1e-14)
        v, rho = rarefaction(p, a, side, g)
        return rho, p, v

    for xi in xi_list:
        if xi < vs:
            if left[0] == "shock":
                out.append(L if xi < left[1] else (left[2], ps, vs))
            else:
                if xi <= left[1]:
                    out.append(L)
                elif xi >= left[2]:
                    out.append((left[3], ps, vs))
                else:
                    out.append(in_fan(xi, L, -1))
        else:
            if right[0] == "shock":
                out.append(R if xi > right[1] else (right[2], ps, vs))
            else:
                if xi >= right[1]:
                    out.append(R)
                elif xi <= right[2]:
                    out.append((right[3], ps, vs))
                else:
                    out.append(in_fan(xi, R, +1))
    return out

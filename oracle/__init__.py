"""Plain FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

This package is the reference the CUDA path is checked against.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it; the product path (``paper_2212_00370_gb300``) never does, and
the two share no code.  The numerics live in plain C (``oracle/*.c``, built
by ``oracle/build.py`` with ``-ffp-contract=off``); this module only marshals
numpy arrays through ctypes.

Paper: Lopez-Miralles, Marti & Perucho 2022, arXiv:2212.00370.  Every C
function cites the section / equation it restates.

Parity pins: see ``tests/test_oracle_*.py``.  All point functions and the
grid update are pinned (printed Table 4 errors, exact Riemann solutions,
closed forms, Lorentz covariance of the four-force, brute-force Jacobians,
conservation).
"""
import ctypes as C
import dataclasses

import numpy as np

from . import build as _build

RECON = {"godunov": 0, "minmod": 1, "mc": 2, "vanleer": 3}
BC = {"outflow": 0, "periodic": 1}

_lib = None


class _Params(C.Structure):
    _fields_ = [
        ("gamma", C.c_double), ("a_rad", C.c_double), ("cfl", C.c_double),
        ("pvm_eps", C.c_double), ("recon", C.c_int), ("beta_mode", C.c_int),
        ("imp_mode", C.c_int), ("pvm_k", C.c_int), ("solver", C.c_int), ("c2p_maxit", C.c_int),
        ("imp_maxit", C.c_int),
        ("imp_tol", C.c_double), ("gfac", C.c_double), ("gm1g", C.c_double),
    ]


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "c2p_calls", "c2p_iters", "c2p_fail", "flux_evals", "pvm_faces", "pvm_fallback",
        "imp_cells", "imp_iters", "imp_resid", "imp_jac", "imp_fail", "imp_matter", "imp_resid_max",
        "fallback_cells", "fallback_flagged", "imp_polish")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class _Grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("dx", C.c_double * 3), ("bc", C.c_int * 3)]


@dataclasses.dataclass
class Params:
    gamma: float = 5.0 / 3.0
    a_rad: float = 1.0
    cfl: float = 0.4
    pvm_eps: float = 1e-8
    recon: str = "vanleer"
    beta: object = True     # True: Eq. beta; False: beta = 1; "radiation": Eq. beta on E_r, F_r only
    implicit: str = "newton"
    c2p_maxit: int = 60
    imp_maxit: int = 50
    imp_tol: float = 1e-10
    pvm_k: int = 3          # PVM-int-2^k: 3 is the paper's PVM-int-8, 4 is PVM-int-16
    solver: str = "pvm"     # "pvm" (Sec. 3.2.2) or "radhll" (Sec. 3.2.1)

    def struct(self):
        p = _Params(self.gamma, self.a_rad, self.cfl, self.pvm_eps, RECON[self.recon],
                    2 if self.beta == "radiation" else (1 if self.beta else 0),
                    {"newton": 0, "picard": 1, "matter": 2}[self.implicit], self.pvm_k,
                    {"pvm": 0, "radhll": 1}[self.solver],
                    self.c2p_maxit, self.imp_maxit, self.imp_tol, 0.0, 0.0)
        lib().or_params_init(C.byref(p))
        return p


@dataclasses.dataclass
class Grid:
    ndim: int
    n: tuple
    dx: tuple
    bc: tuple = ("outflow", "outflow", "outflow")

    def struct(self):
        n = list(self.n) + [1] * (3 - len(self.n))
        dx = list(self.dx) + [1.0] * (3 - len(self.dx))
        bc = [BC[b] if isinstance(b, str) else int(b) for b in self.bc]
        bc = bc + [0] * (3 - len(bc))
        return _Grid(self.ndim, (C.c_int * 3)(*n), (C.c_double * 3)(*dx), (C.c_int * 3)(*bc))

    @property
    def ncells(self):
        return int(np.prod(self.n))


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        P = C.POINTER(_Params)
        S = C.POINTER(Stats)
        G = C.POINTER(_Grid)
        i64, i32p = C.c_int64, C.POINTER(C.c_int32)
        sig = {
            "or_params_init": (None, [P]),
            "or_prim2con_n": (None, [P, i64, dp, dp]),
            "or_prim_Z_n": (None, [P, i64, dp, dp]),
            "or_con2prim_n": (None, [P, i64, dp, dp, dp, dp, i32p, S]),
            "or_flux_n": (None, [P, C.c_int, i64, dp, dp, dp]),
            "or_signal_speed_n": (None, [P, C.c_int, i64, dp, dp]),
            "or_pvm_flux_n": (None, [P, C.c_int, i64, dp, dp, dp, dp, dp, dp, i32p, S]),
            "or_implicit_n": (None, [P, i64, dp, dp, C.c_double, dp, dp, dp, dp, i32p, S]),
            "or_implicit_cn": (None, [P, i64, dp, dp, C.c_double, dp, dp, dp, dp, dp, i32p, S]),
            "or_four_force": (None, [C.c_double, C.c_double, C.c_double, dp, C.c_double,
                                     C.c_double, C.c_double, dp, dp, dp]),
            "or_m1_pressure": (None, [C.c_double, dp, dp]),
            "or_eddington_factor": (C.c_double, [C.c_double]),
            "or_limiter": (C.c_double, [C.c_int, C.c_double, C.c_double]),
            "or_pvm_coefficients": (C.c_int, [C.c_int, dp]),
            "or_reconstruct": (None, [P, dp, dp, dp, dp, dp, C.POINTER(C.c_int)]),
            "or_picard_matrix": (None, [C.c_double, C.c_double, C.c_double, C.c_double, dp,
                                        C.c_double, C.c_double, dp, dp, dp, dp]),
            "or_solve4": (C.c_int, [dp, dp, dp]),
            "or_llf_flux": (None, [P, C.c_int, dp, dp, dp]),
            "or_radhll_flux": (None, [P, C.c_int, dp, dp, C.c_double, C.c_double, dp]),
            "or_mhd_speeds": (None, [P, C.c_int, dp, dp, dp]),
            "or_rad_speeds": (None, [C.c_int, dp, dp, dp]),
            "or_grid_dt": (C.c_double, [P, G, dp]),
            "or_grid_face_flux": (C.c_int, [P, G, C.c_int, dp, dp, dp, dp, dp, S]),
            "or_grid_stage": (C.c_int, [P, G, C.c_int, C.c_double, dp, dp, dp, dp, dp, dp, dp,
                                        i32p, S]),
            "or_grid_step": (C.c_int, [P, G, C.c_double, dp, dp, dp, dp, S]),
            "or_grid_step_c": (C.c_int, [P, G, C.c_double, dp, dp, dp, dp, dp, S]),
            "or_grid_run": (C.c_int, [P, G, C.c_double, C.c_double, C.c_int, dp, dp, dp, dp,
                                      dp, C.POINTER(C.c_int), S]),
            "or_grid_step_ct": (C.c_int, [P, G, C.c_double, dp, dp, dp, dp, dp, dp, S]),
            "or_grid_run_ct": (C.c_int, [P, G, C.c_double, C.c_double, C.c_int, dp, dp, dp, dp, dp,
                                         dp, C.POINTER(C.c_int), S]),
            "or_grid_face_flux_b": (C.c_int, [P, G, C.c_int, dp, dp, dp, dp, dp, dp, S]),
            "or_ct_nfaces": (C.c_int64, [G]),
            "or_ct_faces_from_cells": (None, [G, dp, dp]),
            "or_ct_cells_from_faces": (None, [G, dp, dp, dp]),
            "or_ct_div": (None, [G, dp, dp]),
            "or_ct_canonical": (None, [G, dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i32(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _soa(a):
    """(12,) or (12, n) float64 C-contiguous view; returns (array, n, squeeze)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim == 1:
        return a.reshape(12, 1).copy(), 1, True
    return a.reshape(12, -1), a.reshape(12, -1).shape[1], False


def _out(a, squeeze):
    return a[:, 0] if squeeze else a


def _stats(stats):
    return C.byref(stats) if stats is not None else None


# ------------------------------ point functions ------------------------------
def prim2con(V, P):
    V, n, sq = _soa(V)
    U = np.empty_like(V)
    lib().or_prim2con_n(C.byref(P.struct()), n, _d(V), _d(U))
    return _out(U, sq)


def prim_Z(V, P):
    V, n, sq = _soa(V)
    Z = np.empty(n)
    lib().or_prim_Z_n(C.byref(P.struct()), n, _d(V), _d(Z))
    return Z[0] if sq else Z


def con2prim(U, P, Zguess=None, stats=None):
    U, n, sq = _soa(U)
    V = np.zeros_like(U)
    Z = np.zeros(n)
    st = np.zeros(n, dtype=np.int32)
    zg = None if Zguess is None else np.ascontiguousarray(np.broadcast_to(Zguess, (n,)), dtype=np.float64)
    lib().or_con2prim_n(C.byref(P.struct()), n, _d(U), _d(zg) if zg is not None else None,
                        _d(V), _d(Z), _i32(st), _stats(stats))
    if sq:
        return V[:, 0], Z[0], int(st[0])
    return V, Z, st


def flux(V, U, d, P):
    V, n, sq = _soa(V)
    U, _, _ = _soa(U)
    F = np.empty_like(V)
    lib().or_flux_n(C.byref(P.struct()), d, n, _d(V), _d(U), _d(F))
    return _out(F, sq)


def signal_speed(V, d, P):
    V, n, sq = _soa(V)
    lam = np.empty(n)
    lib().or_signal_speed_n(C.byref(P.struct()), d, n, _d(V), _d(lam))
    return lam[0] if sq else lam


def pvm_flux(VL, VR, tauL, tauR, d, P, stats=None):
    VL, n, sq = _soa(VL)
    VR, _, _ = _soa(VR)
    tL = np.ascontiguousarray(np.broadcast_to(tauL, (n,)), dtype=np.float64)
    tR = np.ascontiguousarray(np.broadcast_to(tauR, (n,)), dtype=np.float64)
    F = np.empty_like(VL)
    U4 = np.empty_like(VL)
    st = np.zeros(n, dtype=np.int32)
    lib().or_pvm_flux_n(C.byref(P.struct()), d, n, _d(VL), _d(VR), _d(tL), _d(tR), _d(F),
                        _d(U4), _i32(st), _stats(stats))
    if sq:
        return F[:, 0], U4[:, 0], int(st[0])
    return F, U4, st


def implicit(Ustar, kappa, sigma, hdt, P, Zguess=None, stats=None):
    Us, n, sq = _soa(Ustar)
    k = np.ascontiguousarray(np.broadcast_to(kappa, (n,)), dtype=np.float64)
    s = np.ascontiguousarray(np.broadcast_to(sigma, (n,)), dtype=np.float64)
    zg = None if Zguess is None else np.ascontiguousarray(np.broadcast_to(Zguess, (n,)), dtype=np.float64)
    U = np.zeros_like(Us)
    V = np.zeros_like(Us)
    st = np.zeros(n, dtype=np.int32)
    lib().or_implicit_n(C.byref(P.struct()), n, _d(k), _d(s), float(hdt), _d(Us),
                        _d(zg) if zg is not None else None, _d(U), _d(V), _i32(st), _stats(stats))
    if sq:
        return U[:, 0], V[:, 0], int(st[0])
    return U, V, st


def implicit_cached(Ustar, kappa, sigma, hdt, P, jcache, Zguess=None, stats=None):
    """The implicit step of n cells with their Jacobian cache jcache ((17, n) float64,
    zero = empty; updated in place, as a grid step does).  Returns (U, V, status)."""
    Us, n, _ = _soa(Ustar)
    assert jcache.shape == (17, n) and jcache.dtype == np.float64 and jcache.flags.c_contiguous
    k = np.ascontiguousarray(np.broadcast_to(kappa, (n,)), dtype=np.float64)
    s = np.ascontiguousarray(np.broadcast_to(sigma, (n,)), dtype=np.float64)
    zg = None if Zguess is None else np.ascontiguousarray(np.broadcast_to(Zguess, (n,)), dtype=np.float64)
    U = np.zeros_like(Us)
    V = np.zeros_like(Us)
    st = np.zeros(n, dtype=np.int32)
    lib().or_implicit_cn(C.byref(P.struct()), n, _d(k), _d(s), float(hdt), _d(Us),
                         _d(zg) if zg is not None else None, _d(U), _d(V), _d(jcache), _i32(st),
                         _stats(stats))
    return U, V, st


def four_force(kappa, sigma, rho, u, W, BP, E, F, Pr):
    u = np.ascontiguousarray(u, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    Pr = np.ascontiguousarray(Pr, dtype=np.float64)
    G = np.empty(4)
    lib().or_four_force(kappa, sigma, rho, _d(u), W, BP, E, _d(F), _d(Pr), _d(G))
    return G


def m1_pressure(E, F):
    F = np.ascontiguousarray(F, dtype=np.float64)
    Pr = np.empty((3, 3))
    lib().or_m1_pressure(float(E), _d(F), _d(Pr))
    return Pr


def eddington_factor(f):
    return lib().or_eddington_factor(float(f))


def pvm_coefficients(k):
    """Horner-order coefficients of p_k from Eq. iterat (degree 2^(k-1) in x^2)."""
    a = np.zeros(9)
    m = lib().or_pvm_coefficients(int(k), _d(a))
    return a[:m + 1]


def limiter(recon, dL, dR):
    return lib().or_limiter(RECON[recon], float(dL), float(dR))


def reconstruct(Vm1, V0, Vp1, P):
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (Vm1, V0, Vp1)]
    Vm = np.empty(12)
    Vp = np.empty(12)
    fb = C.c_int(0)
    lib().or_reconstruct(C.byref(P.struct()), _d(a[0]), _d(a[1]), _d(a[2]), _d(Vm), _d(Vp),
                         C.byref(fb))
    return Vm, Vp, fb.value


def picard_matrix(kappa, sigma, hdt, rho, u, W, BP, Dr, Xs):
    u = np.ascontiguousarray(u, dtype=np.float64)
    Dr = np.ascontiguousarray(Dr, dtype=np.float64)
    Xs = np.ascontiguousarray(Xs, dtype=np.float64)
    Cm = np.empty((4, 4))
    rhs = np.empty(4)
    lib().or_picard_matrix(kappa, sigma, hdt, rho, _d(u), W, BP, _d(Dr), _d(Xs), _d(Cm), _d(rhs))
    return Cm, rhs


def llf_flux(VL, VR, d, P):
    VL = np.ascontiguousarray(VL, dtype=np.float64)
    VR = np.ascontiguousarray(VR, dtype=np.float64)
    F = np.empty(12)
    lib().or_llf_flux(C.byref(P.struct()), d, _d(VL), _d(VR), _d(F))
    return F


def radhll_flux(VL, VR, tauL, tauR, d, P):
    """Radiative HLL flux at one face (Sec. 3.2.1)."""
    VL = np.ascontiguousarray(VL, dtype=np.float64)
    VR = np.ascontiguousarray(VR, dtype=np.float64)
    F = np.empty(12)
    lib().or_radhll_flux(C.byref(P.struct()), d, _d(VL), _d(VR), float(tauL), float(tauR), _d(F))
    return F


def mhd_speeds(V, d, P):
    V = np.ascontiguousarray(V, dtype=np.float64)
    lm, lp = C.c_double(), C.c_double()
    lib().or_mhd_speeds(C.byref(P.struct()), d, _d(V), C.byref(lm), C.byref(lp))
    return lm.value, lp.value


def rad_speeds(V, d):
    V = np.ascontiguousarray(V, dtype=np.float64)
    l1, l3 = C.c_double(), C.c_double()
    lib().or_rad_speeds(d, _d(V), C.byref(l1), C.byref(l3))
    return l1.value, l3.value


def solve4(A, b):
    A = np.ascontiguousarray(A, dtype=np.float64).copy()
    b = np.ascontiguousarray(b, dtype=np.float64).copy()
    x = np.empty(4)
    rc = lib().or_solve4(_d(A), _d(b), _d(x))
    return x, rc


# ------------------------------ grids ------------------------------
def _field(a, N):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.size == 12 * N, (a.shape, N)
    return a


def grid_dt(g, V, P):
    V = _field(V, g.ncells)
    return lib().or_grid_dt(C.byref(P.struct()), C.byref(g.struct()), _d(V))


def face_flux(g, d, U, V, kappa, sigma, P, stats=None):
    N = g.ncells
    U, V = _field(U, N), _field(V, N)
    k = np.ascontiguousarray(kappa, dtype=np.float64).reshape(-1)
    s = np.ascontiguousarray(sigma, dtype=np.float64).reshape(-1)
    m = list(g.n) + [1] * (3 - len(g.n))
    m[d] += 1
    F = np.empty((12, m[2], m[1], m[0]))
    lib().or_grid_face_flux(C.byref(P.struct()), C.byref(g.struct()), d, _d(U), _d(V), _d(k),
                            _d(s), _d(F), _stats(stats))
    return F


def stage(g, s, dt, U0, Us, Vs, kappa, sigma, P, stats=None):
    N = g.ncells
    U0, Us, Vs = _field(U0, N), _field(Us, N), _field(Vs, N)
    k = np.ascontiguousarray(kappa, dtype=np.float64).reshape(-1)
    sg = np.ascontiguousarray(sigma, dtype=np.float64).reshape(-1)
    Uo = np.empty_like(Us)
    Vo = np.empty_like(Vs)
    cs = np.zeros(N, dtype=np.int32)
    nf = lib().or_grid_stage(C.byref(P.struct()), C.byref(g.struct()), s, float(dt), _d(U0),
                             _d(Us), _d(Vs), _d(k), _d(sg), _d(Uo), _d(Vo), _i32(cs), _stats(stats))
    return Uo, Vo, cs, nf


def step(g, dt, U, V, kappa, sigma, P, stats=None, jcache=None, bface=None):
    """One IMEX-RK3 step in place; returns the number of failed cells.  jcache: a
    float64 array of 17 * ncells (zeros = empty) carried between steps, or None.
    bface: the staggered field of constrained transport (2D/3D; ct_nfaces(g)
    values, advanced in place), or None."""
    N = g.ncells
    assert U.flags.c_contiguous and V.flags.c_contiguous and U.dtype == np.float64
    k = np.ascontiguousarray(kappa, dtype=np.float64).reshape(-1)
    s = np.ascontiguousarray(sigma, dtype=np.float64).reshape(-1)
    assert U.size == 12 * N
    if jcache is None and bface is None:
        return lib().or_grid_step(C.byref(P.struct()), C.byref(g.struct()), float(dt), _d(U),
                                  _d(V), _d(k), _d(s), _stats(stats))
    if jcache is None:
        jcache = np.zeros(17 * N)
    assert jcache.size == 17 * N and jcache.dtype == np.float64 and jcache.flags.c_contiguous
    if bface is None:
        return lib().or_grid_step_c(C.byref(P.struct()), C.byref(g.struct()), float(dt), _d(U),
                                    _d(V), _d(k), _d(s), _d(jcache), _stats(stats))
    assert bface.flags.c_contiguous and bface.dtype == np.float64 and bface.size == ct_nfaces(g)
    return lib().or_grid_step_ct(C.byref(P.struct()), C.byref(g.struct()), float(dt), _d(U), _d(V),
                                 _d(bface), _d(k), _d(s), _d(jcache), _stats(stats))


def run(g, t0, t_end, U, V, kappa, sigma, P, max_steps=10 ** 9, stats=None, bface=None):
    """Advance in place to t_end (last step clipped); returns (t, steps, nfail).
    bface: staggered field of constrained transport (advanced in place), or None."""
    N = g.ncells
    assert U.flags.c_contiguous and V.flags.c_contiguous and U.size == 12 * N
    k = np.ascontiguousarray(kappa, dtype=np.float64).reshape(-1)
    s = np.ascontiguousarray(sigma, dtype=np.float64).reshape(-1)
    t = C.c_double(0.0)
    ns = C.c_int(0)
    if bface is not None:
        assert bface.flags.c_contiguous and bface.dtype == np.float64 and bface.size == ct_nfaces(g)
    nf = lib().or_grid_run_ct(C.byref(P.struct()), C.byref(g.struct()), float(t0), float(t_end),
                              int(max_steps), _d(U), _d(V), None if bface is None else _d(bface),
                              _d(k), _d(s), C.byref(t), C.byref(ns), _stats(stats))
    return t.value, ns.value, nf


def ct_nfaces(g):
    """Faces of the staggered field (directions d < ndim, one after the other)."""
    return int(lib().or_ct_nfaces(C.byref(g.struct())))


def ct_faces_from_cells(g, V):
    b = np.empty(ct_nfaces(g))
    lib().or_ct_faces_from_cells(C.byref(g.struct()), _d(np.ascontiguousarray(V)), _d(b))
    return b


def ct_cells_from_faces(g, bface, U, V):
    """Sets the cell-centred B_d (d < ndim) of U and V (in place) to the face means."""
    lib().or_ct_cells_from_faces(C.byref(g.struct()), _d(bface), _d(U), _d(V))


def ct_canonical(g, bface):
    """Periodic duplicate faces (index n_d) take the value of face 0 (in place)."""
    lib().or_ct_canonical(C.byref(g.struct()), _d(bface))


def ct_div(g, bface):
    div = np.empty(g.ncells)
    lib().or_ct_div(C.byref(g.struct()), _d(bface), _d(div))
    return div

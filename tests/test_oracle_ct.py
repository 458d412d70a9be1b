"""Pins of the oracle's constrained transport (CT-contact, Gardiner & Stone 2005;
the method the paper's multi-dimensional runs use, Sec. 4).

  * a face field built as the discrete curl of a vector potential keeps its
    discrete divergence at round-off level over many steps, in 2D and 3D;
  * the magnetic flux through every lattice plane of a periodic box is conserved
    exactly (the EMF differences telescope);
  * a uniform state stays uniform;
  * a planar problem (variation along one axis) run on a 2D/3D grid with CT gives
    the 1D solution: for plane-parallel data the CT-contact corner EMF equals the
    upwind face EMF of the 1D solver (its corrections cancel), so CT reduces to
    the 1D induction update.
"""
import numpy as np
import pytest

import oracle as O


def smooth_state(shape, seed, amp_b=0.3):
    """Smooth periodic primitives on the unit box; B set later from the faces."""
    rng = np.random.default_rng(seed)
    nd = len(shape)
    N = int(np.prod(shape))
    X = np.meshgrid(*[(np.arange(n) + 0.5) / n for n in shape], indexing="ij")
    ph = sum(2 * np.pi * X[k] * (k + 1) for k in range(nd))
    flat = lambda a: np.ascontiguousarray(np.asarray(a).T).reshape(-1)
    V = np.zeros((12, N))
    V[0] = flat(1 + 0.4 * np.sin(ph))
    V[1] = flat(0.3 * np.cos(ph))
    V[2] = flat(0.2 * np.sin(2 * ph))
    V[3] = 0.1
    V[4] = flat(0.6 + 0.3 * np.cos(ph))
    V[7] = flat(0.1 * np.sin(ph))
    V[8] = flat(0.8 + 0.4 * np.sin(ph))
    V[9] = V[8] * flat(0.3 * np.cos(ph))
    V[10] = 0.2 * V[8]
    kappa = 10 ** rng.uniform(-1, 0.5, N)
    sigma = 10 ** rng.uniform(-1, 0.5, N)
    return V, kappa, sigma


def curl_faces(shape, amp=0.3):
    """Face field = discrete curl of an edge vector potential on the periodic unit
    box (exactly divergence-free up to rounding), plus a uniform background.
    2D: A_z at corners.  3D: A_x, A_y, A_z on their edges."""
    nd = len(shape)
    h = [1.0 / n for n in shape]
    if nd == 2:
        nx, ny = shape
        xc = np.arange(nx + 1) * h[0]
        yc = np.arange(ny + 1) * h[1]
        Xc, Yc = np.meshgrid(xc, yc, indexing="ij")              # corners (i-1/2, j-1/2)
        Az = amp / (2 * np.pi) * (np.sin(2 * np.pi * Xc) * np.cos(2 * np.pi * Yc) + 0.5 * np.sin(4 * np.pi * Yc))
        bx = (Az[:, 1:] - Az[:, :-1]) / h[1] + 0.2                # x-faces (nx+1, ny)
        by = -(Az[1:, :] - Az[:-1, :]) / h[0] + 0.1               # y-faces (nx, ny+1)
        return np.concatenate([bx.T.reshape(-1), by.T.reshape(-1)])
    nx, ny, nz = shape
    def ax(n, hh, stag):
        return (np.arange(n + 1) if stag else np.arange(n) + 0.5) * hh
    def pot(X, Y, Z, k):
        return amp / (2 * np.pi) * np.sin(2 * np.pi * (X + 2 * Y + 3 * Z) + k)
    # A_x on x-edges (i, j-1/2, k-1/2): (nx, ny+1, nz+1); A_y on (i-1/2, j, k-1/2); A_z on (i-1/2, j-1/2, k)
    Ax = pot(*np.meshgrid(ax(nx, h[0], 0), ax(ny, h[1], 1), ax(nz, h[2], 1), indexing="ij"), 0.3)
    Ay = pot(*np.meshgrid(ax(nx, h[0], 1), ax(ny, h[1], 0), ax(nz, h[2], 1), indexing="ij"), 1.1)
    Az = pot(*np.meshgrid(ax(nx, h[0], 1), ax(ny, h[1], 1), ax(nz, h[2], 0), indexing="ij"), 2.0)
    bx = (Az[:, 1:, :] - Az[:, :-1, :]) / h[1] - (Ay[:, :, 1:] - Ay[:, :, :-1]) / h[2] + 0.2
    by = (Ax[:, :, 1:] - Ax[:, :, :-1]) / h[2] - (Az[1:, :, :] - Az[:-1, :, :]) / h[0] + 0.1
    bz = (Ay[1:, :, :] - Ay[:-1, :, :]) / h[0] - (Ax[:, 1:, :] - Ax[:, :-1, :]) / h[1] - 0.15
    return np.concatenate([bx.transpose(2, 1, 0).reshape(-1), by.transpose(2, 1, 0).reshape(-1),
                           bz.transpose(2, 1, 0).reshape(-1)])


def periodic_grid(shape):
    nd = len(shape)
    return O.Grid(nd, tuple(shape), tuple(1.0 / n for n in shape), ("periodic",) * nd)


def setup(shape, seed):
    g = periodic_grid(shape)
    P = O.Params(gamma=4 / 3, cfl=0.4)
    V, kappa, sigma = smooth_state(shape, seed)
    b = curl_faces(shape)
    assert b.size == O.ct_nfaces(g)
    O.ct_canonical(g, b)
    U = O.prim2con(V, P)
    O.ct_cells_from_faces(g, b, U, V)
    U = O.prim2con(V, P)
    return g, P, U, V, b, kappa, sigma


@pytest.mark.parametrize("shape,steps", [((24, 20), 12), ((8, 7, 6), 4)])
def test_divergence_stays_at_round_off(shape, steps):
    g, P, U, V, b, kappa, sigma = setup(shape, 3)
    bmax = np.abs(b).max()
    h = min(1.0 / n for n in shape)
    div0 = np.abs(O.ct_div(g, b)).max() * h / bmax
    assert div0 < 1e-13
    jc = np.zeros(17 * g.ncells)
    for _ in range(steps):
        dt = O.grid_dt(g, V, P)
        assert O.step(g, dt, U, V, kappa, sigma, P, jcache=jc, bface=b) == 0
    div = np.abs(O.ct_div(g, b)).max() * h / np.abs(b).max()
    assert div < 1e-12, div
    # the field did change
    assert np.abs(b - curl_faces(shape)).max() > 1e-4


def test_plane_fluxes_are_conserved_2d():
    shape = (20, 16)
    g, P, U, V, b, kappa, sigma = setup(shape, 5)
    nx, ny = shape
    def plane_fluxes(bf):
        bx = bf[:(nx + 1) * ny].reshape(ny, nx + 1)
        by = bf[(nx + 1) * ny:].reshape(ny + 1, nx)
        return bx.sum(axis=0), by.sum(axis=1)    # flux through each x-plane and y-plane
    fx0, fy0 = plane_fluxes(b)
    for _ in range(6):
        dt = O.grid_dt(g, V, P)
        assert O.step(g, dt, U, V, kappa, sigma, P, bface=b) == 0
    fx, fy = plane_fluxes(b)
    scale = np.abs(b).sum()
    assert np.abs(fx - fx0).max() <= 1e-13 * scale and np.abs(fy - fy0).max() <= 1e-13 * scale


def test_uniform_state_stays_uniform():
    shape = (10, 9)
    g = periodic_grid(shape)
    P = O.Params(gamma=4 / 3)
    N = g.ncells
    V = np.zeros((12, N))
    V[0], V[1], V[2], V[4], V[5], V[6], V[7] = 1.0, 0.3, -0.2, 0.5, 0.4, -0.3, 0.2
    V[8], V[9] = 1.0, 0.1
    b = O.ct_faces_from_cells(g, V)
    U = O.prim2con(V, P)
    b0, U0 = b.copy(), U.copy()
    for _ in range(3):
        assert O.step(g, O.grid_dt(g, V, P), U, V, np.zeros(N), np.zeros(N), P, bface=b) == 0
    np.testing.assert_array_equal(b, b0)
    np.testing.assert_array_equal(U, U0)


def _planar(nx, ntrans, ndim, axis, solver, steps=4):
    """A planar Riemann-like smooth profile along `axis` on a periodic ndim grid
    with CT, and the same profile on a 1D grid without CT."""
    rng = np.random.default_rng(7)
    P = O.Params(gamma=4 / 3, cfl=0.4, solver=solver)
    x = (np.arange(nx) + 0.5) / nx
    V1 = np.zeros((12, nx))
    V1[0] = 1 + 0.5 * np.tanh(10 * np.sin(2 * np.pi * x))
    V1[1], V1[2], V1[3] = 0.3 * np.cos(2 * np.pi * x), 0.2 * np.sin(2 * np.pi * x), 0.05
    V1[4] = 0.6 + 0.3 * np.cos(2 * np.pi * x)
    V1[5], V1[6], V1[7] = 0.5, 0.3 * np.sin(2 * np.pi * x), 0.1 * np.cos(2 * np.pi * x)
    V1[8] = 0.8 + 0.3 * np.sin(2 * np.pi * x)
    V1[9], V1[10] = 0.2 * V1[8], 0.1 * V1[8]
    k1, s1 = 10 ** rng.uniform(-1, 0.5, nx), 10 ** rng.uniform(-1, 0.5, nx)
    # 1D reference along x, components permuted so that x maps to `axis`
    g1 = O.Grid(1, (nx,), (1.0 / nx,), ("periodic",))
    U1 = O.prim2con(V1, P)
    Vr = V1.copy()
    # multi-D grid: `axis` carries the profile; vector components rotated accordingly
    perm = list(range(3))
    perm[0], perm[axis] = axis, 0
    shape = [ntrans] * ndim
    shape[axis] = nx
    gN = O.Grid(ndim, tuple(shape), tuple(1.0 / s for s in shape), ("periodic",) * ndim)
    N = gN.ncells
    idx = np.indices(shape[::-1]).reshape(ndim, -1)[::-1][axis]   # position along axis, x fastest
    VN = np.zeros((12, N))
    for q in range(12):
        VN[q] = V1[q][idx]
    for base in (1, 5, 9):   # rotate vectors: component 0 of the 1D problem goes to `axis`
        comp = [V1[base + c][idx] for c in range(3)]
        for c in range(3):
            VN[base + perm[c]] = comp[c]
    kN, sN = k1[idx], s1[idx]
    b = O.ct_faces_from_cells(gN, VN)
    UN = O.prim2con(VN, P)
    jc1, jcN = np.zeros(17 * nx), np.zeros(17 * N)
    for _ in range(steps):
        dt = O.grid_dt(g1, Vr, P)
        assert O.step(g1, dt, U1, Vr, k1, s1, P, jcache=jc1) == 0
        assert O.step(gN, dt, UN, VN, kN, sN, P, jcache=jcN, bface=b) == 0
    ref = np.zeros_like(UN)
    for q in range(12):
        ref[q] = U1[q][idx]
    for base in (1, 5, 9):
        comp = [U1[base + c][idx] for c in range(3)]
        for c in range(3):
            ref[base + perm[c]] = comp[c]
    return UN, ref


@pytest.mark.parametrize("solver,tol", [("radhll", 1e-12), ("pvm", 1e-6)])
@pytest.mark.parametrize("ndim,axis", [(2, 0), (2, 1), (3, 2)])
def test_planar_problem_reduces_to_1d(ndim, axis, solver, tol):
    """Equal in exact arithmetic.  Rad-HLL shows the rounding of the corner
    average; the PVM's eps = 1e-8 products amplify that rounding by 1/eps, so its
    bound is the finite-difference noise level."""
    UN, ref = _planar(32, 4, ndim, axis, solver)
    scale = np.abs(ref).max(axis=1, keepdims=True) + 1e-30
    err = (np.abs(UN - ref) / scale).max()
    print("CT planar vs 1D (%s), max relative difference %.2e" % (solver, err))
    assert err < tol


def test_fallback_under_ct_keeps_the_constraint():
    """The 2D blast at 48^2 over 40 steps: the admissibility fallback fires (its
    Rusanov fluxes enter the edge EMFs) and the implicit solve needs the matter
    form, yet the discrete divergence stays at round-off and the magnetic flux
    through every lattice plane of the periodic box is unchanged."""
    from paper_2212_00370_gb300 import workloads as W
    w = W.blast_2d(48)
    P = O.Params(gamma=w.gamma, a_rad=w.a_rad, cfl=w.cfl)
    g = periodic_grid((48, 48))
    V = np.ascontiguousarray(w.V).copy()
    b = O.ct_faces_from_cells(g, V)
    O.ct_canonical(g, b)
    O.ct_cells_from_faces(g, b, np.zeros_like(V), V)
    U = O.prim2con(V, P)
    nx = ny = 48
    fx0 = b[:(nx + 1) * ny].reshape(ny, nx + 1).sum(axis=0)
    fy0 = b[(nx + 1) * ny:].reshape(ny + 1, nx).sum(axis=1)
    st = O.Stats()
    t, steps, nfail = O.run(g, 0.0, np.inf, U, V, w.kappa, w.sigma, P, max_steps=40, stats=st, bface=b)
    assert nfail == 0 and steps == 40
    assert st.fallback_cells > 0 and st.imp_matter > 0
    h = 1.0 / 48
    assert np.abs(O.ct_div(g, b)).max() * h / np.abs(b).max() < 1e-13
    fx = b[:(nx + 1) * ny].reshape(ny, nx + 1).sum(axis=0)
    fy = b[(nx + 1) * ny:].reshape(ny + 1, nx).sum(axis=1)
    scale = np.abs(b).sum()
    assert np.abs(fx - fx0).max() <= 1e-13 * scale and np.abs(fy - fy0).max() <= 1e-13 * scale


def blast_3d(n, kappa=10.0):
    """A periodic 3D blast on the unit box: rho = 1, p = 0.1 (100 inside r < 0.2),
    B = (0.5, 0, 0), E_r = (p/rho)^4 (a_R = 1), F_r = 0, uniform kappa, sigma = 0."""
    x = (np.arange(n) + 0.5) / n - 0.5
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    flat = lambda a: np.ascontiguousarray(np.asarray(a).transpose(2, 1, 0)).reshape(-1)
    V = np.zeros((12, n ** 3))
    V[0] = 1.0
    V[4] = flat(np.where(X ** 2 + Y ** 2 + Z ** 2 < 0.04, 100.0, 0.1))
    V[5] = 0.5
    V[8] = (V[4] / V[0]) ** 4
    return V, np.full(n ** 3, kappa), np.zeros(n ** 3)


def test_fallback_under_ct_keeps_the_constraint_3d():
    """The same in 3D (12^3 blast, 20 steps): the fallback fires, its first-order
    fluxes enter all three EMF components, and the 3x3x3 block around each flagged
    cell is updated again; the discrete divergence stays at round-off and the flux
    through every lattice plane is unchanged."""
    n = 12
    V, kappa, sigma = blast_3d(n)
    P = O.Params(gamma=4 / 3, a_rad=1.0, cfl=0.4)
    g = periodic_grid((n, n, n))
    b = O.ct_faces_from_cells(g, V)
    O.ct_canonical(g, b)
    O.ct_cells_from_faces(g, b, np.zeros_like(V), V)
    U = O.prim2con(V, P)
    nf = (n + 1) * n * n
    planes = lambda bb: [bb[d * nf:(d + 1) * nf].reshape([n + 1 if e == 2 - d else n for e in range(3)])
                         .sum(axis=tuple(e for e in range(3) if e != 2 - d)) for d in range(3)]
    p0 = planes(b)
    st = O.Stats()
    t, steps, nfail = O.run(g, 0.0, np.inf, U, V, kappa, sigma, P, max_steps=20, stats=st, bface=b)
    assert nfail == 0 and steps == 20 and st.fallback_cells > 0
    assert np.abs(O.ct_div(g, b)).max() / n / np.abs(b).max() < 1e-14
    scale = np.abs(b).sum()
    for a0, a1 in zip(p0, planes(b)):
        assert np.abs(a1 - a0).max() <= 1e-13 * scale

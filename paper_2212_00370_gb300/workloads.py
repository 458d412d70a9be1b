"""Seeded synthetic inputs of the benchmark configurations (primitives only).

This module holds no arithmetic of the method: it draws primitive states
V = (rho, v, p, B, E_r, F_r), opacities and grid sizes from numpy's
``default_rng(seed)``.  Both the oracle and the CUDA path consume its output.
The paper uses no public dataset; every configuration is synthetic with the
shapes and value ranges of the paper's tests (Sec. 4) and of the benchmark
configurations:

  C0  1D radiative shock tube, 400 cells, gamma 5/3, E_r = a_R T^4, kappa = 1.
  C1  4096 independent 1D Riemann problems, N ~ U{128..2048}, gamma 4/3,
      log-uniform rho, p, E_r, kappa, sigma; W ~ U[1,10]; |F_r|/E_r ~ U[0,0.99].
  C2  2D 1024^2 periodic magnetised blast with smooth velocity and log-normal kappa.
  C3  3D 256^3 periodic turbulent box.
  C4  serving mix: Poisson arrivals of 1D (70 %, N ~ U{256..4096}) and planar 2D
      (30 %, side ~ U{128..512}) Riemann problems with C1 states, t_end 0.2.
Seeds: 2212003700 + configuration index unless given.
"""
import dataclasses

import numpy as np

SEED_BASE = 2212003700


@dataclasses.dataclass
class Workload:
    name: str
    grids: list            # list of dicts: ndim, n (3), dx (3), bc (3 strings)
    V: np.ndarray          # (12, ncells) primitives, packed instance after instance
    kappa: np.ndarray      # (ncells,)
    sigma: np.ndarray      # (ncells,)
    t_end: np.ndarray      # (n_inst,)
    gamma: float
    a_rad: float = 1.0
    cfl: float = 0.4

    @property
    def ncells(self):
        return self.V.shape[1]

    @property
    def n_inst(self):
        return len(self.grids)

    def cell_offsets(self):
        sizes = [int(np.prod(g["n"])) for g in self.grids]
        return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)

    def instance(self, i):
        off = self.cell_offsets()
        s = slice(off[i], off[i + 1])
        return self.grids[i], self.V[:, s], self.kappa[s], self.sigma[s]

    def subset(self, idx):
        """A workload made of the listed instances (same states)."""
        parts = [self.instance(i) for i in idx]
        return Workload(self.name + "-subset", [p[0] for p in parts],
                        np.ascontiguousarray(np.concatenate([p[1] for p in parts], axis=1)),
                        np.concatenate([p[2] for p in parts]), np.concatenate([p[3] for p in parts]),
                        self.t_end[list(idx)], self.gamma, self.a_rad, self.cfl)


def grid1d(n, length=1.0, bc="outflow"):
    return {"ndim": 1, "n": (int(n), 1, 1), "dx": (length / n, 1.0, 1.0), "bc": (bc, "outflow", "outflow")}


def shock_tube(n=400, kappa=1.0, a_rad=1.0, uniform_radiation=False):
    """C0: rho 1 / 0.125, p 1 / 0.1, v = 0, B = 0 on [0,1] split at 0.5, gamma 5/3;
    E_r = a_R (p/rho)^4 (local equilibrium), F_r = 0; outflow; t_end 0.4."""
    x = (np.arange(n) + 0.5) / n
    left = x < 0.5
    V = np.zeros((12, n))
    V[0] = np.where(left, 1.0, 0.125)
    V[4] = np.where(left, 1.0, 0.1)
    V[8] = 1.0 if uniform_radiation else a_rad * (V[4] / V[0]) ** 4
    return Workload("C0-shock-tube-%d" % n, [grid1d(n)], V, np.full(n, float(kappa)),
                    np.zeros(n), np.array([0.4]), 5.0 / 3.0, a_rad, 0.4)


def _side_state(rng, Bx):
    rho = 10 ** rng.uniform(-2, 1)
    p = 10 ** rng.uniform(-3, 1)
    W = rng.uniform(1, 10)
    d = rng.normal(size=3)
    v = np.sqrt(1 - 1 / W ** 2) * d / np.linalg.norm(d)
    By, Bz = rng.uniform(-1, 1, 2)
    E = 10 ** rng.uniform(-3, 1)
    f = rng.uniform(0, 0.99)
    e = rng.normal(size=3)
    F = f * E * e / np.linalg.norm(e)
    kappa = 10 ** rng.uniform(-3, 3)
    sigma = 10 ** rng.uniform(-3, 2)
    return np.array([rho, *v, p, Bx, By, Bz, E, *F]), kappa, sigma


def riemann_batch(n_inst=4096, seed=SEED_BASE + 1, nmin=128, nmax=2048, t_end=0.2):
    """C1: independent 1D RRMHD Riemann problems on [0,1] split at 0.5.  Each side:
    rho log-U[1e-2,10], p log-U[1e-3,10], W ~ U[1,10] with isotropic direction,
    B_y, B_z ~ U[-1,1], E_r log-U[1e-3,10], |F_r|/E_r ~ U[0,0.99] isotropic,
    kappa log-U[1e-3,1e3], sigma log-U[1e-3,1e2]; B_x ~ U[-1,1] once per instance
    (the normal field is continuous); N ~ U{nmin..nmax}; gamma 4/3, outflow."""
    rng = np.random.default_rng(seed)
    grids, Vs, ks, ss = [], [], [], []
    for _ in range(n_inst):
        n = int(rng.integers(nmin, nmax + 1))
        Bx = rng.uniform(-1, 1)
        (VL, kL, sL), (VR, kR, sR) = _side_state(rng, Bx), _side_state(rng, Bx)
        left = (np.arange(n) + 0.5) / n < 0.5
        Vs.append(np.where(left[None, :], VL[:, None], VR[:, None]))
        ks.append(np.where(left, kL, kR))
        ss.append(np.where(left, sL, sR))
        grids.append(grid1d(n))
    return Workload("C1-riemann-batch-%d" % n_inst, grids, np.ascontiguousarray(np.concatenate(Vs, 1)),
                    np.concatenate(ks), np.concatenate(ss), np.full(n_inst, float(t_end)), 4.0 / 3.0)


def _smooth_field(rng, shape, nmodes=8, kmax=4):
    """Sum of nmodes random Fourier modes (integer wavevectors, |k| <= kmax) on the
    unit periodic box, normalised to zero mean and unit standard deviation."""
    ndim = len(shape)
    axes = [(np.arange(n) + 0.5) / n for n in shape]
    X = np.meshgrid(*axes, indexing="ij")
    f = np.zeros(shape)
    for _ in range(nmodes):
        while True:
            k = rng.integers(-kmax, kmax + 1, ndim)
            if 0 < np.linalg.norm(k) <= kmax:
                break
        ph = rng.uniform(0, 2 * np.pi)
        f += np.cos(2 * np.pi * sum(k[i] * X[i] for i in range(ndim)) + ph)
    f -= f.mean()
    return f / f.std()


def _pack(field):
    """(nx, ny[, nz]) array indexed [x, y, z] -> flat, x fastest."""
    return np.ascontiguousarray(field.T).reshape(-1)


def blast_2d(n=1024, seed=SEED_BASE + 2, a_rad=1.0):
    """C2: periodic [-0.5,0.5]^2, rho = 1, p = 0.1 (p = 100 for r < 0.1), B = (0.5,0,0),
    smooth velocity (8 Fourier modes per component, peak |v| 0.05), log10 kappa a
    smooth field of mean 0 and std 1.5, sigma = 0, gamma 4/3, E_r = a_R (p/rho)^4, F_r = 0."""
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n - 0.5
    X, Y = np.meshgrid(x, x, indexing="ij")
    p = np.where(X ** 2 + Y ** 2 < 0.01, 100.0, 0.1)
    vx, vy = _smooth_field(rng, (n, n)), _smooth_field(rng, (n, n))
    s = 0.05 / np.sqrt(vx ** 2 + vy ** 2).max()
    V = np.zeros((12, n * n))
    V[0] = 1.0
    V[1], V[2] = _pack(vx * s), _pack(vy * s)
    V[4] = _pack(p)
    V[5] = 0.5
    V[8] = a_rad * (V[4] / V[0]) ** 4
    kappa = 10 ** (1.5 * _pack(_smooth_field(rng, (n, n))))
    g = {"ndim": 2, "n": (n, n, 1), "dx": (1.0 / n, 1.0 / n, 1.0), "bc": ("periodic", "periodic", "outflow")}
    return Workload("C2-blast-2d-%d" % n, [g], V, kappa, np.zeros(n * n), np.array([np.inf]),
                    4.0 / 3.0, a_rad, 0.4)


def turbulent_3d(n=256, seed=SEED_BASE + 3):
    """C3: periodic [0,1]^3, rho = exp(0.5 g), p = 1, divergence-free B = curl A from a
    smooth random vector potential (rms |B| 0.3), Gaussian velocities (rms 0.3, capped at
    |v| 0.95), log10 kappa = 1 + g', sigma = 0.1 kappa, gamma 4/3, E_r = (p/rho)^4, F_r = 0."""
    rng = np.random.default_rng(seed)
    sh = (n, n, n)
    rho = np.exp(0.5 * _smooth_field(rng, sh))
    A = [_smooth_field(rng, sh) for _ in range(3)]
    h = 1.0 / n
    # curl by centred differences on the periodic box
    d = lambda f, ax: (np.roll(f, -1, ax) - np.roll(f, 1, ax)) / (2 * h)
    B = np.array([d(A[2], 1) - d(A[1], 2), d(A[0], 2) - d(A[2], 0), d(A[1], 0) - d(A[0], 1)])
    B *= 0.3 / np.sqrt((B ** 2).sum(0).mean())
    v = np.array([_smooth_field(rng, sh) for _ in range(3)])
    v *= 0.3 / np.sqrt((v ** 2).sum(0).mean())
    vm = np.sqrt((v ** 2).sum(0))
    v = np.where(vm > 0.95, v * 0.95 / np.maximum(vm, 1e-300), v)
    V = np.zeros((12, n ** 3))
    V[0] = _pack(rho)
    for k in range(3):
        V[1 + k] = _pack(v[k])
        V[5 + k] = _pack(B[k])
    V[4] = 1.0
    V[8] = (V[4] / V[0]) ** 4
    kappa = 10 ** (1.0 + _pack(_smooth_field(rng, sh)))
    g = {"ndim": 3, "n": (n, n, n), "dx": (h, h, h), "bc": ("periodic",) * 3}
    return Workload("C3-turbulent-3d-%d" % n, [g], V, kappa, 0.1 * kappa, np.array([np.inf]),
                    4.0 / 3.0, 1.0, 0.4)


def serving_requests(n_req, rate=200.0, seed=SEED_BASE + 4, frac_1d=0.7, n1d=(256, 4096),
                     side2d=(128, 512), t_end=0.2):
    """C4 arrival process: n_req requests with exponential inter-arrival times of
    mean 1/rate seconds; each is 1D with probability frac_1d (N ~ U{n1d}) or a
    planar 2D problem (side ~ U{side2d}).  Returns light specs (arrival time, kind,
    size, per-request seed); ``serving_request`` draws the arrays of one spec.  The
    draws are made request by request, so the first k requests of any n_req >= k are
    the same: a sample of n_req is the start of the full process."""
    rng = np.random.default_rng(seed)
    t = 0.0
    specs = []
    for k in range(n_req):
        t = t + float(rng.exponential(1.0 / rate))
        one_d = rng.uniform() < frac_1d
        size = int(rng.integers(n1d[0], n1d[1] + 1)) if one_d else int(rng.integers(side2d[0], side2d[1] + 1))
        specs.append({"arrival": t, "ndim": 1 if one_d else 2, "size": size,
                      "seed": int(rng.integers(2 ** 62)), "t_end": float(t_end)})
    return specs


def serving_request(spec):
    """Arrays of one C4 request: a Riemann problem split at x = 0.5 with the two
    states drawn as in C1 (normal field B_x shared), outflow on every side; 2D
    requests are planar (uniform in y).  Returns (grid dict, V, kappa, sigma, t_end)."""
    rng = np.random.default_rng(spec["seed"])
    n = spec["size"]
    Bx = rng.uniform(-1, 1)
    (VL, kL, sL), (VR, kR, sR) = _side_state(rng, Bx), _side_state(rng, Bx)
    left = (np.arange(n) + 0.5) / n < 0.5
    if spec["ndim"] == 2:
        left = np.tile(left, n)   # x fastest, n rows
        g = {"ndim": 2, "n": (n, n, 1), "dx": (1.0 / n, 1.0 / n, 1.0), "bc": ("outflow",) * 3}
    else:
        g = grid1d(n)
    V = np.ascontiguousarray(np.where(left[None, :], VL[:, None], VR[:, None]))
    return g, V, np.where(left, kL, kR), np.where(left, sL, sR), spec["t_end"]

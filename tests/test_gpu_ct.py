"""Constrained transport on the GPU against the oracle (CT-contact EMFs).

FP64, bit for bit: the conserved and primitive state and the staggered face
field after several steps, on periodic 2D and 3D grids from a vector-potential
field, and in a mixed batch (1D, 2D outflow, 3D periodic) that steps together.
The discrete divergence of the GPU's field stays at round-off.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import compare_bitwise, oracle_grid, oracle_params
from paper_2212_00370_gb300 import rrmhd
from paper_2212_00370_gb300 import workloads as W
from test_oracle_ct import curl_faces, periodic_grid, smooth_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_00370_gb300 import build
    build.build()


def instance(shape, seed, bc="periodic"):
    """(grid dict, V with B from the faces, face field, kappa, sigma)."""
    nd = len(shape)
    V, kappa, sigma = smooth_state(shape, seed)
    g = {"ndim": nd, "n": tuple(shape) + (1,) * (3 - nd),
         "dx": tuple(1.0 / n for n in shape) + (1.0,) * (3 - nd),
         "bc": (bc,) * nd + ("outflow",) * (3 - nd)}
    og = oracle_grid(g)
    if nd >= 2:
        if bc != "periodic":   # an in-plane field from the cells (not divergence-free)
            V[5], V[6] = 0.3 + 0.1 * V[0], 0.1 * V[4]
        b = curl_faces(shape) if bc == "periodic" else O.ct_faces_from_cells(og, V)
        O.ct_canonical(og, b)
        O.ct_cells_from_faces(og, b, np.zeros_like(V), V)
    else:
        b = np.zeros(0)
    return g, V, b, kappa, sigma


def face_counts(g):
    nd = g["ndim"]
    out = []
    for d in range(3):
        if d >= nd:
            out.append(0)
            continue
        m = list(g["n"])
        m[d] += 1
        out.append(int(np.prod(m)))
    return out


def batch_face_field(insts):
    """Per-instance face fields (directions one after the other) -> batch layout
    (direction-major, instances in order within each direction)."""
    blocks = [[] for _ in range(3)]
    for g, V, b, k, s in insts:
        c = face_counts(g)
        off = 0
        for d in range(3):
            if g["ndim"] >= 2:
                blocks[d].append(b[off:off + c[d]])
                off += c[d]
            else:
                blocks[d].append(np.zeros(c[d]))
    return np.concatenate([np.concatenate(x) if x else np.zeros(0) for x in blocks])


def split_face_field(insts, bb):
    counts = [face_counts(g) for g, *_ in insts]
    starts = [0, 0, 0]
    pos = 0
    for d in range(3):
        starts[d] = pos
        pos += sum(c[d] for c in counts)
    out, cur = [], list(starts)
    for (g, *_), c in zip(insts, counts):
        parts = []
        for d in range(3):
            if g["ndim"] >= 2 and d < g["ndim"]:
                parts.append(bb[cur[d]:cur[d] + c[d]])
            cur[d] += c[d]
        out.append(np.concatenate(parts) if parts else np.zeros(0))
    return out


def run_gpu(insts, steps, **opts):
    w = W.Workload("ct", [x[0] for x in insts], np.ascontiguousarray(np.concatenate([x[1] for x in insts], 1)),
                   np.concatenate([x[3] for x in insts]), np.concatenate([x[4] for x in insts]),
                   np.full(len(insts), np.inf), 4 / 3)
    grids = [rrmhd.make_grid(g["ndim"], g["n"], g["dx"], g["bc"]) for g in w.grids]
    ctx = rrmhd.Context(grids, gamma=w.gamma, a_rad=w.a_rad, cfl=w.cfl, ct=1, lanes=2, **opts)
    ctx.set_opacity(torch.tensor(w.kappa, device="cuda"), torch.tensor(w.sigma, device="cuda"))
    ctx.set_state(torch.tensor(w.V, device="cuda"))
    ctx.set_face_field(torch.tensor(batch_face_field(insts), device="cuda"))
    ctx.set_times(np.zeros(w.n_inst), w.t_end)
    ctx.imex_step(steps)
    U, V = ctx.get_state()
    b = ctx.get_face_field().cpu().numpy()
    st = ctx.inst_status()
    ctx.close()
    return w, U.cpu().numpy(), V.cpu().numpy(), split_face_field(insts, b), st


def run_oracle(g, V, b, kappa, sigma, steps, **pk):
    P = O.Params(gamma=4 / 3, a_rad=1.0, cfl=0.4, **pk)
    V = np.ascontiguousarray(V).copy()
    U = O.prim2con(V, P)
    bb = b.copy() if g["ndim"] >= 2 else None
    t, ns, nf = O.run(oracle_grid(g), 0.0, np.inf, U, V, kappa, sigma, P, max_steps=steps, bface=bb)
    return U, V, bb, nf


def check(insts, steps, **pk):
    w, U, V, bl, st = run_gpu(insts, steps, **pk)
    off = w.cell_offsets()
    for i, (g, V0, b0, k, s) in enumerate(insts):
        Ur, Vr, br, nf = run_oracle(g, V0, b0, k, s, steps, **pk)
        assert nf == 0 and st[i] == 0
        sl = slice(off[i], off[i + 1])
        compare_bitwise(U[:, sl], Ur, f"instance {i} U")
        compare_bitwise(V[:, sl], Vr, f"instance {i} V")
        if g["ndim"] >= 2:
            compare_bitwise(bl[i], br, f"instance {i} face field")
            # CT keeps the discrete divergence of every cell (zero for a curl start)
            og = oracle_grid(g)
            h = min(g["dx"][:g["ndim"]])
            ddiv = np.abs(O.ct_div(og, bl[i]) - O.ct_div(og, b0)).max() * h / np.abs(b0).max()
            assert ddiv < 1e-12, ddiv


@pytest.mark.parametrize("shape,steps", [((24, 20), 4), ((8, 7, 6), 2)])
def test_ct_periodic_bitwise(shape, steps):
    check([instance(shape, 3)], steps)


def test_ct_mixed_batch_bitwise():
    insts = [instance((40,), 1), instance((14, 12), 2, bc="outflow"), instance((6, 5, 7), 4),
             instance((10, 9), 5)]
    check(insts, 3)


def test_ct_radhll_bitwise():
    check([instance((16, 18), 6)], 3, solver="radhll")


def test_ct_fp32_bulk_tracks_the_oracle():
    """FP32-bulk with CT: FP32 face fluxes, FP64 EMFs and face field.  Per-variable
    relative L1 against the FP64 oracle <= 1e-5; the divergence is kept."""
    insts = [instance((24, 20), 3), instance((8, 7, 6), 4)]
    w, U, V, bl, st = run_gpu(insts, 3, precision="fp32_bulk")
    off = w.cell_offsets()
    for i, (g, V0, b0, k, s) in enumerate(insts):
        Ur, Vr, br, nf = run_oracle(g, V0, b0, k, s, 3)
        assert nf == 0 and st[i] == 0
        Ui = U[:, off[i]:off[i + 1]]
        for q in range(12):
            den = np.abs(Ur[q]).sum()
            if den > 0:
                assert np.abs(Ui[q] - Ur[q]).sum() / den < 1e-5, (i, q)
        assert np.abs(bl[i] - br).sum() / np.abs(br).sum() < 1e-5
        og = oracle_grid(g)
        h = min(g["dx"][:g["ndim"]])
        assert np.abs(O.ct_div(og, bl[i])).max() * h / np.abs(bl[i]).max() < 1e-12


def test_ct_option_checks():
    g = rrmhd.make_grid(2, (4, 4), (0.25, 0.25))
    ctx = rrmhd.Context([g])
    with pytest.raises(rrmhd.RRMHDError) as e:
        ctx.set_face_field(torch.zeros(ctx.num_face_field(), dtype=torch.float64, device="cuda"))
    assert e.value.code == 10

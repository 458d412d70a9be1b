"""The seeded generators give admissible states of the stated shapes."""
import numpy as np

from paper_2212_00370_gb300 import workloads as W


def _admissible(V):
    v2 = (V[1:4] ** 2).sum(0)
    F = np.sqrt((V[9:12] ** 2).sum(0))
    assert np.all(V[0] > 0) and np.all(V[4] > 0) and np.all(V[8] > 0)
    assert np.all(v2 < 1) and np.all(F <= V[8])


def test_c0():
    w = W.shock_tube()
    assert w.ncells == 400 and w.gamma == 5 / 3
    _admissible(w.V)
    assert w.V[8, 0] == 1.0 and w.V[8, -1] == (0.1 / 0.125) ** 4


def test_c1_small_is_deterministic_and_admissible():
    a = W.riemann_batch(64, seed=5)
    b = W.riemann_batch(64, seed=5)
    np.testing.assert_array_equal(a.V, b.V)
    _admissible(a.V)
    n = [g["n"][0] for g in a.grids]
    assert min(n) >= 128 and max(n) <= 2048
    assert a.ncells == sum(n)
    W_ = 1 / np.sqrt(1 - (a.V[1:4] ** 2).sum(0))
    assert W_.max() <= 10 + 1e-9
    # continuous normal field within each instance
    off = a.cell_offsets()
    for i in range(a.n_inst):
        bx = a.V[5, off[i]:off[i + 1]]
        assert np.all(bx == bx[0])


def test_c2_c3_small():
    c2 = W.blast_2d(32)
    _admissible(c2.V)
    assert np.abs(c2.V[1:3]).max() <= 0.05 + 1e-12
    c3 = W.turbulent_3d(16)
    _admissible(c3.V)
    assert c3.ncells == 16 ** 3

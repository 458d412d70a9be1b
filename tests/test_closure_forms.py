"""Algebraic forms of the M1 closure (Sec. 2.2, Eq. xi) used by the kernels.

The FP32 kernels write the Eddington tensor as P = a E delta + c F F^T with
c = 3 / (E (2 + s)), s = sqrt(4 - 3 f^2), f = |F|/E.  This is exact: with
3 xi - 1 = 6 f^2 / (2 + s) the literal form E (3 xi - 1) n n^T / 2 becomes c F F^T.
The rewritten form avoids the cancellation of 3 xi - 1 near f = 0.  Checked
symbolically here, and numerically against the oracle's closure.
"""
import numpy as np
import pytest

import oracle as O

sympy = pytest.importorskip("sympy")


def test_three_xi_minus_one_identity():
    f = sympy.symbols("f", nonnegative=True)
    s = sympy.sqrt(4 - 3 * f ** 2)
    xi = (3 + 4 * f ** 2) / (5 + 2 * s)
    assert sympy.simplify(3 * xi - 1 - 6 * f ** 2 / (2 + s)) == 0


def test_rewritten_tensor_matches_the_oracle_closure():
    rng = np.random.default_rng(3)
    for _ in range(200):
        E = 10 ** rng.uniform(-4, 8)
        f = rng.choice([rng.uniform(0, 1), 10 ** rng.uniform(-9, -1)])
        n = rng.normal(size=3)
        F = f * E * n / np.linalg.norm(n)
        s = np.sqrt(4 - 3 * f * f)
        xi = (3 + 4 * f * f) / (5 + 2 * s)
        P = 0.5 * (1 - xi) * E * np.eye(3) + 3.0 / (E * (2 + s)) * np.outer(F, F)
        Po = O.m1_pressure(E, F)
        assert np.allclose(P, Po, rtol=1e-12, atol=1e-12 * E), (E, f)

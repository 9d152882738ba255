"""Pins of the matrix-free kernel sketch oracle and its gradient (CPU only).

Each check is independent of the oracle's own formulas: a two-point case
worked by hand, central finite differences of the loss, and two invariances
of a kernel that depends on x_i - x_j and on r / h only.
"""
import math

import numpy as np
import pytest

from oracle import kernel_grad as kg
from oracle import operators as ops


def test_two_points_by_hand():
    a, h = 0.3, 0.25
    X = np.array([[0.0, 0.0, 0.0], [a, 0.0, 0.0]])
    rng = np.random.default_rng(5)
    R = rng.standard_normal((2, 3))
    dS = rng.standard_normal((2, 3))
    e = math.exp(-a * a / (2 * h * h))
    # S = K R with K = [[1, e], [e, 1]]
    S = kg.kernel_sketch(X, h, R)
    np.testing.assert_allclose(S, np.array([[1.0, e], [e, 1.0]]) @ R, rtol=1e-15, atol=1e-15)
    G = dS @ R.T
    g = G[0, 1] + G[1, 0]
    dX, dh = kg.kernel_sketch_grad(X, h, R, dS)
    want = np.zeros((2, 3))
    want[1, 0] = g * e * (-a / h ** 2)
    want[0, 0] = -want[1, 0]
    np.testing.assert_allclose(dX, want, rtol=1e-13, atol=1e-15)
    assert dh == pytest.approx(g * e * a * a / h ** 3, rel=1e-13)


def test_gram_elementwise():
    rng = np.random.default_rng(1)
    X = rng.random((7, 3))
    h = 0.4
    K, r2 = kg.gram(X, h)
    for i in range(7):
        for j in range(7):
            d2 = sum((X[i, k] - X[j, k]) ** 2 for k in range(3))
            assert r2[i, j] == pytest.approx(d2, rel=1e-14, abs=1e-16)
            assert K[i, j] == pytest.approx(math.exp(-d2 / (2 * h * h)), rel=1e-14)


@pytest.mark.parametrize("h", [0.05, 0.2])
def test_gradient_matches_finite_differences(h):
    rng = np.random.default_rng(11)
    n, d = 40, 16
    X = rng.random((n, 3)) * (6 * h)  # spread over a few widths: no vanishing kernel
    op = ops.Operator("sjlt_block", n, d, 4, 99)
    R = op.dense()
    dS = rng.standard_normal((n, d))
    dX, dh = kg.kernel_sketch_grad(X, h, R, dS)
    coords = [(i, a) for i in (0, 7, 23, 39) for a in range(3)]
    fd, fd_h = kg.fd_grad(X, h, R, dS, coords, step=1e-6 * h)
    got = np.array([dX[i, a] for i, a in coords])
    scale = np.abs(dX).max()
    np.testing.assert_allclose(got, fd, rtol=0, atol=1e-6 * scale)
    assert dh == pytest.approx(fd_h, rel=1e-6)


def test_translation_and_scale_invariance():
    rng = np.random.default_rng(3)
    n, d, h = 30, 8, 0.3
    X = rng.random((n, 3))
    R = ops.Operator("sjlt_graph", n, d, 2, 7).dense()
    dS = rng.standard_normal((n, d))
    dX, dh = kg.kernel_sketch_grad(X, h, R, dS)
    # K depends on x_i - x_j only: shifting every point changes nothing
    np.testing.assert_allclose(dX.sum(axis=0), 0.0, atol=1e-12 * np.abs(dX).max() * n)
    # K depends on X / h only: sum_i x_i . dX_i + h dh = 0 (Euler)
    assert float((X * dX).sum()) + h * dh == pytest.approx(0.0, abs=1e-11 * (abs(h * dh) + 1))
    # and the gradient itself is unchanged by a translation of all points
    dX2, dh2 = kg.kernel_sketch_grad(X + np.array([0.5, -1.0, 2.0]), h, R, dS)
    np.testing.assert_allclose(dX2, dX, rtol=1e-9, atol=1e-12)
    assert dh2 == pytest.approx(dh, rel=1e-9)


def test_sketch_of_identity_is_the_kernel():
    rng = np.random.default_rng(2)
    X = rng.random((9, 3))
    K, _ = kg.gram(X, 0.3)
    np.testing.assert_array_equal(kg.kernel_sketch(X, 0.3, np.eye(9)), K)

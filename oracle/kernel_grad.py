"""Matrix-free kernel sketch and its gradient (oracle; test infrastructure only).

The sketch of a Gaussian kernel matrix that is never formed, S = K(X, X; h) R
with K_ij = exp(-||x_i - x_j||^2 / (2 h^2)), is the random sample of the
matrix-free setting (Sec. 1.1: only products with the matrix are available)
for the kernel matrices of the experiments (Sec. 8.1 uses kernel matrices of
points).  Its gradient with respect to the points X and the width h is this
project's extension (the paper does not differentiate the sketch); it is the
plain chain rule of the definition:

    L(X, h) = <dS, K R> = sum_ij G_ij K_ij,   G = dS R^T,
    dK_ij/dx_i = K_ij (x_j - x_i) / h^2,   dK_ij/dh = K_ij ||x_i - x_j||^2 / h^3,
    dX_i = (1/h^2) sum_j (G_ij + G_ji) K_ij (x_j - x_i),
    dh   = (1/h^3) sum_ij G_ij K_ij ||x_i - x_j||^2.

Everything is FP64 and dense (n x n); numpy's matmul is the only library
primitive.  Pinned by tests/test_oracle_kernel_grad.py: a two-point case
worked by hand, central finite differences of ``loss``, translation
invariance (sum_i dX_i = 0) and scale invariance (h dh = -sum_i x_i . dX_i).
"""
from __future__ import annotations

import numpy as np


def gram(X: np.ndarray, h: float) -> tuple[np.ndarray, np.ndarray]:
    """K(X, X; h) and the squared distances r2_ij (FP64)."""
    X = np.asarray(X, dtype=np.float64)
    diff = X[:, None, :] - X[None, :, :]
    r2 = (diff * diff).sum(axis=2)
    return np.exp(-r2 / (2.0 * h * h)), r2


def kernel_sketch(X: np.ndarray, h: float, R: np.ndarray) -> np.ndarray:
    """S = K(X, X; h) R."""
    K, _ = gram(X, h)
    return K @ np.asarray(R, dtype=np.float64)


def loss(X: np.ndarray, h: float, R: np.ndarray, dS: np.ndarray) -> float:
    """L = <dS, K R>: the scalar whose gradient is the adjoint of the sketch for upstream dS."""
    return float((np.asarray(dS, dtype=np.float64) * kernel_sketch(X, h, R)).sum())


def kernel_sketch_grad(X: np.ndarray, h: float, R: np.ndarray,
                       dS: np.ndarray) -> tuple[np.ndarray, float]:
    """(dL/dX, dL/dh) for L = <dS, K(X, X; h) R>, by the formulas in the module docstring."""
    X = np.asarray(X, dtype=np.float64)
    K, r2 = gram(X, h)
    G = np.asarray(dS, dtype=np.float64) @ np.asarray(R, dtype=np.float64).T
    W = (G + G.T) * K
    # sum_j W_ij (x_j - x_i) = (W X)_i - (sum_j W_ij) x_i
    dX = (W @ X - W.sum(axis=1)[:, None] * X) / (h * h)
    dh = float((G * K * r2).sum() / (h ** 3))
    return dX, dh


def fd_grad(X: np.ndarray, h: float, R: np.ndarray, dS: np.ndarray, coords, step: float = 1e-3):
    """Central finite differences of ``loss``: d/dX[i, a] for (i, a) in ``coords`` and d/dh."""
    X = np.array(X, dtype=np.float64, copy=True)
    out = []
    for i, a in coords:
        x0 = X[i, a]
        X[i, a] = x0 + step
        lp = loss(X, h, R, dS)
        X[i, a] = x0 - step
        lm = loss(X, h, R, dS)
        X[i, a] = x0
        out.append((lp - lm) / (2.0 * step))
    dh = (loss(X, h + step, R, dS) - loss(X, h - step, R, dS)) / (2.0 * step)
    return np.array(out), dh

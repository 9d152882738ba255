"""Sketch products, the kernel-matrix generator and a textbook FWHT (oracle; test infrastructure only).

* ``apply(A, R)``: S = A R and S' = A^T R in FP64 (Sec. 6.3: the sketch of the
  rows and of the columns of A; with real A the conjugate transpose is the
  transpose).  The product is the plain definition; numpy's matmul is the
  library primitive that evaluates it.  ``apply_t(A, R)``: S' alone, for
  rectangular A.  ``complex_s``, ``complex_t``, ``apply_complex``: S = A R
  and S' = A* R (conjugate transpose) for complex A (Sec. 2: A in C^{m x n}).
* ``apply_sjlt_outer(A, cols, signs, scale, d)``: the outer-product form of
  Sec. 6.3 written out: every column A_{:i} is added to or subtracted from the
  solution columns named by row i of R, then the result is scaled once.
* ``apply_sjlt_inner(A, ccs, scale, d)``: the inner-product form of Sec. 6.3
  for A^T R through the compressed column storage of B+ and B-.
* ``kernel_matrix(X, Y, h, shift)``: A_ij = exp(-||x_i - y_j||^2 / (2 h^2)) +
  shift * delta_ij in FP64 (a Gaussian kernel; the paper's covariance problem
  uses an exponential kernel, Sec. 8.1, the workloads here use the Gaussian one).
* ``hadamard(nu)``: unnormalised Sylvester matrix, H_1 = [1],
  H_2m = [[H_m, H_m], [H_m, -H_m]] (Sec. 2.4.2).
* ``fwht(x)``: unnormalised fast Walsh-Hadamard transform along the last axis,
  log2(nu) butterfly stages (the O(n log n) transform of Sec. 7.1).
* ``srht_by_fwht(A, D, mu, d_total)``: S = A D H P sqrt(nu/d) computed through
  the transform of the zero-padded rows (Sec. 7.1, A padded to nu columns).
* ``srht_by_split(A, D, mu, d_total)``: the same product for n not a power of
  two through the two smaller transforms of Sec. 7.1 (Eqs. had1 and hadiden):
  with k = 2^floor(log2 n), n = k + r, p = 2^ceil(log2 r) and q = k / p,
  A H_{2k} = [A_k H_k + T, A_k H_k - T] where T = (A^ H_p)[I ... I] repeats
  the p-point transform of the last r columns (zero-padded to p) q times.
"""
from __future__ import annotations

import math

import numpy as np


def apply(A: np.ndarray, R: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    A = np.asarray(A, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    return A @ R, A.T @ R


def apply_t(A: np.ndarray, R: np.ndarray) -> np.ndarray:
    """S' = A^T R alone (Sec. 6.3, the sketch of the columns), for A of any shape with rows(A) = rows(R)."""
    return np.asarray(A, dtype=np.float64).T @ np.asarray(R, dtype=np.float64)


def complex_s(A: np.ndarray, R: np.ndarray) -> np.ndarray:
    """S = A R for complex A (m x n) and real R (n x d), in complex128."""
    return np.asarray(A, dtype=np.complex128) @ np.asarray(R, dtype=np.float64)


def complex_t(A: np.ndarray, R: np.ndarray) -> np.ndarray:
    """S' = A* R (conjugate transpose, Sec. 6.3 "A* R") for complex A (m x n) and real R (m x d)."""
    return np.asarray(A, dtype=np.complex128).conj().T @ np.asarray(R, dtype=np.float64)


def apply_complex(A: np.ndarray, R: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(A R, A* R) for a square complex A and real R."""
    return complex_s(A, R), complex_t(A, R)


def apply_sjlt_outer(A: np.ndarray, cols: np.ndarray, signs: np.ndarray,
                     scale: float, d: int) -> np.ndarray:
    """S = A R by the column-by-column outer-product sum of Sec. 6.3."""
    A = np.asarray(A, dtype=np.float64)
    S = np.zeros((A.shape[0], d), dtype=np.float64)
    for i in range(A.shape[1]):
        for c, s in zip(cols[i], signs[i]):
            if s > 0:
                S[:, c] += A[:, i]
            else:
                S[:, c] -= A[:, i]
    return S * scale


def apply_sjlt_inner(A: np.ndarray, ccs: dict, scale: float, d: int) -> np.ndarray:
    """S' = A^T R by inner products of the columns of A with the CCS lists."""
    A = np.asarray(A, dtype=np.float64)
    St = np.zeros((A.shape[1], d), dtype=np.float64)
    plus, minus = ccs["plus"], ccs["minus"]
    for j in range(A.shape[1]):
        col = A[:, j]
        for c in range(d):
            rp = plus["row_idx"][plus["col_ptr"][c]:plus["col_ptr"][c + 1]]
            rm = minus["row_idx"][minus["col_ptr"][c]:minus["col_ptr"][c + 1]]
            St[j, c] = col[rp].sum() - col[rm].sum()
    return St * scale


def kernel_matrix(X: np.ndarray, Y: np.ndarray, h: float, shift: float = 0.0) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    d2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(axis=2)
    A = np.exp(-d2 / (2.0 * h * h))
    if shift:
        m = min(A.shape)
        A[np.arange(m), np.arange(m)] += shift
    return A


def kernel_rows(X: np.ndarray, Y: np.ndarray, rows: np.ndarray, h: float,
                shift: float = 0.0) -> np.ndarray:
    """Rows ``rows`` of ``kernel_matrix(X, Y, h, shift)`` without forming it."""
    X = np.asarray(X, dtype=np.float64)[rows]
    out = kernel_matrix(X, Y, h, 0.0)
    if shift:
        for k, r in enumerate(np.asarray(rows)):
            if r < Y.shape[0]:
                out[k, r] += shift
    return out


def hadamard(nu: int) -> np.ndarray:
    H = np.ones((1, 1), dtype=np.float64)
    while H.shape[0] < nu:
        H = np.block([[H, H], [H, -H]])
    return H


def fwht(x: np.ndarray) -> np.ndarray:
    """Unnormalised Walsh-Hadamard transform of the last axis (length a power of 2)."""
    y = np.array(x, dtype=np.float64, copy=True)
    nu = y.shape[-1]
    if nu & (nu - 1):
        raise ValueError("length must be a power of two")
    lead = y.shape[:-1]
    h = 1
    while h < nu:
        y = y.reshape(lead + (nu // (2 * h), 2, h))
        a = y[..., 0, :].copy()
        b = y[..., 1, :].copy()
        y[..., 0, :] = a + b
        y[..., 1, :] = a - b
        y = y.reshape(lead + (nu,))
        h *= 2
    return y


def srht_by_fwht(A: np.ndarray, D: np.ndarray, mu: np.ndarray, d_total: int) -> np.ndarray:
    """S = A D H P (scale 1/sqrt(d)) via the transform of zero-padded rows."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    nu = 1 << max(0, (n - 1).bit_length())
    X = np.zeros((m, nu), dtype=np.float64)
    X[:, :n] = A * np.asarray(D, dtype=np.float64)[None, :]
    Y = fwht(X)
    return Y[:, np.asarray(mu)] / math.sqrt(d_total)


def srht_by_split(A: np.ndarray, D: np.ndarray, mu: np.ndarray, d_total: int) -> np.ndarray:
    """S = A D H P (scale 1/sqrt(d)) for n = k + r, 0 < r < k, by Sec. 7.1's split:
    transforms of orders k and p instead of one of order nu = 2k."""
    A = np.asarray(A, dtype=np.float64) * np.asarray(D, dtype=np.float64)[None, :]
    m, n = A.shape
    k = 1 << (n.bit_length() - 1)  # 2^floor(log2 n)
    r = n - k
    if r == 0:
        raise ValueError("n is a power of two: no split")
    p = 1 << (r - 1).bit_length()  # 2^ceil(log2 r)
    q = k // p
    AkHk = A[:, :k] @ hadamard(k)                       # A_{m,k} H_k
    Ahat = np.zeros((m, p), dtype=np.float64)           # A^ = [A_{m,r}  0_{m,p-r}]
    Ahat[:, :r] = A[:, k:]
    T = (Ahat @ hadamard(p)) @ np.hstack([np.eye(p)] * q)  # A^ H_p [I ... I], m x k
    AH = np.hstack([AkHk + T, AkHk - T])                 # A H_{2k}, Eq. had1
    return AH[:, np.asarray(mu)] / math.sqrt(d_total)

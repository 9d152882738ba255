"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds no sketching arithmetic: it only draws points, orders them and
draws dense test matrices.  Everything here is host-side numpy.

Workloads (shapes follow the paper's test problems, Sec. 8.1, and the kernel
matrices used to exercise the sketch):

* points uniform in [0,1]^3, drawn from numpy's Philox bit generator with a
  fixed seed (seed = 20230203 + workload index unless a test picks its own);
* an optional recursive median bisection ordering of the points (the paper
  orders its covariance test problem by recursive bisection, Sec. 8.1): split
  on the coordinate of largest extent (lowest axis index on ties), stable sort by
  (coordinate, original index), left child gets floor(m/2) points, stop at a
  leaf of <= ``leaf`` points;
* dense Gaussian N(0,1) test matrices for parity cases that isolate the sketch
  from the kernel-matrix generator.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20230203


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def points(count: int, seed: int, dtype=np.float32) -> np.ndarray:
    """``count`` x 3 points uniform in [0,1]^3, C-contiguous, of ``dtype``."""
    p = _rng(seed).random((count, 3))
    return np.ascontiguousarray(p.astype(dtype))


def bisection_order(p: np.ndarray, leaf: int = 64) -> np.ndarray:
    """Permutation that orders ``p`` by recursive median bisection.

    Returns an int64 index array ``perm`` so that ``p[perm]`` is the ordered
    point set.  Iterative (explicit stack) so deep trees do not recurse.
    """
    m = p.shape[0]
    perm = np.arange(m, dtype=np.int64)
    out = np.empty(m, dtype=np.int64)
    stack = [(0, m, perm)]
    while stack:
        lo, hi, idx = stack.pop()
        cnt = hi - lo
        if cnt <= leaf:
            out[lo:hi] = idx
            continue
        sub = p[idx].astype(np.float64)
        ext = sub.max(axis=0) - sub.min(axis=0)
        axis = int(np.argmax(ext))  # argmax returns the lowest index on ties
        # stable sort by (coordinate, original index)
        order = np.lexsort((idx, sub[:, axis]))
        idx = idx[order]
        half = cnt // 2
        # push right first so the left child is finished first (order irrelevant
        # for the result, which is written by position)
        stack.append((lo + half, hi, idx[half:]))
        stack.append((lo, lo + half, idx[:half]))
    return out


def dense_matrix(rows: int, cols: int, seed: int, dtype=np.float64) -> np.ndarray:
    """rows x cols matrix with i.i.d. N(0,1) entries, C-contiguous."""
    return np.ascontiguousarray(_rng(seed).standard_normal((rows, cols)).astype(dtype))


def low_rank_matrix(n: int, rank: int, seed: int, dtype=np.float64) -> np.ndarray:
    """n x n matrix U V^T of exact rank ``rank`` (U, V with N(0,1) entries)."""
    g = _rng(seed)
    u = g.standard_normal((n, rank))
    v = g.standard_normal((n, rank))
    return np.ascontiguousarray((u @ v.T).astype(dtype))


def spectrum_matrix(n: int, sigma: np.ndarray, seed: int, dtype=np.float64) -> np.ndarray:
    """n x n matrix with prescribed singular values ``sigma`` (length n).

    Built as U diag(sigma) V^T from the Q factors of two Gaussian matrices.
    """
    g = _rng(seed)
    u, _ = np.linalg.qr(g.standard_normal((n, n)))
    v, _ = np.linalg.qr(g.standard_normal((n, n)))
    return np.ascontiguousarray(((u * sigma) @ v.T).astype(dtype))


def hss_test_matrix(n: int, leaf: int, rank: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Symmetric n x n matrix blockdiag(D_1, ..., D_b) + U C U^T with dense
    symmetric diagonal blocks of ``leaf`` rows (the last one ragged), U n x rank
    and C rank x rank symmetric, all N(0,1): every off-diagonal block of any
    contiguous row range has rank <= ``rank``."""
    g = _rng(seed)
    A = np.zeros((n, n))
    for lo in range(0, n, leaf):
        hi = min(n, lo + leaf)
        b = g.standard_normal((hi - lo, hi - lo))
        A[lo:hi, lo:hi] = b + b.T
    u = g.standard_normal((n, rank))
    c = g.standard_normal((rank, rank))
    A += u @ (c + c.T) @ u.T / n
    return np.ascontiguousarray(A.astype(dtype))


# --- workload descriptors -------------------------------------------------
# The five workloads, by what they are.  Sizes are the full ones; tests shrink
# them where the oracle has to finish in seconds.
WORKLOADS = {
    "sjlt_fp64_n2048": dict(n=2048, d=128, alpha=4, h=0.2, shift=1e-2, dtype="f64",
                            symmetric=True, ordered=True, leaf=64, seed=BASE_SEED + 0),
    "kernel_fp32_n32768": dict(n=32768, d=256, alpha=4, h=0.1, shift=0.0, dtype="f32",
                               symmetric=False, ordered=False, seed=BASE_SEED + 1,
                               d0=128, dd=64, d_max=512),
    "precision_fp32_n65536": dict(n=65536, d=512, h=0.05, shift=0.0, dtype="f32",
                                  symmetric=True, ordered=False, seed=BASE_SEED + 2),
}

"""Global adaptive sketching loop (oracle; test infrastructure only).

Follows Algorithm 1 (HSSCompressAdaptive) restricted to the global sketch of A,
which is this project's reading of the stopping test's scope (the paper applies
it per HSS node, with eps / level(tau)):

1. R <- JL-Operator(d0 + Delta-d, n); S <- A R (and S' <- A^T R).
2. Q <- orthonormal basis of the range of S(:, 1:d).  Sec. 3 defines S^ as
   the projection of the new columns onto the orthogonal complement of the
   current sketch; when S(:, 1:d) is rank deficient (an SJLT column without
   entries, an exactly low-rank A) a d-column QR factor would also span
   directions outside that range, so the basis is the left singular vectors
   of S(:, 1:d) above the numerical rank threshold sigma_1 max(m, d) eps
   (numpy's matrix_rank default; an SVD is the library step).
3. S~ <- S(:, d+1 : d+Delta-d)             (the last Delta-d columns).
4. S^ <- (I - Q Q^T)^2 S~                  (two steps of block Gram-Schmidt,
   the remark after Eq. (3.1)).
5. stop when ||S^||_F < eps_abs or ||S^||_F < eps_rel ||S~||_F
   (Eq. (3.1); no 1/sqrt(d) factor, the remark before it).
6. otherwise R <- [R  R_bar], d <- d + Delta-d, S <- A R, and repeat, while the
   grown R keeps at most d_max columns.

S is recomputed from the grown R at every step (the plain definition), so the
CUDA path's incremental update (rescale old columns, sketch only the new ones)
is checked against it.
When both S and S' are tested, the loop stops when both tests pass.
"""
from __future__ import annotations

import numpy as np

from .operators import Operator
from .sketch import apply


def project_twice(Q: np.ndarray, B: np.ndarray) -> np.ndarray:
    """(I - Q Q^T)^2 B, two block Gram-Schmidt passes."""
    B = B - Q @ (Q.T @ B)
    return B - Q @ (Q.T @ B)


def range_basis(M: np.ndarray) -> np.ndarray:
    """Orthonormal basis of the range of M: its left singular vectors whose
    singular values exceed sigma_1 max(M.shape) eps (FP64)."""
    if M.shape[0] == 0 or M.shape[1] == 0:  # an empty matrix has an empty range
        return np.zeros((M.shape[0], 0))
    U, sv, _ = np.linalg.svd(M, full_matrices=False)
    if sv[0] == 0.0:
        return U[:, :0]
    r = int(np.count_nonzero(sv > sv[0] * max(M.shape) * np.finfo(np.float64).eps))
    return U[:, :r]


def norm_test(S: np.ndarray, d: int, dd: int, eps_rel: float, eps_abs: float):
    """One stopping test on the columns of S: returns (stop, ||S^||_F, ||S~||_F)."""
    Q = range_basis(np.asarray(S[:, :d], dtype=np.float64))
    St = S[:, d:d + dd]
    Sh = project_twice(Q, St)
    nh = float(np.linalg.norm(Sh))
    nt = float(np.linalg.norm(St))
    stop = (nh < eps_abs) or (nh < eps_rel * nt)
    return stop, nh, nt


def norm_tests(S: np.ndarray, d0: int, dd: int, d_end: int):
    """Every test of norm_test on one sketch: for b0 = d0, d0 + dd, ...,
    d_end - dd, (||S^||_F, ||S~||_F) of S~ = S[:, b0 : b0 + dd] against the
    range of S[:, :b0].  The same definitions as norm_test, with the range
    basis grown block by block: range(S[:, :b0 + dd]) is range(S[:, :b0])
    plus the range of the projected block S^, whose directions are kept above
    ||S[:, :d_end]||_F max(m, b) eps (the Frobenius norm bounds the sigma_1 of
    norm_test's threshold from above; the two differ only for directions at
    the FP64 rounding level of S)."""
    S = np.asarray(S, dtype=np.float64)
    m = S.shape[0]
    eps = np.finfo(np.float64).eps
    s1 = float(np.linalg.norm(S[:, :d_end]))
    Q = range_basis(S[:, :d0])
    out = []
    for b0 in range(d0, d_end - dd + 1, dd):
        W = S[:, b0:b0 + dd]
        Sh = project_twice(Q, W) if Q.shape[1] else W.copy()
        out.append((float(np.linalg.norm(Sh)), float(np.linalg.norm(W))))
        U, sv, _ = np.linalg.svd(Sh, full_matrices=False)
        keep = sv > s1 * max(m, b0 + dd) * eps
        Q = np.hstack([Q, U[:, keep]])
    return out


def adaptive(A: np.ndarray, kind: str, d0: int, dd: int, alpha: int, seed: int,
             d_max: int, eps_rel: float, eps_abs: float, which: str = "both"):
    """Run the loop; returns a dict with the operator, final S, S', the
    per-test history [(d, stop, nh_S, nt_S, nh_St, nt_St)], and 'converged'."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("square A expected")
    if d0 + dd > d_max:
        raise ValueError("d0 + Delta-d exceeds d_max")
    op = Operator(kind, n, d0 + dd, alpha, seed)
    d = d0
    history = []
    while True:
        S, St = apply(A, op.dense())
        stop_s, nh_s, nt_s = norm_test(S, d, dd, eps_rel, eps_abs)
        if which == "S":
            stop_t, nh_t, nt_t = True, 0.0, 0.0
        else:
            stop_t, nh_t, nt_t = norm_test(St, d, dd, eps_rel, eps_abs)
        stop = stop_s and stop_t
        history.append((d, stop, nh_s, nt_s, nh_t, nt_t))
        if stop:
            return dict(op=op, S=S, St=St, history=history, converged=True)
        if op.d_total + dd > d_max:
            return dict(op=op, S=S, St=St, history=history, converged=False)
        op.increment(dd)
        d += dd

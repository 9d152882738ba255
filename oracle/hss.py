"""Algorithm 1 (HSSCompressAdaptive, Supplementary D) per HSS node, in FP64 (oracle; test infrastructure only).

For a symmetric A (n x n) and a binary cluster tree of contiguous index
ranges, the adaptive loop compresses every node from the one global sketch
S = A R:

* leaf tau:     D_tau = A(I_tau, I_tau);  S_tau(:, iota) = S(I_tau, iota) - D_tau R(I_tau, iota)
* internal tau: B_tau = A(I~_nu1, I~_nu2);
                S_tau(:, iota) = [S_nu1(J_nu1, iota) - B_tau R_nu2(:, iota);
                                  S_nu2(J_nu2, iota) - B_tau^T R_nu1(:, iota)]
  (iota = 1 : d + dd on a node's first visit, the new dd columns later).
* a node not yet compressed: Q_tau = QR(S_tau(:, 1:d)) on its first visit;
  S~ = S_tau(:, d+1 : d+dd), S^ = (I - Q Q^T)^2 S~ (two block Gram-Schmidt
  passes, the remark after Eq. (3.1)); with eps^tau = eps / level(tau):
  compress when ||S^|| < eps_a^tau or ||S^|| < eps_r^tau ||S~||; otherwise
  {Q^, Om^} = QR(S^), Q_tau <- [Q_tau, Q^], and compress when
  min |diag Om^| < eps_a^tau or < eps_r^tau |(Om_tau)_11| (the rank-deficiency
  test); otherwise the node needs more columns.
* compress: {U_tau^T, J_tau} = ID(S_tau^T, eps_r^tau, eps_a^tau), the row
  interpolative decomposition S_tau ~ U_tau S_tau(J_tau, :) from a
  column-pivoted QR of S_tau^T (scipy's LAPACK geqp3, a library step): rank k
  = the diagonal entries |R_ii| above eps_a^tau and eps_r^tau |R_11|,
  U_tau^T = [I, R11^{-1} R12] P^T.
* a compressed node: R_tau(:, iota) = U_tau^T R(I_tau, iota) (leaf) or
  U_tau^T [R_nu1; R_nu2](:, iota); I~_tau = I_tau(J_tau) or [I~_nu1, I~_nu2](J_tau).
* a node that needs more columns ends the sweep: R <- [R  JL(dd)],
  S <- [S  A R_bar], d <- d + dd, and the next sweep starts again from the leaves.

Readings (where Algorithm 1 leaves a choice): the topological order is level by
level, leaves first, and the nodes of one level are visited together (the
appendix compresses the leaves "in parallel"), so a sweep ends after the first
level that has a node needing more columns; the loop stops unconverged when the
next increment would give R more than d_max columns; Q_tau of the first visit
is the range basis of S_tau(:, 1:d) (as in oracle.adaptive.norm_test); a
block with ||S~|| = 0 passes the test; R_bar keeps its own scale (the
operator's per-block scaling), so appending it leaves the earlier columns of R,
and every S_tau and R_tau formed from them, unchanged.  The root holds
B_root = A(I~_1, I~_2).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .adaptive import project_twice, range_basis
from .operators import Operator


class Node:
    def __init__(self, lo: int, hi: int, level: int):
        self.lo, self.hi, self.level = lo, hi, level
        self.children: list[Node] = []
        self.state = "untouched"
        self.S = None      # local sketch S_tau (rows x columns so far)
        self.Q = None      # orthonormal basis of the tested columns' range
        self.om11 = 0.0    # |(Om_tau)_11|
        self.U = None      # U_tau (rows x k)
        self.J = None      # J_tau (positions within the node's local rows)
        self.R = None      # R_tau (k x columns so far)
        self.It = None     # I~_tau (global indices, k)
        self.D = None      # leaf: A(I, I)
        self.B = None      # internal: A(I~_nu1, I~_nu2)

    @property
    def leaf(self) -> bool:
        return not self.children


def cluster_tree(n: int, leaf: int) -> Node:
    """Binary tree over [0, n): a node of more than `leaf` indices splits into
    halves (the left one floor(m / 2))."""
    def build(lo, hi, level):
        nd = Node(lo, hi, level)
        if hi - lo > leaf:
            mid = lo + (hi - lo) // 2
            nd.children = [build(lo, mid, level + 1), build(mid, hi, level + 1)]
        return nd
    return build(0, n, 0)


def levels(root: Node) -> list[list[Node]]:
    out: list[list[Node]] = []
    stack = [root]
    while stack:
        nd = stack.pop()
        while len(out) <= nd.level:
            out.append([])
        out[nd.level].append(nd)
        stack.extend(reversed(nd.children))
    return out


def row_id(S: np.ndarray, eps_r: float, eps_a: float):
    """S ~ U S(J, :): column-pivoted QR of S^T, rank by the diagonal of R."""
    m = S.shape[0]
    if m == 0 or S.shape[1] == 0:
        return np.zeros((m, 0)), np.zeros(0, dtype=np.int64)
    _, Rf, P = sla.qr(S.T, mode="economic", pivoting=True)
    diag = np.abs(np.diag(Rf))
    if diag.size == 0 or diag[0] == 0.0:
        return np.zeros((m, 0)), np.zeros(0, dtype=np.int64)
    k = int(np.count_nonzero((diag > eps_a) & (diag > eps_r * diag[0])))
    k = max(k, 0)
    R11, R12 = Rf[:k, :k], Rf[:k, k:]
    X = sla.solve_triangular(R11, R12) if k else np.zeros((0, m))
    Ut = np.zeros((k, m))
    Ut[:, P[:k]] = np.eye(k)
    Ut[:, P[k:]] = X
    return Ut.T, np.asarray(P[:k], dtype=np.int64)


def compress_adaptive(A: np.ndarray, leaf: int, kind: str, d0: int, dd: int, alpha: int, seed: int,
                      d_max: int, eps_rel: float, eps_abs: float):
    """Run Algorithm 1; returns dict(root, levels, d, converged, sweeps, op, tests)
    with every node's generators, and the history of (sweep, level, node lo, passed/failed/rank)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("square (symmetric) A expected")
    root = cluster_tree(n, leaf)
    lv = levels(root)
    op = Operator(kind, n, d0 + dd, alpha, seed, scale="block")
    R = op.dense()
    S = A @ R
    d = d0
    history = []
    sweep = 0
    converged = False
    while True:
        grow = False
        for L in range(len(lv) - 1, 0, -1):
            need_more = False
            for nd in lv[L]:
                first = nd.state == "untouched"
                iota = slice(0, d + dd) if first else slice(d, d + dd)
                if nd.leaf:
                    if first:
                        nd.D = A[nd.lo:nd.hi, nd.lo:nd.hi]
                    loc = S[nd.lo:nd.hi, iota] - nd.D @ R[nd.lo:nd.hi, iota]
                else:
                    c1, c2 = nd.children
                    if first:
                        nd.B = A[np.ix_(c1.It, c2.It)]
                    loc = np.vstack([c1.S[c1.J, iota] - nd.B @ c2.R[:, iota],
                                     c2.S[c2.J, iota] - nd.B.T @ c1.R[:, iota]])
                nd.S = loc if first else np.hstack([nd.S, loc])
                if nd.state != "compressed":
                    er, ea = eps_rel / nd.level, eps_abs / nd.level
                    if first:
                        nd.Q = range_basis(nd.S[:, :d])
                        nd.om11 = float(np.linalg.norm(nd.S[:, 0])) if d > 0 else 0.0
                    St = nd.S[:, d:d + dd]
                    Sh = project_twice(nd.Q, St) if nd.Q.shape[1] else St.copy()
                    nh, nt = float(np.linalg.norm(Sh)), float(np.linalg.norm(St))
                    compress = nt == 0.0 or nh < ea or nh < er * nt
                    outcome = "passed"
                    if not compress:
                        Qh, Omh = np.linalg.qr(Sh)
                        nd.Q = np.hstack([nd.Q, Qh])
                        mind = float(np.abs(np.diag(Omh)).min()) if Omh.size else 0.0
                        compress = mind < ea or mind < er * nd.om11
                        outcome = "rank" if compress else "failed"
                    history.append((sweep, L, nd.lo, outcome, nh, nt))
                    if compress:
                        nd.U, nd.J = row_id(nd.S, er, ea)
                        nd.state = "compressed"
                        # R_tau and I~_tau over every column so far
                        if nd.leaf:
                            nd.R = nd.U.T @ R[nd.lo:nd.hi, :d + dd]
                            nd.It = np.arange(nd.lo, nd.hi)[nd.J]
                        else:
                            c1, c2 = nd.children
                            nd.R = nd.U.T @ np.vstack([c1.R[:, :d + dd], c2.R[:, :d + dd]])
                            nd.It = np.concatenate([c1.It, c2.It])[nd.J]
                        continue
                    nd.state = "partial"
                    need_more = True
                    continue
                # compressed before this sweep: extend R_tau by the new columns
                if nd.leaf:
                    new = nd.U.T @ R[nd.lo:nd.hi, iota]
                else:
                    c1, c2 = nd.children
                    new = nd.U.T @ np.vstack([c1.R[:, iota], c2.R[:, iota]])
                nd.R = np.hstack([nd.R, new])
            if need_more:
                grow = True
                break
        if not grow:
            c1, c2 = root.children if root.children else (None, None)
            if c1 is not None:
                root.B = A[np.ix_(c1.It, c2.It)]
            else:
                root.D = A
            root.state = "compressed"
            converged = True
            break
        if op.d_total + dd > d_max:
            break
        op.increment(dd)
        R = op.dense()
        S = A @ R
        d += dd
        sweep += 1
    return dict(root=root, levels=lv, d=d, converged=converged, sweeps=sweep + 1, op=op, history=history)


def reconstruct(root: Node, n: int) -> np.ndarray:
    """The dense matrix the HSS generators represent: D at the leaves, and for
    each internal node A(I_nu1, I_nu2) ~ Ub_nu1 B Ub_nu2^T (and its transpose),
    Ub the nested bases (Ub_leaf = U, Ub_tau = diag(Ub_nu1, Ub_nu2) U_tau)."""
    H = np.zeros((n, n))

    def ubig(nd):
        if nd.leaf:
            return nd.U
        c1, c2 = nd.children
        U1, U2 = ubig(c1), ubig(c2)
        blk = np.zeros((U1.shape[0] + U2.shape[0], U1.shape[1] + U2.shape[1]))
        blk[:U1.shape[0], :U1.shape[1]] = U1
        blk[U1.shape[0]:, U1.shape[1]:] = U2
        return blk @ nd.U

    def fill(nd):
        if nd.leaf:
            H[nd.lo:nd.hi, nd.lo:nd.hi] = nd.D
            return
        c1, c2 = nd.children
        off = ubig(c1) @ nd.B @ ubig(c2).T
        H[c1.lo:c1.hi, c2.lo:c2.hi] = off
        H[c2.lo:c2.hi, c1.lo:c1.hi] = off.T
        fill(c1)
        fill(c2)

    fill(root)
    return H


def hss_ranks(root: Node) -> dict:
    """Rank k_tau of every non-root node, keyed by (level, lo)."""
    out = {}
    stack = list(root.children)
    while stack:
        nd = stack.pop()
        out[(nd.level, nd.lo)] = 0 if nd.J is None else int(nd.J.size)
        stack.extend(nd.children)
    return out

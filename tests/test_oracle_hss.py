"""Pins for the per-node adaptive loop of Algorithm 1 (oracle.hss; CPU only).

* row_id: an exactly rank-k block gives rank k, S = U S(J, :) to rounding,
  identity rows of U at J.
* A matrix blockdiag + U C U^T of off-diagonal rank r < d0 (an exact HSS
  matrix) converges in one sweep, every node's rank is r, the generators
  reconstruct A to rounding, and each local sketch equals the Hankel block
  times R formed directly: A(I_tau, I_tau^c) R(I_tau^c, :) for a leaf,
  A([I~_nu1; I~_nu2], I_tau^c) R(I_tau^c, :) for an internal node.
* With r between d0 and d0 + dd the first tests fail, R grows once, and the
  rank-deficiency test (min |diag Om^| ~ 0) compresses every node.
* A Gaussian kernel matrix on bisection-ordered points: the Hankel blocks are
  reproduced by the nested bases, Ubig_tau A(I~_tau, I_tau^c), within a
  tolerance that shrinks with eps; more columns for a smaller eps.
* A flat-spectrum matrix never converges and stops at d_max.
"""
import numpy as np
import pytest

from oracle import hss
from oracle import sketch as osk
from paper_2302_01977_gb300 import inputs


def nested_basis(nd):
    if nd.leaf:
        return nd.U
    c1, c2 = nd.children
    U1, U2 = nested_basis(c1), nested_basis(c2)
    blk = np.zeros((U1.shape[0] + U2.shape[0], U1.shape[1] + U2.shape[1]))
    blk[:U1.shape[0], :U1.shape[1]] = U1
    blk[U1.shape[0]:, U1.shape[1]:] = U2
    return blk @ nd.U


def nodes(res):
    return [nd for L in res["levels"][1:] for nd in L]


def complement(n, nd):
    return np.concatenate([np.arange(0, nd.lo), np.arange(nd.hi, n)])


def test_row_id_exact_rank():
    g = np.random.default_rng(3)
    S = g.standard_normal((60, 5)) @ g.standard_normal((5, 40))
    U, J = hss.row_id(S, 1e-10, 1e-300)
    assert J.size == 5 and U.shape == (60, 5)
    assert np.linalg.norm(S - U @ S[J]) <= 1e-12 * np.linalg.norm(S)
    assert np.allclose(U[J], np.eye(5), atol=1e-14)
    U0, J0 = hss.row_id(np.zeros((7, 3)), 1e-10, 1e-300)
    assert J0.size == 0 and U0.shape == (7, 0)


@pytest.mark.parametrize("kind,alpha", [("sjlt_block", 4), ("gauss", 1), ("srht", 1)])
def test_exact_hss_one_sweep(kind, alpha):
    n, leaf, r = 512, 64, 12
    A = inputs.hss_test_matrix(n, leaf, r, seed=5)
    res = hss.compress_adaptive(A, leaf, kind, d0=32, dd=16, alpha=alpha, seed=6, d_max=256,
                                eps_rel=1e-10, eps_abs=1e-300)
    assert res["converged"] and res["sweeps"] == 1 and res["d"] == 32
    assert set(hss.hss_ranks(res["root"]).values()) == {r}
    H = hss.reconstruct(res["root"], n)
    assert np.linalg.norm(H - A) <= 1e-11 * np.linalg.norm(A)
    R = res["op"].dense()
    for nd in nodes(res):
        c = complement(n, nd)
        rows = np.arange(nd.lo, nd.hi) if nd.leaf else \
            np.concatenate([nd.children[0].It, nd.children[1].It])
        direct = A[np.ix_(rows, c)] @ R[c]
        assert np.linalg.norm(nd.S - direct) <= 1e-11 * np.linalg.norm(direct), (nd.level, nd.lo)
        # the nested basis reproduces the Hankel block from its skeleton rows
        Hk = A[np.ix_(np.arange(nd.lo, nd.hi), c)]
        assert np.linalg.norm(Hk - nested_basis(nd) @ A[np.ix_(nd.It, c)]) <= 1e-10 * np.linalg.norm(Hk)


def test_rank_between_d_and_d_plus_dd_restarts_once():
    n, leaf, r = 512, 64, 40
    A = inputs.hss_test_matrix(n, leaf, r, seed=7)
    res = hss.compress_adaptive(A, leaf, "gauss", d0=16, dd=16, alpha=1, seed=8, d_max=256,
                                eps_rel=1e-10, eps_abs=1e-300)
    assert res["converged"] and res["sweeps"] == 2 and res["d"] == 32
    first = [h for h in res["history"] if h[0] == 0]
    second = [h for h in res["history"] if h[0] == 1]
    # sweep 0 stops after the leaf level, where every leaf fails its test
    assert {h[1] for h in first} == {3} and {h[3] for h in first} == {"failed"}
    # sweep 1: every node compresses through the rank-deficiency test
    assert len(second) == 14 and {h[3] for h in second} == {"rank"}
    assert set(hss.hss_ranks(res["root"]).values()) == {r}
    H = hss.reconstruct(res["root"], n)
    assert np.linalg.norm(H - A) <= 1e-11 * np.linalg.norm(A)


def kernel_case(n=1024, leaf=64, h=0.2):
    X = inputs.points(n, seed=11).astype(np.float64)
    X = X[inputs.bisection_order(X, leaf)]
    return osk.kernel_matrix(X, X, h, 1e-2)


def test_kernel_matrix_nested_bases_and_eps():
    n, leaf = 1024, 64
    A = kernel_case(n, leaf)
    errs, ds = [], []
    for eps in (1e-3, 1e-7):
        res = hss.compress_adaptive(A, leaf, "sjlt_block", d0=32, dd=16, alpha=4, seed=12,
                                    d_max=512, eps_rel=eps, eps_abs=1e-300)
        assert res["converged"]
        worst = 0.0
        for nd in nodes(res):
            c = complement(n, nd)
            Hk = A[np.ix_(np.arange(nd.lo, nd.hi), c)]
            e = np.linalg.norm(Hk - nested_basis(nd) @ A[np.ix_(nd.It, c)]) / np.linalg.norm(Hk)
            worst = max(worst, e)
        errs.append(worst)
        ds.append(res["d"])
        H = hss.reconstruct(res["root"], n)
        assert np.linalg.norm(H - A) <= 100 * eps * np.linalg.norm(A)
    assert errs[1] < errs[0] / 100 and errs[1] < 1e-5
    assert ds[0] < ds[1]


def test_flat_spectrum_stops_at_d_max():
    n, leaf = 256, 64
    g = np.random.default_rng(13)
    B = g.standard_normal((n, n))
    A = B + B.T
    res = hss.compress_adaptive(A, leaf, "gauss", d0=16, dd=16, alpha=1, seed=14, d_max=64,
                                eps_rel=1e-8, eps_abs=1e-300)
    assert not res["converged"] and res["op"].d_total == 64 and res["d"] == 48


def test_single_leaf_tree():
    A = inputs.hss_test_matrix(48, 64, 3, seed=15)
    res = hss.compress_adaptive(A, 64, "gauss", d0=8, dd=8, alpha=1, seed=16, d_max=64,
                                eps_rel=1e-6, eps_abs=1e-300)
    assert res["converged"] and res["history"] == []
    assert np.array_equal(hss.reconstruct(res["root"], 48), A)


def test_level_scaled_tolerance():
    """A leaf at level 2 is tested against eps / 2: its first test, with the
    ratio rho = ||S^|| / ||S~|| of its local sketch formed directly
    (A(I, I^c) R(I^c, :), tested by oracle.adaptive.norm_test), fails at
    eps = 1.5 rho and passes at eps = 2.5 rho."""
    from oracle import adaptive as ad
    from oracle.operators import Operator
    n, leaf, d0, dd = 256, 64, 24, 8
    A = kernel_case(n, leaf, h=0.3)
    R = Operator("gauss", n, d0 + dd, 1, 17, scale="block").dense()
    c = np.arange(64, n)
    S_loc = A[np.ix_(np.arange(64), c)] @ R[c]
    _, nh, nt = ad.norm_test(S_loc, d0, dd, 0.0, 0.0)
    rho = nh / nt
    assert 1e-8 < rho < 1e-1
    for f, want in ((1.5, False), (2.5, True)):
        res = hss.compress_adaptive(A, leaf, "gauss", d0=d0, dd=dd, alpha=1, seed=17, d_max=128,
                                    eps_rel=f * rho, eps_abs=1e-300)
        h0 = [h for h in res["history"] if h[0] == 0 and h[1] == 2 and h[2] == 0][0]
        assert abs(h0[4] / h0[5] - rho) <= 1e-10 * rho
        assert (h0[3] == "passed") == want, (f, h0)


@pytest.mark.parametrize("n,leaf", [(1, 1), (7, 8), (64, 64), (65, 64), (1000, 37), (2048, 64), (3001, 100)])
def test_cluster_tree_partition_and_split_rule(n, leaf):
    """The tree's leaves are consecutive index ranges covering [0, n) in order,
    no leaf holds more than `leaf` indices, every split node holds more and
    gives its left child floor(m / 2) indices, and a node's level is its depth
    (checked by a walk written independently of the tree's construction)."""
    root = hss.cluster_tree(n, leaf)
    leaves, seen = [], 0

    def walk(nd, depth):
        nonlocal seen
        assert nd.level == depth and nd.hi > nd.lo
        m = nd.hi - nd.lo
        if not nd.children:
            assert m <= leaf and nd.lo == seen
            seen = nd.hi
            leaves.append(m)
            return
        assert m > leaf and len(nd.children) == 2
        a, b = nd.children
        assert (a.lo, a.hi, b.lo, b.hi) == (nd.lo, nd.lo + m // 2, nd.lo + m // 2, nd.hi)
        walk(a, depth + 1)
        walk(b, depth + 1)

    walk(root, 0)
    assert seen == n and sum(leaves) == n
    # levels() lists every node once, by depth, left to right
    lv = hss.levels(root)
    assert [nd.level for L in lv for nd in L] == sorted(nd.level for L in lv for nd in L)
    for L in lv:
        assert [nd.lo for nd in L] == sorted(nd.lo for nd in L)
    assert sum(len(L) for L in lv) == 2 * len(leaves) - 1
    # for n = leaf * 2^j the tree is perfect with j + 1 levels
    if n % leaf == 0 and ((n // leaf) & (n // leaf - 1)) == 0:
        assert len(lv) == (n // leaf).bit_length() and set(leaves) == {leaf}

"""Pins for the oracle's JL operators and sketch products (CPU only).

Each check is a fact the paper or the mathematics fixes, not a retyped formula:
nonzero counts and values (Sec. 2.4.3), the Sec. 6.1 worked example, the
Sylvester recursion and H H^T = nu I (Sec. 2.4.2), R^T R = (n/d) I for an SRHT
of power-of-two order, the FWHT route agreeing with the element formula,
E||x^T R||^2 = ||x||^2 (Definition 2.2), A = I giving R back, and brute-force
triple loops at n <= 64.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import operators as ops
from oracle import sketch as sk
from paper_2302_01977_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- SJLT ----------------------------------------------------------------

@pytest.mark.parametrize("n,d,alpha", [(64, 16, 4), (100, 24, 3), (257, 128, 4), (33, 8, 8), (50, 5, 1)])
def test_sjlt_block_structure(n, d, alpha):
    op = ops.Operator("sjlt_block", n, d, alpha, seed=11)
    R = op.dense()
    nz = R != 0
    assert (nz.sum(axis=1) == alpha).all()
    assert np.allclose(np.abs(R[nz]), 1.0 / math.sqrt(alpha), rtol=0, atol=0)
    chunk = d // alpha
    for k in range(alpha):  # exactly one nonzero per chunk
        assert (nz[:, k * chunk:(k + 1) * chunk].sum(axis=1) == 1).all()
    assert abs((R ** 2).sum() - n) < 1e-9
    cols, signs = op.sjlt_entries()
    assert set(np.unique(signs).tolist()) <= {-1, 1}


@pytest.mark.parametrize("n,d,alpha", [(64, 16, 4), (200, 128, 4), (40, 7, 7), (31, 9, 2)])
def test_sjlt_graph_structure(n, d, alpha):
    op = ops.Operator("sjlt_graph", n, d, alpha, seed=5)
    cols, signs = op.sjlt_entries()
    assert (np.diff(cols, axis=1) > 0).all()  # distinct and ascending
    assert cols.min() >= 0 and cols.max() < d
    R = op.dense()
    assert ((R != 0).sum(axis=1) == alpha).all()
    assert abs((R ** 2).sum() - n) < 1e-9


def test_sjlt_positions_uniform_and_signs_balanced():
    n, d, alpha = 20000, 64, 4
    cols, signs = ops.Operator("sjlt_block", n, d, alpha, seed=3).sjlt_entries()
    rel = cols - (np.arange(alpha) * (d // alpha))[None, :]
    counts = np.bincount(rel.ravel(), minlength=d // alpha)
    expect = n * alpha / (d // alpha)
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 60  # 15 dof: P(chi2 > 60) ~ 1e-7
    assert abs((signs == 1).mean() - 0.5) < 0.01


def test_sjlt_worked_example_crs_ccs():
    ex = json.load(open(os.path.join(GOLDEN, "sjlt_worked_example.json")))
    R = np.array(ex["R_times_sqrt_alpha"])
    rows, colsk = np.nonzero(R)
    n, d = R.shape
    alpha = ex["alpha"]
    cols = colsk.reshape(n, alpha)
    signs = np.sign(R[rows, colsk]).astype(np.int8).reshape(n, alpha)
    st = ops.crs_ccs(cols, signs, d)
    for name, key in (("plus", "B_plus"), ("minus", "B_minus")):
        B = np.zeros((n, d), dtype=int)
        crs = st[name]
        for i in range(n):
            B[i, crs["col_idx"][crs["row_ptr"][i]:crs["row_ptr"][i + 1]]] = 1
        assert (B == np.array(ex[key])).all()
        B2 = np.zeros((n, d), dtype=int)
        for c in range(d):
            B2[crs["row_idx"][crs["col_ptr"][c]:crs["col_ptr"][c + 1]], c] = 1
        assert (B2 == np.array(ex[key])).all()
    # R = (B+ - B-)/sqrt(alpha)
    Rs = (np.array(ex["B_plus"]) - np.array(ex["B_minus"])) / math.sqrt(alpha)
    assert np.array_equal(Rs, R / math.sqrt(alpha))


@pytest.mark.parametrize("kind", ["sjlt_block", "sjlt_graph"])
def test_sjlt_outer_and_inner_forms_brute_force(kind):
    n, d, alpha = 48, 16, 4
    A = inputs.dense_matrix(n, n, seed=1)
    op = ops.Operator(kind, n, d, alpha, seed=9)
    cols, signs = op.sjlt_entries()
    S_outer = sk.apply_sjlt_outer(A, cols, signs, op.scale(), d)
    St_inner = sk.apply_sjlt_inner(A, ops.crs_ccs(cols, signs, d), op.scale(), d)
    R = op.dense()
    S_bf = np.zeros((n, d))
    St_bf = np.zeros((n, d))
    for i in range(n):
        for c in range(d):
            S_bf[i, c] = sum(A[i, j] * R[j, c] for j in range(n))
            St_bf[i, c] = sum(A[j, i] * R[j, c] for j in range(n))
    S, St = sk.apply(A, R)
    for X in (S_outer, S):
        assert np.allclose(X, S_bf, rtol=1e-13, atol=1e-13)
    for X in (St_inner, St):
        assert np.allclose(X, St_bf, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind,alpha", [("sjlt_block", 4), ("srht", 1), ("gauss", 1)])
def test_apply_t_rectangular_brute_force(kind, alpha):
    """S' = A^T R for a rectangular, nonsymmetric A (m x n, R m x d): a triple
    loop over S'[j, c] = sum_i A[i, j] R[i, c], a unit matrix e_i e_j^T that
    must move row i of R to row j of S', and the shape, which a transposed
    operand would change."""
    m, n, d = 40, 23, 8
    A = inputs.dense_matrix(m, n, seed=12)
    R = ops.Operator(kind, m, d, alpha, seed=13).dense()
    St = sk.apply_t(A, R)
    assert St.shape == (n, d)
    bf = np.zeros((n, d))
    for j in range(n):
        for c in range(d):
            bf[j, c] = sum(A[i, j] * R[i, c] for i in range(m))
    assert np.allclose(St, bf, rtol=1e-13, atol=1e-13)
    E = np.zeros((m, n))
    E[31, 5] = 1.0
    pick = sk.apply_t(E, R)
    expect = np.zeros((n, d))
    expect[5] = R[31]
    assert np.array_equal(pick, expect)
    with pytest.raises(ValueError):
        sk.apply_t(A.T, R)  # rows(A) must equal rows(R)


# --- SRHT ----------------------------------------------------------------

@pytest.mark.parametrize("nu", [1, 2, 4, 16, 64])
def test_hadamard_recursion_orthogonality(nu):
    H = sk.hadamard(nu)
    assert np.array_equal(H @ H.T, nu * np.eye(nu))
    i = np.arange(nu)[:, None]
    j = np.arange(nu)[None, :]
    assert np.array_equal(H, np.where(ops.popcount_parity(i & j) == 1, -1.0, 1.0))


def test_fwht_is_hadamard_product():
    x = inputs.dense_matrix(5, 64, seed=2)
    assert np.allclose(sk.fwht(x), x @ sk.hadamard(64).T, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n,d", [(64, 16), (128, 128), (32, 5)])
def test_srht_orthogonal_columns_power_of_two(n, d):
    op = ops.Operator("srht", n, d, seed=4)
    R = op.dense()
    assert np.allclose(R.T @ R, (n / d) * np.eye(d), rtol=0, atol=1e-12)
    mu = op.srht_samples()
    assert len(set(mu.tolist())) == d and mu.min() >= 0 and mu.max() < n
    assert abs((R ** 2).sum() - n) < 1e-9


@pytest.mark.parametrize("n,d", [(64, 16), (50, 12), (37, 32)])
def test_srht_fwht_route_equals_element_formula(n, d):
    A = inputs.dense_matrix(9, n, seed=8)
    op = ops.Operator("srht", n, d, seed=21)
    S_def = A @ op.dense()
    S_fwht = sk.srht_by_fwht(A, op.srht_diag(), op.srht_samples(), op.d_total)
    assert np.allclose(S_def, S_fwht, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n", [3, 5, 6, 12, 100, 130, 777, 1100])
def test_srht_split_equals_element_formula_and_padded_transform(n):
    """Sec. 7.1's H_k / H_p split of a non-power-of-two order gives the product with
    R from the element formula of Sec. 7.2 and the transform of zero-padded rows."""
    d = min(16, 1 << (n - 1).bit_length())
    op = ops.Operator("srht", n, d, 1, seed=n)
    A = np.random.default_rng(n).standard_normal((7, n))
    S_split = sk.srht_by_split(A, op.srht_diag(), op.srht_samples(), op.d_total)
    assert np.allclose(S_split, A @ op.dense(), rtol=0, atol=1e-12 * max(1.0, np.abs(A).sum()))
    S_pad = sk.srht_by_fwht(A, op.srht_diag(), op.srht_samples(), op.d_total)
    assert np.allclose(S_split, S_pad, rtol=0, atol=1e-12 * max(1.0, np.abs(A).sum()))


def test_srht_split_tail_is_a_periodic_transform():
    """Eq. hadiden: the padded order-k transform of a vector whose nonzeros are its
    first r <= p entries repeats its order-p transform k/p times."""
    k, r = 64, 11
    p = 16
    x = np.zeros(k)
    x[:r] = np.random.default_rng(1).standard_normal(r)
    y = sk.fwht(x)
    assert np.allclose(y, np.tile(sk.fwht(x[:p]), k // p), rtol=0, atol=1e-12)
    with pytest.raises(ValueError):
        sk.srht_by_split(np.ones((2, 8)), np.ones(8), np.arange(4), 4)


def test_srht_nu_too_small_rejected():
    with pytest.raises(ValueError):
        ops.Operator("srht", 8, 9)
    op = ops.Operator("srht", 8, 6)
    with pytest.raises(ValueError):
        op.increment(3)


# --- Gaussian ------------------------------------------------------------

def test_gaussian_distribution():
    from scipy import stats
    z = ops.gaussian_z(4000, 0, 64, seed=12).ravel()
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # even/odd columns (cos and sin halves of one Box-Muller pair) uncorrelated
    zz = ops.gaussian_z(20000, 0, 2, seed=13)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 5 / math.sqrt(20000)


def test_gaussian_columns_independent_of_width():
    a = ops.gaussian_z(30, 0, 10, seed=1)
    b = ops.gaussian_z(30, 3, 7, seed=1)
    assert np.array_equal(a[:, 3:7], b)


# --- all operators -------------------------------------------------------

KIND_ARGS = [("sjlt_block", 4), ("sjlt_graph", 4), ("srht", 1), ("gauss", 1)]


@pytest.mark.parametrize("kind,alpha", KIND_ARGS)
def test_identity_returns_R(kind, alpha):
    n, d = 64, 16
    op = ops.Operator(kind, n, d, alpha, seed=77)
    R = op.dense()
    S, St = sk.apply(np.eye(n), R)
    assert np.array_equal(S, R) and np.array_equal(St, R)


@pytest.mark.parametrize("kind,alpha", KIND_ARGS)
def test_unit_matrix_picks_row(kind, alpha):
    n, d = 40, 8
    op = ops.Operator(kind, n, d, alpha, seed=78)
    R = op.dense()
    E = np.zeros((n, n))
    E[3, 17] = 1.0
    S, St = sk.apply(E, R)
    expect = np.zeros((n, d))
    expect[3] = R[17]
    assert np.array_equal(S, expect)
    expect_t = np.zeros((n, d))
    expect_t[17] = R[3]
    assert np.array_equal(St, expect_t)


@pytest.mark.parametrize("kind,alpha", KIND_ARGS)
def test_symmetric_A_gives_equal_sketches(kind, alpha):
    n, d = 64, 16
    X = inputs.dense_matrix(n, n, seed=5)
    A = X + X.T
    S, St = sk.apply(A, ops.Operator(kind, n, d, alpha, seed=3).dense())
    assert np.allclose(S, St, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("kind,alpha", KIND_ARGS)
def test_jl_norm_expectation_monte_carlo(kind, alpha):
    """E ||x^T R||^2 = ||x||^2 (Definition 2.2 with eps -> expectation)."""
    n, d, T = 64, 16, 400
    x = inputs.dense_matrix(1, n, seed=6)[0]
    vals = np.array([((x @ ops.Operator(kind, n, d, alpha, seed=s).dense()) ** 2).sum() for s in range(T)])
    mean, sd = vals.mean(), vals.std(ddof=1)
    nx = (x ** 2).sum()
    assert abs(mean - nx) < 5 * sd / math.sqrt(T)


@pytest.mark.parametrize("kind,alpha", KIND_ARGS)
def test_increment_rescales_and_appends(kind, alpha):
    n, d0, dd = 64, 16, 8
    base = ops.Operator(kind, n, d0, alpha, seed=31)
    grown = ops.Operator(kind, n, d0, alpha, seed=31)
    grown.increment(dd)
    R0, R1 = base.dense(), grown.dense()
    assert R1.shape == (n, d0 + dd)
    ratio = grown.scale() / base.scale()
    assert np.allclose(R1[:, :d0], R0 * ratio, rtol=1e-15, atol=0)
    # the grown operator is again a JL operator of the new width
    if kind.startswith("sjlt"):
        assert ((R1[:, d0:] != 0).sum(axis=1) == alpha).all()
        assert abs((R1 ** 2).sum() - n) < 1e-9
    if kind == "srht":
        assert np.allclose(R1.T @ R1, (n / (d0 + dd)) * np.eye(d0 + dd), atol=1e-12)


def test_invalid_operator_arguments():
    with pytest.raises(ValueError):
        ops.Operator("sjlt_block", 10, 10, 3)
    with pytest.raises(ValueError):
        ops.Operator("sjlt_graph", 10, 3, 4)
    with pytest.raises(ValueError):
        ops.Operator("nope", 10, 3, 1)
    with pytest.raises(ValueError):
        ops.Operator("gauss", 0, 3, 1)


# --- kernel matrix and input ordering -------------------------------------

def test_kernel_matrix_brute_force_and_symmetry():
    X = inputs.points(20, seed=1, dtype=np.float64)
    Y = inputs.points(15, seed=2, dtype=np.float64)
    A = sk.kernel_matrix(X, Y, 0.3, 0.0)
    for i in range(20):
        for j in range(15):
            r2 = sum((X[i, k] - Y[j, k]) ** 2 for k in range(3))
            assert abs(A[i, j] - math.exp(-r2 / (2 * 0.09))) < 1e-15
    As = sk.kernel_matrix(X, X, 0.2, 1e-2)
    assert np.array_equal(As, As.T)
    assert np.allclose(np.diag(As), 1.0 + 1e-2, rtol=0, atol=1e-15)
    rows = np.array([0, 7, 19])
    assert np.array_equal(sk.kernel_rows(X, X, rows, 0.2, 1e-2), As[rows])


def test_bisection_order_is_a_valid_median_split():
    P = inputs.points(1000, seed=3, dtype=np.float64)
    perm = inputs.bisection_order(P, leaf=64)
    assert np.array_equal(np.sort(perm), np.arange(1000))
    # top-level split: on the widest axis, left half <= right half
    Q = P[perm]
    axis = int(np.argmax(P.max(0) - P.min(0)))
    assert Q[:500, axis].max() <= Q[500:, axis].min()


def test_apply_complex_against_real_parts():
    """S = A R and S' = A* R for A = B + iC equal B R + i C R and B^T R - i C^T R
    (R real), and reduce to the real products for real A."""
    from oracle import sketch as osk
    rng = np.random.default_rng(21)
    B, C = rng.standard_normal((7, 9)), rng.standard_normal((7, 9))
    R9, R7 = rng.standard_normal((9, 4)), rng.standard_normal((7, 4))
    S = osk.complex_s(B + 1j * C, R9)
    np.testing.assert_allclose(S, B @ R9 + 1j * (C @ R9), rtol=1e-14, atol=1e-14)
    St = osk.complex_t(B + 1j * C, R7)
    np.testing.assert_allclose(St, B.T @ R7 - 1j * (C.T @ R7), rtol=1e-14, atol=1e-14)
    A = rng.standard_normal((6, 6))
    R = rng.standard_normal((6, 3))
    S, St = osk.apply_complex(A, R)
    S0, St0 = osk.apply(A, R)
    np.testing.assert_allclose(S, S0, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(St, St0, rtol=1e-14, atol=1e-14)
    # entry by entry: S'_jc = sum_i conj(A_ij) R_ic
    Z = B[:, :7] + 1j * C[:, :7]
    St = osk.complex_t(Z, R7)
    for j in range(7):
        for c in range(4):
            want = sum(np.conj(Z[i, j]) * R7[i, c] for i in range(7))
            assert abs(St[j, c] - want) <= 1e-13


# --- creation flags: per-block scale (Algorithm 1's independent JL(Delta-d)) and
# --- SRHT sampling with replacement (Sec. 2.4.2, "independently and uniformly")

@pytest.mark.parametrize("kind,alpha", [("sjlt_block", 4), ("sjlt_graph", 4), ("srht", 1), ("gauss", 1)])
def test_block_scale_each_block_is_its_own_jl_operator(kind, alpha):
    n, d0, dd = 96, 24, 8
    ren = ops.Operator(kind, n, d0, alpha, seed=21)
    blk = ops.Operator(kind, n, d0, alpha, seed=21, scale="block")
    for _ in range(2):
        ren.increment(dd)
        blk.increment(dd)
    Rr, Rb = ren.dense(), blk.dense()
    widths = [d0, dd, dd]
    c0 = 0
    for w in widths:
        cols = slice(c0, c0 + w)
        nz = Rb[:, cols][Rb[:, cols] != 0]
        if kind.startswith("sjlt"):
            assert np.allclose(np.abs(nz), 1.0 / math.sqrt(alpha), rtol=0, atol=1e-15)
            assert np.count_nonzero(Rb[:, cols], axis=1).tolist() == [alpha] * n
        elif kind == "srht":
            assert np.allclose(np.abs(Rb[:, cols]), 1.0 / math.sqrt(w), rtol=0, atol=1e-15)
        # the same random draws as the renormalized operator, another scale per block
        ratio = math.sqrt(3) if kind.startswith("sjlt") else math.sqrt((d0 + 2 * dd) / w)
        assert np.allclose(Rb[:, cols], Rr[:, cols] * ratio, rtol=1e-14, atol=0)
        c0 += w


def test_block_scale_gaussian_block_variance():
    n, d0, dd = 4000, 64, 16
    op = ops.Operator("gauss", n, d0, seed=5, scale="block")
    op.increment(dd)
    R = op.dense()
    for cols, w in ((slice(0, d0), d0), (slice(d0, d0 + dd), dd)):
        v = R[:, cols].var()
        k = n * w
        assert abs(v * w - 1.0) < 5 * math.sqrt(2.0 / k)  # variance 1/w_b within 5 sigma


def test_srht_with_replacement_draws():
    nu, count, seed = 64, 200, 8
    rep = ops.srht_samples(nu, count, seed, replace=True)
    assert rep.shape == (count,) and rep.min() >= 0 and rep.max() < nu  # more than nu columns allowed
    # the sample without replacement is this sequence with its repeats removed, in order
    first = list(dict.fromkeys(rep.tolist()))
    k = min(len(first), nu)
    assert ops.srht_samples(nu, k, seed).tolist() == first[:k]
    # repeats at the rate of independent uniform draws: E[distinct] = nu (1 - (1 - 1/nu)^count)
    distinct = []
    for s in range(200):
        distinct.append(len(set(ops.srht_samples(nu, 40, 1000 + s, replace=True).tolist())))
    e = nu * (1 - (1 - 1 / nu) ** 40)
    assert abs(np.mean(distinct) - e) < 5 * np.std(distinct) / math.sqrt(len(distinct))
    # uniform over [0, nu): chi-square over many draws
    big = ops.srht_samples(nu, 64 * 200, 77, replace=True)
    cnt = np.bincount(big, minlength=nu)
    chi2 = ((cnt - 200.0) ** 2 / 200.0).sum()
    assert chi2 < nu - 1 + 5 * math.sqrt(2 * (nu - 1))
    with pytest.raises(ValueError):
        ops.srht_samples(nu, nu + 1, seed)


def test_srht_with_replacement_operator():
    n, d = 40, 80  # nu = 64 < d: only possible with replacement
    op = ops.Operator("srht", n, d, seed=3, replace=True)
    R = op.dense()
    mu = op.srht_samples()
    assert np.allclose(np.abs(R), 1.0 / math.sqrt(d), rtol=0, atol=1e-15)
    # a repeated sample gives a repeated column (the element formula depends on mu_j only)
    a, b = [(i, j) for i in range(d) for j in range(i + 1, d) if mu[i] == mu[j]][0]
    assert np.array_equal(R[:, a], R[:, b])
    # E ||x^T R||^2 = ||x||^2 over the random signs D (Definition 2.2), Monte Carlo, 5 sigma
    x = inputs.dense_matrix(1, n, seed=4)[0]
    vals = np.array([np.sum((x @ ops.Operator("srht", n, d, seed=s, replace=True).dense()) ** 2)
                     for s in range(300)])
    assert abs(vals.mean() - x @ x) < 5 * vals.std() / math.sqrt(vals.size)
    with pytest.raises(ValueError):
        ops.Operator("srht", n, d, seed=3)  # without replacement d <= nu
    with pytest.raises(ValueError):
        ops.Operator("gauss", n, 8, seed=3, replace=True)


def test_next_pow2_is_the_least_power_of_two_not_below_n():
    for n in range(1, 5000):
        p = ops.next_pow2(n)
        assert p >= n and p & (p - 1) == 0 and (p == 1 or p // 2 < n)
    assert ops.next_pow2(1 << 40) == 1 << 40 and ops.next_pow2((1 << 40) + 1) == 1 << 41


@pytest.mark.parametrize("construction,width,alpha", [("block", 64, 4), ("block", 12, 3), ("graph", 64, 4),
                                                      ("graph", 5, 5), ("graph", 32, 1)])
def test_sjlt_block_draws_structure(construction, width, alpha):
    """Sec. 2.4.3: each row holds alpha +-1 entries; the block construction puts
    one in each of alpha chunks of width / alpha columns, the graph construction
    alpha distinct columns (sorted); draws of another block or seed differ."""
    n = 3000
    cols, signs = ops.sjlt_block_draws(n, width, alpha, seed=5, block=2, construction=construction)
    assert cols.shape == (n, alpha) and signs.shape == (n, alpha)
    assert cols.min() >= 0 and cols.max() < width
    assert set(np.unique(signs)) <= {-1, 1}
    if construction == "block":
        span = width // alpha
        assert np.array_equal(cols // span, np.broadcast_to(np.arange(alpha), (n, alpha)))
    else:
        assert (np.diff(cols, axis=1) > 0).all()
        if alpha == width:
            assert (cols == np.arange(width)).all()
    # both signs and (where there is a choice) every position occur
    assert (signs == 1).any() and (signs == -1).any()
    if construction == "graph" and alpha < width:
        assert np.unique(cols).size == width
    c2, s2 = ops.sjlt_block_draws(n, width, alpha, seed=5, block=3, construction=construction)
    c3, s3 = ops.sjlt_block_draws(n, width, alpha, seed=6, block=2, construction=construction)
    assert not (np.array_equal(c2, cols) and np.array_equal(s2, signs))
    assert not (np.array_equal(c3, cols) and np.array_equal(s3, signs))
    c4, s4 = ops.sjlt_block_draws(n, width, alpha, seed=5, block=2, construction=construction)
    assert np.array_equal(c4, cols) and np.array_equal(s4, signs)


def test_sjlt_block_draws_refuses_bad_arguments():
    with pytest.raises(ValueError):
        ops.sjlt_block_draws(10, 8, 2, 1, 0, "other")
    with pytest.raises(ValueError):
        ops.sjlt_block_draws(10, 8, 0, 1, 0, "graph")
    with pytest.raises(ValueError):
        ops.sjlt_block_draws(10, 8, 9, 1, 0, "graph")
    with pytest.raises(ValueError):
        ops.sjlt_block_draws(10, 10, 3, 1, 0, "block")

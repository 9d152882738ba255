"""The tcgen05 bf16 split path (prec = SK_PREC_BF16X2) against the FP64 oracle.

FP32 data; SRHT and Gaussian operators.  Two gates per case:

* relative Frobenius error <= 1e-5 against the oracle applied to the same
  FP32 matrix widened to FP64;
* an elementwise bound.  With a = a_hi + a_lo + r_a, |r_a| <= 2^-16 |a| (two
  bf16 roundings, unit roundoff 2^-8 each), and likewise for the Gaussian z,
  the terms the kernel keeps differ from a*z by at most about 3 * 2^-16 |a z|
  (the dropped a_lo z_lo and the two residuals); the FP32 accumulation adds
  at most chain * 2^-23 relative, chain <= 1024 products.  So every output
  obeys |S - S_ref| <= 2.5e-4 * (|A| |R|), while a dropped or doubled term
  (2^-9 relative) breaks it.

Shapes span several 128-row tiles with ragged tails in M, K and d, two
column tiles (d > 256), increments whose first column is not a multiple of 4
(scalar epilogue), and enough tiles that the stream-K split gives tiles two
contributing CTAs.
"""
import numpy as np
import pytest

from oracle import operators as ops
from oracle import sketch as osk
from paper_2302_01977_gb300 import inputs
from tests.util import TOL, dev_padded, ensure_built, host, rel_fro

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ELEM_BOUND = 2.5e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def jlmod():
    from paper_2302_01977_gb300 import jlsketch as jl
    return jl


def run(kind, A_np, which, d, seed, incs=()):
    """Sketch FP32 A with the split path; returns the output and the oracle's R."""
    jl = jlmod()
    rows, cols = A_np.shape
    n = cols if which == jl.SK_S else rows
    out_rows = rows if which == jl.SK_S else cols
    dmax = d + sum(incs)
    A = dev_padded(A_np, torch.float32)
    h = jl.sketch_create(kind, n, d, 1, seed, dmax)
    try:
        O = torch.full((out_rows, dmax), np.nan, dtype=torch.float32, device="cuda")
        kw = {"S": O} if which == jl.SK_S else {"St": O}
        jl.sketch_apply(h, A, which=which, prec=jl.SK_PREC_BF16X2, **kw)
        for dd in incs:
            jl.sketch_increment(h, dd)
            jl.sketch_apply_increment(h, A, which=which, prec=jl.SK_PREC_BF16X2, **kw)
        torch.cuda.synchronize()
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)
    op = ops.Operator(kind, n, d, 1, seed)
    for dd in incs:
        op.increment(dd)
    return host(O), op.dense()


def check(kind, A_np, which, d, seed, incs=()):
    jl = jlmod()
    got, R = run(kind, A_np, which, d, seed, incs)
    A64 = A_np.astype(np.float64)
    B = A64 if which == jl.SK_S else A64.T
    ref = B @ R
    assert np.isfinite(got).all()
    err = rel_fro(got, ref)
    assert err <= TOL["bf16x2"], err
    bound = ELEM_BOUND * (np.abs(B) @ np.abs(R))
    assert (np.abs(got - ref) <= bound).all()
    return err


@pytest.mark.parametrize("kind", ["srht", "gauss"])
@pytest.mark.parametrize("n,d", [(64, 16), (1000, 100), (2048, 128), (1537, 72), (777, 300)])
def test_tc_square_both(kind, n, d):
    A = inputs.dense_matrix(n, n, seed=n + 7 * d).astype(np.float32)
    jl = jlmod()
    check(kind, A, jl.SK_S, d, 11 * n + d)
    check(kind, A, jl.SK_ST, d, 11 * n + d)


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_tc_kernel_matrix_d512(kind):
    """A Gaussian-kernel matrix (the paper's test matrices) with two 256-column tiles."""
    n, d = 4096, 512
    X = inputs.points(n, seed=5)
    A = osk.kernel_matrix(X, X, 1.0).astype(np.float32)
    jl = jlmod()
    check(kind, A, jl.SK_S, d, 3)
    check(kind, A, jl.SK_ST, d, 3)


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_tc_increments_unaligned(kind):
    """Increments whose first column is 50 and 64: scalar and vector epilogues."""
    n = 1200
    A = inputs.dense_matrix(n, n, seed=8).astype(np.float32)
    jl = jlmod()
    check(kind, A, jl.SK_S, 50, 21, incs=(14, 33))
    check(kind, A, jl.SK_ST, 50, 21, incs=(14, 33))


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_tc_stream_k_split(kind):
    """More 128-row tiles than SMs: CTA ranges cut tiles, two partial sums per cell."""
    rows, n, d = 20000, 1500, 64
    A = inputs.dense_matrix(rows, n, seed=9).astype(np.float32)
    jl = jlmod()
    check(kind, A, jl.SK_S, d, 4)
    check(kind, np.ascontiguousarray(A.T), jl.SK_ST, d, 4)


def test_tc_deterministic():
    """Two runs give identical bits (at most two contributions per cell)."""
    rows, n, d = 20000, 1500, 64
    A = inputs.dense_matrix(rows, n, seed=10).astype(np.float32)
    jl = jlmod()
    g1, _ = run("gauss", A, jl.SK_S, d, 6)
    g2, _ = run("gauss", A, jl.SK_S, d, 6)
    assert np.array_equal(g1, g2)


def test_tc_rejects_fp64_and_sjlt_fp8():
    jl = jlmod()
    A = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    S = torch.zeros((64, 16), dtype=torch.float64, device="cuda")
    h = jl.sketch_create("gauss", 64, 16, 1, 1, 16)
    try:
        with pytest.raises(jl.JLSketchError) as e:
            jl.sketch_apply(h, A, which=jl.SK_S, prec=jl.SK_PREC_BF16X2, S=S)
        assert e.value.status == jl.SK_ERR_DTYPE
    finally:
        jl.sketch_destroy(h)
    A32 = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    S32 = torch.zeros((64, 16), dtype=torch.float32, device="cuda")
    h = jl.sketch_create("sjlt_block", 64, 16, 4, 1, 16)
    try:
        with pytest.raises(jl.JLSketchError) as e:
            jl.sketch_apply(h, A32, which=jl.SK_S, prec=jl.SK_PREC_FP8, S=S32)
        assert e.value.status == jl.SK_ERR_DTYPE
    finally:
        jl.sketch_destroy(h)


@pytest.mark.parametrize("route", ["tc", "sjlt", "pick"])
@pytest.mark.parametrize("kind,alpha", [("sjlt_block", 4), ("sjlt_graph", 3)])
def test_sjlt_bf16x2_routes(kind, alpha, route, monkeypatch):
    """SJLT products with SK_PREC_BF16X2 through the tensor-core +-1 product
    (R's {0, +-1} plane exact in bf16, A split hi + lo), the SJLT kernels, or
    whichever measures faster, with an increment: S and S' against the FP64
    oracle (1e-5 relative Frobenius; each term of the split within 2.5e-4 of
    |A||R| elementwise)."""
    jl = jlmod()
    if route != "pick":
        monkeypatch.setenv("JLS_SJLT_ROUTE", route)
    m, n, d, dd = 900, 1500, 96, 32
    A_np = inputs.dense_matrix(m, n, seed=31).astype(np.float32)
    A = dev_padded(A_np, torch.float32)
    Ae = host(A).astype(np.float64)
    for which, rows_r in ((jl.SK_S, n), (jl.SK_ST, m)):
        h = jl.sketch_create(kind, rows_r, d, alpha, 41, d + dd)
        try:
            out_rows = m if which == jl.SK_S else n
            O = torch.full((out_rows, d + dd), np.nan, dtype=torch.float32, device="cuda")
            kw = {"S": O} if which == jl.SK_S else {"St": O}
            jl.sketch_apply(h, A, which=which, prec=jl.SK_PREC_BF16X2, **kw)
            jl.sketch_increment(h, dd)
            jl.sketch_apply_increment(h, A, which=which, prec=jl.SK_PREC_BF16X2, **kw)
            jl.sketch_device_status(h)
        finally:
            jl.sketch_destroy(h)
        op = ops.Operator(kind, rows_r, d, alpha, 41)
        op.increment(dd)
        R = op.dense()
        want = Ae @ R if which == jl.SK_S else Ae.T @ R
        got = host(O).astype(np.float64)
        assert rel_fro(got, want) <= TOL["bf16x2"]
        bound = (np.abs(Ae) @ np.abs(R)) if which == jl.SK_S else (np.abs(Ae).T @ np.abs(R))
        assert np.all(np.abs(got - want) <= ELEM_BOUND * bound + 1e-30)


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_full_size_bf16x2_sampled_rows(kind):
    """The benchmark's n = 32768 FP32 kernel matrix (X != Y, h = 0.1), d = 256,
    SK_PREC_BF16X2 as the benchmark runs it (the SRHT S product may take the row
    FWHT, whichever route measured faster); the oracle recomputes 128 sampled
    rows of S and of S' in FP64."""
    from paper_2302_01977_gb300 import jlsketch as jl
    w = inputs.WORKLOADS["kernel_fp32_n32768"]
    n, d = w["n"], w["d"]
    X = inputs.points(n, seed=w["seed"])
    Y = inputs.points(n, seed=w["seed"] + 1000)
    A = torch.empty((n, n), dtype=torch.float32, device="cuda")
    jl.kernel_matrix(jl.generator(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), w["h"]), A)
    h = jl.sketch_create(kind, n, d, 1, w["seed"] + 3, d)
    try:
        S = torch.full((n, d), np.nan, dtype=torch.float32, device="cuda")
        St = torch.full((n, d), np.nan, dtype=torch.float32, device="cuda")
        jl.sketch_apply(h, A, jl.SK_S, jl.SK_PREC_BF16X2, S=S)
        jl.sketch_apply(h, A, jl.SK_ST, jl.SK_PREC_BF16X2, St=St)
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)
    rows = np.sort(np.random.default_rng(2).choice(n, 128, replace=False))
    R = ops.Operator(kind, n, d, 1, w["seed"] + 3).dense()
    A_rows = osk.kernel_matrix(X[rows], Y, w["h"]).astype(np.float32).astype(np.float64)
    A_cols = osk.kernel_matrix(X, Y[rows], w["h"]).T.astype(np.float32).astype(np.float64)
    assert rel_fro(host(S)[rows], A_rows @ R) <= TOL["bf16x2"]
    assert rel_fro(host(St)[rows], A_cols @ R) <= TOL["bf16x2"]
    assert torch.isfinite(S).all() and torch.isfinite(St).all()

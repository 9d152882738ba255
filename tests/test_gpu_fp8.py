"""The tcgen05 scaled-FP8 path (prec = SK_PREC_FP8) against the FP64 oracle.

FP32 data; SRHT and Gaussian operators.  Two gates per case:

* relative Frobenius error <= 2e-2 against the oracle applied to the same
  FP32 matrix widened to FP64;
* an elementwise bound.  A value a of a tile with scale s = amax / 448 is
  held as e4m3 terms y_hi + y_lo of a / s; e4m3 has three mantissa bits, so
  |a - s (y_hi + y_lo)| <= 2^-8 |a| + 2^-10 s (the second term is half the
  subnormal spacing), and likewise for z.  With the dropped y_lo w_lo term the
  kept products differ from a z by at most about 3 * 2^-8 |a z| plus those
  floors, so
      |S - S_ref| <= 0.02 (|A| |R|) + 1e-5 (max|A| |1| |R| + max|R| |A| |1|),
  while a dropped or doubled term (2^-4 relative) breaks it.
"""
import numpy as np
import pytest

from oracle import operators as ops
from oracle import sketch as osk
from paper_2302_01977_gb300 import inputs
from tests.util import dev_padded, ensure_built, host, rel_fro

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_FP8 = 2e-2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def jlmod():
    from paper_2302_01977_gb300 import jlsketch as jl
    return jl


def run(kind, A_np, which, d, seed, incs=()):
    """Sketch FP32 A with the FP8 path; returns the output and the oracle's R."""
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
        jl.sketch_apply(h, A, which=which, prec=jl.SK_PREC_FP8, **kw)
        for dd in incs:
            jl.sketch_increment(h, dd)
            jl.sketch_apply_increment(h, A, which=which, prec=jl.SK_PREC_FP8, **kw)
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
    assert err <= TOL_FP8, err
    aB, aR = np.abs(B), np.abs(R)
    bound = (0.02 * (aB @ aR) + 1e-5 * aB.max() * aR.sum(axis=0, keepdims=True)
             + 1e-5 * aR.max() * aB.sum(axis=1, keepdims=True))
    assert (np.abs(got - ref) <= bound).all()
    return err


@pytest.mark.parametrize("kind", ["srht", "gauss"])
@pytest.mark.parametrize("n,d", [(64, 16), (1000, 100), (2048, 128), (1537, 72), (777, 300)])
def test_fp8_square_both(kind, n, d):
    A = inputs.dense_matrix(n, n, seed=n + 5 * d).astype(np.float32)
    jl = jlmod()
    e1 = check(kind, A, jl.SK_S, d, 13 * n + d)
    e2 = check(kind, A, jl.SK_ST, d, 13 * n + d)
    assert max(e1, e2) < 5e-3  # the split keeps about eight significant bits


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_fp8_kernel_matrix_d512(kind):
    """A Gaussian-kernel matrix with two 256-column tiles and many tiny entries."""
    n, d = 4096, 512
    X = inputs.points(n, seed=6)
    A = osk.kernel_matrix(X, X, 0.3).astype(np.float32)
    jl = jlmod()
    check(kind, A, jl.SK_S, d, 4)
    check(kind, A, jl.SK_ST, d, 4)


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_fp8_increments_unaligned(kind):
    """Increments whose first column is 50 and 64: scalar and vector epilogues;
    earlier columns keep their quantization."""
    n = 1200
    A = inputs.dense_matrix(n, n, seed=18).astype(np.float32)
    jl = jlmod()
    check(kind, A, jl.SK_S, 50, 22, incs=(14, 33))
    check(kind, A, jl.SK_ST, 50, 22, incs=(14, 33))


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_fp8_stream_k_split(kind):
    """More 128-row tiles than SMs: CTA ranges cut tiles, two partial sums per cell."""
    rows, n, d = 20000, 1500, 64
    A = inputs.dense_matrix(rows, n, seed=19).astype(np.float32)
    jl = jlmod()
    check(kind, A, jl.SK_S, d, 5)
    check(kind, np.ascontiguousarray(A.T), jl.SK_ST, d, 5)


def test_fp8_wide_dynamic_range():
    """Rows scaled over 30 orders of magnitude: the 64 x 128 scale tiles keep
    each tile's values in e4m3's range, so the relative error stays small."""
    n, d = 1024, 64
    A = inputs.dense_matrix(n, n, seed=20)
    A *= np.logspace(-15, 15, n)[:, None]
    A = A.astype(np.float32)
    jl = jlmod()
    got, R = run("gauss", A, jl.SK_S, d, 8)
    ref = A.astype(np.float64) @ R
    # per 64-row block, the block's own relative error
    for r0 in range(0, n, 64):
        assert rel_fro(got[r0:r0 + 64], ref[r0:r0 + 64]) < 5e-3


def test_fp8_rejects_fp64_and_sjlt():
    jl = jlmod()
    A = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    S = torch.zeros((64, 16), dtype=torch.float64, device="cuda")
    h = jl.sketch_create("gauss", 64, 16, 1, 1, 16)
    try:
        with pytest.raises(jl.JLSketchError) as e:
            jl.sketch_apply(h, A, which=jl.SK_S, prec=jl.SK_PREC_FP8, S=S)
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

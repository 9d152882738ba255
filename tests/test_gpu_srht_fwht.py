"""SRHT S = A R through the row FWHT (Sec. 7.1) against the FP64 oracle.

FP32 data with nu = 2^ceil(log2 n) in [2^14, 2^16] has two routes, the FWHT
and the +-1 product; the first apply of a shape times both and keeps the
faster.  These tests check the result against the oracle (relative Frobenius
error <= 1e-5) whichever route was kept, and check that the FWHT is the one
kept where it must win by a wide margin (FP32 CUDA-core product of 4096 rows,
n = 16384, d = 256: about 34 GFLOP against one read of 268 MB).  Shapes cover
one, two and four 16384-value segments (the top bits folded in while
loading), zero padding (n not a power of two) and increments whose first
column is not a multiple of 4.  For n = k + r not a power of two, Sec. 7.1's
split (transforms of orders k and p = 2^ceil(log2 r)) is checked against the
oracle and against the zero-padded transform of the same shape, with the FWHT
route pinned (JLS_SRHT_ROUTE=fwht).
"""
import numpy as np
import pytest

from oracle import operators as ops
from paper_2302_01977_gb300 import inputs
from tests.util import TOL, dev_padded, ensure_built, host, rel_fro

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def jlmod():
    from paper_2302_01977_gb300 import jlsketch as jl
    return jl


def nu_of(n):
    return 1 << (int(n) - 1).bit_length()


def run(A_np, d, seed, prec, incs=()):
    jl = jlmod()
    rows, n = A_np.shape
    dmax = d + sum(incs)
    A = dev_padded(A_np, torch.float32)
    h = jl.sketch_create("srht", n, d, 1, seed, dmax)
    try:
        S = torch.full((rows, dmax), np.nan, dtype=torch.float32, device="cuda")
        jl.sketch_apply(h, A, which=jl.SK_S, prec=prec, S=S)
        for dd in incs:
            jl.sketch_increment(h, dd)
            jl.sketch_apply_increment(h, A, which=jl.SK_S, prec=prec, S=S)
        torch.cuda.synchronize()
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)
    op = ops.Operator("srht", n, d, 1, seed)
    for dd in incs:
        op.increment(dd)
    return host(S), op.dense()


@pytest.mark.parametrize("rows,n,d", [(4096, 16384, 256), (1000, 20000, 100), (600, 40000, 64)])
def test_fwht_native_parity(rows, n, d):
    jl = jlmod()
    A = inputs.dense_matrix(rows, n, seed=n + d).astype(np.float32)
    S, R = run(A, d, 7 + n, jl.SK_PREC_NATIVE)
    assert rel_fro(S, A.astype(np.float64) @ R) <= TOL["f32"]
    route = jl.sketch_srht_route(nu_of(n), rows, n, d, jl.SK_PREC_NATIVE)
    assert route in (0, 1)
    if (rows, n, d) == (4096, 16384, 256):
        assert route == 1


def test_fwht_bf16x2_request_parity():
    jl = jlmod()
    rows, n, d = 2048, 32768, 256
    X = inputs.points(n, seed=3)
    A = np.exp(-((X[:rows, None, :] - X[None, :, :]) ** 2).sum(-1) / (2 * 0.1 ** 2)).astype(np.float32)
    S, R = run(A, d, 11, jl.SK_PREC_BF16X2)
    assert rel_fro(S, A.astype(np.float64) @ R) <= TOL["bf16x2"]
    assert jl.sketch_srht_route(nu_of(n), rows, n, d, jl.SK_PREC_BF16X2) in (0, 1)


def test_fwht_increments_unaligned():
    jl = jlmod()
    rows, n = 700, 17000
    A = inputs.dense_matrix(rows, n, seed=5).astype(np.float32)
    S, R = run(A, 50, 13, jl.SK_PREC_NATIVE, incs=(14, 33))
    assert rel_fro(S, A.astype(np.float64) @ R) <= TOL["f32"]


def test_fwht_identity_rows_give_R():
    """Rows of the identity: S = R (each output a single +-1/sqrt(d) term)."""
    jl = jlmod()
    n, d = 16384, 32
    A = np.zeros((256, n), dtype=np.float32)
    cols = np.arange(0, n, n // 256)
    A[np.arange(256), cols] = 1.0
    S, R = run(A, d, 17, jl.SK_PREC_NATIVE)
    assert np.array_equal(S.astype(np.float64), np.float32(R[cols]).astype(np.float64))


SPLIT_SHAPES = [(512, 16384 + 3000, 256),   # k = 2^14, p = 4096
                (300, 16384 + 1, 64),       # r = 1: p = 1
                (256, 16384 + 8192, 128),   # r = 8192: the largest tail
                (200, 32768 + 5000, 100),   # k = 2^15 (two segments), p = 8192
                (256, 16384 + 8193, 64)]    # r > 8192: the zero-padded transform


@pytest.mark.parametrize("rows,n,d", SPLIT_SHAPES)
def test_fwht_split_parity(rows, n, d, monkeypatch):
    jl = jlmod()
    monkeypatch.setenv("JLS_SRHT_ROUTE", "fwht")
    A = inputs.dense_matrix(rows, n, seed=n + 1).astype(np.float32)
    S_split, R = run(A, d, 23 + n, jl.SK_PREC_NATIVE)
    ref = A.astype(np.float64) @ R
    assert rel_fro(S_split, ref) <= TOL["f32"]
    monkeypatch.setenv("JLS_SRHT_SPLIT", "0")
    S_pad, _ = run(A, d, 23 + n, jl.SK_PREC_NATIVE)
    assert rel_fro(S_pad, ref) <= TOL["f32"]
    assert rel_fro(S_split, S_pad) <= TOL["f32"]


def test_fwht_split_increments_unaligned(monkeypatch):
    jl = jlmod()
    monkeypatch.setenv("JLS_SRHT_ROUTE", "fwht")
    rows, n = 300, 16384 + 2500
    A = inputs.dense_matrix(rows, n, seed=9).astype(np.float32)
    S, R = run(A, 37, 29, jl.SK_PREC_NATIVE, incs=(10, 21))
    assert rel_fro(S, A.astype(np.float64) @ R) <= TOL["f32"]

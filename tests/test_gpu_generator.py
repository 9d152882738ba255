"""sketch_apply with a kernel generator: S = K(X, Y) R and S' = K(X, Y)^T R
without the caller forming K.

The result is compared with the oracle applied to the same K as the device
computes it (K is also formed explicitly by kernel_matrix and read back), at
the FP64 / FP32 tolerances.  Shapes with more rows (or columns, for S') than
one scratch block (20480 rows) exercise the block loop and the diagonal
shift's placement in later blocks; S' exercises K(Y, X) = K^T.
"""
import numpy as np
import pytest

from oracle import operators as ops
from paper_2302_01977_gb300 import inputs
from tests.util import TOL, dev, ensure_built, host, rel_fro

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def jlmod():
    from paper_2302_01977_gb300 import jlsketch as jl
    return jl


def explicit_K(jl, Xd, Yd, h, shift, tdt):
    K = torch.empty((Xd.shape[0], Yd.shape[0]), dtype=tdt, device="cuda")
    jl.kernel_matrix(jl.generator(Xd, Yd, h, shift), K)
    return host(K).astype(np.float64)


@pytest.mark.parametrize("kind,alpha", [("sjlt_block", 4), ("srht", 1), ("gauss", 1)])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_generator_both_small(kind, alpha, dtype):
    jl = jlmod()
    tdt = torch.float32 if dtype == "f32" else torch.float64
    npdt = np.float32 if dtype == "f32" else np.float64
    m, n, d = 700, 700, 64
    X = inputs.points(m, seed=1, dtype=npdt)
    Y = inputs.points(n, seed=2, dtype=npdt)
    Xd, Yd = dev(X), dev(Y)
    K = explicit_K(jl, Xd, Yd, 0.2, 1e-2, tdt)
    h = jl.sketch_create(kind, n, d, alpha, 5, d)
    try:
        S = torch.full((m, d), np.nan, dtype=tdt, device="cuda")
        St = torch.full((n, d), np.nan, dtype=tdt, device="cuda")
        jl.sketch_apply(h, jl.generator(Xd, Yd, 0.2, 1e-2), which=jl.SK_BOTH, S=S, St=St)
        torch.cuda.synchronize()
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)
    R = ops.Operator(kind, n, d, alpha, 5).dense()
    assert rel_fro(host(S), K @ R) <= TOL[dtype]
    assert rel_fro(host(St), K.T @ R) <= TOL[dtype]


@pytest.mark.parametrize("kind,alpha,prec", [("sjlt_block", 4, 0), ("gauss", 1, 3)])
def test_generator_several_blocks(kind, alpha, prec):
    """45000 rows: three scratch blocks for S; S' of the 600 x 45000 transpose."""
    jl = jlmod()
    m, n, d = 45000, 600, 64
    X = inputs.points(m, seed=3)
    Y = inputs.points(n, seed=4)
    Xd, Yd = dev(X), dev(Y)
    K = explicit_K(jl, Xd, Yd, 0.1, 0.5, torch.float32)  # the shift lands on rows 0..599 only
    h = jl.sketch_create(kind, n, d, alpha, 6, d)
    try:
        S = torch.full((m, d), np.nan, dtype=torch.float32, device="cuda")
        jl.sketch_apply(h, jl.generator(Xd, Yd, 0.1, 0.5), which=jl.SK_S, prec=prec, S=S)
        torch.cuda.synchronize()
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)
    R = ops.Operator(kind, n, d, alpha, 6).dense()
    assert rel_fro(host(S), K @ R) <= TOL["f32"]
    # S' of the transpose: K2 = K(Y, X) is 600 x 45000, S' = K2^T R2 has 45000 rows
    K2 = K.T
    h = jl.sketch_create(kind, n, d, alpha, 7, d)
    try:
        St = torch.full((m, d), np.nan, dtype=torch.float32, device="cuda")
        jl.sketch_apply(h, jl.generator(Yd, Xd, 0.1, 0.5), which=jl.SK_ST, prec=prec, St=St)
        torch.cuda.synchronize()
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)
    R2 = ops.Operator(kind, n, d, alpha, 7).dense()
    assert rel_fro(host(St), K2.T @ R2) <= TOL["f32"]


def test_generator_increment():
    jl = jlmod()
    m = n = 1500
    X = inputs.points(m, seed=8)
    Xd = dev(X)
    K = explicit_K(jl, Xd, Xd, 0.15, 1e-3, torch.float32)
    h = jl.sketch_create("srht", n, 40, 1, 9, 104)
    try:
        S = torch.full((m, 104), np.nan, dtype=torch.float32, device="cuda")
        g = jl.generator(Xd, Xd, 0.15, 1e-3)
        jl.sketch_apply(h, g, which=jl.SK_S, S=S)
        jl.sketch_increment(h, 64)
        jl.sketch_apply_increment(h, g, which=jl.SK_S, S=S)
        torch.cuda.synchronize()
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)
    op = ops.Operator("srht", n, 40, 1, 9)
    op.increment(64)
    assert rel_fro(host(S), K @ op.dense()) <= TOL["f32"]

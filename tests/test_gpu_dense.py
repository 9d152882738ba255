"""SRHT and Gaussian sketches on the GPU against the FP64 oracle.

CUDA-core path (FP64, FP32) and, when built, the tcgen05 bf16 hi+lo split
path (FP32 data).  Tolerances: 1e-12 FP64, 1e-5 FP32 and bf16x2 (relative
Frobenius), against the oracle applied to the same matrix widened to FP64.
"""
import numpy as np
import pytest

from oracle import operators as ops
from oracle import sketch as osk
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


def sketch(kind, A_np, d, seed, dtype, prec=0, incs=(), which=3):
    jl = jlmod()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    m, n = A_np.shape
    A = dev_padded(A_np, tdt)
    dmax = d + sum(incs)
    h = jl.sketch_create(kind, n, d, 1, seed, dmax)
    try:
        S = torch.full((m, dmax), np.nan, dtype=tdt, device="cuda")
        St = torch.full((n, dmax), np.nan, dtype=tdt, device="cuda")
        Sa = S if which & 1 else None
        Sta = St if which & 2 else None
        jl.sketch_apply(h, A, which=which, prec=prec, S=Sa, St=Sta)
        for dd in incs:
            jl.sketch_increment(h, dd)
            jl.sketch_apply_increment(h, A, which=which, prec=prec, S=Sa, St=Sta)
        torch.cuda.synchronize()
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)
    return host(S), host(St)


@pytest.mark.parametrize("kind", ["srht", "gauss"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,d", [(64, 16), (1000, 100), (2048, 128), (1537, 72)])
def test_dense_native_parity(kind, dtype, n, d):
    A = inputs.dense_matrix(n, n, seed=n + 3 * d)
    if dtype == "f32":
        A = A.astype(np.float32)
    seed = 31 * n + d
    S, St = sketch(kind, A, d, seed, dtype)
    R = ops.Operator(kind, n, d, 1, seed).dense()
    S0, St0 = osk.apply(A.astype(np.float64), R)
    assert rel_fro(S, S0) <= TOL[dtype]
    assert rel_fro(St, St0) <= TOL[dtype]


@pytest.mark.parametrize("kind", ["srht", "gauss"])
def test_dense_increments(kind):
    n, d0, incs = 900, 48, (16, 32)
    A = inputs.dense_matrix(n, n, seed=4)
    S, St = sketch(kind, A, d0, 17, "f64", incs=incs)
    op = ops.Operator(kind, n, d0, 1, 17)
    for dd in incs:
        op.increment(dd)
    S0, St0 = osk.apply(A, op.dense())
    assert rel_fro(S, S0) <= TOL["f64"]
    assert rel_fro(St, St0) <= TOL["f64"]


def test_srht_matches_fwht_route():
    """The element-formula sketch equals the transform of the padded rows (Sec. 7.1)."""
    n, d = 1000, 64
    A = inputs.dense_matrix(50, n, seed=2)
    S, _ = sketch("srht", A, d, 5, "f64", which=1)
    op = ops.Operator("srht", n, d, 1, 5)
    ref = osk.srht_by_fwht(A, op.srht_diag(), op.srht_samples(), d)
    assert rel_fro(S, ref) <= TOL["f64"]


def test_gauss_fp32_plane_values():
    """A = I gives S = R: the FP32 Gaussian plane (Box-Muller with FP32
    transcendentals) matches the FP64 draw of the oracle to a few FP32 ulps."""
    n, d = 4096, 64
    A = np.eye(n, dtype=np.float32)
    S, _ = sketch("gauss", A, d, 77, "f32", which=1)
    R = ops.Operator("gauss", n, d, 1, 77).dense()
    assert np.max(np.abs(S[:, :d] - R)) <= 1e-6 * np.max(np.abs(R))

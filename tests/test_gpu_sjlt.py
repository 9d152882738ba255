"""SJLT sketches on the GPU against the FP64 oracle (Sec. 6.3).

Tolerances (relative Frobenius error): 1e-12 for FP64, 1e-5 for FP32.  FP32
cases compare against the oracle applied to the same FP32 matrix widened to
FP64.  Sizes span several tiles (512 rows of R per FP32 tile, 256 per FP64
tile) with ragged tails, and the full n = 32768 workload is checked on sampled
rows that the oracle computes one by one.
"""
import numpy as np
import pytest

from oracle import operators as ops
from oracle import sketch as osk
from paper_2302_01977_gb300 import inputs
from tests.util import TOL, dev, dev_padded, ensure_built, host, rel_fro

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def jlmod():
    from paper_2302_01977_gb300 import jlsketch as jl
    return jl


def run_apply(kind, A_np, d, alpha, seed, dtype, which=3, incs=(), ld_pad=0, s_pad=0):
    """Sketch A_np on the GPU (explicit matrix) after the given increments."""
    jl = jlmod()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    m, n = A_np.shape
    A = dev_padded(np.pad(A_np, ((0, 0), (0, ld_pad))), tdt)[:, :n]
    dmax = d + sum(incs)
    h = jl.sketch_create(kind, n if which & 1 else m, d, alpha, seed, dmax)
    try:
        for dd in incs:
            jl.sketch_increment(h, dd)
        S = torch.full((m, dmax + s_pad), np.nan, dtype=tdt, device="cuda")
        St = torch.full((n, dmax + s_pad), np.nan, dtype=tdt, device="cuda")
        jl.sketch_apply(h, A, which=which, S=S if which & 1 else None, St=St if which & 2 else None)
        torch.cuda.synchronize()
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)
    return host(S[:, :dmax]), host(St[:, :dmax])


@pytest.mark.parametrize("kind", ["sjlt_block", "sjlt_graph"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,d,alpha", [(64, 16, 4), (1000, 128, 4), (1537, 200, 8), (2048, 64, 1), (700, 512, 4)])
def test_sjlt_parity(kind, dtype, n, d, alpha):
    if kind == "sjlt_block" and d % alpha:
        pytest.skip("block construction needs alpha | d")
    A = inputs.dense_matrix(n, n, seed=n + d)
    if dtype == "f32":
        A = A.astype(np.float32)
    seed = 7 * n + d
    S, St = run_apply(kind, A, d, alpha, seed, dtype)
    R = ops.Operator(kind, n, d, alpha, seed).dense()
    S0, St0 = osk.apply(A.astype(np.float64), R)
    assert rel_fro(S, S0) <= TOL[dtype]
    assert rel_fro(St, St0) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_identity_returns_R_exactly(dtype):
    n, d, alpha = 600, 64, 4
    S, St = run_apply("sjlt_block", np.eye(n), d, alpha, 3, dtype)
    R = ops.Operator("sjlt_block", n, d, alpha, 3).dense()
    Rc = R.astype(np.float32).astype(np.float64) if dtype == "f32" else R
    assert np.array_equal(S, Rc) and np.array_equal(St, Rc)


@pytest.mark.parametrize("which", [1, 2])
def test_rectangular_and_padded(which):
    """S = A R with A m x n (m != n) and S' = A^T R with A n x m; padded lds."""
    n, m, d, alpha = 900, 333, 96, 4
    A = inputs.dense_matrix(m, n, seed=5) if which == 1 else inputs.dense_matrix(n, m, seed=5)
    S, St = run_apply("sjlt_block", A, d, alpha, 11, "f64", which=which, ld_pad=12, s_pad=5)
    R = ops.Operator("sjlt_block", n, d, alpha, 11).dense()
    if which == 1:
        assert rel_fro(S, A @ R) <= TOL["f64"]
    else:
        assert rel_fro(St, A.T @ R) <= TOL["f64"]


@pytest.mark.parametrize("kind", ["sjlt_block", "sjlt_graph"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_increments_match_grown_operator(kind, dtype):
    """apply, then increment + apply_increment twice == oracle S of the grown R."""
    jl = jlmod()
    n, d0, dd, alpha, seed = 1101, 64, 32, 4, 99
    tdt = torch.float64 if dtype == "f64" else torch.float32
    A_np = inputs.dense_matrix(n, n, seed=8)
    if dtype == "f32":
        A_np = A_np.astype(np.float32)
    A = dev_padded(A_np, tdt)
    h = jl.sketch_create(kind, n, d0, alpha, seed, d0 + 2 * dd)
    op = ops.Operator(kind, n, d0, alpha, seed)
    try:
        S = torch.zeros((n, d0 + 2 * dd), dtype=tdt, device="cuda")
        St = torch.zeros_like(S)
        jl.sketch_apply(h, A, S=S, St=St)
        for _ in range(2):
            jl.sketch_increment(h, dd)
            op.increment(dd)
            jl.sketch_apply_increment(h, A, S=S, St=St)
            w = op.d_total
            S0, St0 = osk.apply(A_np.astype(np.float64), op.dense())
            assert rel_fro(host(S[:, :w]), S0) <= TOL[dtype]
            assert rel_fro(host(St[:, :w]), St0) <= TOL[dtype]
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)


def test_kernel_matrix_fp64_n2048_graph_sjlt():
    """The FP64 workload: 2048 bisection-ordered points, h = 0.2, shift 1e-2,
    graph SJLT d = 128, alpha = 4; full S and S' against the oracle."""
    jl = jlmod()
    w = inputs.WORKLOADS["sjlt_fp64_n2048"]
    P = inputs.points(w["n"], seed=w["seed"], dtype=np.float64)
    P = P[inputs.bisection_order(P, leaf=w["leaf"])]
    Pd = dev(P)
    n = w["n"]
    A = torch.empty((n, n), dtype=torch.float64, device="cuda")
    jl.kernel_matrix(jl.generator(Pd, Pd, w["h"], w["shift"]), A)
    S, St = run_apply("sjlt_graph", host(A), w["d"], w["alpha"], w["seed"], "f64")
    A0 = osk.kernel_matrix(P, P, w["h"], w["shift"])
    R = ops.Operator("sjlt_graph", n, w["d"], w["alpha"], w["seed"]).dense()
    S0, St0 = osk.apply(A0, R)
    assert rel_fro(S, S0) <= TOL["f64"]
    assert rel_fro(St, St0) <= TOL["f64"]
    assert rel_fro(St, S) <= TOL["f64"]  # symmetric A


def test_full_size_fp32_sampled_rows():
    """n = 32768 FP32 kernel matrix (X != Y, h = 0.1), block SJLT d = 256,
    alpha = 4, in the launch configuration the benchmark times; the oracle
    recomputes 192 sampled rows of S and of S' in FP64."""
    jl = jlmod()
    w = inputs.WORKLOADS["kernel_fp32_n32768"]
    n, d, alpha = w["n"], w["d"], w["alpha"]
    X = inputs.points(n, seed=w["seed"])
    Y = inputs.points(n, seed=w["seed"] + 1000)
    A = torch.empty((n, n), dtype=torch.float32, device="cuda")
    jl.kernel_matrix(jl.generator(dev(X), dev(Y), w["h"]), A)
    h = jl.sketch_create("sjlt_block", n, d, alpha, w["seed"], d)
    try:
        S = torch.empty((n, d), dtype=torch.float32, device="cuda")
        St = torch.empty_like(S)
        jl.sketch_apply(h, A, S=S, St=St)
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(n, 192, replace=False))
    R = ops.Operator("sjlt_block", n, d, alpha, w["seed"]).dense()
    A_rows = osk.kernel_matrix(X[rows], Y, w["h"])            # rows of A
    A_cols = osk.kernel_matrix(X, Y[rows], w["h"]).T          # rows of A^T
    assert rel_fro(host(S)[rows], A_rows @ R) <= TOL["f32"]
    assert rel_fro(host(St)[rows], A_cols @ R) <= TOL["f32"]
    # every row is finite (no tile left unwritten)
    assert np.isfinite(host(S)).all() and np.isfinite(host(St)).all()


def test_unaligned_leading_dimension_rejected():
    """TMA needs 16-byte row pitches: an odd FP32 leading dimension is refused."""
    jl = jlmod()
    n = 129
    A = dev(np.ones((n, n), dtype=np.float32))  # ld = 129 floats = 516 bytes
    h = jl.sketch_create("sjlt_block", n, 16, 4, 1, 16)
    try:
        S = torch.zeros((n, 16), dtype=torch.float32, device="cuda")
        with pytest.raises(jl.JLSketchError) as e:
            jl.sketch_apply(h, A, which=1, S=S)
        assert e.value.status == jl.SK_ERR_ALIGN
    finally:
        jl.sketch_destroy(h)

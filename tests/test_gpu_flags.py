"""The creation flags on the GPU against the oracle.

SK_SCALE_BLOCK: every block of R keeps the scale of a JL operator of its own
width (Algorithm 1 appends an independent JL(Delta-d)); the sketch of the
grown operator, built by sketch_apply and sketch_apply_increment, must equal
the oracle's A R and A^T R with oracle.operators.Operator(scale="block"), and
the exported R its dense R.  SK_SRHT_REPLACE: SRHT columns sampled with
replacement (Sec. 2.4.2); the sampled indices must equal the oracle's bit for
bit (more than nu of them, repeats included) and the sketches its products.
Tolerances as elsewhere: 1e-12 (FP64), 1e-5 (FP32, bf16 split) relative
Frobenius.
"""
import numpy as np
import pytest

from oracle import adaptive as oad
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


BLOCK_CASES = [(k, a, "native", dt) for k, a in (("sjlt_block", 4), ("sjlt_graph", 3), ("srht", 1), ("gauss", 1))
               for dt in ("f64", "f32")] + [("srht", 1, "bf16x2", "f32"), ("gauss", 1, "bf16x2", "f32")]


@pytest.mark.parametrize("kind,alpha,prec,dtype", BLOCK_CASES)
def test_block_scale_apply_and_increments(kind, alpha, prec, dtype):
    jl = jlmod()
    m, n, d0, incs = 700, 1500, 48, [24, 24]
    A_np = inputs.dense_matrix(m, n, seed=3)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    A = dev_padded(A_np, tdt)
    Ae = host(A).astype(np.float64)  # A as the device holds it
    p = jl.SK_PREC_BF16X2 if prec == "bf16x2" else jl.SK_PREC_NATIVE
    d_max = d0 + sum(incs)
    seed = 91
    with jl.Sketch(kind, n, d0, alpha, seed, d_max=d_max, flags=jl.SK_SCALE_BLOCK) as op:
        S = torch.zeros((m, d_max), dtype=tdt, device="cuda")
        jl.sketch_apply(op.h, A, jl.SK_S, p, S=S)
        ref = ops.Operator(kind, n, d0, alpha, seed, scale="block")
        for dd in incs:
            jl.sketch_increment(op.h, dd)
            jl.sketch_apply_increment(op.h, A, jl.SK_S, p, S=S)
            ref.increment(dd)
        jl.sketch_device_status(op.h)
        R = ref.dense()
        got_R = jl.sketch_export(op.h, dense=True)["R"]
    if kind == "gauss":  # values through log and sincos: equal to rounding (1e-12 of max |R|)
        assert np.abs(got_R - R).max() <= 1e-12 * np.abs(R).max()
    else:
        assert np.array_equal(got_R, R)
    want = Ae @ R
    tol = TOL[dtype] if prec == "native" else TOL["bf16x2"]
    assert rel_fro(host(S), want) <= tol


@pytest.mark.parametrize("kind,alpha", [("sjlt_block", 4), ("srht", 1), ("gauss", 1)])
def test_block_scale_transpose_and_relative_test(kind, alpha):
    """S' = A^T R with block scale, and the stopping test on it: the relative
    test is scale-free per block, so its ratio equals the oracle's on the
    block-scaled sketch."""
    jl = jlmod()
    n, d0, dd = 900, 32, 16
    A_np = inputs.spectrum_matrix(n, 0.8 ** np.arange(n), seed=4)
    A = dev_padded(A_np, torch.float64)
    with jl.Sketch(kind, n, d0 + dd, alpha, 7, d_max=d0 + 2 * dd, flags=jl.SK_SCALE_BLOCK) as op:
        St = torch.zeros((n, d0 + 2 * dd), dtype=torch.float64, device="cuda")
        jl.sketch_apply(op.h, A, jl.SK_ST, jl.SK_PREC_NATIVE, St=St)
        jl.sketch_increment(op.h, dd)
        jl.sketch_apply_increment(op.h, A, jl.SK_ST, jl.SK_PREC_NATIVE, St=St)
        stop, nh, nt = jl.adaptive_norm_test(op.h, 1, St, dd, 1e-3, 0.0)
        jl.sketch_device_status(op.h)
    ref = ops.Operator(kind, n, d0 + dd, alpha, 7, scale="block")
    ref.increment(dd)
    want = osk.apply_t(A_np, ref.dense())
    assert rel_fro(host(St), want) <= 1e-12
    _, nh0, nt0 = oad.norm_test(want, d0 + dd, dd, 1e-3, 0.0)
    assert abs(nt - nt0) <= 1e-9 * nt0 and abs(nh - nh0) <= 1e-9 * nt0


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_srht_with_replacement(dtype):
    jl = jlmod()
    n, d, dd = 1000, 1100, 64  # nu = 1024 < d: only with replacement
    A_np = inputs.dense_matrix(300, n, seed=8)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    A = dev_padded(A_np, tdt)
    Ae = host(A).astype(np.float64)
    with jl.Sketch("srht", n, d, 1, 55, d_max=d + dd, flags=jl.SK_SRHT_REPLACE) as op:
        S = torch.zeros((300, d + dd), dtype=tdt, device="cuda")
        jl.sketch_apply(op.h, A, jl.SK_S, jl.SK_PREC_NATIVE, S=S)
        jl.sketch_increment(op.h, dd)
        jl.sketch_apply_increment(op.h, A, jl.SK_S, jl.SK_PREC_NATIVE, S=S)
        jl.sketch_device_status(op.h)
        ex = jl.sketch_export(op.h, dense=True)
    ref = ops.Operator("srht", n, d, 1, 55, replace=True)
    ref.increment(dd)
    mu = ref.srht_samples()
    assert np.array_equal(ex["mu"].astype(np.int64), mu)
    assert np.array_equal(ex["diag"].astype(np.int64), ref.srht_diag().astype(np.int64))
    assert len(set(mu.tolist())) < mu.size  # repeats are kept
    R = ref.dense()
    assert np.array_equal(ex["R"], R)
    assert rel_fro(host(S), Ae @ R) <= TOL[dtype]


def test_flags_argument_checks():
    jl = jlmod()
    with pytest.raises(jl.JLSketchError):
        jl.sketch_create("gauss", 64, 16, flags=jl.SK_SRHT_REPLACE)  # SRHT only
    with pytest.raises(jl.JLSketchError):
        jl.sketch_create("srht", 64, 16, flags=8)  # unknown bit
    with pytest.raises(jl.JLSketchError):
        jl.sketch_create("srht", 64, 80)  # without replacement d <= nu
    h = jl.sketch_create("srht", 64, 80, flags=jl.SK_SRHT_REPLACE)
    jl.sketch_destroy(h)

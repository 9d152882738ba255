"""Operator generation on the GPU against the oracle (bit-exact integers).

SJLT column/sign arrays, SRHT signs and sampled columns must equal the
oracle's exactly (same Philox streams, independently implemented); the dense
R the kernels use must equal the oracle's R (exactly for SJLT/SRHT in FP64,
to 1e-12 for the Gaussian values, whose log/sincos differ between libm and
CUDA by rounding only).
"""
import numpy as np
import pytest

from oracle import operators as ops
from tests.util import ensure_built

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def jlmod():
    from paper_2302_01977_gb300 import jlsketch as jl
    return jl


CASES = [
    ("sjlt_block", 64, 16, 4, [8]),
    ("sjlt_block", 1000, 128, 4, [64, 64]),
    ("sjlt_block", 32768, 256, 4, []),
    ("sjlt_block", 777, 48, 8, [16]),
    ("sjlt_graph", 2048, 128, 4, [32]),
    ("sjlt_graph", 513, 7, 7, [9]),
    ("sjlt_graph", 300, 64, 1, []),
    ("srht", 64, 16, 1, [8, 8]),
    ("srht", 1000, 100, 1, [50]),
    ("srht", 32768, 256, 1, [64]),
    ("gauss", 257, 33, 1, [7]),
    ("gauss", 64, 16, 1, []),
]


@pytest.mark.parametrize("kind,n,d,alpha,incs", CASES)
def test_operator_arrays_bit_exact(kind, n, d, alpha, incs):
    jl = jlmod()
    seed = 20230203 + n + d
    dmax = d + sum(incs)
    h = jl.sketch_create(kind, n, d, alpha, seed, dmax)
    op = ops.Operator(kind, n, d, alpha, seed)
    try:
        for dd in incs:
            jl.sketch_increment(h, dd)
            op.increment(dd)
        dims = jl.sketch_dims(h)
        assert dims["d_total"] == op.d_total and dims["blocks"] == len(op.blocks)
        ex = jl.sketch_export(h, dense=n * dmax <= 2_000_000)
        if kind.startswith("sjlt"):
            cols, signs = op.sjlt_entries()
            assert np.array_equal(ex["cols"], cols)
            assert np.array_equal(ex["signs"], signs)
        if kind == "srht":
            assert np.array_equal(ex["diag"], op.srht_diag())
            assert np.array_equal(ex["mu"], op.srht_samples())
        if "R" in ex:
            R = op.dense()
            if kind == "gauss":
                assert np.max(np.abs(ex["R"] - R)) <= 1e-12 * np.max(np.abs(R))
            else:
                assert np.array_equal(ex["R"], R)
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)


def test_increment_limits():
    jl = jlmod()
    h = jl.sketch_create("sjlt_block", 128, 16, 4, 1, 24)
    try:
        with pytest.raises(jl.JLSketchError) as e:
            jl.sketch_increment(h, 12)  # 28 > d_max
        assert e.value.status == jl.SK_ERR_D_MAX
        with pytest.raises(jl.JLSketchError) as e:
            jl.sketch_increment(h, 6)  # alpha does not divide
        assert e.value.status == jl.SK_ERR_INVALID_ARG
        jl.sketch_increment(h, 8)
        assert jl.sketch_dims(h)["d_total"] == 24
    finally:
        jl.sketch_destroy(h)

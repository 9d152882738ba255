"""Adaptive increments and the stopping test on the GPU against the oracle.

The oracle recomputes S = A R for the grown operator and tests with a
Householder QR basis; the GPU rescales old columns, sketches only the new ones
and keeps an incrementally orthonormalised basis.  The norms ||S^||_F and
||S~||_F must agree (FP64: 1e-9 of ||S~||; FP32: 1e-5 of ||S~||) and the loop
must take the same decisions where the ratio is not within that margin of
eps_rel.
"""
import numpy as np
import pytest

from oracle import adaptive as oad
from paper_2302_01977_gb300 import inputs
from tests.util import dev_padded, ensure_built, same_s_check

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def gpu_loop(A_np, dtype, **kw):
    from paper_2302_01977_gb300 import jlsketch as jl
    from paper_2302_01977_gb300.adaptive import adaptive_sketch
    tdt = torch.float64 if dtype == "f64" else torch.float32
    res = adaptive_sketch(dev_padded(A_np, tdt), **kw)
    try:
        jl.sketch_device_status(res["handle"])
    finally:
        jl.sketch_destroy(res["handle"])
    return res


KINDS = [("sjlt_block", 4), ("sjlt_graph", 4), ("srht", 1), ("gauss", 1)]


@pytest.mark.parametrize("kind,alpha", KINDS)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_loop_matches_oracle(kind, alpha, dtype):
    n = 600
    sigma = 0.8 ** np.arange(n)
    A = inputs.spectrum_matrix(n, sigma, seed=3)
    if dtype == "f32":
        A = A.astype(np.float32)
    kw = dict(kind=kind, d0=16, dd=16, alpha=alpha, seed=4, d_max=160, eps_rel=1e-4, eps_abs=1e-300)
    res = gpu_loop(A, dtype, **kw)
    ref = oad.adaptive(A.astype(np.float64), kw["kind"], kw["d0"], kw["dd"], alpha, kw["seed"], kw["d_max"],
                       kw["eps_rel"], kw["eps_abs"])
    tol = 1e-9 if dtype == "f64" else 1e-5
    steps = min(len(res["history"]), len(ref["history"]))
    for k in range(steps):
        d, stop, nh, nt, nht, ntt = res["history"][k]
        d0, stop0, nh0, nt0, nht0, ntt0 = ref["history"][k]
        assert d == d0
        assert abs(nt - nt0) <= tol * nt0 and abs(ntt - ntt0) <= tol * ntt0
        assert abs(nh - nh0) <= tol * nt0 and abs(nht - nht0) <= tol * ntt0
        near = min(abs(nh0 / nt0 - kw["eps_rel"]), abs(nht0 / ntt0 - kw["eps_rel"])) <= 2 * tol
        if not near:
            assert stop == stop0
        else:
            break
    else:
        assert len(res["history"]) == len(ref["history"])
        assert res["converged"] == ref["converged"]


@pytest.mark.parametrize("kind,alpha", KINDS)
def test_low_rank_stops_at_first_test(kind, alpha):
    n, r = 512, 10
    A = inputs.low_rank_matrix(n, r, seed=9)
    res = gpu_loop(A, "f64", kind=kind, d0=32, dd=16, alpha=alpha, seed=2, d_max=96, eps_rel=1e-8,
                   eps_abs=1e-300)
    assert res["converged"] and len(res["history"]) == 1
    d, stop, nh, nt, nht, ntt = res["history"][0]
    assert nh < 1e-11 * nt and nht < 1e-11 * ntt


def test_flat_spectrum_runs_to_d_max():
    n = 400
    A = inputs.spectrum_matrix(n, np.ones(n), seed=7)
    res = gpu_loop(A, "f64", kind="gauss", d0=16, dd=16, alpha=1, seed=8, d_max=64, eps_rel=1e-6,
                   eps_abs=1e-300)
    assert not res["converged"] and res["d"] == 64
    assert [hh[0] for hh in res["history"]] == [16, 32, 48]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_pair_equals_two_single_tests(dtype):
    """adaptive_norm_test_pair (S and S' on two streams) returns what two
    adaptive_norm_test calls return, increment after increment (same kernels,
    same order of sums: equal to the last bit)."""
    from paper_2302_01977_gb300 import jlsketch as jl
    n, d0, dd, d_max = 640, 32, 32, 192
    A = inputs.spectrum_matrix(n, 0.9 ** np.arange(n), seed=12)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Ad = dev_padded(A.astype(np.float64), tdt)
    outs = []
    for pair in (True, False):
        h = jl.sketch_create("sjlt_block", n, d0 + dd, 4, 21, d_max)
        try:
            S = torch.zeros((n, d_max), dtype=tdt, device="cuda")
            St = torch.zeros((n, d_max), dtype=tdt, device="cuda")
            jl.sketch_apply(h, Ad, jl.SK_BOTH, 0, S=S, St=St)
            res, w = [], d0 + dd
            while w <= d_max:
                if pair:
                    r = jl.adaptive_norm_test_pair(h, S[:, :w], St[:, :w], dd, 1e-12, 0.0)
                else:
                    r = (jl.adaptive_norm_test(h, 0, S[:, :w], dd, 1e-12, 0.0),
                         jl.adaptive_norm_test(h, 1, St[:, :w], dd, 1e-12, 0.0))
                res.append(r)
                if w + dd > d_max:
                    break
                jl.sketch_increment(h, dd)
                jl.sketch_apply_increment(h, Ad, jl.SK_BOTH, 0, S=S, St=St)
                w += dd
            jl.sketch_device_status(h)
            outs.append(res)
        finally:
            jl.sketch_destroy(h)
    assert len(outs[0]) == len(outs[1]) == 5
    assert outs[0] == outs[1]


@pytest.mark.parametrize("kind,alpha", [("sjlt_block", 4), ("gauss", 1)])
def test_tight_tolerance_decisions_on_the_device_sketch(kind, alpha):
    """eps_rel = 1e-6 on an FP32 kernel matrix (X != Y): every test of S and of
    S' against the FP64 test on the sketch as the device held it at that test
    (a copy taken after each test), decisions outside a 1 % band around
    eps_rel, ratios within 1 % plus the device arithmetic's resolution."""
    from paper_2302_01977_gb300 import jlsketch as jl
    n, d0, dd, d_max, eps = 2048, 64, 32, 448, 1e-6
    X = torch.from_numpy(inputs.points(n, seed=31)).cuda()
    Y = torch.from_numpy(inputs.points(n, seed=32)).cuda()
    A = torch.empty((n, n), dtype=torch.float32, device="cuda")
    jl.kernel_matrix(jl.generator(X, Y, 0.3), A)
    h = jl.sketch_create(kind, n, d0 + dd, alpha, 41, d_max)
    snaps, stopped = [], False
    try:
        S = torch.zeros((n, d_max), device="cuda")
        St = torch.zeros((n, d_max), device="cuda")
        jl.sketch_apply(h, A, jl.SK_BOTH, jl.SK_PREC_NATIVE, S=S, St=St)
        w = d0 + dd
        while True:
            rs, rt = jl.adaptive_norm_test_pair(h, S[:, :w], St[:, :w], dd, eps, 0.0)
            snaps.append((w, S[:, :w].double().cpu().numpy(), St[:, :w].double().cpu().numpy(), rs, rt))
            if (rs[0] and rt[0]) or w + dd > d_max:
                stopped = rs[0] and rt[0]
                break
            jl.sketch_increment(h, dd)
            jl.sketch_apply_increment(h, A, jl.SK_BOTH, jl.SK_PREC_NATIVE, S=S, St=St)
            w += dd
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)
    assert stopped  # this kernel converges within d_max
    for w, Sn, Stn, rs, rt in snaps:
        same_s_check(Sn, [(w - dd, rs[0], rs[1], rs[2])], dd, eps, what=("S", w))
        same_s_check(Stn, [(w - dd, rt[0], rt[1], rt[2])], dd, eps, what=("St", w))

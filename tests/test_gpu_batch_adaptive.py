"""Algorithm 1's adaptive loop for every instance of a batch, run on the device
(sketch, stopping test of Eq. (3.1), decision, renumbering; no host round
trips), against the FP64 oracle loop instance by instance.

For instance i the oracle runs oracle.adaptive on A_i^T (so its S is S'_i =
A_i^T R_i) with the same operator (same seed, JL(d0 + dd) grown by dd).  The
GPU must take the same decisions (where the oracle's ratio ||S^||/||S~|| is not
within the FP32 margin of eps_rel), reach the same width, report the last
test's norms within 1e-5 of ||S~||_F, and leave S'_i[:, :d] equal to the
oracle's final sketch within 1e-5 (relative Frobenius).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adaptive as oad  # noqa: E402
from oracle import operators as ops  # noqa: E402
from paper_2302_01977_gb300 import inputs  # noqa: E402
from paper_2302_01977_gb300 import jlsketch as jl  # noqa: E402
from tests.util import ensure_built  # noqa: E402
from tests.util import batch_same_s as util_batch_same_s  # noqa: E402

pytestmark = pytest.mark.gpu

SENTINEL = 12345.0
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def make(specs, dd, seed):
    """specs: (kind, n, d0, alpha, increments, h, amplitude); square nonsymmetric
    A_i = amplitude * K(Y_i, X_i; h), so S'_i = A_i^T R_i differs from A_i R_i."""
    out = []
    for k, (kind, n, d0, alpha, incs, h, amp) in enumerate(specs):
        X = torch.from_numpy(inputs.points(n, seed=seed + 2 * k)).cuda()
        Y = torch.from_numpy(inputs.points(n, seed=seed + 2 * k + 1)).cuda()
        A = torch.empty((n, n), device="cuda")
        jl.kernel_matrix(jl.generator(Y, X, h), A)
        A *= amp
        d_max = d0 + (incs + 1) * dd
        op = jl.Sketch(kind, n, d0 + dd, alpha, 500 + k, d_max=d_max)
        for _ in range(incs):
            jl.sketch_increment(op.h, dd)
        St = torch.full((n, d_max), SENTINEL, device="cuda")
        out.append(dict(kind=kind, n=n, d0=d0, alpha=alpha, d_max=d_max, op=op, A=A, St=St, seed=500 + k))
    return out


def oracle_loop(x, dd, eps_rel, eps_abs):
    At = x["A"].double().cpu().numpy().T.copy()
    return oad.adaptive(At, x["kind"], x["d0"], dd, x["alpha"], x["seed"], x["d_max"], eps_rel, eps_abs,
                        which="S")


def compare(inst, res, dd, eps_rel, eps_abs, max_rounds=None):
    for i, x in enumerate(inst):
        ref = oracle_loop(x, dd, eps_rel, eps_abs)
        hist = ref["history"]
        if max_rounds is not None and len(hist) > max_rounds:
            hist = hist[:max_rounds]
            state_ref = 0
        else:
            state_ref = 1 if ref["converged"] else 2
        # decisions are compared up to the first test that sits within the FP32 margin of
        # a threshold (eps_rel of the ratio, or eps_abs of ||S^||)
        near = [h[3] > 0 and (abs(h[2] / h[3] - eps_rel) <= 2 * TOL or abs(h[2] - eps_abs) <= 2 * TOL * h[3])
                for h in hist]
        if any(near):
            assert res["tests"][i] >= near.index(True) + 1, (i, res["tests"][i], near)
            continue
        assert res["tests"][i] == len(hist), (i, res["tests"][i], len(hist))
        assert res["state"][i] == state_ref, (i, res["state"][i], state_ref)
        d_last = hist[-1][0] + dd
        assert res["d"][i] == d_last, (i, res["d"][i], d_last)
        nh0, nt0 = hist[-1][2], hist[-1][3]
        assert abs(res["nt"][i] - nt0) <= TOL * nt0, (i, res["nt"][i], nt0)
        assert abs(res["nh"][i] - nh0) <= TOL * nt0, (i, res["nh"][i], nh0, nt0)
        # the sketch the loop leaves: S'_i[:, :d] at the scale of R_i[:, :d]
        d = int(res["d"][i])
        if max_rounds is None or state_ref != 0:
            got = x["St"][:, :d].double().cpu().numpy()
            want = ref["S"][:, :d]
            err = np.linalg.norm(got - want) / np.linalg.norm(want)
            assert err <= TOL, (i, err)
        # columns past what the loop (and the tuner's runs) wrote are untouched
        rest = x["St"][:, max(d, x["d0"] + 2 * dd):].cpu().numpy()
        assert np.all(rest == SENTINEL)


SPECS_32 = [("sjlt_block", 256, 64, 4, 4, 0.5, 1.0),    # smooth: stops at once
            ("sjlt_block", 448, 32, 4, 5, 0.12, 1.0),
            ("sjlt_graph", 1000, 64, 3, 4, 0.08, 1.0),  # rows not a multiple of 16 per CTA
            ("sjlt_block", 2048, 128, 4, 3, 0.2, 1.0),
            ("sjlt_block", 132, 0, 2, 2, 0.3, 1.0),     # d0 = 0: the first test has no basis
            ("sjlt_block", 512, 96, 4, 2, 0.03, 1.0),   # rough kernel: runs out of increments
            ("sjlt_block", 640, 64, 4, 3, 0.3, 1e-9)]   # tiny entries: the absolute test stops it


@pytest.mark.parametrize("eps_rel", [1e-2, 1e-4])
def test_adaptive_batch_matches_oracle(eps_rel):
    dd, eps_abs = 32, 1e-7
    inst = make(SPECS_32, dd, seed=41)
    items = [(x["op"].h, x["A"], x["St"], 0, x["d0"] + dd) for x in inst]
    with jl.Batch(items) as B:
        B.adaptive_setup([x["d0"] for x in inst], dd, eps_rel, eps_abs)
        for x in inst:  # the tuner's runs wrote the first two ranges: start from the sentinel again
            x["St"].fill_(SENTINEL)
        B.adaptive_run()
        res = B.adaptive_result()
    compare(inst, res, dd, eps_rel, eps_abs)
    for x in inst:
        x["op"].close()


def test_adaptive_batch_small_increments_and_round_limit():
    dd, eps_rel, eps_abs = 16, 1e-3, 0.0
    specs = [("sjlt_block", 300, 8, 4, 6, 0.1, 1.0), ("sjlt_graph", 784, 48, 4, 6, 0.15, 1.0),
             ("sjlt_block", 1200, 16, 4, 6, 0.25, 1.0),
             ("sjlt_block", 272, 16, 4, 0, 0.05, 1.0)]  # no increment: one test, then out of columns
    inst = make(specs, dd, seed=77)
    items = [(x["op"].h, x["A"], x["St"], 0, x["d0"] + dd) for x in inst]
    with jl.Batch(items) as B:
        B.adaptive_setup([x["d0"] for x in inst], dd, eps_rel, eps_abs)
        for x in inst:
            x["St"].fill_(SENTINEL)
        B.adaptive_run(max_rounds=2)
        res2 = B.adaptive_result()
        compare(inst, res2, dd, eps_rel, eps_abs, max_rounds=2)
        for x in inst:
            x["St"].fill_(SENTINEL)
        B.adaptive_run()
        res = B.adaptive_result()
        compare(inst, res, dd, eps_rel, eps_abs)
    for x in inst:
        x["op"].close()


def test_adaptive_batch_graph_replay():
    dd, eps_rel = 32, 1e-3
    specs = [("sjlt_block", 512, 64, 4, 4, 0.1, 1.0), ("sjlt_block", 1024, 128, 4, 3, 0.2, 1.0),
             ("sjlt_block", 384, 32, 4, 5, 0.06, 1.0)]
    inst = make(specs, dd, seed=5)
    items = [(x["op"].h, x["A"], x["St"], 0, x["d0"] + dd) for x in inst]
    with jl.Batch(items) as B:
        B.adaptive_setup([x["d0"] for x in inst], dd, eps_rel)
        B.adaptive_run()
        first = B.adaptive_result()
        snap = [x["St"].clone() for x in inst]
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            B.adaptive_run(stream=s)  # warm-up on the capture stream
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            B.adaptive_run(stream=s)
        for _ in range(2):
            for x in inst:
                x["St"].fill_(SENTINEL)
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            res = B.adaptive_result()
            # the same decisions; the sums agree to FP32 rounding (the batched sketch adds
            # the partial sums of CTAs that share a block of outputs atomically, in any order)
            for k in ("d", "state", "tests"):
                assert np.array_equal(res[k], first[k]), k
            for k in ("nh", "nt"):
                assert np.all(np.abs(res[k] - first[k]) <= TOL * first["nt"]), k
            for i, (x, y) in enumerate(zip(inst, snap)):
                d = int(res["d"][i])
                assert torch.allclose(x["St"][:, :d], y[:, :d], rtol=1e-5, atol=1e-5 * float(y[:, :d].abs().max()))
    compare(inst, first, dd, eps_rel, 0.0)
    for x in inst:
        x["op"].close()


def test_adaptive_batch_argument_checks():
    dd = 32
    inst = make([("sjlt_block", 256, 64, 4, 2, 0.2, 1.0)], dd, seed=3)
    x = inst[0]
    with jl.Batch([(x["op"].h, x["A"], x["St"], 0, x["d0"] + dd)]) as B:
        with pytest.raises(jl.JLSketchError):
            B.adaptive_setup([x["d0"]], 24 + 16, 1e-3)  # dd > 32
        with pytest.raises(jl.JLSketchError):
            B.adaptive_setup([x["d0"] + 8], dd, 1e-3)  # first block is not d0 + dd wide
        with pytest.raises(jl.JLSketchError):
            B.adaptive_setup([x["d0"]], 16, 1e-3)  # increments are not dd wide
        with pytest.raises(jl.JLSketchError):
            B.adaptive_run()  # no setup
    x["op"].close()


def batch_same_s(x, res, i, dd, eps_rel):
    d = int(res["d"][i])
    return util_batch_same_s(x["St"][:, :d].double().cpu().numpy(), x["d0"], dd, d, int(res["state"][i]),
                             res["nh"][i], res["nt"][i], eps_rel, srht=False, what=i)


@pytest.mark.parametrize("eps_rel", [1e-6])
def test_adaptive_batch_tight_tolerance_same_sketch(eps_rel):
    """eps_rel = 1e-6 on the small specifications: the decisions against the
    FP64 test on the device's own sketch, and the sketch against the FP64 A^T R."""
    dd, eps_abs = 32, 0.0
    specs = [("sjlt_block", 256, 64, 4, 4, 0.5, 1.0), ("sjlt_block", 448, 32, 4, 7, 0.2, 1.0),
             ("sjlt_graph", 1000, 64, 3, 6, 0.3, 1.0), ("sjlt_block", 2048, 128, 4, 5, 0.25, 1.0),
             ("sjlt_block", 1088, 96, 4, 6, 0.35, 1.0), ("sjlt_block", 512, 96, 4, 2, 0.03, 1.0)]
    inst = make(specs, dd, seed=19)
    items = [(x["op"].h, x["A"], x["St"], 0, x["d0"] + dd) for x in inst]
    with jl.Batch(items) as B:
        B.adaptive_setup([x["d0"] for x in inst], dd, eps_rel, eps_abs)
        B.adaptive_run()
        res = B.adaptive_result()
    for i, x in enumerate(inst):
        batch_same_s(x, res, i, dd, eps_rel)
        d = int(res["d"][i])
        R = ops.Operator(x["kind"], x["n"], x["d0"] + dd, x["alpha"], x["seed"])
        for _ in range((d - x["d0"] - dd) // dd):
            R.increment(dd)
        want = x["A"].double().cpu().numpy().T @ R.dense()
        got = x["St"][:, :d].double().cpu().numpy()
        assert np.linalg.norm(got - want) <= TOL * np.linalg.norm(want), i
    assert set(np.unique(res["state"])) <= {1, 2}
    assert 1 in set(res["state"]) and 2 in set(res["state"])
    for x in inst:
        x["op"].close()


@pytest.mark.parametrize("eps_rel", [1e-6, 1e-3])
def test_adaptive_batch_wide_basis(eps_rel):
    """Bases wider than the 512 columns whose Q^T W stays in shared memory (the
    loop runs to d_max = n for rough kernels): Q^T W goes through each
    instance's global G in chunks of 512 columns.  Decisions and the last
    ratio against the FP64 test on the device's sketch, the sketch against the
    FP64 A^T R."""
    dd = 32
    specs = [("sjlt_block", 800, 64, 4, 22, 0.03, 1.0),    # rough: every increment, basis up to 768 columns
             ("sjlt_block", 704, 32, 4, 20, 0.12, 1.0),
             ("sjlt_graph", 640, 96, 4, 16, 0.05, 1.0)]
    inst = make(specs, dd, seed=23)
    items = [(x["op"].h, x["A"], x["St"], 0, x["d0"] + dd) for x in inst]
    with jl.Batch(items) as B:
        B.adaptive_setup([x["d0"] for x in inst], dd, eps_rel, 0.0)
        B.adaptive_run()
        res = B.adaptive_result()
    assert int(res["d"][0]) - dd > 512  # the first instance's basis passed 512 columns
    for i, x in enumerate(inst):
        batch_same_s(x, res, i, dd, eps_rel)
        d = int(res["d"][i])
        R = ops.Operator(x["kind"], x["n"], x["d0"] + dd, x["alpha"], x["seed"])
        for _ in range((d - x["d0"] - dd) // dd):
            R.increment(dd)
        want = x["A"].double().cpu().numpy().T @ R.dense()
        got = x["St"][:, :d].double().cpu().numpy()
        assert np.linalg.norm(got - want) <= TOL * np.linalg.norm(want), i
    for x in inst:
        x["op"].close()


def test_adaptive_batch_full_size_1024():
    """The benchmark's batched adaptive workload in the launch configuration it
    times: 1024 kernel matrices K(X_i, X_i; h_i), n_i over multiples of 64 in
    [256, 4096], d0_i in {64, 128, 256}, dd = 32, eps_rel = 1e-6, increments up
    to d_max_i = n_i (at least d0_i + dd).  Every instance must end in a valid
    state (the width a whole number of increments, the number of tests to
    match, converged only with ||S^|| below eps_rel ||S~||, out of increments
    only at d_max).  On 24 sampled instances (16 with n_i <= 1024, 8 larger)
    every decision equals the FP64 test's on the device's sketch outside a 1 %
    band around eps_rel, and the last test's ratio agrees with it; on the 16
    smaller ones the final S'_i[:, :d_i] also equals the FP64 A_i^T R_i[:, :d_i]."""
    count, dd, alpha, eps_rel, seed = 1024, 32, 4, 1e-6, 20230203 + 3
    rng = np.random.default_rng(seed)
    ns = 64 * rng.integers(256 // 64, 4096 // 64 + 1, size=count)
    hs = rng.uniform(0.05, 0.5, size=count)
    d0s = rng.choice((64, 128, 256), size=count)
    inst = []
    for i in range(count):
        n = int(ns[i])
        X = torch.from_numpy(inputs.points(n, seed=seed + 17 * i)).cuda()
        A = torch.empty((n, n), device="cuda")
        jl.kernel_matrix(jl.generator(X, X, float(hs[i])), A)
        incs = max(0, (n - int(d0s[i])) // dd - 1)
        d_max = int(d0s[i]) + (incs + 1) * dd
        op = jl.Sketch("sjlt_block", n, int(d0s[i]) + dd, alpha, seed + i, d_max=d_max)
        for _ in range(incs):
            jl.sketch_increment(op.h, dd)
        inst.append(dict(op=op, A=A, St=torch.empty((n, d_max), device="cuda"), n=n, d0=int(d0s[i]), d_max=d_max))
    items = [(x["op"].h, x["A"], x["St"], 0, x["d0"] + dd) for x in inst]
    with jl.Batch(items) as B:
        B.adaptive_setup([x["d0"] for x in inst], dd, eps_rel, 0.0)
        B.adaptive_run()
        res = B.adaptive_result()
    d, state, tests, nh, nt = res["d"], res["state"], res["tests"], res["nh"], res["nt"]
    d0 = np.array([x["d0"] for x in inst])
    d_max = np.array([x["d_max"] for x in inst])
    assert set(np.unique(state)) <= {1, 2}
    assert np.all((d - d0 - dd) % dd == 0) and np.all(d >= d0 + dd) and np.all(d <= d_max)
    assert np.array_equal(tests, (d - d0 - dd) // dd + 1)
    assert np.all(nt > 0)
    assert np.all(nh[state == 1] < eps_rel * nt[state == 1])
    assert np.all(d[state == 2] == d_max[state == 2])
    pick = np.random.default_rng(5)
    small = [i for i in range(count) if inst[i]["n"] <= 1024]
    large = [i for i in range(count) if inst[i]["n"] > 1024]
    chosen_small = pick.choice(small, 16, replace=False)
    for i in list(chosen_small) + list(pick.choice(large, 8, replace=False)):
        batch_same_s(inst[i], res, int(i), dd, eps_rel)
    for i in chosen_small:
        x, di = inst[i], int(d[i])
        R = ops.Operator("sjlt_block", x["n"], x["d0"] + dd, alpha, seed + int(i))
        for _ in range((di - x["d0"] - dd) // dd):
            R.increment(dd)
        ref = x["A"].double().cpu().numpy().T @ R.dense()
        got = x["St"][:, :di].double().cpu().numpy()
        assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref), i
    for x in inst:
        x["op"].close()

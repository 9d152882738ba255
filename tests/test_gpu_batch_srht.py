"""Batched SRHT sketches: many uneven S_i = A_i R_i (row transforms of orders
nu_i <= 4096) in one persistent launch, checked instance by instance against
the FP64 oracle (A_i R_i with R_i = D H P / sqrt(d) formed densely from its
definition), through set() changes and CUDA-graph replays."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import operators as ops  # noqa: E402
from oracle import sketch as osk  # noqa: E402
from paper_2302_01977_gb300 import inputs  # noqa: E402
from paper_2302_01977_gb300 import jlsketch as jl  # noqa: E402
from tests.util import ensure_built  # noqa: E402

pytestmark = pytest.mark.gpu

SENTINEL = 12345.0
TOL = 1e-5  # relative Frobenius, FP32 sums


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def make(specs, seed):
    """specs: (rows, n, d0, increments, dd, h); A_i = K(Y_i, X_i; h) is rows x n."""
    out = []
    for k, (rows, n, d0, incs, dd, h) in enumerate(specs):
        X = torch.from_numpy(inputs.points(n, seed=seed + 2 * k)).cuda()
        Y = torch.from_numpy(inputs.points(rows, seed=seed + 2 * k + 1)).cuda()
        A = torch.empty((rows, n), device="cuda")
        jl.kernel_matrix(jl.generator(Y, X, h), A)
        d = d0 + incs * dd
        op = jl.Sketch("srht", n, d0, 1, 300 + k, d_max=d)
        for _ in range(incs):
            jl.sketch_increment(op.h, dd)
        S = torch.full((rows, d), SENTINEL, device="cuda")
        out.append(dict(op=op, A=A, S=S, n=n, d0=d0, d=d, dd=dd, incs=incs, seed=300 + k))
    return out


def oracle_s(x):
    """A_i R_i with R_i from the oracle's definition (same seed and increments)."""
    R = ops.Operator("srht", x["n"], x["d0"], 1, x["seed"])
    for _ in range(x["incs"]):
        R.increment(x["dd"])
    return osk.apply_t(x["A"].double().cpu().numpy().T, R.dense())  # (A^T)^T R = A R


def check(x, lo, hi, ref=None):
    got = x["S"].double().cpu().numpy()
    ref = oracle_s(x) if ref is None else ref
    err = np.linalg.norm(got[:, lo:hi] - ref[:, lo:hi]) / np.linalg.norm(ref[:, lo:hi])
    assert err <= TOL, (x["n"], lo, hi, err)
    outside = np.concatenate([got[:, :lo].ravel(), got[:, hi:].ravel()])
    assert np.all(outside == SENTINEL)


# every transform order from 1 to 4096, powers of two and ragged n, square and
# rectangular A, ranges of one column up to 160
SPECS = [(40, 1, 1, 0, 1, 0.3), (64, 100, 16, 1, 8, 0.2), (256, 256, 64, 2, 32, 0.3), (300, 300, 32, 1, 32, 0.1),
         (512, 512, 96, 1, 32, 0.2), (37, 700, 64, 2, 32, 0.05), (1024, 1024, 128, 1, 32, 0.2),
         (200, 1500, 160, 0, 32, 0.1), (2048, 2048, 64, 3, 32, 0.3), (333, 3000, 100, 1, 28, 0.08),
         (4096, 4096, 128, 1, 32, 0.2)]


def test_srht_batch_matches_oracle():
    inst = make(SPECS, seed=11)
    items = [(x["op"].h, x["A"], x["S"], 0, x["d"]) for x in inst]
    with jl.SrhtBatch(items) as B:
        for x in inst:  # the tuner's runs wrote every range: start from the sentinel again
            x["S"].fill_(SENTINEL)
        B.run()
        torch.cuda.synchronize()
        info = B.info()
    assert info["ctas_per_sm"] in (3, 6, 12)
    assert info["units"] == sum(x["A"].shape[0] for x in inst)
    for x in inst:
        check(x, 0, x["d"])
        x["op"].close()


@pytest.mark.parametrize("n", [65, 300, 576, 700, 1088, 1500, 2112, 3000])
def test_srht_batch_split_equals_padded_transform(n, monkeypatch):
    """Rows with n = k + r, 0 < r <= k / 2 (k = nu / 2) can take Sec. 7.1's
    split (orders k and p = 2^ceil(log2 r), two passes); JLS_SRHT_SPLIT=1 pins
    it on and =0 pins the zero-padded rows of order nu (by default the batch's
    tuner times both).  Both equal the oracle's A R and each other to FP32
    rounding."""
    outs = []
    for split in ("0", "1"):
        monkeypatch.setenv("JLS_SRHT_SPLIT", split)
        inst = make([(150, n, 48, 1, 16, 0.15)], seed=100 + n)
        x = inst[0]
        with jl.SrhtBatch([(x["op"].h, x["A"], x["S"], 0, x["d"])]) as B:
            B.run()
            torch.cuda.synchronize()
            assert B.info()["split"] == (split == "1")
        check(x, 0, x["d"])
        outs.append(x["S"].double().cpu().numpy())
        x["op"].close()
    assert np.linalg.norm(outs[1] - outs[0]) <= 1e-6 * np.linalg.norm(outs[0])


def test_srht_batch_graph_replay_of_increments():
    specs = [(512, 512, 64, 3, 32, 0.2), (384, 384, 128, 3, 32, 0.1), (1000, 1000, 96, 3, 32, 0.3),
             (2500, 2500, 64, 3, 32, 0.05)]
    inst = make(specs, seed=23)
    refs = [oracle_s(x) for x in inst]
    items = [(x["op"].h, x["A"], x["S"], 0, x["d0"] + x["dd"]) for x in inst]
    with jl.SrhtBatch(items) as B:
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            B.run(stream=s)  # warm-up on the capture stream
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            B.run(stream=s)
        for r in range(1, 3):  # increments r = 1, 2: columns [d0 + r dd, d0 + (r + 1) dd)
            lo = [x["d0"] + r * x["dd"] for x in inst]
            hi = [x["d0"] + (r + 1) * x["dd"] for x in inst]
            for x in inst:
                x["S"].fill_(SENTINEL)
            torch.cuda.synchronize()
            B.set(lo, hi)
            g.replay()
            torch.cuda.synchronize()
            for x, a, b, ref in zip(inst, lo, hi, refs):
                check(x, a, b, ref)
        # an empty range leaves that instance out of the run
        for x in inst:
            x["S"].fill_(SENTINEL)
        torch.cuda.synchronize()
        B.set([0, 5, 0, 0], [0, 5, inst[2]["d"], 0])
        assert B.info()["units"] == inst[2]["A"].shape[0]
        g.replay()
        torch.cuda.synchronize()
        for k, x in enumerate(inst):
            if k == 2:
                check(x, 0, x["d"], refs[2])
            else:
                assert torch.all(x["S"] == SENTINEL)
    for x in inst:
        x["op"].close()


def test_srht_batch_deterministic():
    inst = make([(700, 700, 64, 0, 32, 0.2), (1200, 1200, 96, 0, 32, 0.1)], seed=5)
    items = [(x["op"].h, x["A"], x["S"], 0, x["d"]) for x in inst]
    with jl.SrhtBatch(items) as B:
        B.run()
        first = [x["S"].clone() for x in inst]
        B.run()
        torch.cuda.synchronize()
        for x, f in zip(inst, first):
            assert torch.equal(x["S"], f)
    for x in inst:
        x["op"].close()


def test_srht_batch_argument_checks():
    inst = make([(256, 256, 32, 0, 32, 0.2)], seed=3)
    x = inst[0]
    with pytest.raises(jl.JLSketchError):
        jl.SrhtBatch([(x["op"].h, x["A"], x["S"], 0, x["d"] + 1)])  # beyond d_total
    sj = jl.Sketch("sjlt_block", 256, 32, 4, 1)
    with pytest.raises(jl.JLSketchError):
        jl.SrhtBatch([(sj.h, x["A"], x["S"], 0, 8)])  # not an SRHT operator
    sj.close()
    big = jl.Sketch("srht", 5000, 16, 1, 2)
    A5 = torch.zeros((4, 5000), device="cuda")
    S5 = torch.zeros((4, 16), device="cuda")
    with pytest.raises(jl.JLSketchError) as e:
        jl.SrhtBatch([(big.h, A5, S5, 0, 16)])  # order 8192 > 4096
    assert e.value.status == jl.SK_ERR_UNSUPPORTED
    big.close()
    with jl.SrhtBatch([(x["op"].h, x["A"], x["S"], 0, 16)]) as B:
        with pytest.raises(jl.JLSketchError):
            B.set([0], [x["d"] + 4])
        with pytest.raises(jl.JLSketchError):
            B.set([9], [8])
    x["op"].close()


def test_srht_batch_full_size_1024():
    """The batching workload's instances with SRHT operators: 1024 kernel matrices
    K(X_i, X_i; h_i), n_i over multiples of 64 in [256, 4096], d0_i in {64, 128, 256} (at most
    nu_i - 64: an SRHT samples at most nu_i columns),
    the first sketch of d0_i + 32 columns in one launch, then one 32-column increment
    replayed from a CUDA graph; 16 sampled instances (sampled rows) against the oracle."""
    count, dd, seed = 1024, 32, 20230203 + 3
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
        nu = 1 << (n - 1).bit_length()
        d0 = min(int(d0s[i]), nu - 2 * dd)  # the SRHT samples at most nu columns (n_i = 256, d0_i = 256)
        d = d0 + 2 * dd
        op = jl.Sketch("srht", n, d0 + dd, 1, seed + i, d_max=d)
        jl.sketch_increment(op.h, dd)
        inst.append(dict(op=op, A=A, S=torch.full((n, d), SENTINEL, device="cuda"), n=n, d0=d0, d=d))
    items = [(x["op"].h, x["A"], x["S"], 0, x["d0"] + dd) for x in inst]
    with jl.SrhtBatch(items) as B:
        B.run()
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=s):
            B.run(stream=s)
        torch.cuda.synchronize()
        B.set([x["d0"] + dd for x in inst], [x["d"] for x in inst])
        g.replay()
        torch.cuda.synchronize()
    pick = np.random.default_rng(9).choice(count, 16, replace=False)
    for i in pick:
        x = inst[int(i)]
        R = ops.Operator("srht", x["n"], x["d0"] + dd, 1, seed + int(i))
        R.increment(dd)
        rows = np.random.default_rng(int(i)).choice(x["n"], 64, replace=False)
        ref = osk.apply_t(x["A"][torch.from_numpy(rows).cuda()].double().cpu().numpy().T, R.dense())
        got = x["S"][torch.from_numpy(rows).cuda()].double().cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= TOL, (int(i), err)
    for x in inst:
        x["op"].close()


# ---- Algorithm 1 on the device for SRHT batches ------------------------------------------
from oracle import adaptive as oad  # noqa: E402


def make_adaptive(specs, dd, seed):
    """specs: (n, d0, increments, h, amplitude); symmetric A_i = amplitude * K(X_i, X_i; h)."""
    out = []
    for k, (n, d0, incs, h, amp) in enumerate(specs):
        X = torch.from_numpy(inputs.points(n, seed=seed + k)).cuda()
        A = torch.empty((n, n), device="cuda")
        jl.kernel_matrix(jl.generator(X, X, h), A)
        A *= amp
        d_max = d0 + (incs + 1) * dd
        op = jl.Sketch("srht", n, d0 + dd, 1, 700 + k, d_max=d_max)
        for _ in range(incs):
            jl.sketch_increment(op.h, dd)
        S = torch.full((n, d_max), SENTINEL, device="cuda")
        out.append(dict(op=op, A=A, S=S, n=n, d0=d0, d_max=d_max, seed=700 + k))
    return out


def compare_adaptive(inst, res, dd, eps_rel, eps_abs):
    for i, x in enumerate(inst):
        ref = oad.adaptive(x["A"].double().cpu().numpy(), "srht", x["d0"], dd, 1, x["seed"], x["d_max"], eps_rel,
                           eps_abs, which="S")
        hist = ref["history"]
        # decisions are compared up to the first test within the FP32 margin of a threshold
        near = [h[3] > 0 and (abs(h[2] / h[3] - eps_rel) <= 2 * TOL or abs(h[2] - eps_abs) <= 2 * TOL * h[3])
                for h in hist]
        if any(near):
            assert res["tests"][i] >= near.index(True) + 1, (i, res["tests"][i], near)
            continue
        assert res["tests"][i] == len(hist), (i, res["tests"][i], len(hist))
        assert res["state"][i] == (1 if ref["converged"] else 2), (i, res["state"][i])
        d = hist[-1][0] + dd
        assert res["d"][i] == d, (i, res["d"][i], d)
        nh0, nt0 = hist[-1][2], hist[-1][3]
        assert abs(res["nt"][i] - nt0) <= TOL * nt0, (i, res["nt"][i], nt0)
        assert abs(res["nh"][i] - nh0) <= TOL * nt0, (i, res["nh"][i], nh0, nt0)
        got = x["S"][:, :d].double().cpu().numpy()
        want = ref["S"][:, :d]
        assert np.linalg.norm(got - want) <= TOL * np.linalg.norm(want), i
        assert torch.all(x["S"][:, d:] == SENTINEL)


SPECS_ADAPT = [(256, 64, 4, 0.5, 1.0),     # smooth: stops at once
               (448, 32, 5, 0.12, 1.0),
               (1000, 64, 4, 0.08, 1.0),   # order 1024, ragged rows
               (2048, 128, 3, 0.2, 1.0),
               (512, 96, 2, 0.03, 1.0),    # rough kernel: runs out of columns
               (640, 64, 3, 0.3, 1e-9)]    # tiny entries: the absolute test stops it


@pytest.mark.parametrize("eps_rel", [1e-2, 1e-4])
def test_srht_batch_adaptive_matches_oracle(eps_rel):
    dd, eps_abs = 32, 1e-7
    inst = make_adaptive(SPECS_ADAPT, dd, seed=61)
    items = [(x["op"].h, x["A"], x["S"], 0, x["d0"] + dd) for x in inst]
    with jl.SrhtBatch(items) as B:
        B.adaptive_setup([x["d0"] for x in inst], dd, eps_rel, eps_abs)
        for x in inst:  # the tuner's runs wrote the first range: start from the sentinel again
            x["S"].fill_(SENTINEL)
        B.adaptive_run()
        res = B.adaptive_result()
        # the whole loop replayed from one captured CUDA graph gives the same result
        first = [x["S"].clone() for x in inst]
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=s):
            B.adaptive_run(stream=s)
        for x in inst:
            x["S"].fill_(SENTINEL)
        torch.cuda.synchronize()
        g.replay()
        res2 = B.adaptive_result(stream=s)
    compare_adaptive(inst, res, dd, eps_rel, eps_abs)
    for k in ("d", "state", "tests"):
        assert np.array_equal(res[k], res2[k])
    for x, f in zip(inst, first):
        assert torch.equal(x["S"], f)
        x["op"].close()


@pytest.mark.parametrize("split", ["0", "1"])
def test_srht_batch_adaptive_tight_tolerance_same_sketch(split, monkeypatch):
    """eps_rel = 1e-6: each decision against the FP64 test on the device's own
    sketch (outside a 1 % band around eps_rel), the last test's ratio within
    1 % plus the device arithmetic's resolution; with the rows zero-padded and
    with Sec. 7.1's split (n = 1088, 1000, 448 qualify)."""
    from tests.util import batch_same_s
    monkeypatch.setenv("JLS_SRHT_SPLIT", split)
    dd, eps_rel = 32, 1e-6
    specs = [(256, 64, 4, 0.5, 1.0), (448, 32, 7, 0.2, 1.0), (1000, 64, 6, 0.3, 1.0), (2048, 128, 5, 0.25, 1.0),
             (1088, 96, 6, 0.35, 1.0), (512, 96, 2, 0.03, 1.0)]
    inst = make_adaptive(specs, dd, seed=67)
    items = [(x["op"].h, x["A"], x["S"], 0, x["d0"] + dd) for x in inst]
    with jl.SrhtBatch(items) as B:
        B.adaptive_setup([x["d0"] for x in inst], dd, eps_rel, 0.0)
        B.adaptive_run()
        res = B.adaptive_result()
    for i, x in enumerate(inst):
        d = int(res["d"][i])
        batch_same_s(x["S"][:, :d].double().cpu().numpy(), x["d0"], dd, d, int(res["state"][i]), res["nh"][i],
                     res["nt"][i], eps_rel, srht=True, what=i)
    assert 1 in set(res["state"])
    for x in inst:
        x["op"].close()


def test_srht_batch_adaptive_argument_checks():
    dd = 32
    inst = make_adaptive([(300, 64, 2, 0.2, 1.0)], dd, seed=3)
    x = inst[0]
    with jl.SrhtBatch([(x["op"].h, x["A"], x["S"], 0, 96)]) as B:
        with pytest.raises(jl.JLSketchError):
            B.adaptive_setup([32], dd, 1e-3)  # the first block is d0 + dd = 96 wide, not 64
        with pytest.raises(jl.JLSketchError):
            B.adaptive_setup([64], 40, 1e-3)  # dd > 32
        with pytest.raises(jl.JLSketchError):
            B.adaptive_run()  # no setup yet
    x["op"].close()

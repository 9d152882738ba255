"""Batched SJLT sketches: many uneven S'_i = A_i^T R_i in one persistent launch,
checked instance by instance against the FP64 oracle (A_i^T R_i with R_i formed
densely from the exported operator), through set() changes and CUDA-graph
replays."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sketch as osk  # noqa: E402
from paper_2302_01977_gb300 import inputs  # noqa: E402
from paper_2302_01977_gb300 import jlsketch as jl  # noqa: E402

pytestmark = pytest.mark.gpu

SENTINEL = 12345.0


def make_instances(specs, seed=7):
    """specs: (kind, rows n_i, cols m_i, d0, alpha, increments of dd, dd)."""
    out = []
    for k, (kind, n, m, d0, alpha, incs, dd) in enumerate(specs):
        X = torch.from_numpy(inputs.points(m, seed=seed + 2 * k)).cuda()
        Y = torch.from_numpy(inputs.points(n, seed=seed + 2 * k + 1)).cuda()
        A = torch.empty((n, m), device="cuda")
        jl.kernel_matrix(jl.generator(Y, X, 0.05 + 0.05 * (k % 8)), A)
        op = jl.Sketch(kind, n, d0, alpha, 100 + k, d_max=d0 + incs * dd)
        for _ in range(incs):
            jl.sketch_increment(op.h, dd)
        d = d0 + incs * dd
        St = torch.full((m, d), SENTINEL, device="cuda")
        out.append(dict(op=op, A=A, St=St, d0=d0, d=d, dd=dd))
    return out


def oracle_cols(inst, lo, hi):
    R = jl.sketch_export(inst["op"].h, dense=True)["R"]
    return osk.apply_t(inst["A"].double().cpu().numpy(), R)[:, lo:hi]


def check(inst, lo, hi, tol=1e-5):
    got = inst["St"].double().cpu().numpy()
    ref = oracle_cols(inst, lo, hi)
    err = np.linalg.norm(got[:, lo:hi] - ref) / np.linalg.norm(ref)
    assert err <= tol, (lo, hi, err)
    outside = np.concatenate([got[:, :lo].ravel(), got[:, hi:].ravel()])
    assert np.all(outside == SENTINEL)


# (rows may be any size; the row pitch of A, cols * 4 bytes, must be a multiple of 16 for TMA)
SPECS = [("sjlt_block", 256, 256, 64, 4, 2, 32), ("sjlt_block", 448, 448, 128, 4, 1, 32),
         ("sjlt_graph", 320, 200, 48, 3, 1, 24), ("sjlt_block", 1000, 1000, 256, 4, 1, 32),
         ("sjlt_block", 64, 132, 32, 2, 0, 8), ("sjlt_block", 2048, 2048, 128, 4, 3, 32),
         ("sjlt_graph", 777, 780, 96, 4, 2, 16), ("sjlt_block", 130, 1500, 64, 4, 0, 32)]


def test_batch_first_sketch_and_increments():
    inst = make_instances(SPECS)
    # first run: Algorithm 1's first sketch, columns [0, d0 + dd) (or [0, d) without increments)
    lo = [0] * len(inst)
    hi = [min(x["d"], x["d0"] + x["dd"]) for x in inst]
    items = [(x["op"].h, x["A"], x["St"], a, b) for x, a, b in zip(inst, lo, hi)]
    with jl.Batch(items) as B:
        info = B.info()
        shapes = {24: 0, 20: 1, 16: 2, 32: 3}  # the autotuner's shapes, in the order of tuned_ms
        assert info["warps"] in shapes
        eligible = [t for t in info["tuned_ms"] if t >= 0]
        assert eligible and info["tuned_ms"][shapes[info["warps"]]] == min(eligible)
        B.run()
        B.status()
        for x, a, b in zip(inst, lo, hi):
            check(x, a, b)
        # later increments: the next dd columns of the instances that have one; the rest inactive
        active = [1 if x["d"] >= x["d0"] + 2 * x["dd"] else 0 for x in inst]
        lo2 = [x["d0"] + x["dd"] if on else 0 for x, on in zip(inst, active)]
        hi2 = [x["d0"] + 2 * x["dd"] if on else 1 for x, on in zip(inst, active)]
        for x in inst:
            x["St"].fill_(SENTINEL)
        B.set(active, lo2, hi2)
        B.tune()  # narrow ranges: the 32 x 2 shape becomes eligible
        assert B.info()["tuned_ms"][3] >= 0
        for x in inst:
            x["St"].fill_(SENTINEL)
        B.run()
        B.status()
        for x, on, a, b in zip(inst, active, lo2, hi2):
            if on:
                check(x, a, b)
            else:
                assert torch.all(x["St"] == SENTINEL)
    for x in inst:
        x["op"].close()


def test_batch_cuda_graph_replay():
    specs = [("sjlt_block", 512, 512, 64, 4, 3, 32), ("sjlt_block", 384, 384, 128, 4, 3, 32),
             ("sjlt_block", 1024, 1024, 256, 4, 3, 32)]
    inst = make_instances(specs, seed=31)
    items = [(x["op"].h, x["A"], x["St"], 0, x["d0"] + x["dd"]) for x in inst]
    with jl.Batch(items) as B:
        B.run()
        torch.cuda.synchronize()
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
                x["St"].fill_(SENTINEL)
            torch.cuda.synchronize()
            B.set([1] * len(inst), lo, hi)
            g.replay()
            torch.cuda.synchronize()
            B.status()
            for x, a, b in zip(inst, lo, hi):
                check(x, a, b)
    for x in inst:
        x["op"].close()


def test_batch_argument_checks():
    inst = make_instances([("sjlt_block", 256, 256, 64, 4, 0, 32)], seed=3)
    x = inst[0]
    with pytest.raises(jl.JLSketchError):
        jl.Batch([(x["op"].h, x["A"], x["St"], 0, x["d"] + 1)])  # beyond d_total
    A2 = torch.zeros((256, 257), device="cuda")[:, :256]
    with pytest.raises(jl.JLSketchError):
        jl.Batch([(x["op"].h, A2, x["St"], 0, 8)])  # ld * 4 is not a multiple of 16
    with pytest.raises(jl.JLSketchError):
        jl.Batch([(x["op"].h, x["A"][:200], x["St"], 0, 8)])  # rows != n
    with jl.Batch([(x["op"].h, x["A"], x["St"], 0, 16)]) as B:
        with pytest.raises(jl.JLSketchError):
            B.set(None, [0], [x["d"] + 4])
    x["op"].close()

"""Decision study of the batched adaptive loop (GPU; not collected by pytest).

Runs Algorithm 1 on the 1024-instance batching workload (eps_rel = 1e-6, dd = 32,
up to 8 increments) and, for 256 sampled instances, compares each decision with
the FP64 ratios ||S^||_F / ||S~||_F of Eq. (3.1).  Those ratios come from one
Householder QR of the FP64 sketch A_i^T R_i (R_i formed by the oracle): for the
tested columns b_k, the diagonal block R[b_k, b_k] of the QR factor is their part
orthogonal to every earlier column, so ||S^|| = ||R[b_k, b_k]||_F.  Prints the
disagreements and writes the rows to a JSON file.

    python tests/decision_study.py [out.json]
"""
import json
import os
import sys
import time

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import operators as ops  # noqa: E402
from paper_2302_01977_gb300 import inputs  # noqa: E402
from paper_2302_01977_gb300 import jlsketch as jl  # noqa: E402

count, dd, incs, alpha, eps_rel, seed = 1024, 32, 8, 4, 1e-6, 20230203 + 3
rng = np.random.default_rng(seed)
ns = 64 * rng.integers(256 // 64, 4096 // 64 + 1, size=count)
hs = rng.uniform(0.05, 0.5, size=count)
d0s = rng.choice((64, 128, 256), size=count)
torch.cuda.set_device(0)
inst = []
for i in range(count):
    n = int(ns[i])
    X = torch.from_numpy(inputs.points(n, seed=seed + 17 * i)).cuda()
    A = torch.empty((n, n), device="cuda")
    jl.kernel_matrix(jl.generator(X, X, float(hs[i])), A)
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
d, state, tests, nh, nt = (np.asarray(res[k]) for k in ("d", "state", "tests", "nh", "nt"))
print("converged", int((state == 1).sum()), "out", int((state == 2).sum()), flush=True)

sample = np.random.default_rng(7).choice(count, 256, replace=False)
rows = []
t0 = time.time()
for i in sample:
    x = inst[i]
    n, d0 = x["n"], x["d0"]
    R = ops.Operator("sjlt_block", n, d0 + dd, alpha, seed + int(i))
    for _ in range(incs):
        R.increment(dd)
    Sf = x["A"].double().cpu().numpy().T @ R.dense()
    Rq = np.linalg.qr(Sf, mode="r")
    ratios = []
    for k in range(incs + 1):
        b0 = d0 + k * dd
        ratios.append(float(np.linalg.norm(Rq[b0:b0 + dd, b0:b0 + dd]) / np.linalg.norm(Sf[:, b0:b0 + dd])))
    ok = [k for k, r in enumerate(ratios) if r < eps_rel]
    o_tests = ok[0] + 1 if ok else incs + 1
    o_state = 1 if ok else 2
    rows.append(dict(i=int(i), n=n, h=float(hs[i]), d0=d0, gpu_state=int(state[i]), gpu_tests=int(tests[i]),
                     gpu_ratio=float(nh[i] / nt[i]), o_state=o_state, o_tests=o_tests, ratios=ratios))
print("oracle time", time.time() - t0, flush=True)
agree = sum(r["gpu_state"] == r["o_state"] and r["gpu_tests"] == r["o_tests"] for r in rows)
print("agree", agree, "of", len(rows))
for r in rows:
    if not (r["gpu_state"] == r["o_state"] and r["gpu_tests"] == r["o_tests"]):
        k = r["gpu_tests"] - 1
        print(r["i"], r["n"], round(r["h"], 3), r["d0"], "gpu", r["gpu_state"], r["gpu_tests"],
              "%.2e" % r["gpu_ratio"], "oracle", r["o_state"], r["o_tests"],
              "oracle ratio at gpu stop %.2e" % r["ratios"][k],
              "min oracle ratio %.2e" % min(r["ratios"]))
out = sys.argv[1] if len(sys.argv) > 1 else "decisions.json"
with open(out, "w") as f:
    json.dump(dict(converged=int((state == 1).sum()), rows=rows), f)

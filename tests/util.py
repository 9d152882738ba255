"""Helpers shared by the GPU parity tests."""
import numpy as np

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16x2": 1e-5}


def rel_fro(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def dev(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def ensure_built():
    import os
    from paper_2302_01977_gb300 import jlsketch as jl
    if not os.path.exists(jl.LIB_PATH):
        from paper_2302_01977_gb300 import build
        build.build()
    return jl.lib()

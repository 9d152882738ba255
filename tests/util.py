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


def dev_padded(x, dtype):
    """Device copy of a 2-D array whose leading dimension is rounded up to 16
    bytes (the library's alignment contract); returns the (rows, cols) view."""
    import torch
    x = np.ascontiguousarray(x)
    m, n = x.shape
    es = 8 if dtype == torch.float64 else 4
    ld = (n * es + 15) // 16 * 16 // es
    buf = torch.zeros((m, ld), dtype=dtype, device="cuda")
    buf[:, :n] = torch.from_numpy(x).to(dtype).cuda()
    return buf[:, :n]


def host(t):
    return t.detach().cpu().numpy()


def ensure_built():
    import os
    from paper_2302_01977_gb300 import jlsketch as jl
    if not os.path.exists(jl.LIB_PATH):
        from paper_2302_01977_gb300 import build
        build.build()
    return jl.lib()

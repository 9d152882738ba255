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


# Stopping-test parity on the device's own sketch.  The FP32 sketch carries its
# own rounding (about 1e-7 of S, in every direction), so near eps_rel = 1e-6 the
# decision is that of the test applied to the sketch the device holds: the FP64
# oracle's test (oracle.adaptive.norm_test) is run on that sketch, widened to
# FP64, as the FP32 matrix A itself is.  A decision must agree wherever the
# FP64 ratio ||S^|| / ||S~|| is more than BAND (relative) away from eps_rel;
# the ratio itself must agree within RTOL of it, after a floor FLOOR combined
# in quadrature: the device's ratio is that of a residual carrying, besides
# S^, the error of its FP32 basis of the earlier columns, which represents
# their span only to about 1e-7 of the block (a CPU model of the arithmetic
# reads 1-2e-7 ratios 1-3 % high), so |r - r0| <= RTOL r0 + FLOOR^2 / (r + r0).
# Near eps_rel = 1e-6 the floor adds at most 0.5 %.
SAME_S_BAND = 1e-2
SAME_S_RTOL = 1e-2
SAME_S_FLOOR = 1e-7


def same_s_check(S, tests, dd, eps_rel, what="", atol_extra=0.0, ref=None):
    """S: the device sketch (FP64 copy of its FP32 values), with at least the
    columns the last test covers; tests: [(b0, stop, nh, nt)] in order, the
    device's test of columns [b0, b0 + dd) against the basis of [0, b0) and
    its decision (nh, nt None where the device does not report them).
    atol_extra: a bound on how far S has moved since the device tested it
    (one FP32 rescale of every column moves the ratio by at most 2^-23).
    ref: the oracle's (||S^||, ||S~||) of each test if already computed.
    Returns the FP64 ratios."""
    from oracle import adaptive as oad
    ratios = []
    for k, (b0, stop, nh, nt) in enumerate(tests):
        if ref is not None:
            nh0, nt0 = ref[k]
        else:
            _, nh0, nt0 = oad.norm_test(S[:, :b0 + dd], b0, dd, eps_rel, 0.0)
        r0 = nh0 / nt0 if nt0 > 0 else 0.0
        ratios.append(r0)
        if nt is not None:
            assert abs(nt - nt0) <= 1e-5 * nt0, (what, b0, nt, nt0)
            r = nh / nt
            floor = SAME_S_FLOOR ** 2 / max(r + r0, 1e-300)
            assert abs(r - r0) <= SAME_S_RTOL * r0 + floor + atol_extra, (what, b0, r, r0)
        if abs(r0 - eps_rel) > SAME_S_BAND * eps_rel:
            assert bool(stop) == (r0 < eps_rel), (what, b0, stop, r0)
    return ratios


def batch_same_s(S, d0, dd, d, state, nh, nt, eps_rel, srht=False, what=""):
    """same_s_check for one instance of a batched adaptive run: S is its final
    sketch (FP64 copy of the device's S_i[:, :d]), tests at columns d0, d0 + dd,
    ..., d - dd, the loop went on after all but the last, the last stopped iff
    state == 1 (converged), and the device reports the last test's norms.  The
    run rescales the finished columns once by a uniform factor (1/sqrt(blocks)
    for SJLT, sqrt((d0 + dd) / d) for SRHT), which moves the ratios by at most
    2^-23 unless the factor is a power of two."""
    b0s = list(range(d0, d, dd))
    tests = [(b0, False, None, None) for b0 in b0s[:-1]]
    tests.append((b0s[-1], state == 1, float(nh), float(nt)))
    first_w = d0 + dd
    f2 = first_w / d if srht else 1.0 / (1 + (d - first_w) // dd)
    e = np.log2(f2)
    exact = float(e).is_integer() and int(e) % 2 == 0
    from oracle import adaptive as oad
    ref = oad.norm_tests(S, d0, dd, d)  # every test of the run at once
    return same_s_check(S, tests, dd, eps_rel, what=what, atol_extra=0.0 if exact else 2.0 ** -23, ref=ref)

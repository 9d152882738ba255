"""Global adaptive sketching driven through the C ABI (host control flow only).

Algorithm 1 restricted to the global sketch: R <- JL(d0 + Delta-d); S <- A R
(and S' <- A^T R); then repeat the Frobenius stopping test on the last Delta-d
columns and, while it fails and the grown R stays within d_max columns, append
Delta-d columns and sketch only those (sketch_increment +
sketch_apply_increment).  Every arithmetic step is a libjlsketch kernel; this
module only sequences the calls and collects the norms.
"""
from __future__ import annotations

from . import jlsketch as jl


def adaptive_sketch(A, kind, d0: int, dd: int, alpha: int = 1, seed: int = 0, d_max: int = 512,
                    eps_rel: float = 1e-2, eps_abs: float = 1e-8, which: int = jl.SK_BOTH,
                    prec: int = jl.SK_PREC_NATIVE, S=None, St=None, stream=None):
    """Run the loop on explicit matrix ``A`` (square torch CUDA tensor).

    Returns dict(handle=..., S=..., St=..., d=final width, converged=bool,
    history=[(d, stop, nh_S, nt_S, nh_St, nt_St), ...]).  The caller owns the
    handle (``jl.sketch_destroy``).  S / St may be preallocated with at least
    d_max columns.
    """
    import torch
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("square A expected")
    if d0 + dd > d_max:
        raise ValueError("d0 + Delta-d exceeds d_max")
    if S is None and which & jl.SK_S:
        S = torch.empty((n, d_max), dtype=A.dtype, device=A.device)
    if St is None and which & jl.SK_ST:
        St = torch.empty((n, d_max), dtype=A.dtype, device=A.device)
    h = jl.sketch_create(kind, n, d0 + dd, alpha, seed, d_max, stream)
    jl.sketch_apply(h, A, which, prec, S, St, stream)
    d = d0
    history = []
    while True:
        w = d + dd
        stop_s, nh_s, nt_s = (True, 0.0, 0.0)
        stop_t, nh_t, nt_t = (True, 0.0, 0.0)
        if which == jl.SK_BOTH:  # the two tests overlap on two streams
            (stop_s, nh_s, nt_s), (stop_t, nh_t, nt_t) = jl.adaptive_norm_test_pair(
                h, S[:, :w], St[:, :w], dd, eps_rel, eps_abs, stream)
        elif which & jl.SK_S:
            stop_s, nh_s, nt_s = jl.adaptive_norm_test(h, 0, S[:, :w], dd, eps_rel, eps_abs, stream)
        elif which & jl.SK_ST:
            stop_t, nh_t, nt_t = jl.adaptive_norm_test(h, 1, St[:, :w], dd, eps_rel, eps_abs, stream)
        stop = stop_s and stop_t
        history.append((d, stop, nh_s, nt_s, nh_t, nt_t))
        if stop:
            return dict(handle=h, S=S, St=St, d=w, converged=True, history=history)
        if w + dd > d_max:
            return dict(handle=h, S=S, St=St, d=w, converged=False, history=history)
        jl.sketch_increment(h, dd, stream)
        jl.sketch_apply_increment(h, A, which, prec, S, St, stream)
        d += dd

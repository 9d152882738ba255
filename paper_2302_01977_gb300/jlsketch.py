"""Thin ctypes binding of libjlsketch (include/jlsketch.h).

Argument marshalling only: every step of the sketching path runs in the CUDA
library.  Functions carry the C names; tensors are torch CUDA tensors (row-major
2-D, unit column stride) whose ``data_ptr()`` is passed through, and streams
default to torch's current stream.  A non-zero status raises ``JLSketchError``.
If the shared library has not been built the first call raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjlsketch.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "jlsketch.h")

# constants (mirrors include/jlsketch.h; tests check the two agree)
SK_OK = 0
SK_ERR_INVALID_ARG = -1
SK_ERR_ALIGN = -2
SK_ERR_DTYPE = -3
SK_ERR_NOMEM = -4
SK_ERR_D_MAX = -5
SK_ERR_STATE = -6
SK_ERR_TIMEOUT = -7
SK_ERR_DEVICE = -8
SK_ERR_UNSUPPORTED = -9
SK_SJLT_GRAPH = 1
SK_SJLT_BLOCK = 2
SK_SRHT = 3
SK_GAUSS = 4
SK_F64 = 1
SK_F32 = 2
SK_C64 = 3
SK_PREC_NATIVE = 0
SK_PREC_BF16X2 = 3
SK_PREC_FP8 = 4
SK_S = 1
SK_ST = 2
SK_BOTH = 3
SK_SCALE_BLOCK = 1
SK_SRHT_REPLACE = 2
SK_HSS_U = 1
SK_HSS_J = 2
SK_HSS_IT = 3
SK_HSS_D = 4
SK_HSS_B = 5
SK_HSS_S = 6
SK_HSS_R = 7

KIND_NAMES = {"sjlt_graph": SK_SJLT_GRAPH, "sjlt_block": SK_SJLT_BLOCK, "srht": SK_SRHT, "gauss": SK_GAUSS}

EXPORTS = ["sketch_create", "sketch_create_flags", "sketch_sjlt_route", "sketch_increment", "sketch_apply", "sketch_apply_increment",
           "adaptive_norm_test", "adaptive_norm_test_pair", "sketch_project_norms_noalloc", "kernel_matrix", "sketch_kernel_apply",
           "sketch_kernel_adjoint", "sketch_batch_create", "sketch_batch_set", "sketch_batch_run",
           "sketch_batch_tune", "sketch_batch_adaptive_setup", "sketch_batch_adaptive_run",
           "sketch_batch_adaptive_result",
           "sketch_batch_info", "sketch_batch_status", "sketch_batch_destroy", "sketch_srht_batch_create",
           "sketch_srht_batch_set", "sketch_srht_batch_run", "sketch_srht_batch_info",
           "sketch_srht_batch_adaptive_setup", "sketch_srht_batch_adaptive_run", "sketch_srht_batch_adaptive_result",
           "sketch_srht_batch_destroy",
           "sketch_dims", "sketch_export",
           "sketch_device_status", "sketch_selftest_wait", "sketch_launch_count", "sketch_srht_route",
           "sketch_destroy",
           "sketch_strerror",
           "hss_compress_adaptive", "hss_info", "hss_node", "hss_node_get", "hss_history", "hss_launch_count",
           "hss_profile", "hss_destroy"]


class JLSketchError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {sketch_strerror(status)} (status {status})")


class SkBatchItem(ctypes.Structure):
    _fields_ = [("op", ctypes.c_void_p), ("A", ctypes.c_void_p), ("rows", ctypes.c_int64),
                ("cols", ctypes.c_int64), ("ld", ctypes.c_int64), ("St", ctypes.c_void_p),
                ("ldSt", ctypes.c_int64), ("c_lo", ctypes.c_int32), ("c_hi", ctypes.c_int32),
                ("scale", ctypes.c_double)]


class SkSrhtBatchItem(ctypes.Structure):
    _fields_ = [("op", ctypes.c_void_p), ("A", ctypes.c_void_p), ("rows", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("S", ctypes.c_void_p), ("ldS", ctypes.c_int64),
                ("c_lo", ctypes.c_int32), ("c_hi", ctypes.c_int32), ("scale", ctypes.c_double)]


class SkMatrix(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("generator", ctypes.c_int32),
                ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("ld", ctypes.c_int64),
                ("X", ctypes.c_void_p), ("Y", ctypes.c_void_p),
                ("h", ctypes.c_double), ("shift", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libjlsketch.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(the sketching path has no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "sketch_create": (i32, [P(vp), i32, i64, i32, i32, u64, i32, vp]),
        "sketch_create_flags": (i32, [P(vp), i32, i64, i32, i32, u64, i32, ctypes.c_uint32, vp]),
        "sketch_increment": (i32, [vp, i32, vp]),
        "sketch_apply": (i32, [vp, P(SkMatrix), i32, i32, vp, i64, vp, i64, vp]),
        "sketch_apply_increment": (i32, [vp, P(SkMatrix), i32, i32, vp, i64, vp, i64, vp]),
        "adaptive_norm_test": (i32, [vp, i32, vp, i64, i64, i32, i32, dbl, dbl, P(i32), P(dbl), P(dbl), vp]),
        "adaptive_norm_test_pair": (i32, [vp, vp, i64, i64, vp, i64, i64, i32, i32, dbl, dbl, P(i32), P(dbl),
                                          P(dbl), vp]),
        "sketch_project_norms_noalloc": (i32, [vp, i64, i32, vp, i64, i64, i32, i32, vp, i64, dbl, dbl, P(i32),
                                               P(dbl), P(dbl), vp]),
        "kernel_matrix": (i32, [P(SkMatrix), vp, i64, vp]),
        "sketch_kernel_apply": (i32, [vp, vp, i64, vp, dbl, dbl, vp, i64, vp]),
        "sketch_kernel_adjoint": (i32, [vp, vp, dbl, vp, i64, vp, vp, vp]),
        "sketch_batch_create": (i32, [P(vp), P(SkBatchItem), i32, vp]),
        "sketch_batch_set": (i32, [vp, vp, vp, vp]),
        "sketch_batch_run": (i32, [vp, vp]),
        "sketch_batch_tune": (i32, [vp, vp]),
        "sketch_batch_adaptive_setup": (i32, [vp, P(i32), i32, ctypes.c_double, ctypes.c_double, vp]),
        "sketch_batch_adaptive_run": (i32, [vp, i32, vp]),
        "sketch_batch_adaptive_result": (i32, [vp, P(i32), P(i32), P(i32), P(ctypes.c_double),
                                               P(ctypes.c_double), vp]),
        "sketch_batch_info": (i32, [vp, P(i32), P(i32), P(i64), P(ctypes.c_float)]),
        "sketch_batch_status": (i32, [vp, vp]),
        "sketch_batch_destroy": (None, [vp]),
        "sketch_srht_batch_create": (i32, [P(vp), P(SkSrhtBatchItem), i32, vp]),
        "sketch_srht_batch_set": (i32, [vp, vp, vp]),
        "sketch_srht_batch_run": (i32, [vp, vp]),
        "sketch_srht_batch_info": (i32, [vp, P(i32), P(i64), P(ctypes.c_float), P(i32)]),
        "sketch_srht_batch_adaptive_setup": (i32, [vp, P(i32), i32, ctypes.c_double, ctypes.c_double, vp]),
        "sketch_srht_batch_adaptive_run": (i32, [vp, i32, vp]),
        "sketch_srht_batch_adaptive_result": (i32, [vp, P(i32), P(i32), P(i32), P(ctypes.c_double),
                                                    P(ctypes.c_double), vp]),
        "sketch_srht_batch_destroy": (None, [vp]),
        "sketch_selftest_wait": (i32, [vp]),
        "sketch_dims": (i32, [vp, P(i32), P(i64), P(i32), P(i32), P(i32)]),
        "sketch_export": (i32, [vp, vp, vp, vp, vp, vp, i32]),
        "sketch_device_status": (i32, [vp, vp]),
        "sketch_launch_count": (i64, []),
        "sketch_srht_route": (i32, [i64, i64, i64, i32, i32]),
        "sketch_sjlt_route": (i32, [i32, i64, i64, i64, i32, i32]),
        "sketch_destroy": (None, [vp]),
        "sketch_strerror": (ctypes.c_char_p, [i32]),
        "hss_compress_adaptive": (i32, [P(vp), vp, i64, i64, i32, i32, i32, i32, i32, u64, i32, dbl, dbl, vp]),
        "hss_info": (i32, [vp, P(i32), P(i32), P(i32), P(i32), P(i32), P(i32)]),
        "hss_node": (i32, [vp, i32, P(i64), P(i32)]),
        "hss_node_get": (i32, [vp, i32, i32, vp]),
        "hss_history": (i32, [vp, vp, vp]),
        "hss_launch_count": (i64, [vp]),
        "hss_profile": (i32, [vp, vp, vp, vp, vp]),
        "hss_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def header_constants() -> dict:
    """#define SK_* values parsed from include/jlsketch.h."""
    out = {}
    for line in open(HEADER):
        m = re.match(r"#define\s+(SK_\w+)\s+(-?\d+)", line)
        if m:
            out[m.group(1)] = int(m.group(2))
    return out


def sketch_strerror(status: int) -> str:
    try:
        return lib().sketch_strerror(int(status)).decode()
    except RuntimeError:
        return f"status {status}"


def _check(rc: int, where: str) -> None:
    if rc != SK_OK:
        raise JLSketchError(rc, where)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return SK_F32
    if t.dtype == torch.float64:
        return SK_F64
    if t.dtype == torch.complex64:
        return SK_C64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _check_2d(t, name):
    if t.dim() != 2 or t.stride(1) != 1 or not t.is_cuda:
        raise ValueError(f"{name} must be a 2-D CUDA tensor with unit column stride")


def matrix(A) -> SkMatrix:
    """Descriptor of an explicit row-major matrix held in a CUDA tensor."""
    if isinstance(A, SkMatrix):
        return A
    _check_2d(A, "A")
    return SkMatrix(dtype=_dtype_code(A), generator=0, rows=A.shape[0], cols=A.shape[1],
                    A=A.data_ptr(), ld=A.stride(0), X=None, Y=None, h=0.0, shift=0.0)


def generator(X, Y, h: float, shift: float = 0.0) -> SkMatrix:
    """Descriptor of A_ij = exp(-||x_i - y_j||^2/(2h^2)) + shift [i == j]."""
    for t, nm in ((X, "X"), (Y, "Y")):
        if t.dim() != 2 or t.shape[1] != 3 or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"{nm} must be a contiguous CUDA tensor of shape (m, 3)")
    return SkMatrix(dtype=_dtype_code(X), generator=1, rows=X.shape[0], cols=Y.shape[0], A=None, ld=0,
                    X=X.data_ptr(), Y=Y.data_ptr(), h=float(h), shift=float(shift))


def sketch_create(kind, n: int, d: int, alpha: int = 1, seed: int = 0, d_max: int | None = None,
                  stream=None, flags: int = 0) -> ctypes.c_void_p:
    """flags: 0 (sketch_create), or SK_SCALE_BLOCK | SK_SRHT_REPLACE (sketch_create_flags)."""
    k = KIND_NAMES.get(kind, kind) if isinstance(kind, str) else int(kind)
    h = ctypes.c_void_p()
    dm = int(d if d_max is None else d_max)
    if flags:
        rc = lib().sketch_create_flags(ctypes.byref(h), k, int(n), int(d), int(alpha), int(seed) & (2**64 - 1), dm,
                                       int(flags), _stream(stream))
    else:
        rc = lib().sketch_create(ctypes.byref(h), k, int(n), int(d), int(alpha), int(seed) & (2**64 - 1), dm,
                                 _stream(stream))
    _check(rc, "sketch_create_flags" if flags else "sketch_create")
    return h


def sketch_increment(h, delta_d: int, stream=None) -> None:
    _check(lib().sketch_increment(h, int(delta_d), _stream(stream)), "sketch_increment")


def _apply(fn, name, h, A, which, prec, S, St, stream):
    desc = matrix(A)
    sp, lds, stp, ldst = None, 0, None, 0
    if S is not None:
        _check_2d(S, "S")
        sp, lds = S.data_ptr(), S.stride(0)
    if St is not None:
        _check_2d(St, "St")
        stp, ldst = St.data_ptr(), St.stride(0)
    _check(fn(h, ctypes.byref(desc), int(which), int(prec), sp, lds, stp, ldst, _stream(stream)), name)


def sketch_apply(h, A, which: int = SK_BOTH, prec: int = SK_PREC_NATIVE, S=None, St=None, stream=None) -> None:
    _apply(lib().sketch_apply, "sketch_apply", h, A, which, prec, S, St, stream)


def sketch_apply_increment(h, A, which: int = SK_BOTH, prec: int = SK_PREC_NATIVE, S=None, St=None,
                           stream=None) -> None:
    _apply(lib().sketch_apply_increment, "sketch_apply_increment", h, A, which, prec, S, St, stream)


def adaptive_norm_test(h, slot: int, S, delta_d: int, eps_rel: float, eps_abs: float, stream=None):
    """Returns (stop, ||S^||_F, ||S~||_F)."""
    _check_2d(S, "S")
    stop = ctypes.c_int32()
    nh = ctypes.c_double()
    nt = ctypes.c_double()
    rc = lib().adaptive_norm_test(h, int(slot), S.data_ptr(), S.shape[0], S.stride(0), _dtype_code(S),
                                  int(delta_d), float(eps_rel), float(eps_abs), ctypes.byref(stop),
                                  ctypes.byref(nh), ctypes.byref(nt), _stream(stream))
    _check(rc, "adaptive_norm_test")
    return bool(stop.value), nh.value, nt.value


def adaptive_norm_test_pair(h, S, St, delta_d: int, eps_rel: float, eps_abs: float, stream=None):
    """Both tests at once (S on `stream`, S' on the handle's second stream); returns
    ((stop, ||S^||, ||S~||) for S, the same for S')."""
    _check_2d(S, "S")
    _check_2d(St, "St")
    if _dtype_code(S) != _dtype_code(St):
        raise ValueError("S and St must have the same dtype")
    stop = (ctypes.c_int32 * 2)()
    nh = (ctypes.c_double * 2)()
    nt = (ctypes.c_double * 2)()
    rc = lib().adaptive_norm_test_pair(h, S.data_ptr(), S.shape[0], S.stride(0), St.data_ptr(), St.shape[0],
                                       St.stride(0), _dtype_code(S), int(delta_d), float(eps_rel), float(eps_abs),
                                       stop, nh, nt, _stream(stream))
    _check(rc, "adaptive_norm_test_pair")
    return (bool(stop[0]), nh[0], nt[0]), (bool(stop[1]), nh[1], nt[1])


def _noalloc_shapes(Q, S_tilde, S_hat):
    """Shape and dtype agreement of the allocation-free call's operands.  The C
    side sees only pointers and S_tilde's shape and dtype, so an S_hat or a Q
    with fewer rows, or of another dtype, would be read or written past its end
    on the device; such calls are refused here."""
    for t, name in ((S_tilde, "S_tilde"), (S_hat, "S_hat")) + (((Q, "Q"),) if Q is not None else ()):
        if t.dim() != 2:
            raise ValueError(f"{name} must be 2-D")
    rows, b = S_tilde.shape
    if S_hat.shape[0] != rows or S_hat.shape[1] < b:
        raise ValueError(f"S_hat must have S_tilde's {rows} rows and at least its {b} columns")
    if S_hat.dtype != S_tilde.dtype:
        raise ValueError("S_hat must have S_tilde's dtype")
    if Q is not None:
        if Q.shape[0] != rows:
            raise ValueError(f"Q must have S_tilde's {rows} rows")
        if Q.dtype != S_tilde.dtype:
            raise ValueError("Q must have S_tilde's dtype")


def sketch_project_norms_noalloc(Q, S_tilde, S_hat, eps_rel: float, eps_abs: float, stream=None):
    """(I - Q Q^T)^2 S_tilde into S_hat without device allocation; returns
    (stop, ||S_hat||_F, ||S_tilde||_F).  Q may be None for an empty basis."""
    _noalloc_shapes(Q, S_tilde, S_hat)
    _check_2d(S_tilde, "S_tilde")
    _check_2d(S_hat, "S_hat")
    q_ptr, ldq, qc = None, 0, 0
    if Q is not None:
        _check_2d(Q, "Q")
        q_ptr, ldq, qc = Q.data_ptr(), Q.stride(0), Q.shape[1]
    stop = ctypes.c_int32()
    nh = ctypes.c_double()
    nt = ctypes.c_double()
    rc = lib().sketch_project_norms_noalloc(q_ptr, ldq, qc, S_tilde.data_ptr(), S_tilde.stride(0),
                                            S_tilde.shape[0], S_tilde.shape[1], _dtype_code(S_tilde),
                                            S_hat.data_ptr(), S_hat.stride(0), float(eps_rel), float(eps_abs),
                                            ctypes.byref(stop), ctypes.byref(nh), ctypes.byref(nt), _stream(stream))
    _check(rc, "sketch_project_norms_noalloc")
    return bool(stop.value), nh.value, nt.value


def kernel_matrix(gen: SkMatrix, A, stream=None) -> None:
    _check_2d(A, "A")
    _check(lib().kernel_matrix(ctypes.byref(gen), A.data_ptr(), A.stride(0), _stream(stream)), "kernel_matrix")


def _check_points(t, name):
    import torch
    if t.dim() != 2 or t.shape[1] != 3 or not t.is_contiguous() or not t.is_cuda or t.dtype != torch.float32:
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of shape (m, 3)")


def sketch_kernel_apply(h, X, Y, h_bw: float, S, shift: float = 0.0, stream=None) -> None:
    """S = K(X, Y; h) R (+ shift on the diagonal), K never formed (SJLT handles, FP32)."""
    _check_points(X, "X")
    _check_points(Y, "Y")
    _check_2d(S, "S")
    _check(lib().sketch_kernel_apply(h, X.data_ptr(), X.shape[0], Y.data_ptr(), float(h_bw), float(shift),
                                     S.data_ptr(), S.stride(0), _stream(stream)), "sketch_kernel_apply")


def sketch_kernel_adjoint(h, X, h_bw: float, dS, dX, dh, stream=None) -> None:
    """dX (n x 3) and dh (one float64 on the device) of <dS, K(X, X; h) R>."""
    _check_points(X, "X")
    _check_points(dX, "dX")
    _check_2d(dS, "dS")
    _check(lib().sketch_kernel_adjoint(h, X.data_ptr(), float(h_bw), dS.data_ptr(), dS.stride(0), dX.data_ptr(),
                                       dh.data_ptr(), _stream(stream)), "sketch_kernel_adjoint")


class Batch:
    """Many S'_i = A_i^T R_i (columns [c_lo_i, c_hi_i) of SJLT handles) in one persistent launch.

    ``items``: sequence of (op_handle, A, St, c_lo, c_hi) with A and St float32 CUDA tensors.
    The tensors must outlive the batch.  ``run()`` is asynchronous and capturable in a
    CUDA graph; ``set(active, c_lo, c_hi)`` changes what the next run (or replay) does.
    """

    def __init__(self, items, stream=None):
        arr = (SkBatchItem * len(items))()
        self._keep = []
        for k, (op, A, St, lo, hi) in enumerate(items):
            _check_2d(A, "A")
            _check_2d(St, "St")
            self._keep.append((A, St))
            arr[k] = SkBatchItem(op=op, A=A.data_ptr(), rows=A.shape[0], cols=A.shape[1], ld=A.stride(0),
                                 St=St.data_ptr(), ldSt=St.stride(0), c_lo=int(lo), c_hi=int(hi), scale=0.0)
        self.count = len(items)
        self.b = ctypes.c_void_p()
        _check(lib().sketch_batch_create(ctypes.byref(self.b), arr, self.count, _stream(stream)),
               "sketch_batch_create")

    def set(self, active=None, c_lo=None, c_hi=None) -> None:
        def arr(x):
            if x is None:
                return None
            a = np.ascontiguousarray(np.asarray(x, dtype=np.int32))
            if a.shape != (self.count,):
                raise ValueError("one value per instance")
            return a
        a, lo, hi = arr(active), arr(c_lo), arr(c_hi)
        p = lambda x: None if x is None else x.ctypes.data  # noqa: E731
        _check(lib().sketch_batch_set(self.b, p(a), p(lo), p(hi)), "sketch_batch_set")

    def run(self, stream=None) -> None:
        _check(lib().sketch_batch_run(self.b, _stream(stream)), "sketch_batch_run")

    def tune(self, stream=None) -> None:
        """Re-pick the kernel shape by timing the current ranges (synchronizes; not capturable)."""
        _check(lib().sketch_batch_tune(self.b, _stream(stream)), "sketch_batch_tune")

    def adaptive_setup(self, d0, dd: int, eps_rel: float, eps_abs: float = 0.0, stream=None) -> None:
        """Prepare Algorithm 1's loop per instance (operators JL(d0_i + dd) grown by dd-column
        increments up to the columns the loop may use); synchronizes, not capturable."""
        a = np.ascontiguousarray(np.asarray(d0, dtype=np.int32))
        if a.shape != (self.count,):
            raise ValueError("one d0 per instance")
        _check(lib().sketch_batch_adaptive_setup(self.b, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                 int(dd), float(eps_rel), float(eps_abs), _stream(stream)),
               "sketch_batch_adaptive_setup")

    def adaptive_run(self, max_rounds: int = 0, stream=None) -> None:
        """Enqueue the whole adaptive loop (asynchronous; capturable in one CUDA graph)."""
        _check(lib().sketch_batch_adaptive_run(self.b, int(max_rounds), _stream(stream)),
               "sketch_batch_adaptive_run")

    def adaptive_result(self, stream=None) -> dict:
        """Per instance: d (columns sketched), state (1 converged, 2 out of increments, 0 still
        running), tests taken, and the last test's ||S^||_F and ||S~||_F."""
        n = self.count
        d, st, t = (np.zeros(n, np.int32) for _ in range(3))
        nh, nt = np.zeros(n), np.zeros(n)
        pi = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))  # noqa: E731
        pd = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
        _check(lib().sketch_batch_adaptive_result(self.b, pi(d), pi(st), pi(t), pd(nh), pd(nt), _stream(stream)),
               "sketch_batch_adaptive_result")
        return dict(d=d, state=st, tests=t, nh=nh, nt=nt)

    def info(self) -> dict:
        w, nb, u = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        ms = (ctypes.c_float * 4)()
        _check(lib().sketch_batch_info(self.b, ctypes.byref(w), ctypes.byref(nb), ctypes.byref(u), ms),
               "sketch_batch_info")
        return dict(warps=w.value, cols_per_warp=nb.value, units=u.value, tuned_ms=[round(x, 4) for x in ms])

    def status(self, stream=None) -> None:
        _check(lib().sketch_batch_status(self.b, _stream(stream)), "sketch_batch_status")

    def close(self):
        if self.b:
            lib().sketch_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SrhtBatch:
    """Many S_i = A_i R_i (columns [c_lo_i, c_hi_i) of SRHT handles, orders nu_i <= 4096) in
    one persistent launch.

    ``items``: sequence of (op_handle, A, S, c_lo, c_hi) with A (rows x n_i) and S float32
    CUDA tensors that outlive the batch.  ``run()`` is asynchronous and capturable in a CUDA
    graph; ``set(c_lo, c_hi)`` changes the ranges of the next run (or replay).
    """

    def __init__(self, items, stream=None):
        arr = (SkSrhtBatchItem * len(items))()
        self._keep = []
        for k, (op, A, S, lo, hi) in enumerate(items):
            _check_2d(A, "A")
            _check_2d(S, "S")
            if str(A.dtype) != "torch.float32" or str(S.dtype) != "torch.float32":
                raise ValueError("A and S must be float32")
            self._keep.append((A, S))
            arr[k] = SkSrhtBatchItem(op=op, A=A.data_ptr(), rows=A.shape[0], ld=A.stride(0), S=S.data_ptr(),
                                     ldS=S.stride(0), c_lo=int(lo), c_hi=int(hi), scale=0.0)
        self.count = len(items)
        self.b = ctypes.c_void_p()
        _check(lib().sketch_srht_batch_create(ctypes.byref(self.b), arr, self.count, _stream(stream)),
               "sketch_srht_batch_create")

    def set(self, c_lo=None, c_hi=None) -> None:
        def arr(x):
            if x is None:
                return None
            a = np.ascontiguousarray(np.asarray(x, dtype=np.int32))
            if a.shape != (self.count,):
                raise ValueError("one value per instance")
            return a
        lo, hi = arr(c_lo), arr(c_hi)
        p = lambda x: None if x is None else x.ctypes.data  # noqa: E731
        _check(lib().sketch_srht_batch_set(self.b, p(lo), p(hi)), "sketch_srht_batch_set")

    def run(self, stream=None) -> None:
        _check(lib().sketch_srht_batch_run(self.b, _stream(stream)), "sketch_srht_batch_run")

    def adaptive_setup(self, d0, dd: int, eps_rel: float, eps_abs: float = 0.0, stream=None) -> None:
        """Prepare Algorithm 1's loop per instance (operators SRHT(d0_i + dd) grown by dd-column
        increments up to the columns the loop may use); synchronizes, not capturable."""
        a = np.ascontiguousarray(np.asarray(d0, dtype=np.int32))
        if a.shape != (self.count,):
            raise ValueError("one d0 per instance")
        _check(lib().sketch_srht_batch_adaptive_setup(self.b, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                      int(dd), float(eps_rel), float(eps_abs), _stream(stream)),
               "sketch_srht_batch_adaptive_setup")

    def adaptive_run(self, max_rounds: int = 0, stream=None) -> None:
        """Enqueue the whole adaptive loop (asynchronous; capturable in one CUDA graph)."""
        _check(lib().sketch_srht_batch_adaptive_run(self.b, int(max_rounds), _stream(stream)),
               "sketch_srht_batch_adaptive_run")

    def adaptive_result(self, stream=None) -> dict:
        """Per instance: d, state (1 converged, 2 out of columns, 0 still running), tests, and
        the last test's ||S^||_F and ||S~||_F."""
        n = self.count
        d, st, t = (np.zeros(n, np.int32) for _ in range(3))
        nh, nt = np.zeros(n), np.zeros(n)
        pi = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))  # noqa: E731
        pd = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
        _check(lib().sketch_srht_batch_adaptive_result(self.b, pi(d), pi(st), pi(t), pd(nh), pd(nt),
                                                       _stream(stream)), "sketch_srht_batch_adaptive_result")
        return dict(d=d, state=st, tests=t, nh=nh, nt=nt)

    def info(self) -> dict:
        c, u, sp = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
        ms = (ctypes.c_float * 6)()
        _check(lib().sketch_srht_batch_info(self.b, ctypes.byref(c), ctypes.byref(u), ms, ctypes.byref(sp)),
               "sketch_srht_batch_info")
        return dict(ctas_per_sm=c.value, units=u.value, split=bool(sp.value), tuned_ms=[round(x, 4) for x in ms])

    def close(self):
        if self.b:
            lib().sketch_srht_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sketch_dims(h) -> dict:
    kind, d, alpha, blocks = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    n = ctypes.c_int64()
    _check(lib().sketch_dims(h, ctypes.byref(kind), ctypes.byref(n), ctypes.byref(d), ctypes.byref(alpha),
                             ctypes.byref(blocks)), "sketch_dims")
    return dict(kind=kind.value, n=n.value, d_total=d.value, alpha=alpha.value, blocks=blocks.value)


def sketch_export(h, dense: bool = False, dense_dtype: int = SK_F64) -> dict:
    """Host copies: SJLT cols/signs, SRHT diag/mu, and optionally dense R."""
    dims = sketch_dims(h)
    n, d, a, B, kind = dims["n"], dims["d_total"], dims["alpha"], dims["blocks"], dims["kind"]
    out = {}
    cols = signs = diag = mu = R = None
    if kind in (SK_SJLT_GRAPH, SK_SJLT_BLOCK):
        cols = np.zeros((n, a * B), dtype=np.int32)
        signs = np.zeros((n, a * B), dtype=np.int8)
        out.update(cols=cols, signs=signs)
    if kind == SK_SRHT:
        diag = np.zeros(n, dtype=np.int8)
        mu = np.zeros(d, dtype=np.int32)
        out.update(diag=diag, mu=mu)
    if dense:
        R = np.zeros((n, d), dtype=np.float64 if dense_dtype == SK_F64 else np.float32)
        out["R"] = R
    ptr = lambda x: None if x is None else x.ctypes.data  # noqa: E731
    _check(lib().sketch_export(h, ptr(cols), ptr(signs), ptr(diag), ptr(mu), ptr(R), int(dense_dtype)),
           "sketch_export")
    return out


def sketch_device_status(h, stream=None) -> None:
    _check(lib().sketch_device_status(h, _stream(stream)), "sketch_device_status")


def sketch_launch_count() -> int:
    return int(lib().sketch_launch_count())


def sketch_srht_route(nu: int, rows: int, cols: int, width: int, prec: int) -> int:
    """1: row FWHT, 0: +-1 product, -1: shape not measured yet (SRHT S = A R)."""
    return int(lib().sketch_srht_route(int(nu), int(rows), int(cols), int(width), int(prec)))


def sketch_sjlt_route(kind, n: int, rows: int, cols: int, width: int, which: int) -> int:
    """1 tensor-core +-1 product, 0 SJLT kernels, -1 not measured (SK_PREC_BF16X2 products of FP32 data)."""
    k = KIND_NAMES.get(kind, kind) if isinstance(kind, str) else int(kind)
    return int(lib().sketch_sjlt_route(k, int(n), int(rows), int(cols), int(width), int(which)))


def sketch_destroy(h) -> None:
    if h:
        lib().sketch_destroy(h)


class Sketch:
    """Owning wrapper of a handle (closes it on exit / garbage collection)."""

    def __init__(self, kind, n, d, alpha=1, seed=0, d_max=None, stream=None, flags=0):
        self.h = sketch_create(kind, n, d, alpha, seed, d_max, stream, flags)

    def close(self):
        if self.h:
            sketch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sketch_selftest_wait(stream=None) -> int:
    """Run the bounded-wait self test; returns the status code (SK_ERR_TIMEOUT expected)."""
    return int(lib().sketch_selftest_wait(_stream(stream)))


# --- per-node adaptive HSS compression (Algorithm 1) ------------------------
OUTCOMES = {0: "passed", 1: "rank", 2: "failed"}


class Hss:
    """hss_compress_adaptive on a symmetric FP64 device matrix A (n x n); the
    generators are read back to the host on request."""

    def __init__(self, A, leaf: int, kind, d0: int, dd: int, alpha: int = 1, seed: int = 0,
                 d_max: int = 512, eps_rel: float = 1e-6, eps_abs: float = 0.0, stream=None):
        import torch
        _check_2d(A, "A")
        if A.dtype != torch.float64 or A.shape[0] != A.shape[1]:
            raise TypeError("A must be a square float64 CUDA tensor")
        k = KIND_NAMES[kind] if isinstance(kind, str) else int(kind)
        h = ctypes.c_void_p()
        _check(lib().hss_compress_adaptive(ctypes.byref(h), A.data_ptr(), A.shape[0], A.stride(0), int(leaf), k,
                                           int(d0), int(dd), int(alpha), int(seed), int(d_max), float(eps_rel),
                                           float(eps_abs), _stream(stream)), "hss_compress_adaptive")
        self.h = h.value
        self.n = A.shape[0]
        self.dd = int(dd)

    def info(self) -> dict:
        v = [ctypes.c_int32() for _ in range(6)]
        _check(lib().hss_info(self.h, *[ctypes.byref(x) for x in v]), "hss_info")
        keys = ("nodes", "d", "d_total", "sweeps", "converged", "tests")
        return {k: x.value for k, x in zip(keys, v)}

    def node(self, i: int) -> dict:
        lohi = (ctypes.c_int64 * 2)()
        inf = (ctypes.c_int32 * 7)()
        _check(lib().hss_node(self.h, int(i), lohi, inf), "hss_node")
        return dict(lo=lohi[0], hi=lohi[1], level=inf[0], parent=inf[1], c1=inf[2], c2=inf[3], state=inf[4],
                    m=inf[5], k=inf[6])

    def get(self, i: int, what: int, shape, dtype, order: str = "F") -> np.ndarray:
        """One generator of node i as a host array of `shape` (column-major
        unless order == "C")."""
        out = np.zeros(int(np.prod(shape)), dtype=dtype)
        if out.size:
            _check(lib().hss_node_get(self.h, int(i), int(what), out.ctypes.data), "hss_node_get")
        if len(shape) != 2:
            return out
        return out.reshape(shape) if order == "C" else out.reshape(tuple(reversed(shape))).T

    def generators(self, i: int) -> dict:
        """U, J, It, R, S (and D for a leaf, B for a node with children) of node i."""
        nd = self.node(i)
        out = dict(nd)
        m, k = nd["m"], nd["k"]
        w = self.columns()
        if nd["state"] == 2 and i != 0:
            out["U"] = self.get(i, SK_HSS_U, (m, k), np.float64, order="C")
            out["J"] = self.get(i, SK_HSS_J, (k,), np.int32)
            out["It"] = self.get(i, SK_HSS_IT, (k,), np.int32)
            out["R"] = self.get(i, SK_HSS_R, (k, w), np.float64)
        if i != 0 and nd["state"] != 0:
            out["S"] = self.get(i, SK_HSS_S, (m, w), np.float64)
        if nd["c1"] < 0:
            if nd["state"] != 0:
                out["D"] = self.get(i, SK_HSS_D, (m, m), np.float64)
        elif nd["state"] == 2:
            k1, k2 = self.node(nd["c1"])["k"], self.node(nd["c2"])["k"]
            out["B"] = self.get(i, SK_HSS_B, (k1, k2), np.float64)
        return out

    def columns(self) -> int:
        """Columns of S_tau and R_tau held: d + Delta-d of the last sweep."""
        return self.info()["d"] + self.dd

    def history(self) -> list:
        t = self.info()["tests"]
        ints = np.zeros(4 * max(t, 1), dtype=np.int32)
        reals = np.zeros(3 * max(t, 1), dtype=np.float64)
        _check(lib().hss_history(self.h, ints.ctypes.data, reals.ctypes.data), "hss_history")
        return [(int(ints[4 * u]), int(ints[4 * u + 1]), int(ints[4 * u + 2]), OUTCOMES[int(ints[4 * u + 3])],
                 float(reals[3 * u]), float(reals[3 * u + 1]), float(reals[3 * u + 2])) for u in range(t)]

    def launches(self) -> int:
        return int(lib().hss_launch_count(self.h))

    PROFILE_KINDS = ("gather", "local_sketch", "test", "id", "r_tau", "global_sketch")

    def profile(self) -> dict:
        """Per kind of work: device ms, algorithmic FP64 FLOPs, launches, average SMs held."""
        ms = np.zeros(6)
        fl = np.zeros(6)
        ln = np.zeros(6, dtype=np.int64)
        sm = np.zeros(6)
        _check(lib().hss_profile(self.h, ms.ctypes.data, fl.ctypes.data, ln.ctypes.data, sm.ctypes.data),
               "hss_profile")
        return {k: dict(ms=float(ms[i]), flops=float(fl[i]), launches=int(ln[i]),
                        avg_sms=float(sm[i] / ms[i]) if ms[i] > 0 else 0.0)
                for i, k in enumerate(self.PROFILE_KINDS)}

    def close(self):
        if self.h:
            lib().hss_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

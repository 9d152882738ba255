"""The C ABI library loads and exports every entry point include/jlsketch.h
declares; constants agree; host-side argument checks and the no-GPU path
return the documented status codes (no compute call is made here)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2302_01977_gb300 import jlsketch as jl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(jl.LIB_PATH):
        from paper_2302_01977_gb300 import build
        build.build()
    return jl.lib()


def declared_functions():
    text = open(jl.HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|int64_t|void|const char\*)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(jl.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", jl.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(L, name)


def test_constants_match_header():
    hc = jl.header_constants()
    for name, val in hc.items():
        assert getattr(jl, name) == val, name
    assert len(hc) >= 20


def test_strerror_covers_codes(L):
    for code in range(0, -10, -1):
        s = jl.sketch_strerror(code)
        assert s and s != "unknown status"
    assert jl.sketch_strerror(-99) == "unknown status"


def test_create_argument_checks(L):
    h = ctypes.c_void_p()
    bad = [
        (0, 64, 16, 4, 16),            # kind
        (jl.SK_SJLT_BLOCK, 0, 16, 4, 16),   # n
        (jl.SK_SJLT_BLOCK, 64, 0, 4, 16),   # d
        (jl.SK_SJLT_BLOCK, 64, 16, 3, 16),  # alpha does not divide d
        (jl.SK_SJLT_GRAPH, 64, 4, 8, 16),   # alpha > d
        (jl.SK_SJLT_GRAPH, 64, 64, 33, 64),  # alpha > 32
        (jl.SK_GAUSS, 64, 16, 1, 8),        # d_max < d
        (jl.SK_SRHT, 64, 16, 1, 128),       # d_max > nu
        (jl.SK_GAUSS, 64, 16, 1, 9000),     # d_max > 8192
    ]
    for kind, n, d, a, dmax in bad:
        assert L.sketch_create(ctypes.byref(h), kind, n, d, a, 1, dmax, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_create(None, jl.SK_GAUSS, 64, 16, 1, 1, 16, None) == jl.SK_ERR_INVALID_ARG


def test_null_handle_calls(L):
    assert L.sketch_increment(None, 4, None) == jl.SK_ERR_INVALID_ARG
    m = jl.SkMatrix()
    assert L.sketch_apply(None, ctypes.byref(m), 1, 0, None, 0, None, 0, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_dims(None, None, None, None, None, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_device_status(None, None) == jl.SK_ERR_INVALID_ARG
    L.sketch_destroy(None)  # no-op
    assert L.kernel_matrix(None, None, 0, None) == jl.SK_ERR_INVALID_ARG
    # batches and their adaptive loop
    assert L.sketch_batch_create(None, None, 0, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_batch_run(None, None) == jl.SK_ERR_INVALID_ARG
    d0 = (ctypes.c_int32 * 1)(32)
    assert L.sketch_batch_adaptive_setup(None, d0, 32, 1e-3, 0.0, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_batch_adaptive_run(None, 0, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_batch_adaptive_result(None, None, None, None, None, None, None) == jl.SK_ERR_INVALID_ARG
    L.sketch_batch_destroy(None)  # no-op
    # batches of SRHT sketches
    assert L.sketch_srht_batch_create(None, None, 0, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_srht_batch_set(None, None, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_srht_batch_run(None, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_srht_batch_info(None, None, None, None, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_srht_batch_adaptive_setup(None, d0, 32, 1e-3, 0.0, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_srht_batch_adaptive_run(None, 0, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_srht_batch_adaptive_result(None, None, None, None, None, None, None) == jl.SK_ERR_INVALID_ARG
    L.sketch_srht_batch_destroy(None)  # no-op


def test_no_gpu_fails_loudly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert L.sketch_create(ctypes.byref(h), jl.SK_GAUSS, 64, 16, 1, 1, 16, None) == jl.SK_ERR_DEVICE
    assert L.sketch_selftest_wait(None) == jl.SK_ERR_DEVICE
    with pytest.raises(jl.JLSketchError):
        jl.sketch_create("gauss", 64, 16, stream=0)


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(jl, "_lib", None)
    monkeypatch.setattr(jl, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        jl.lib()


def test_noalloc_wrapper_refuses_mismatched_operands():
    """The allocation-free call's C side sees only pointers and S_tilde's shape
    and dtype; the binding refuses operands that would be read or written past
    their ends (checked on CPU tensors: the refusal comes before any device use)."""
    import torch
    St = torch.zeros((64, 8), dtype=torch.float32)
    ok_hat = torch.zeros((64, 8), dtype=torch.float32)
    ok_q = torch.zeros((64, 16), dtype=torch.float32)
    bad = [
        (ok_q, St, torch.zeros((63, 8)), "rows"),                      # S_hat has fewer rows
        (ok_q, St, torch.zeros((64, 7)), "columns"),                   # S_hat has fewer columns
        (ok_q, St, torch.zeros((64, 8), dtype=torch.float64), "dtype"),  # S_hat of another dtype
        (torch.zeros((60, 16)), St, ok_hat, "rows"),                   # Q has fewer rows
        (torch.zeros((64, 16), dtype=torch.float64), St, ok_hat, "dtype"),  # Q of another dtype
        (ok_q, torch.zeros(64), ok_hat, "2-D"),                        # S_tilde not 2-D
    ]
    for Q, S_t, S_h, what in bad:
        with pytest.raises(ValueError, match=what):
            jl.sketch_project_norms_noalloc(Q, S_t, S_h, 1e-2, 0.0)
    # consistent operands pass the shape checks and stop at the device check
    with pytest.raises(ValueError, match="CUDA"):
        jl.sketch_project_norms_noalloc(ok_q, St, ok_hat, 1e-2, 0.0)
    with pytest.raises(ValueError, match="CUDA"):
        jl.sketch_project_norms_noalloc(None, St, torch.zeros((64, 9)), 1e-2, 0.0)


def test_create_flags_argument_checks(L):
    """Flag checks come before any device use (no GPU needed)."""
    h = ctypes.c_void_p()
    assert L.sketch_create_flags(ctypes.byref(h), jl.SK_GAUSS, 64, 16, 1, 1, 16, jl.SK_SRHT_REPLACE,
                                 None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_create_flags(ctypes.byref(h), jl.SK_SRHT, 64, 16, 1, 1, 16, 4, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_create_flags(ctypes.byref(h), jl.SK_SRHT, 64, 16, 1, 1, 80, 0, None) == jl.SK_ERR_INVALID_ARG
    assert L.sketch_create_flags(None, jl.SK_SRHT, 64, 16, 1, 1, 16, 0, None) == jl.SK_ERR_INVALID_ARG


def test_hss_argument_checks(L):
    """hss_compress_adaptive refuses bad sizes, tolerances and alignment before it touches a device."""
    h = ctypes.c_void_p()
    A = ctypes.c_void_p(1 << 20)  # never dereferenced: every case below is refused first
    good = dict(n=512, lda=512, leaf=64, kind=jl.SK_GAUSS, d0=16, dd=16, alpha=1, d_max=64, er=1e-6, ea=0.0)
    bad = [dict(n=0), dict(lda=100), dict(leaf=0), dict(leaf=5000), dict(d0=0), dict(dd=0), dict(d_max=16),
           dict(d_max=4096), dict(d_max=63), dict(er=-1.0), dict(ea=float("nan"))]
    for b in bad:
        a = dict(good, **b)
        rc = L.hss_compress_adaptive(ctypes.byref(h), A, a["n"], a["lda"], a["leaf"], a["kind"], a["d0"], a["dd"],
                                     a["alpha"], 1, a["d_max"], a["er"], a["ea"], None)
        assert rc == jl.SK_ERR_INVALID_ARG, b
    a = good
    assert L.hss_compress_adaptive(None, A, 512, 512, 64, jl.SK_GAUSS, 16, 16, 1, 1, 64, 1e-6, 0.0,
                                   None) == jl.SK_ERR_INVALID_ARG
    assert L.hss_compress_adaptive(ctypes.byref(h), None, 512, 512, 64, jl.SK_GAUSS, 16, 16, 1, 1, 64, 1e-6, 0.0,
                                   None) == jl.SK_ERR_INVALID_ARG
    # A not 16-byte aligned, or a leading dimension whose rows are not
    assert L.hss_compress_adaptive(ctypes.byref(h), ctypes.c_void_p((1 << 20) + 8), 512, 512, 64, jl.SK_GAUSS, 16,
                                   16, 1, 1, 64, 1e-6, 0.0, None) == jl.SK_ERR_ALIGN
    assert L.hss_compress_adaptive(ctypes.byref(h), A, 512, 513, 64, jl.SK_GAUSS, 16, 16, 1, 1, 64, 1e-6, 0.0,
                                   None) == jl.SK_ERR_ALIGN


def test_hss_null_handle_calls(L):
    i32 = ctypes.c_int32()
    assert L.hss_info(None, ctypes.byref(i32), None, None, None, None, None) == jl.SK_ERR_INVALID_ARG
    assert L.hss_node(None, 0, None, None) == jl.SK_ERR_INVALID_ARG
    assert L.hss_node_get(None, 0, jl.SK_HSS_U, ctypes.c_void_p(1 << 20)) == jl.SK_ERR_INVALID_ARG
    assert L.hss_history(None, None, None) == jl.SK_ERR_INVALID_ARG
    assert L.hss_profile(None, None, None, None, None) == jl.SK_ERR_INVALID_ARG
    assert L.hss_launch_count(None) == 0
    L.hss_destroy(None)  # no-op


def test_hss_no_gpu_fails_loudly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert L.hss_compress_adaptive(ctypes.byref(h), ctypes.c_void_p(1 << 20), 512, 512, 64, jl.SK_GAUSS, 16, 16, 1,
                                   1, 64, 1e-6, 0.0, None) == jl.SK_ERR_DEVICE

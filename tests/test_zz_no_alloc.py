"""The allocation-free projection/norms entry point against adaptive_norm_test.

sketch_project_norms_noalloc serves callers that cannot allocate device memory
(processes whose device memory belongs to another allocator or a fixed pool).
Here it is called through the C ABI twice in a row (before and after an
increment) and its norms and stop decision are compared with the handle-based
adaptive_norm_test on the same sketch, to the parity tolerances used elsewhere
(FP64 1e-9 of ||S~||_F, FP32 1e-5); around the second call the device's free
memory must not change.  The basis it needs is built on the host
with numpy from the GPU sketch.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2302_01977_gb300 import inputs
from tests.util import dev_padded, ensure_built, host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_adaptive_norm_test_twice(dtype):
    from paper_2302_01977_gb300 import jlsketch as jl
    tdt = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-9 if dtype == "f64" else 1e-5
    n, d0, dd = 1500, 32, 16
    A_np = inputs.spectrum_matrix(n, 0.85 ** np.arange(n), seed=11)
    A = dev_padded(A_np, tdt)
    h = jl.sketch_create("gauss", n, d0 + dd, 1, 5, d0 + 2 * dd)
    try:
        S = torch.zeros((n, d0 + 2 * dd), dtype=tdt, device="cuda")
        jl.sketch_apply(h, A, jl.SK_S, S=S)
        d = d0
        for call in range(2):
            w = d + dd
            stop0, nh0, nt0 = jl.adaptive_norm_test(h, 0, S[:, :w], dd, 1e-3, 1e-30)
            Sh = host(S[:, :w]).astype(np.float64)
            Q = np.linalg.qr(Sh[:, :d])[0]
            Qd = torch.from_numpy(np.ascontiguousarray(Q)).to(tdt).cuda()
            S_hat = torch.full((n, dd), np.nan, dtype=tdt, device="cuda")
            if call == 1:  # every kernel of the call has run once: nothing is loaded lazily now
                torch.cuda.synchronize()
                free0 = torch.cuda.mem_get_info()[0]
            stop1, nh1, nt1 = jl.sketch_project_norms_noalloc(Qd, S[:, d:w], S_hat, 1e-3, 1e-30)
            if call == 1:  # the call took no device memory
                torch.cuda.synchronize()
                assert torch.cuda.mem_get_info()[0] == free0
            assert abs(nt1 - nt0) <= tol * nt0
            assert abs(nh1 - nh0) <= tol * nt0
            if abs(nh0 / nt0 - 1e-3) > 2 * tol:
                assert stop1 == stop0
            # the returned block is the projection: orthogonal to Q, norm as reported
            P = host(S_hat).astype(np.float64)
            assert np.abs(Q.T @ P).max() <= 10 * tol * nt0
            assert abs(np.linalg.norm(P) - nh1) <= tol * nt0
            if call == 0:
                jl.sketch_increment(h, dd)
                jl.sketch_apply_increment(h, A, jl.SK_S, S=S)
                d += dd
        jl.sketch_device_status(h)
    finally:
        jl.sketch_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2302_01977_gb300 import jlsketch as jl
    S = torch.zeros((128, 65), dtype=torch.float32, device="cuda")
    out = torch.zeros_like(S)
    with pytest.raises(jl.JLSketchError) as e:
        jl.sketch_project_norms_noalloc(None, S, out, 1e-2, 0.0)
    assert e.value.status == jl.SK_ERR_INVALID_ARG
    Q = torch.zeros((128, 1025), dtype=torch.float32, device="cuda")
    S2 = torch.zeros((128, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(jl.JLSketchError) as e:
        jl.sketch_project_norms_noalloc(Q, S2, torch.zeros_like(S2), 1e-2, 0.0)
    assert e.value.status == jl.SK_ERR_INVALID_ARG

"""Complex A (interleaved FP32 parts) with real SJLT, SRHT and Gaussian
operators: S = A R and S' = A* R (the conjugate transpose of Sec. 6.3)
against the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sketch as osk  # noqa: E402
from paper_2302_01977_gb300 import inputs  # noqa: E402
from paper_2302_01977_gb300 import jlsketch as jl  # noqa: E402

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def helmholtz(n, kappa, seed):
    """A_ij = exp(i kappa r_ij) / (1 + kappa r_ij) for points uniform in [0,1]^3 (symmetric, complex)."""
    X = torch.from_numpy(inputs.points(n, seed=seed)).cuda().double()
    r = torch.cdist(X, X)
    return (torch.exp(1j * kappa * r) / (1.0 + kappa * r)).to(torch.complex64).contiguous()


@pytest.mark.parametrize("kind,n,d,alpha", [("sjlt_block", 1000, 64, 4), ("sjlt_graph", 514, 40, 3),
                                            ("sjlt_block", 2048, 256, 4)])
def test_complex_sketch_matches_oracle(kind, n, d, alpha):
    g = torch.Generator().manual_seed(n)
    A = torch.complex(torch.randn(n, n, generator=g), torch.randn(n, n, generator=g)).cuda()
    with jl.Sketch(kind, n, d, alpha, 5) as op:
        S = torch.empty((n, d), dtype=torch.complex64, device="cuda")
        St = torch.empty_like(S)
        jl.sketch_apply(op.h, A, jl.SK_BOTH, S=S, St=St)
        jl.sketch_device_status(op.h)
        R = jl.sketch_export(op.h, dense=True)["R"]
    S0, St0 = osk.apply_complex(A.cpu().numpy(), R)
    assert rel(S.cpu().numpy().astype(np.complex128), S0) <= 1e-5
    assert rel(St.cpu().numpy().astype(np.complex128), St0) <= 1e-5


def test_complex_rectangular_and_increment():
    m, n, d, dd = 300, 1000, 64, 32
    g = torch.Generator().manual_seed(3)
    A = torch.complex(torch.randn(m, n, generator=g), torch.randn(m, n, generator=g)).cuda()
    with jl.Sketch("sjlt_block", n, d, 4, 9, d_max=d + dd) as op:
        S = torch.full((m, d + dd), 7.0 + 7.0j, dtype=torch.complex64, device="cuda")
        jl.sketch_apply(op.h, A, jl.SK_S, S=S)
        jl.sketch_increment(op.h, dd)
        jl.sketch_apply_increment(op.h, A, jl.SK_S, S=S)
        jl.sketch_device_status(op.h)
        R = jl.sketch_export(op.h, dense=True)["R"]
    S0 = osk.complex_s(A.cpu().numpy(), R)
    assert rel(S.cpu().numpy().astype(np.complex128), S0) <= 1e-5
    # S' of the same A needs rows == n of R: a separate operator over the m rows
    with jl.Sketch("sjlt_block", m, d, 4, 11) as op2:
        St = torch.empty((n, d), dtype=torch.complex64, device="cuda")
        jl.sketch_apply(op2.h, A, jl.SK_ST, St=St)
        jl.sketch_device_status(op2.h)
        R2 = jl.sketch_export(op2.h, dense=True)["R"]
    St0 = osk.complex_t(A.cpu().numpy(), R2)
    assert rel(St.cpu().numpy().astype(np.complex128), St0) <= 1e-5


def test_complex_helmholtz_symmetry():
    """A symmetric complex A (A^T = A) gives A* R = conj(A R)."""
    n = 1536
    A = helmholtz(n, 20.0, 4)
    with jl.Sketch("sjlt_block", n, 128, 4, 13) as op:
        S = torch.empty((n, 128), dtype=torch.complex64, device="cuda")
        St = torch.empty_like(S)
        jl.sketch_apply(op.h, A, jl.SK_BOTH, S=S, St=St)
        jl.sketch_device_status(op.h)
    assert torch.linalg.norm(St - S.conj()) <= 1e-5 * torch.linalg.norm(S)


def test_complex_rejected_where_not_built():
    n = 256
    A = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    S = torch.empty((n, 32), dtype=torch.complex64, device="cuda")
    with jl.Sketch("sjlt_block", n, 32, 4, 1) as op:  # SJLT sums stay in FP32
        with pytest.raises(jl.JLSketchError):
            jl.sketch_apply(op.h, A, jl.SK_S, jl.SK_PREC_BF16X2, S=S)


# ---- SRHT and Gaussian operators on complex A: CUDA cores (FP32 sums) and the bf16 split on tensor cores

@pytest.mark.parametrize("kind,prec", [("srht", jl.SK_PREC_NATIVE), ("srht", jl.SK_PREC_BF16X2),
                                       ("gauss", jl.SK_PREC_NATIVE), ("gauss", jl.SK_PREC_BF16X2)])
@pytest.mark.parametrize("m,n,d", [(1000, 1000, 64), (300, 1500, 96)])
def test_complex_dense_operators(kind, prec, m, n, d):
    """S = A R and S' = A* R for complex A (rectangular, ragged sizes) with an
    SRHT or Gaussian R, then one increment, against the FP64 oracle with the
    exported R; the bf16 split keeps each product term within 2^-16 of A's."""
    dd = 32
    g = torch.Generator().manual_seed(m + n)
    A = torch.complex(torch.randn(m, n, generator=g), torch.randn(m, n, generator=g)).cuda()
    with jl.Sketch(kind, n, d, 1, 13, d_max=d + dd) as op:
        S = torch.full((m, d + dd), 7.0 + 7.0j, dtype=torch.complex64, device="cuda")
        jl.sketch_apply(op.h, A, jl.SK_S, prec, S=S)
        jl.sketch_increment(op.h, dd)
        jl.sketch_apply_increment(op.h, A, jl.SK_S, prec, S=S)
        jl.sketch_device_status(op.h)
        R = jl.sketch_export(op.h, dense=True)["R"]
    S0 = osk.complex_s(A.cpu().numpy(), R)
    assert rel(S.cpu().numpy().astype(np.complex128), S0) <= 1e-5
    with jl.Sketch(kind, m, d, 1, 17, d_max=d + dd) as op2:
        St = torch.full((n, d + dd), 7.0 + 7.0j, dtype=torch.complex64, device="cuda")
        jl.sketch_apply(op2.h, A, jl.SK_ST, prec, St=St)
        jl.sketch_increment(op2.h, dd)
        jl.sketch_apply_increment(op2.h, A, jl.SK_ST, prec, St=St)
        jl.sketch_device_status(op2.h)
        R2 = jl.sketch_export(op2.h, dense=True)["R"]
    St0 = osk.complex_t(A.cpu().numpy(), R2)
    assert rel(St.cpu().numpy().astype(np.complex128), St0) <= 1e-5


def test_complex_dense_helmholtz_conjugate_symmetry():
    """For the symmetric complex Helmholtz kernel, A* R = conj(A R) for any real
    R: the S' route (transpose product, conjugating interleave) and the S route
    (expanded operator) must agree to FP32 rounding."""
    n, d = 2048, 128
    A = helmholtz(n, 20.0, 3)
    for kind in ("srht", "gauss"):
        for prec in (jl.SK_PREC_NATIVE, jl.SK_PREC_BF16X2):
            with jl.Sketch(kind, n, d, 1, 21) as op:
                S = torch.empty((n, d), dtype=torch.complex64, device="cuda")
                St = torch.empty_like(S)
                jl.sketch_apply(op.h, A, jl.SK_BOTH, prec, S=S, St=St)
                jl.sketch_device_status(op.h)
            assert rel(St.cpu().numpy(), np.conj(S.cpu().numpy())) <= 2e-5, (kind, prec)


def test_complex_refuses_fp8():
    A = torch.zeros((64, 64), dtype=torch.complex64, device="cuda")
    with jl.Sketch("gauss", 64, 16, 1, 1) as op:
        S = torch.empty((64, 16), dtype=torch.complex64, device="cuda")
        with pytest.raises(jl.JLSketchError) as e:
            jl.sketch_apply(op.h, A, jl.SK_S, jl.SK_PREC_FP8, S=S)
        assert e.value.status == jl.SK_ERR_DTYPE

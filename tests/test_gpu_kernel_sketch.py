"""Matrix-free kernel sketch S = K(X, X; h) R and its adjoint (dX, dh) against
the FP64 oracle, central finite differences of the oracle's loss, and
properties that hold at any size (checked at the full n = 262144 size)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import kernel_grad as kg  # noqa: E402
from oracle import sketch as osk  # noqa: E402
from paper_2302_01977_gb300 import inputs  # noqa: E402
from paper_2302_01977_gb300 import jlsketch as jl  # noqa: E402
from paper_2302_01977_gb300.kernel_sketch import kernel_sketch  # noqa: E402

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def points(n, seed):
    return inputs.points(n, seed=seed).astype(np.float32)


def dense_R(op):
    return jl.sketch_export(op.h, dense=True)["R"]


@pytest.mark.parametrize("kind,n,d,alpha,h", [("sjlt_block", 1000, 64, 4, 0.2), ("sjlt_block", 4096, 256, 4, 0.05),
                                              ("sjlt_graph", 777, 48, 3, 0.1)])
def test_forward_matches_oracle(kind, n, d, alpha, h):
    X = points(n, 3)
    with jl.Sketch(kind, n, d, alpha, 41) as op:
        Xd = torch.from_numpy(X).cuda()
        S = torch.empty((n, d), device="cuda")
        jl.sketch_kernel_apply(op.h, Xd, Xd, h, S)
        jl.sketch_device_status(op.h)
        ref = kg.kernel_sketch(X.astype(np.float64), h, dense_R(op))
    assert rel(S.cpu().numpy(), ref) <= 1e-5


def test_forward_two_point_sets_shift_and_increment():
    n, m, h, shift = 900, 650, 0.15, 0.01
    X, Y = points(m, 5), points(n, 6)
    with jl.Sketch("sjlt_block", n, 32, 4, 8, d_max=96) as op:
        jl.sketch_increment(op.h, 32)
        S = torch.empty((m, 64), device="cuda")
        jl.sketch_kernel_apply(op.h, torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), h, S, shift=shift)
        jl.sketch_device_status(op.h)
        ref = osk.kernel_matrix(X.astype(np.float64), Y.astype(np.float64), h, shift) @ dense_R(op)
    assert rel(S.cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("kind,n,d,alpha,h,inc", [("sjlt_block", 4096, 256, 4, 0.05, 0),
                                                  ("sjlt_block", 1000, 64, 4, 0.2, 0),
                                                  ("sjlt_graph", 700, 40, 2, 0.15, 24)])
def test_adjoint_matches_oracle_gradient(kind, n, d, alpha, h, inc):
    X = points(n, 9)
    rng = np.random.default_rng(17)
    dS = rng.standard_normal((n, d + inc)).astype(np.float32)
    with jl.Sketch(kind, n, d, alpha, 23, d_max=d + inc) as op:
        if inc:
            jl.sketch_increment(op.h, inc)
        Xd = torch.from_numpy(X).cuda()
        dX = torch.empty_like(Xd)
        dh = torch.empty(1, dtype=torch.float64, device="cuda")
        jl.sketch_kernel_adjoint(op.h, Xd, h, torch.from_numpy(dS).cuda(), dX, dh)
        jl.sketch_device_status(op.h)
        gX, gh = kg.kernel_sketch_grad(X.astype(np.float64), h, dense_R(op), dS.astype(np.float64))
    assert rel(dX.cpu().numpy(), gX) <= 1e-4
    assert abs(float(dh.item()) - gh) <= 1e-4 * abs(gh)


def test_autograd_against_central_differences():
    """X.grad and h.grad through torch.autograd against FP64 central
    differences (step 1e-3) of the oracle's loss, on a 512-point problem."""
    n, d, h0 = 512, 32, 0.1
    X = points(n, 12)
    rng = np.random.default_rng(4)
    dS = rng.standard_normal((n, d)).astype(np.float32)
    with jl.Sketch("sjlt_block", n, d, 4, 77) as op:
        Xt = torch.from_numpy(X).cuda().requires_grad_(True)
        ht = torch.tensor(h0, dtype=torch.float32, device="cuda", requires_grad=True)
        S = kernel_sketch(Xt, ht, op)
        (S * torch.from_numpy(dS).cuda()).sum().backward()
        R = dense_R(op)
    coords = [(i, a) for i in (0, 101, 300, 511) for a in range(3)]
    fd, fd_h = kg.fd_grad(X.astype(np.float64), h0, R, dS.astype(np.float64), coords, step=1e-3)
    got = np.array([Xt.grad[i, a].item() for i, a in coords])
    scale = np.abs(Xt.grad.cpu().numpy()).max()
    np.testing.assert_allclose(got, fd, rtol=0, atol=2e-3 * scale)
    assert float(ht.grad.item()) == pytest.approx(fd_h, rel=2e-3)


def test_full_size_sampled_rows_and_invariants():
    """n = 262144, d = 256, alpha = 4, h = 0.05 (the differentiation workload):
    sampled rows of S and of dX against the FP64 oracle computed row by row,
    and the translation / scale invariances of the gradient."""
    n, d, h = 262144, 256, 0.05
    X = inputs.points(n, seed=20230203 + 4).astype(np.float32)
    rng = np.random.default_rng(99)
    with jl.Sketch("sjlt_block", n, d, 4, 20230207) as op:
        Xd = torch.from_numpy(X).cuda()
        S = torch.empty((n, d), device="cuda")
        jl.sketch_kernel_apply(op.h, Xd, Xd, h, S)
        dSd = torch.randn((n, d), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
        dX = torch.empty_like(Xd)
        dh = torch.empty(1, dtype=torch.float64, device="cuda")
        jl.sketch_kernel_adjoint(op.h, Xd, h, dSd, dX, dh)
        jl.sketch_device_status(op.h)
        ex = jl.sketch_export(op.h)
    cols, signs = ex["cols"].astype(np.int64), ex["signs"].astype(np.float64)
    scale = 0.5
    X64 = X.astype(np.float64)
    dS = dSd.cpu().numpy().astype(np.float64)
    S_h, dX_h = S.cpu().numpy(), dX.cpu().numpy().astype(np.float64)
    for i in rng.choice(n, 8, replace=False):
        r2 = ((X64 - X64[i]) ** 2).sum(axis=1)
        k = np.exp(-r2 / (2 * h * h))
        row = np.zeros(d)
        for a in range(4):
            np.add.at(row, cols[:, a], k * signs[:, a] * scale)
        assert rel(S_h[i], row) <= 1e-5
        # dX_i = (1/h^2) sum_j (G_ij + G_ji) K_ij (x_j - x_i)
        g_ij = scale * (dS[i][cols] * signs).sum(axis=1)                      # <dS_i, R_j> for all j
        g_ji = scale * (dS[:, cols[i]] * signs[i][None, :]).sum(axis=1)       # <dS_j, R_i> for all j
        want = (((g_ij + g_ji) * k)[:, None] * (X64 - X64[i])).sum(axis=0) / h ** 2
        assert np.linalg.norm(dX_h[i] - want) <= 1e-4 * np.linalg.norm(want) + 1e-6 * np.abs(dX_h).max()
    gh = float(dh.item())
    # K depends on differences: sum_i dX_i = 0; on X / h: h dh + sum_i x_i . dX_i = 0
    tot = np.abs(dX_h).sum(axis=0)
    assert np.all(np.abs(dX_h.sum(axis=0)) <= 1e-4 * tot)
    assert abs(h * gh + float((X64 * dX_h).sum())) <= 1e-4 * (abs(h * gh) + float(np.abs(X64 * dX_h).sum()))

"""The device kernel-matrix generator against the oracle's FP64 formula.

FP64: |dA| <= (4 + 8|arg|) * 2^-52 * A_64: exp rounding plus the argument, which
carries about four roundings (squares and sum, 1/(2h^2), the product).
FP32: the device works in FP32 (distance and expf), so the bound is a few ulp
plus the argument's rounding: |dA| <= (4 + 2|arg|) * 2^-23 * A_64 + 1e-37.
"""
import numpy as np
import pytest

from oracle import sketch as osk
from paper_2302_01977_gb300 import inputs
from tests.util import dev, ensure_built, host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("m,n,h,shift", [(300, 2100, 0.1, 0.0), (1025, 1025, 0.2, 1e-2), (7, 3, 0.5, 2.0)])
def test_kernel_matrix(dtype, m, n, h, shift):
    from paper_2302_01977_gb300 import jlsketch as jl
    npdt = np.float64 if dtype == "f64" else np.float32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    X = inputs.points(m, seed=m, dtype=npdt)
    Y = inputs.points(n, seed=n + 1, dtype=npdt) if m != n else X
    A = torch.full((m, n + 4), np.nan, dtype=tdt, device="cuda")
    jl.kernel_matrix(jl.generator(dev(X), dev(Y), h, shift), A)
    got = host(A)[:, :n]
    ref = osk.kernel_matrix(X, Y, h, shift)
    d2 = ((X.astype(np.float64)[:, None, :] - Y.astype(np.float64)[None]) ** 2).sum(-1)
    arg = d2 / (2 * h * h)
    if dtype == "f64":
        assert np.all(np.abs(got - ref) <= (4 + 8 * arg) * 2.0 ** -52 * ref)
    else:
        bound = (4 + 8 * arg) * 2.0 ** -23 * ref + 1e-37
        assert np.all(np.abs(got - ref) <= bound)

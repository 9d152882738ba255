"""Pins for the oracle's adaptive loop (CPU only).

* An exactly rank-r matrix with r < d0 has no range left for the new columns:
  the first test must stop with ||S^|| ~ 0 (Sec. 3, Eq. (3.1)).
* A matrix with a prescribed geometric singular spectrum reaches a larger d for
  a smaller eps_rel (the test is monotone in its tolerance).
* The two-pass projection leaves a block orthogonal to Q.
* With a rank-deficient S(:, 1:d) (a zero column, a repeated column) the test
  projects onto the orthogonal complement of the range of S(:, 1:d) (Sec. 3),
  with a closed-form ||S^||.
* A full-rank matrix with a flat spectrum never passes a tight test and stops
  at d_max without converging.
* norm_tests (every test of one sketch, the range basis grown block by block)
  equals norm_test test by test, on decaying, rank-deficient and exactly
  low-rank sketches.
"""
import numpy as np
import pytest

from oracle import adaptive as ad
from paper_2302_01977_gb300 import inputs

KINDS = [("sjlt_block", 4), ("sjlt_graph", 4), ("srht", 1), ("gauss", 1)]


@pytest.mark.parametrize("kind,alpha", KINDS)
def test_low_rank_stops_first_test(kind, alpha):
    n, r = 128, 12
    A = inputs.low_rank_matrix(n, r, seed=1)
    res = ad.adaptive(A, kind, d0=32, dd=16, alpha=alpha, seed=2, d_max=96,
                      eps_rel=1e-8, eps_abs=1e-30)
    assert res["converged"] and len(res["history"]) == 1
    d, stop, nh, nt, nh_t, nt_t = res["history"][0]
    assert nh < 1e-12 * nt and nh_t < 1e-12 * nt_t


@pytest.mark.parametrize("kind,alpha", KINDS)
def test_d_reached_monotone_in_eps(kind, alpha):
    n = 128
    sigma = 0.7 ** np.arange(n)
    A = inputs.spectrum_matrix(n, sigma, seed=3)
    reached = []
    for eps in (1e-1, 1e-3, 1e-6):
        res = ad.adaptive(A, kind, d0=8, dd=8, alpha=alpha, seed=4, d_max=128,
                          eps_rel=eps, eps_abs=1e-300, which="S")
        reached.append(res["op"].d_total)
    assert reached[0] <= reached[1] <= reached[2]
    assert reached[0] < reached[2]


def test_projection_orthogonal():
    Q, _ = np.linalg.qr(inputs.dense_matrix(200, 30, seed=5))
    B = inputs.dense_matrix(200, 7, seed=6)
    P = ad.project_twice(Q, B)
    assert np.abs(Q.T @ P).max() < 1e-13 * np.abs(B).max()
    # projecting a block already in range(Q) gives zero
    assert np.abs(ad.project_twice(Q, Q @ B[:30])).max() < 1e-13


def test_flat_spectrum_hits_d_max():
    n = 96
    A = inputs.spectrum_matrix(n, np.ones(n), seed=7)
    res = ad.adaptive(A, "gauss", d0=16, dd=16, alpha=1, seed=8, d_max=64,
                      eps_rel=1e-6, eps_abs=1e-300)
    assert not res["converged"]
    assert res["op"].d_total == 64
    assert [h[0] for h in res["history"]] == [16, 32, 48]


def test_absolute_tolerance_stops():
    n = 64
    A = 1e-12 * inputs.dense_matrix(n, n, seed=9)
    res = ad.adaptive(A, "sjlt_block", d0=16, dd=8, alpha=4, seed=1, d_max=64,
                      eps_rel=1e-12, eps_abs=1e-6)
    assert res["converged"] and len(res["history"]) == 1


def test_rank_deficient_sketch_projects_on_its_range():
    """S(:, 1:6) = [u1, u2, 0, u3, 2 u1, u4] has rank 4; the tested block
    [v1 + u2, 3 v2] with v1, v2 orthogonal to span(u) has ||S^|| = sqrt(10)
    and ||S~|| = sqrt(11) exactly.  A 6-column QR factor of S(:, 1:6) would
    span two directions outside its range and could take parts of v1, v2."""
    n = 50
    B, _ = np.linalg.qr(inputs.dense_matrix(n, 6, seed=10))
    u, v = B[:, :4], B[:, 4:]
    S = np.column_stack([u[:, 0], u[:, 1], np.zeros(n), u[:, 2], 2 * u[:, 0], u[:, 3],
                         v[:, 0] + u[:, 1], 3 * v[:, 1]])
    assert ad.range_basis(S[:, :6]).shape[1] == 4
    stop, nh, nt = ad.norm_test(S, 6, 2, 0.5, 0.0)
    assert abs(nh - np.sqrt(10.0)) < 1e-13 and abs(nt - np.sqrt(11.0)) < 1e-13
    assert not stop  # sqrt(10 / 11) > 0.5
    assert ad.range_basis(np.zeros((n, 3))).shape[1] == 0


@pytest.mark.parametrize("case", ["decay", "zero_cols", "low_rank"])
def test_norm_tests_equal_norm_test(case):
    rng = np.random.default_rng(12)
    m, d0, dd, d_end = 300, 24, 8, 120
    if case == "decay":
        A = inputs.spectrum_matrix(m, 0.85 ** np.arange(m), seed=13)
        S = A @ rng.standard_normal((m, d_end))
    elif case == "zero_cols":
        S = inputs.spectrum_matrix(m, 0.9 ** np.arange(m), seed=14) @ rng.standard_normal((m, d_end))
        S[:, [3, 30, 31, 77]] = 0.0  # columns without entries
        S[:, 50] = 2.0 * S[:, 10]    # a repeated direction
    else:
        S = inputs.low_rank_matrix(m, 40, seed=15) @ rng.standard_normal((m, d_end))
    got = ad.norm_tests(S, d0, dd, d_end)
    for k, b0 in enumerate(range(d0, d_end - dd + 1, dd)):
        _, nh, nt = ad.norm_test(S, b0, dd, 0.0, 0.0)
        assert abs(got[k][1] - nt) <= 1e-12 * nt
        assert abs(got[k][0] - nh) <= 1e-9 * nt + 1e-9 * nh, (case, b0, got[k][0], nh)

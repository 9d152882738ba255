"""Pins for the oracle's counter-based generator (CPU only).

Philox4x64-10 is checked against numpy's independent implementation
(numpy.random.Philox, which pre-increments its counter); the 128-bit product
and Lemire's bounded draws are checked against Python integers.
"""
import numpy as np
import pytest

from oracle import rng

M64 = (1 << 64) - 1


@pytest.mark.parametrize("key,ctr", [
    ((0, 0), (0, 0, 0, 0)),
    ((1, 2), (5, 0, 0, 0)),
    ((20230203, rng.TAG_SJLT | 3), (123456, 7, 0, 0)),
    ((M64, M64), (M64 - 1, M64, 17, 3)),
    ((0xDEADBEEF, rng.TAG_GAUSS), (2**40 + 5, 2**33, 9, 1)),
])
def test_philox_matches_numpy(key, ctr):
    ours = rng.philox4x64_10(*[np.uint64(c) for c in ctr], np.uint64(key[0]), np.uint64(key[1]))
    # numpy increments the 256-bit counter before producing a block
    prev = list(ctr)
    for i in range(4):  # 256-bit decrement, wrapping at zero
        if prev[i] > 0:
            prev[i] -= 1
            break
        prev[i] = M64
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(prev, dtype=np.uint64))
    ref = bg.random_raw(4)
    assert [int(x) for x in ours] == [int(x) for x in ref]


def test_philox_vectorised_equals_scalar():
    ctr = np.arange(1000, dtype=np.uint64) * np.uint64(7919)
    w = rng.philox4x64_10(ctr, np.uint64(3), 0, 0, np.uint64(99), np.uint64(5))
    for k in (0, 1, 517, 999):
        s = rng.philox4x64_10(ctr[k], np.uint64(3), 0, 0, np.uint64(99), np.uint64(5))
        assert [int(a[k]) for a in w] == [int(x) for x in s]


def test_mulhilo_matches_bigint():
    g = np.random.Generator(np.random.Philox(1))
    a = g.integers(0, 2**63, size=2000, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    b = g.integers(0, 2**63, size=2000, dtype=np.uint64) * np.uint64(2)
    hi, lo = rng.mulhilo64(a, b)
    for k in range(0, 2000, 37):
        p = int(a[k]) * int(b[k])
        assert int(hi[k]) == p >> 64 and int(lo[k]) == p & M64
    hi, lo = rng.mulhilo64(np.uint64(M64), np.uint64(M64))
    assert int(hi) == (M64 * M64) >> 64 and int(lo) == (M64 * M64) & M64


@pytest.mark.parametrize("s", [1, 2, 3, 7, 48, 64, 100, 32768, 2**31 + 11, 2**63 + 5])
def test_lemire_definition(s):
    g = np.random.Generator(np.random.Philox(s))
    words = g.integers(0, 2**64 - 1, size=500, dtype=np.uint64, endpoint=True)
    words = np.concatenate([words, np.array([0, 1, M64, s, (2**64 % s)], dtype=np.uint64)])
    v, ok = rng.lemire(words, s)
    t = (2**64) % s
    for w, vv, kk in zip(words.tolist(), v.tolist(), ok.tolist()):
        p = w * s
        assert vv == p >> 64
        assert kk == (not ((p & M64) < t))
        assert 0 <= vv < s


def test_lemire_power_of_two_is_shift():
    words = np.random.Generator(np.random.Philox(7)).integers(0, 2**64 - 1, 1000, dtype=np.uint64, endpoint=True)
    v, ok = rng.lemire(words, 64)
    assert ok.all()
    assert (v == (words >> np.uint64(58))).all()


def test_uniform_and_sign_helpers():
    assert rng.u53(np.uint64(0)) == 0.0
    assert rng.u53_open0(np.uint64(0)) == 2.0 ** -53
    assert rng.u53_open0(np.uint64(M64)) == 1.0
    assert rng.u53(np.uint64(M64)) == 1.0 - 2.0 ** -53
    assert int(rng.sign_of(np.uint64(1 << 63))) == -1
    assert int(rng.sign_of(np.uint64((1 << 63) - 1))) == 1

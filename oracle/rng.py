"""Counter-based random numbers for the oracle (test infrastructure only).

The paper draws its operators with ``std::minstd_rand`` (Sec. 8.3.1) and does not
say how streams are laid out.  This project's reading: every random quantity is
a pure function of (seed, tag, counter) through Philox4x64-10 (Salmon, Moraes,
Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), so that the
host oracle and the device kernels draw identical integers independently.

* ``philox4x64_10(c0, c1, c2, c3, k0, k1)`` -> four 64-bit words.  Ten rounds of
  the Philox S-box with multipliers 0xD2E7470EE14C6C93 / 0xCA5A826395121157 and
  Weyl key increments 0x9E3779B97F4A7C15 / 0xBB67AE8584CAA73B.
* ``lemire(word, s)`` -> (value in [0, s), accepted).  Lemire's multiply-shift
  with rejection (D. Lemire, "Fast random integer generation in an interval",
  ACM TOMACS 2019): value = floor(word * s / 2^64); reject when the low 64 bits
  of the product are below (2^64 - s) mod s.
* uniform doubles from the top 53 bits of a word.

All functions are vectorised over numpy uint64 arrays.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

# stream tags (high 32 bits: ASCII name; low bits: block index where used)
TAG_SJLT = 0x534A4C54 << 32      # "SJLT", | block index
TAG_SRHT_D = 0x53524844 << 32    # "SRHD"
TAG_SRHT_MU = 0x5352484D << 32   # "SRHM"
TAG_GAUSS = 0x47415553 << 32     # "GAUS"


def _u64(x) -> np.ndarray:
    return np.asarray(x, dtype=np.uint64)


def mulhilo64(a, b):
    """Full 64x64 -> 128-bit product of uint64 arrays: returns (hi, lo)."""
    a = _u64(a)
    b = _u64(b)
    with np.errstate(over="ignore"):
        a_lo = a & _MASK32
        a_hi = a >> _S32
        b_lo = b & _MASK32
        b_hi = b >> _S32
        ll = a_lo * b_lo
        lh = a_lo * b_hi
        hl = a_hi * b_lo
        hh = a_hi * b_hi
        mid = (ll >> _S32) + (lh & _MASK32) + (hl & _MASK32)
        hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
        lo = a * b
    return hi, lo


def philox4x64_10(c0, c1, c2, c3, k0, k1):
    """Philox4x64 with 10 rounds on (broadcast) uint64 arrays."""
    x0, x1, x2, x3 = np.broadcast_arrays(_u64(c0), _u64(c1), _u64(c2), _u64(c3))
    x0, x1, x2, x3 = x0.copy(), x1.copy(), x2.copy(), x3.copy()
    k0 = _u64(k0).copy()
    k1 = _u64(k1).copy()
    with np.errstate(over="ignore"):
        for r in range(10):
            hi0, lo0 = mulhilo64(M0, x0)
            hi1, lo1 = mulhilo64(M1, x2)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
            if r < 9:
                k0 = k0 + W0
                k1 = k1 + W1
    return x0, x1, x2, x3


def lemire(word, s):
    """Bounded integer in [0, s) from a 64-bit word; returns (value, accepted)."""
    word = _u64(word)
    s_arr = _u64(s)
    hi, lo = mulhilo64(word, s_arr)
    with np.errstate(over="ignore"):
        # (2^64 - s) mod s, computed as (-s) mod s in uint64 arithmetic
        thresh = (np.uint64(0) - s_arr) % s_arr
    accepted = ~((lo < s_arr) & (lo < thresh))
    return hi, accepted


def u53_open0(word):
    """Uniform double in (0, 1] from the top 53 bits of ``word``."""
    return ((_u64(word) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53


def u53(word):
    """Uniform double in [0, 1) from the top 53 bits of ``word``."""
    return (_u64(word) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def sign_of(word):
    """+1 / -1 (int8) from the top bit of ``word``: set bit means -1."""
    return np.where((_u64(word) >> np.uint64(63)) != 0, -1, 1).astype(np.int8)

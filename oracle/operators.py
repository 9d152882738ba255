"""JL sketching operators formed from their definitions (oracle; test infrastructure only).

Operators and the sections they follow:

* Gaussian (Sec. 2.4.1): R in R^{n x d}, i.i.d. N(0, 1/d).
* SRHT (Sec. 2.4.2 and Sec. 7.2): R = D H P with
  D a Rademacher diagonal, H the normalized Sylvester-Hadamard matrix of order
  nu = 2^ceil(log2 n) (zero padding of A to nu columns), and P selecting d
  columns with scale sqrt(nu/d); element-wise R_ij = d_i (-1)^(i . mu_j)/sqrt(d)
  (the element formula of Sec. 7.2), i . mu the dot product of the base-2 digits of the 0-based
  indices.
* SJLT (Sec. 2.4.3): alpha nonzeros of value +-1/sqrt(alpha) per row; graph
  construction = alpha distinct positions uniform in [d]; block construction =
  one position uniform in each of the alpha chunks of d/alpha columns.  The
  data structure R = (B+ - B-)/sqrt(alpha) with B+ and B- kept in CRS and CCS
  without value arrays follows Sec. 6.1.
* Increments (Sec. 6.2 "Adaptive SJLT sketching", Algorithm 1): Delta-d columns
  are appended and the scaling factor adjusted.

Readings where the paper is silent:

* Random streams: Philox4x64-10 keyed by (seed, tag), see ``oracle.rng``.
  SJLT row i, block b: draws t = 0, 1, 2, ... at counter (i, t, 0, 0) with key
  (seed, TAG_SJLT | b); chunk/slot k takes the next accepted draw: position =
  lemire(word0, width), rejected draws (Lemire rejection, or a repeated column
  in the graph construction) are skipped; sign = top bit of word1 (set = -1).
  Graph rows are stored ascending by column, each sign travelling with its
  column.
* SRHT: d_i from the top bit of word0 at counter (i, 0, 0, 0), key
  (seed, TAG_SRHT_D); the sampled columns mu are the first distinct values of
  lemire(word0, nu) over counters (t, 0, 0, 0), key (seed, TAG_SRHT_MU), in order
  of first appearance (sampling without replacement).  Increments continue the
  same sequence and keep D, so the grown operator is again D H P.
* Gaussian: column c uses counter (i, c >> 1, 0, 0), key (seed, TAG_GAUSS):
  u1 = (w0 >> 11 + 1) 2^-53 in (0, 1], u2 = (w1 >> 11) 2^-53 in [0, 1),
  z = sqrt(-2 ln u1) * cos(2 pi u2) for even c and * sin(2 pi u2) for odd c
  (Box-Muller), R_ic = z_ic / sqrt(d_total).
* Scale after increments (scale="renorm", the default): the grown R is
  rescaled to be one JL operator of the new width: SJLT values
  +-1/sqrt(alpha * blocks), SRHT 1/sqrt(d_total), Gaussian variance 1/d_total.
  scale="block": each block keeps the scale of a JL operator of its own width,
  as Algorithm 1 appends an independent JL(Delta-d): SJLT +-1/sqrt(alpha) in
  every block, SRHT 1/sqrt(w_b) and Gaussian variance 1/w_b for a block of
  width w_b.
* SRHT sampling with replacement (replace=True): mu_j is the j-th accepted
  draw lemire(word0, nu) over the same counters, repeats kept ("independently
  and uniformly", Sec. 2.4.2), so more than nu columns may be drawn.
"""
from __future__ import annotations

import math

import numpy as np

from . import rng

KINDS = ("sjlt_graph", "sjlt_block", "srht", "gauss")


def popcount_parity(x: np.ndarray) -> np.ndarray:
    """Parity (0/1) of the number of set bits of non-negative int64 ``x``:
    (-1)^(i . mu) with i . mu the base-2 digit dot product (the element formula of Sec. 7.2)."""
    x = np.asarray(x, dtype=np.int64)
    if hasattr(np, "bitwise_count"):
        return (np.bitwise_count(x) & 1).astype(np.int64)
    x = x.copy()
    for sh in (32, 16, 8, 4, 2, 1):
        x ^= x >> sh
    return x & 1


def next_pow2(n: int) -> int:
    return 1 << max(0, (int(n) - 1).bit_length())


def sjlt_block_draws(n: int, width: int, alpha: int, seed: int, block: int,
                     construction: str) -> tuple[np.ndarray, np.ndarray]:
    """Positions (relative to the block) and signs of one SJLT block.

    Returns ``cols`` (n, alpha) int64 in [0, width) and ``signs`` (n, alpha)
    int8 in {+1, -1}.  Graph rows are sorted ascending by column.
    """
    if construction not in ("graph", "block"):
        raise ValueError(construction)
    if alpha < 1 or alpha > width:
        raise ValueError("need 1 <= alpha <= width")
    if construction == "block" and width % alpha:
        raise ValueError("block construction needs alpha | width")
    span = width // alpha if construction == "block" else width
    key0 = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    key1 = np.uint64(rng.TAG_SJLT | block)
    rows = np.arange(n, dtype=np.uint64)
    t = np.zeros(n, dtype=np.uint64)
    cols = np.zeros((n, alpha), dtype=np.int64)
    signs = np.zeros((n, alpha), dtype=np.int8)
    for k in range(alpha):
        pending = np.arange(n)
        while pending.size:
            w0, w1, _, _ = rng.philox4x64_10(rows[pending], t[pending], 0, 0, key0, key1)
            t[pending] += np.uint64(1)
            v, ok = rng.lemire(w0, span)
            v = v.astype(np.int64)
            if construction == "graph" and k > 0:
                dup = (cols[pending, :k] == v[:, None]).any(axis=1)
                ok = ok & ~dup
            acc = pending[ok]
            cols[acc, k] = (k * span + v[ok]) if construction == "block" else v[ok]
            signs[acc, k] = rng.sign_of(w1[ok])
            pending = pending[~ok]
    if construction == "graph":
        order = np.argsort(cols, axis=1, kind="stable")
        cols = np.take_along_axis(cols, order, axis=1)
        signs = np.take_along_axis(signs, order, axis=1)
    return cols, signs


def srht_diag(n: int, seed: int) -> np.ndarray:
    """Rademacher diagonal d_i (int8 +-1)."""
    w0, _, _, _ = rng.philox4x64_10(np.arange(n, dtype=np.uint64), 0, 0, 0,
                                    np.uint64(seed & 0xFFFFFFFFFFFFFFFF),
                                    np.uint64(rng.TAG_SRHT_D))
    return rng.sign_of(w0)


def srht_samples(nu: int, count: int, seed: int, replace: bool = False) -> np.ndarray:
    """First ``count`` distinct draws of lemire(word0, nu) in order (int64);
    with ``replace`` the first ``count`` accepted draws, repeats kept."""
    if count > nu and not replace:
        raise ValueError("cannot sample more distinct columns than nu")
    chosen: list[int] = []
    seen = set()
    t = 0
    batch = max(64, 2 * count)
    key0 = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    key1 = np.uint64(rng.TAG_SRHT_MU)
    while len(chosen) < count:
        ctr = np.arange(t, t + batch, dtype=np.uint64)
        w0, _, _, _ = rng.philox4x64_10(ctr, 0, 0, 0, key0, key1)
        v, ok = rng.lemire(w0, nu)
        for val, good in zip(v.tolist(), ok.tolist()):
            if good and (replace or val not in seen):
                seen.add(val)
                chosen.append(val)
                if len(chosen) == count:
                    break
        t += batch
    return np.asarray(chosen, dtype=np.int64)


def gaussian_z(n: int, c_begin: int, c_end: int, seed: int) -> np.ndarray:
    """Standard normal z_ic for rows [0, n) and columns [c_begin, c_end)."""
    cols = np.arange(c_begin, c_end, dtype=np.int64)
    out = np.empty((n, cols.size), dtype=np.float64)
    rows = np.arange(n, dtype=np.uint64)[:, None]
    pairs = (cols >> 1).astype(np.uint64)[None, :]
    w0, w1, _, _ = rng.philox4x64_10(rows, pairs, 0, 0,
                                     np.uint64(seed & 0xFFFFFFFFFFFFFFFF),
                                     np.uint64(rng.TAG_GAUSS))
    u1 = rng.u53_open0(w0)
    u2 = rng.u53(w1)
    rad = np.sqrt(-2.0 * np.log(u1))
    even = (cols % 2 == 0)[None, :]
    out[:] = np.where(even, rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2))
    return out


class Operator:
    """A JL operator R (n x d_total) grown by increments, formed from definitions."""

    def __init__(self, kind: str, n: int, d: int, alpha: int = 1, seed: int = 0, scale: str = "renorm",
                 replace: bool = False):
        if kind not in KINDS:
            raise ValueError(kind)
        if n < 1 or d < 1:
            raise ValueError("n and d must be positive")
        if scale not in ("renorm", "block"):
            raise ValueError(scale)
        if replace and kind != "srht":
            raise ValueError("sampling with replacement is an SRHT option")
        self.scale_mode = scale
        self.replace = bool(replace)
        self.kind = kind
        self.n = int(n)
        self.alpha = int(alpha)
        self.seed = int(seed)
        self.blocks: list[int] = []
        self.nu = next_pow2(n)
        self._check_block(d)
        self.blocks.append(int(d))

    # -- structure ---------------------------------------------------------
    def _check_block(self, w: int) -> None:
        if self.kind.startswith("sjlt"):
            if self.alpha < 1 or self.alpha > w:
                raise ValueError("SJLT needs 1 <= alpha <= block width")
            if self.kind == "sjlt_block" and w % self.alpha:
                raise ValueError("block construction needs alpha | width")
        if self.kind == "srht" and not self.replace and self.d_total + w > self.nu:
            raise ValueError("SRHT cannot sample more than nu columns")

    @property
    def d_total(self) -> int:
        return int(sum(self.blocks))

    def increment(self, dd: int) -> None:
        """Append ``dd`` columns (Algorithm 1, R <- [R  R_bar])."""
        if dd < 1:
            raise ValueError("increment must be positive")
        self._check_block(dd)
        self.blocks.append(int(dd))

    def scale(self) -> float:
        """The scale of every column (renorm), or of the last block's columns (block)."""
        if self.kind.startswith("sjlt"):
            return 1.0 / math.sqrt(self.alpha * (1 if self.scale_mode == "block" else len(self.blocks)))
        if self.scale_mode == "block":
            return 1.0 / math.sqrt(self.blocks[-1])
        return 1.0 / math.sqrt(self.d_total)

    def column_scales(self) -> np.ndarray:
        """Scale of each of the d_total columns."""
        if self.scale_mode == "renorm" or self.kind.startswith("sjlt"):
            return np.full(self.d_total, self.scale())
        return np.concatenate([np.full(w, 1.0 / math.sqrt(w)) for w in self.blocks])

    # -- random parts ------------------------------------------------------
    def sjlt_entries(self) -> tuple[np.ndarray, np.ndarray]:
        """(cols, signs), each (n, alpha * blocks); block b's entries are
        columns [alpha*b, alpha*(b+1)) and carry global column indices."""
        construction = "graph" if self.kind == "sjlt_graph" else "block"
        cols, signs, off = [], [], 0
        for b, w in enumerate(self.blocks):
            c, s = sjlt_block_draws(self.n, w, self.alpha, self.seed, b, construction)
            cols.append(c + off)
            signs.append(s)
            off += w
        return np.concatenate(cols, axis=1), np.concatenate(signs, axis=1)

    def srht_diag(self) -> np.ndarray:
        return srht_diag(self.n, self.seed)

    def srht_samples(self) -> np.ndarray:
        return srht_samples(self.nu, self.d_total, self.seed, self.replace)

    def gaussian_z(self) -> np.ndarray:
        return gaussian_z(self.n, 0, self.d_total, self.seed)

    # -- dense form --------------------------------------------------------
    def dense(self) -> np.ndarray:
        """R (n x d_total) in FP64, from the element definitions."""
        n, d = self.n, self.d_total
        if self.kind.startswith("sjlt"):
            cols, signs = self.sjlt_entries()
            R = np.zeros((n, d), dtype=np.float64)
            rows = np.repeat(np.arange(n), cols.shape[1])
            R[rows, cols.ravel()] = signs.ravel().astype(np.float64)
            return R * self.column_scales()[None, :]
        if self.kind == "srht":
            D = self.srht_diag().astype(np.float64)
            mu = self.srht_samples()
            i = np.arange(n, dtype=np.int64)[:, None]
            H = np.where(popcount_parity(i & mu[None, :]) == 1, -1.0, 1.0)
            return D[:, None] * H * self.column_scales()[None, :]
        return self.gaussian_z() * self.column_scales()[None, :]


def crs_ccs(cols: np.ndarray, signs: np.ndarray, d: int):
    """The Sec. 6.1 data structure: R = s (B+ - B-) with B+ and B- in CRS and CCS.

    Returns a dict with, for each of 'plus' and 'minus': 'row_ptr', 'col_idx'
    (CRS, columns ascending within a row) and 'col_ptr', 'row_idx' (CCS, rows
    ascending within a column).  No value arrays: the entries are all one.
    """
    n = cols.shape[0]
    out = {}
    for name, sgn in (("plus", 1), ("minus", -1)):
        mask = signs == sgn
        r, k = np.nonzero(mask)
        c = cols[r, k]
        order = np.lexsort((c, r))
        r_crs, c_crs = r[order], c[order]
        row_ptr = np.zeros(n + 1, dtype=np.int64)
        np.add.at(row_ptr, r_crs + 1, 1)
        row_ptr = np.cumsum(row_ptr)
        order = np.lexsort((r, c))
        r_ccs, c_ccs = r[order], c[order]
        col_ptr = np.zeros(d + 1, dtype=np.int64)
        np.add.at(col_ptr, c_ccs + 1, 1)
        col_ptr = np.cumsum(col_ptr)
        out[name] = dict(row_ptr=row_ptr, col_idx=c_crs.astype(np.int64),
                         col_ptr=col_ptr, row_idx=r_ccs.astype(np.int64))
    return out

"""Seeded, counter-based synthetic columns for the query-processor workloads.

This module is shared by the CPU oracle tests and by the CUDA-path tests and
benchmark: both sides receive the *same* host arrays.  It holds none of the
query arithmetic (no predicate, join, grouping or aggregation code) -- only
random draws and the column recipes.

Draws
-----
* ``draw(seed, col_id, rows)``: SplitMix64 (Steele, Lea & Flood, "Fast
  splittable pseudorandom number generators", OOPSLA 2014) applied to the
  counter ``seed ^ (col_id << 56) ^ row``, so every row of every column can be
  produced independently and in any order.
* ``uniform_int``: multiply-high range reduction of the top 32 bits
  (Lemire, "Fast random integer generation in an interval", TOMACS 2019):
  ``lo + ((v >> 32) * span >> 32)`` with ``span = hi - lo + 1 <= 2**32``.
* ``zipf_ranks``: inverse-CDF sampling of ranks ``r in [1, N]`` with
  ``P(r) ~ r**-s`` from a float64 CDF table.
* ``feistel_perm``: a seeded bijection on ``[0, N)`` -- a 4-round balanced
  Feistel network on ``2*h`` bits (``2**(2h) >= N``) with cycle-walking.

Column recipes follow the analytical-table shapes of the paper's evaluation
(Section 6: TPC-H lineitem-like fact rows and a keyed dimension table); the
generated values are synthetic stand-ins, not benchmark data.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

DEFAULT_SEED = 20220301
_M64 = (1 << 64) - 1
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)

# Column ids of the fact-table recipe (fixed so that any subset can be drawn).
COL_KEY, COL_PRICE, COL_DISCOUNT, COL_QUANTITY, COL_DATE, COL_FLAG, COL_STATUS = range(7)
COL_FK, COL_VALUE = 8, 9
COL_ZIPF = 10
DATE_DAYS = 2557  # 7 years of int32 day numbers [0, 2556]

_CHUNK = 1 << 22


def _threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser of ``x + golden`` (uint64 in, uint64 out)."""
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        return z ^ (z >> np.uint64(31))


def _counter_base(seed: int, col_id: int) -> np.uint64:
    return np.uint64((int(seed) ^ (int(col_id) << 56)) & _M64)


def draw(seed: int, col_id: int, row0: int, n: int) -> np.ndarray:
    """Raw 64-bit draws for rows ``[row0, row0 + n)`` of column ``col_id``."""
    rows = np.arange(row0, row0 + n, dtype=np.uint64)
    return splitmix64(rows ^ _counter_base(seed, col_id))


def _chunked(n: int, fn, dtype) -> np.ndarray:
    """Fill an array of ``n`` elements by calling ``fn(row0, count)`` per chunk."""
    out = np.empty(n, dtype=dtype)
    if n <= _CHUNK:
        if n:
            out[:] = fn(0, n)
        return out

    def work(r0):
        c = min(_CHUNK, n - r0)
        out[r0:r0 + c] = fn(r0, c)

    with ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(work, range(0, n, _CHUNK)))
    return out


def uniform_int(seed: int, col_id: int, n: int, lo: int, hi: int, dtype, row0: int = 0) -> np.ndarray:
    """Integers uniform on ``[lo, hi]`` (inclusive), ``hi - lo + 1 <= 2**32``."""
    span = hi - lo + 1
    if not (0 < span <= (1 << 32)):
        raise ValueError("span must be in (0, 2**32]")

    def fn(r0, c):
        v = draw(seed, col_id, row0 + r0, c) >> np.uint64(32)
        with np.errstate(over="ignore"):
            off = (v * np.uint64(span)) >> np.uint64(32)
        return (off.astype(np.int64) + lo).astype(dtype)

    return _chunked(n, fn, dtype)


def unit_float(seed: int, col_id: int, row0: int, n: int) -> np.ndarray:
    """Float64 uniform on [0, 1) from the top 53 bits of the draw."""
    return (draw(seed, col_id, row0, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


_ZIPF_CDF_CACHE: dict = {}


def zipf_cdf(N: int, s: float) -> np.ndarray:
    key = (int(N), float(s))
    if key not in _ZIPF_CDF_CACHE:
        w = np.arange(1, N + 1, dtype=np.float64) ** (-float(s))
        c = np.cumsum(w)
        _ZIPF_CDF_CACHE[key] = c / c[-1]
    return _ZIPF_CDF_CACHE[key]


def zipf_ranks(seed: int, col_id: int, n: int, N: int, s: float, row0: int = 0) -> np.ndarray:
    """Zero-based ranks ``r - 1`` with ``P(r) ~ r**-s`` on ``[1, N]`` (int64)."""
    cdf = zipf_cdf(N, s)

    def fn(r0, c):
        u = unit_float(seed, col_id, row0 + r0, c)
        idx = np.searchsorted(cdf, u, side="right")
        return np.minimum(idx, N - 1).astype(np.int64)

    return _chunked(n, fn, np.int64)


def feistel_perm(seed: int, N: int, x: np.ndarray) -> np.ndarray:
    """Seeded bijection on ``[0, N)``, applied element-wise to ``x`` (int64)."""
    x = np.asarray(x, dtype=np.int64)
    if N <= 1:
        return np.zeros_like(x)
    bits = max(2, math.ceil(math.log2(N)))
    h = (bits + 1) // 2
    mask = np.uint64((1 << h) - 1)
    keys = [np.uint64(int(splitmix64(np.array([seed ^ (0xFE15 << 40) ^ r], dtype=np.uint64))[0])) for r in range(4)]

    def once(y: np.ndarray) -> np.ndarray:
        L = (y >> np.uint64(h)) & mask
        R = y & mask
        for k in keys:
            F = splitmix64(R ^ k) & mask
            L, R = R, L ^ F
        return (L << np.uint64(h)) | R

    y = once(x.astype(np.uint64))
    bad = y >= np.uint64(N)
    while bad.any():
        y[bad] = once(y[bad])
        bad = y >= np.uint64(N)
    return y.astype(np.int64)


# ---------------------------------------------------------------------------
# Table recipes
# ---------------------------------------------------------------------------

def fact_table(n: int, seed: int = DEFAULT_SEED, cols=None, row0: int = 0) -> dict:
    """Lineitem-like fact rows (all integer; decimals are x100 fixed point).

    key i32 U[0,1e5); price i64 U[100,1e7]; discount i64 U[0,10];
    quantity i32 U[1,50]; date i32 U[0,2556]; flag u8 U{0,1,2}; status u8 U{0,1}.
    """
    want = set(cols) if cols is not None else {"key", "price", "discount", "quantity", "date", "flag", "status"}
    out = {}
    if "key" in want:
        out["key"] = uniform_int(seed, COL_KEY, n, 0, 99_999, np.int32, row0)
    if "price" in want:
        out["price"] = uniform_int(seed, COL_PRICE, n, 100, 10_000_000, np.int64, row0)
    if "discount" in want:
        out["discount"] = uniform_int(seed, COL_DISCOUNT, n, 0, 10, np.int64, row0)
    if "quantity" in want:
        out["quantity"] = uniform_int(seed, COL_QUANTITY, n, 1, 50, np.int32, row0)
    if "date" in want:
        out["date"] = uniform_int(seed, COL_DATE, n, 0, DATE_DAYS - 1, np.int32, row0)
    if "flag" in want:
        out["flag"] = uniform_int(seed, COL_FLAG, n, 0, 2, np.uint8, row0)
    if "status" in want:
        out["status"] = uniform_int(seed, COL_STATUS, n, 0, 1, np.uint8, row0)
    return out


SPARSE_MULT = 1_000_003  # odd: multiplication by it is a bijection modulo 2**31


def key_values(idx: np.ndarray, nkeys: int, seed: int, sparse: bool) -> np.ndarray:
    """The int32 join key of key index ``idx`` in ``[0, nkeys)``.

    Dense keys are the indices themselves.  Sparse keys scatter the indices
    over ``[0, 2**31)``: ``(pi(idx) * 1_000_003) mod 2**31`` with ``pi`` a seeded
    bijection on ``[0, nkeys)``; distinct indices give distinct keys (the
    multiplier is odd, so it permutes the residues modulo ``2**31``), and the
    keys span far more than twice their number, so no table can be
    direct-mapped over them."""
    idx = np.asarray(idx, dtype=np.int64)
    if not sparse:
        return idx.astype(np.int32)
    perm = feistel_perm(seed ^ 0x5BA55, nkeys, idx)
    return ((perm * SPARSE_MULT) & ((1 << 31) - 1)).astype(np.int32)


def dim_table(nb: int, ngroups: int, seed: int = DEFAULT_SEED, sparse: bool = False, dup: int = 1) -> dict:
    """Dimension rows: row i has key index i // dup (``dup`` rows per key; the
    last key may have fewer), its key from ``key_values`` (dense: 0..nkeys-1),
    and payload = pi(i) mod ngroups with pi a seeded bijection on [0, nb)."""
    rows = np.arange(nb, dtype=np.int64)
    nkeys = (nb + dup - 1) // dup
    key = key_values(rows // dup, nkeys, seed, sparse)
    payload = feistel_perm(seed ^ 0xD1A, nb, rows) % ngroups
    return {"key": key, "payload": payload.astype(np.int32)}


def probe_table(n: int, nb: int, seed: int = DEFAULT_SEED, zipf_s: float = 0.5, sparse: bool = False) -> dict:
    """Probe rows: fk = the key of key index pi'(Zipf(s) rank) over nb key
    indices (``key_values``; dense: the index itself); value i64 U[100,1e7]."""
    ranks = zipf_ranks(seed, COL_ZIPF, n, nb, zipf_s)

    def keys(r0, c):
        return key_values(feistel_perm(seed ^ 0x21FF, nb, ranks[r0:r0 + c]), nb, seed, sparse)

    fk = _chunked(n, keys, np.int32)
    value = uniform_int(seed, COL_VALUE, n, 100, 10_000_000, np.int64)
    return {"fk": fk, "value": value}


def log_uniform_int(seed: int, col_id: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Integers log-uniform on [lo, hi]."""
    u = unit_float(seed, col_id, 0, n)
    v = np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    return np.clip(np.floor(v).astype(np.int64), lo, hi)


COL_WORDS, COL_WORD0 = 20, 21  # string column draws: word count, then one column per word slot
STR_WIDTH = 24
STR_VOCAB = 32


def string_vocab(seed: int = DEFAULT_SEED) -> list:
    """``STR_VOCAB`` synthetic lowercase words of 3 to 7 letters (a seeded draw, no natural-language list)."""
    lens = uniform_int(seed, 30, STR_VOCAB, 3, 7, np.int64)
    letters = uniform_int(seed, 31, STR_VOCAB * 7, 0, 25, np.int64).reshape(STR_VOCAB, 7)
    return [bytes((97 + letters[i, :lens[i]]).astype(np.uint8)) for i in range(STR_VOCAB)]


def string_column(n: int, seed: int = DEFAULT_SEED, width: int = STR_WIDTH, row0: int = 0) -> np.ndarray:
    """A string column: each row 1 to 3 words of the seeded vocabulary joined by one space, as an
    ``(n, width)`` uint8 array right-padded with 0 (the paper's (n x m) character tensor, Section 4.1).
    ``width`` >= 23 holds every row; a smaller width cuts rows at ``width`` bytes (no padding byte left)."""
    vocab = string_vocab(seed)
    wl = np.array([len(w) for w in vocab], np.int64)
    wb = np.zeros((STR_VOCAB, 7), np.uint8)
    for i, w in enumerate(vocab):
        wb[i, :len(w)] = np.frombuffer(w, np.uint8)
    k = uniform_int(seed, COL_WORDS, n, 1, 3, np.int64, row0)
    out = np.zeros((n, width + 8), np.uint8)   # slack for the last word, cut below
    pos = np.zeros(n, np.int64)
    rows = np.arange(n)
    for slot in range(3):
        w = uniform_int(seed, COL_WORD0 + slot, n, 0, STR_VOCAB - 1, np.int64, row0)
        act = slot < k
        if slot:
            sp = act & (pos < width + 7)
            out[rows[sp], pos[sp]] = 32
            pos = pos + act
        for j in range(7):
            m = act & (j < wl[w]) & (pos + j < width + 8)
            out[rows[m], (pos + j)[m]] = wb[w[m], j]
        pos = pos + np.where(act, wl[w], 0)
    return np.ascontiguousarray(out[:, :width])

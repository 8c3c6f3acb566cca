"""The counter-based column generators of ``datagen`` in PyTorch, for building
large resident tables directly in device memory.  Every value equals the
NumPy generator's for the same (seed, column, row): the SplitMix64 finaliser
and the multiply-high range reduction are computed in int64 with
two's-complement wrap-around and explicit masks for the logical shifts.
Like ``datagen`` itself, this holds no query arithmetic."""
from __future__ import annotations

import torch

from datagen import (COL_DATE, COL_DISCOUNT, COL_FLAG, COL_KEY, COL_PRICE, COL_QUANTITY, COL_STATUS, DATE_DAYS,
                     DEFAULT_SEED)

_M64 = (1 << 64) - 1


def _s64(u: int) -> int:
    """uint64 constant as the int64 with the same bits."""
    u &= _M64
    return u - (1 << 64) if u >= (1 << 63) else u


_GOLDEN = _s64(0x9E3779B97F4A7C15)
_MIX1 = _s64(0xBF58476D1CE4E5B9)
_MIX2 = _s64(0x94D049BB133111EB)


def _srl(x: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def splitmix64(x: torch.Tensor) -> torch.Tensor:
    z = x + _GOLDEN
    z = (z ^ _srl(z, 30)) * _MIX1
    z = (z ^ _srl(z, 27)) * _MIX2
    return z ^ _srl(z, 31)


def draw(seed: int, col_id: int, row0: int, n: int, device) -> torch.Tensor:
    base = _s64((int(seed) ^ (int(col_id) << 56)) & _M64)
    rows = torch.arange(row0, row0 + n, dtype=torch.int64, device=device)
    return splitmix64(rows ^ base)


def uniform_int(seed: int, col_id: int, n: int, lo: int, hi: int, dtype, device, row0: int = 0,
                chunk: int = 1 << 26) -> torch.Tensor:
    span = hi - lo + 1
    if not (0 < span <= (1 << 32)):
        raise ValueError("span must be in (0, 2**32]")
    out = torch.empty(n, dtype=dtype, device=device)
    for c0 in range(0, n, chunk):
        c = min(chunk, n - c0)
        v = _srl(draw(seed, col_id, row0 + c0, c, device), 32)        # < 2**32
        off = _srl(v * span, 32)                                        # product wraps mod 2**64
        out[c0:c0 + c] = (off + lo).to(dtype)
    return out


def fact_table(n: int, seed: int = DEFAULT_SEED, cols=None, device="cuda", row0: int = 0) -> dict:
    """The fact-table recipe of ``datagen.fact_table``, as device tensors."""
    want = set(cols) if cols is not None else {"key", "price", "discount", "quantity", "date", "flag", "status"}
    spec = {"key": (COL_KEY, 0, 99_999, torch.int32), "price": (COL_PRICE, 100, 10_000_000, torch.int64),
            "discount": (COL_DISCOUNT, 0, 10, torch.int64), "quantity": (COL_QUANTITY, 1, 50, torch.int32),
            "date": (COL_DATE, 0, DATE_DAYS - 1, torch.int32), "flag": (COL_FLAG, 0, 2, torch.uint8),
            "status": (COL_STATUS, 0, 1, torch.uint8)}
    return {k: uniform_int(seed, cid, n, lo, hi, dt, device, row0) for k, (cid, lo, hi, dt) in spec.items()
            if k in want}

"""Helpers for the GPU parity tests: upload seeded host columns, run the C ABI."""
import numpy as np


def dev():
    import torch
    return torch.device("cuda:0")


def up(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def zeros(n, dtype):
    import torch
    return torch.zeros(max(int(n), 1), dtype=dtype, device=dev())


def gpu_filter(ctx, host_cols, preds, sum_expr=None, capacity=None, want_ids=True, stream=None):
    """Run tqp_filter on host columns; returns (ids or None, count, sum, status)."""
    import torch
    import paper_2203_01877_gb300 as tqp
    cols = [up(a) for a in host_cols]
    table = tqp.TableRef(cols)
    n = len(host_cols[0])
    cap = n if capacity is None else capacity
    ids = zeros(cap, torch.int32) if want_ids else None
    cnt = torch.full((1,), -7, dtype=torch.int64, device=dev())
    s = torch.full((1,), -7, dtype=torch.int64, device=dev()) if sum_expr is not None else None
    tqp.tqp_filter(ctx, table, preds, sum_expr, s, ids, cap if want_ids else 0, cnt, stream)
    status = ctx.status(stream)
    k = int(cnt.item())
    out_ids = ids[:min(k, cap)].cpu().numpy() if want_ids else None
    return out_ids, k, (int(s.item()) if s is not None else None), status

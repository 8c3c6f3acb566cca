"""Run one plan spec (the oracle's vocabulary) through tqp_run_plan / tqp_run_plans."""
import numpy as np


def gpu_plan_prepare(fact, preds=(), dim=None, fact_fk=0, dim_key=0, group_cols=(), aggs=(), sum_expr=None,
                     topk=0, topk_agg=0, want_row_ids=False, capacity_groups=None, max_groups=0, dim_ref=None,
                     prepared=None, join_kind="inner", fact_ref=None):
    """dim_ref: an existing TableRef of `dim` (needed with `prepared`, which was built on it); fact_ref: an
    existing TableRef of `fact` (plans sharing one uploaded table)."""
    import torch
    import paper_2203_01877_gb300 as tqp
    from tests.gpu_util import up
    F = fact_ref if fact_ref is not None else tqp.TableRef([up(c) for c in fact])
    D = dim_ref if dim_ref is not None else (tqp.TableRef([up(c) for c in dim]) if dim is not None else None)
    nf = len(fact[0])
    ngc, na = len(group_cols), len(aggs)
    capg = capacity_groups if capacity_groups is not None else (topk if topk else max(64, min(nf, 1 << 16)))
    dev = "cuda:0"
    bufs = {
        "row_ids": torch.zeros(max(nf, 1), dtype=torch.int32, device=dev) if want_row_ids else None,
        "num_rows": torch.full((1,), -7, dtype=torch.int64, device=dev),
        "sum": torch.full((1,), -7, dtype=torch.int64, device=dev) if sum_expr is not None else None,
        "keys": torch.zeros(max(capg * ngc, 1), dtype=torch.int64, device=dev),
        "ivals": torch.zeros(max(capg * na, 1), dtype=torch.int64, device=dev),
        "fvals": torch.zeros(max(capg * na, 1), dtype=torch.float64, device=dev),
        "num_groups": torch.full((1,), -7, dtype=torch.int64, device=dev),
        "total_groups": torch.full((1,), -7, dtype=torch.int64, device=dev),
        "num_joined": torch.full((1,), -7, dtype=torch.int64, device=dev),
    }
    plan = tqp.make_plan(F, preds, D, fact_fk, dim_key, group_cols, aggs, sum_expr, topk, topk_agg,
                         emit_row_ids=want_row_ids, max_groups=max_groups, prepared=prepared, join_kind=join_kind)
    res = tqp.make_result(bufs["row_ids"], nf if want_row_ids else 0, bufs["num_rows"], bufs["sum"], bufs["keys"],
                          bufs["ivals"], bufs["fvals"], capg, bufs["num_groups"], bufs["total_groups"],
                          bufs["num_joined"])
    return plan, res, bufs, (F, D), (ngc, na, want_row_ids, sum_expr is not None, ngc + na > 0)


def gpu_plan_collect(bufs, shape):
    ngc, na, want_ids, has_sum, grouped = shape
    out = {"num_rows": int(bufs["num_rows"].item()), "num_pairs": int(bufs["num_joined"].item())}
    if want_ids:
        out["row_ids"] = bufs["row_ids"][:out["num_rows"]].cpu().numpy()
    if has_sum:
        out["sum"] = int(bufs["sum"].item())
    if grouped:
        G = int(bufs["num_groups"].item())
        out["num_groups"] = G
        out["total_groups"] = int(bufs["total_groups"].item())
        if G >= 0:
            out["keys"] = bufs["keys"][:G * ngc].reshape(G, ngc).cpu().numpy()
            out["ivals"] = bufs["ivals"][:G * na].reshape(G, na).cpu().numpy()
            out["fvals"] = bufs["fvals"][:G * na].reshape(G, na).cpu().numpy()
    return out


def gpu_plan(ctx, **spec):
    import paper_2203_01877_gb300 as tqp
    plan, res, bufs, keep, shape = gpu_plan_prepare(**spec)
    tqp.tqp_run_plan(ctx, plan, res)
    st = ctx.status()
    out = gpu_plan_collect(bufs, shape)
    out["status"] = st
    return out


def compare(got, want, shape_spec):
    """Element-by-element comparison of a GPU plan result with the oracle's."""
    assert got["status"] == 0
    assert got["num_rows"] == want["num_rows"]
    if shape_spec.get("dim") is not None:
        assert got["num_pairs"] == want["num_pairs"]
    if shape_spec.get("want_row_ids"):
        assert np.array_equal(got["row_ids"], want["row_ids"])
    if shape_spec.get("sum_expr") is not None:
        assert got["sum"] == want["sum"]
    if len(shape_spec.get("group_cols", ())) + len(shape_spec.get("aggs", ())) > 0:
        assert got["num_groups"] == want["num_groups"]
        assert got["total_groups"] == want["total_groups"]
        assert np.array_equal(got["keys"], want["keys"])
        assert np.array_equal(got["ivals"], want["ivals"])
        assert np.array_equal(got["fvals"].view(np.int64), want["fvals"].view(np.int64))


_CACHE = {}


def hashed_join_inputs(n_probe=60_000_000, n_build=1_500_000, n_groups=150_000, dup=1, seed=None):
    """The join + group workload over SPARSE build keys (unique int32 keys scattered over [0, 2**31), so the
    library must use its hashed table): build n_build rows (dup rows per key), payload = 150K groups, probe
    n_probe Zipf(0.5) foreign keys over the build keys.  Cached per process (generation takes seconds)."""
    import datagen
    key = (n_probe, n_build, n_groups, dup, seed)
    if key not in _CACHE:
        s = datagen.DEFAULT_SEED + 2 if seed is None else seed
        dim = datagen.dim_table(n_build, n_groups, seed=s, sparse=True, dup=dup)
        pr = datagen.probe_table(n_probe, (n_build + dup - 1) // dup, seed=s, sparse=True)
        _CACHE.clear()
        _CACHE[key] = (dim, pr)
    return _CACHE[key]


def oracle_groups_sample(dim, pr, groups, aggs, group_col_payload=3):
    """The oracle's per-group result for the payload groups in `groups` only: the dimension is restricted to the
    rows of those groups, which leaves each of their aggregates unchanged (a group's joined rows all come from
    its own dimension rows) and lets the oracle run over the full probe side in seconds."""
    import numpy as np
    import oracle
    keep = np.isin(dim["payload"], np.asarray(groups))
    sub = [dim["key"][keep], dim["payload"][keep]]
    return oracle.run_plan(fact=[pr["fk"], pr["value"]], dim=sub, fact_fk=0, dim_key=0,
                           group_cols=[group_col_payload], aggs=aggs, want_pairs=False, cap_groups=None,
                           want_row_ids=False)

#!/usr/bin/env python3
"""Benchmark of the query-processor hot path on GB300 (one JSON line).

Workload (one step = the whole filter -> compaction -> projection-sum path):
60M synthetic lineitem-like rows (date i32, discount i64 x100, quantity i32,
price i64 x100), predicates 731 <= date < 1096, 5 <= discount <= 7,
quantity < 24 (~1.8% pass), outputs the ascending int32 row ids of passing
rows and the exact int64 SUM(price * discount).  Inputs (1.44 GB) exceed the
L2 cache, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tqp|reference]

Under torchrun each rank runs its own 60M-row problem (weak scaling, no
data-path collective); rank 0 prints max-over-ranks timing.  --impl reference
times the CPU oracle on the host cores instead (bounded samples).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import datagen  # noqa: E402

N_ROWS = 60_000_000
PREDS = [(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)]
EXPR = [("col", 3), ("col", 1), "mul"]
WORKLOAD = ("filter-project-reduce: 60M rows (date i32, discount i64, quantity i32, price i64); "
            "731<=date<1096 AND 5<=discount<=7 AND quantity<24; ascending int32 row ids + SUM(price*discount)")
PROFILE_MD = os.path.join(ROOT, "profiles", "k_filter_q6_60M.md")
KERNEL_SRCS = ["filter.cu", "bodies.cuh", "engine.cuh", "common.cuh"]


def gen_host(rank: int):
    t = datagen.fact_table(N_ROWS, seed=datagen.DEFAULT_SEED + 1 + 1000 * rank,
                           cols=["date", "discount", "quantity", "price"])
    return [t["date"], t["discount"], t["quantity"], t["price"]]


def algorithmic_bytes(n: int, k: int) -> int:
    # predicate columns read once (4 + 8 + 4 B/row); price gathered and a row id
    # written for every passing row (8 + 4 B)
    return n * 16 + k * 12


def kernel_src_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SRCS:
        with open(os.path.join(ROOT, "paper_2203_01877_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernel source."""
    try:
        txt = open(PROFILE_MD).read()
    except OSError:
        return None
    vals = {}
    for ln in txt.splitlines():
        if ":" in ln and ln.strip().startswith("- "):
            k, v = ln.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_src_sha") != kernel_src_hash():
        return None
    try:
        return int(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    """The host CPU's model name (x86 /proc/cpuinfo, else lscpu, e.g. an Arm Neoverse core)."""
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_rate(cols, min_seconds: float, rows_cap: int | None = None, threads: int = 1):
    """Rows/s of the CPU oracle on the same columns (threads > 1: its row-range variant on that many
    threads), paper protocol style: at most 10 runs, median of the later half."""
    import oracle
    if rows_cap is not None and rows_cap < len(cols[0]):
        cols = [c[:rows_cap] for c in cols]
    n = len(cols[0])
    times = []
    t_end = time.perf_counter() + min_seconds
    while len(times) < 3 or time.perf_counter() < t_end:
        t0 = time.perf_counter()
        oracle.filter_rows(cols, PREDS, EXPR, threads=threads)
        times.append(time.perf_counter() - t0)
        if len(times) >= 10:
            break
    tail = times[len(times) // 2:]
    return n / statistics.median(tail), n, len(times), sum(times)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cols = gen_host(0)
    cores = host_cores()
    # calibrate on 8M rows, then size each step's sample so the whole run takes ~2 minutes
    rate, _, _, _ = oracle_rate(cols, 0.0, rows_cap=8_000_000, threads=cores)
    total_steps = max(1, args.steps + args.warmup)
    sample = int(max(100_000, min(N_ROWS, rate * 120.0 / total_steps)))
    import oracle
    sub = [c[:sample] for c in cols]
    for _ in range(args.warmup):
        oracle.filter_rows(sub, PREDS, EXPR, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.filter_rows(sub, PREDS, EXPR, threads=cores)
    dt = time.perf_counter() - t0
    value = sample * args.steps / dt
    line = {
        "impl": "reference", "metric": "rows/s", "value": value, "unit": "rows/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded counter-based generators)",
        "config": {"workload": WORKLOAD, "rows": N_ROWS},
        "cpu_baseline": {"value": value, "unit": "rows/s", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"first {sample} rows of the 60M-row workload per step, the oracle's row loop "
                                   f"over {cores} contiguous row ranges on {cores} threads"},
        "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _time_launches(torch, fn, reps, flush=None, stream=None):
    """Median CUDA-event time (ms) of fn() over reps launches, after 3 warm-ups;
    `flush` (untimed) runs before each timed launch."""
    for _ in range(3):
        fn()
    times = []
    for _ in range(reps):
        if flush is not None:
            flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def _time_burst(torch, fn, reps, stream=None):
    """Mean CUDA-event time (ms) of fn() over `reps` back-to-back calls after 3 warm-ups: the host enqueues
    ahead, so per-call host work overlaps the device (the device-limited rate of repeated calls)."""
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def oracle_plan_rate(spec, rows, seconds):
    """Rows/s of the CPU oracle's plan evaluator (one thread) on `spec`: runs until `seconds` pass (at least
    twice), median of the later half."""
    import oracle
    times = []
    t_end = time.perf_counter() + seconds
    while len(times) < 2 or (time.perf_counter() < t_end and len(times) < 8):
        t0 = time.perf_counter()
        oracle.run_plan(want_pairs=False, cap_groups=None, **spec)
        times.append(time.perf_counter() - t0)
    return rows / statistics.median(times[len(times) // 2:]), len(times)


def secondary_workloads(tqp, torch, dev, local, reps, cpu_seconds=0.0):
    """The other two analytical shapes, timed per launch (reported beside the headline), each with the CPU
    oracle timed on the same inputs (the 1M-row aggregate in full, the join on a 6M-row probe sample)."""
    out = {}
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # 512 MB > L2

    def flush():
        flush_buf.fill_(1)

    # 1M-row six-group aggregation: date <= 2450, GROUP BY (flag, status)
    n = 1_000_000
    t = datagen.fact_table(n, seed=datagen.DEFAULT_SEED)
    cols = [torch.from_numpy(t[k]).to(dev) for k in ("date", "flag", "status", "quantity", "price", "discount")]
    table = tqp.TableRef(cols)
    ctx = tqp.Context(local, 64 << 20)
    ctx.set_autotune(True)
    aggs = [("sum", [("col", 3)]), ("sum", [("col", 4)]),
            ("sum", [("col", 4), ("const", 100), ("col", 5), "sub", "mul"]), ("count", None), ("avg", [("col", 4)])]
    keys = torch.zeros(64 * 2, dtype=torch.int64, device=dev)
    iv = torch.zeros(64 * 5, dtype=torch.int64, device=dev)
    fv = torch.zeros(64 * 5, dtype=torch.float64, device=dev)
    ng = torch.zeros(1, dtype=torch.int64, device=dev)

    def q1():
        tqp.tqp_groupby_agg(ctx, table, [(0, "le", 2450)], [1, 2], aggs, keys, iv, fv, 64, ng, stream)

    # the generic kernel, then the kernel compiled for this query's shape (a prepared query: the
    # compile, once per shape, happens in the first untimed call)
    ctx.set_jit(0)
    generic = {"ms_l2_resident": _time_launches(torch, q1, reps),
               "ms_after_l2_flush": _time_launches(torch, q1, max(5, reps // 4), flush=flush),
               "ms_back_to_back": _time_burst(torch, q1, 50, stream=stream)}
    ctx.set_jit(2)
    jit0 = tqp.tqp_jit_stats()["launches"]
    hot = _time_launches(torch, q1, reps)
    cold = _time_launches(torch, q1, max(5, reps // 4), flush=flush)
    burst = _time_burst(torch, q1, 50, stream=stream)
    specialised = tqp.tqp_jit_stats()["launches"] > jit0
    ctx.check(stream)
    out["groupby_1M_6groups"] = {
        "workload": "1M rows; date<=2450; GROUP BY (flag u8, status u8): SUM(qty), SUM(price), "
                    "SUM(price*(100-disc)), COUNT, AVG(price); keys ascending",
        "ms_l2_resident": hot, "ms_after_l2_flush": cold, "rows_per_s": n / (cold / 1e3),
        "ms_back_to_back": burst, "rows_per_s_back_to_back": n / (burst / 1e3),
        "timing": "ms_l2_resident / ms_after_l2_flush: one call between synchronisations (host work included); "
                  "ms_back_to_back: 50 calls enqueued back to back (host work overlapped, table L2-resident)",
        "algorithmic_bytes": n * 26, "achieved_gbs_after_flush": n * 26 / (cold / 1e3) / 1e9,
        "groups": int(ng.item()),
        "kernel": "compiled for the query's shape at run time" if specialised else "generic",
        "generic_kernel": generic}
    if cpu_seconds > 0:
        spec = dict(fact=[t[k] for k in ("date", "flag", "status", "quantity", "price", "discount")],
                    preds=[(0, "le", 2450)], group_cols=[1, 2], aggs=aggs, want_row_ids=False)
        rate, runs = oracle_plan_rate(spec, n, cpu_seconds)
        out["groupby_1M_6groups"]["cpu_baseline"] = {"value": rate, "unit": "rows/s", "cores": 1, "kind": "oracle",
                                                     "sample": f"the full 1M-row workload, {runs} runs"}
    ctx.close()

    # hash join + 150K-group aggregation + top-100
    nb, ngr, npr = 1_500_000, 150_000, 60_000_000
    dim = datagen.dim_table(nb, ngr, seed=datagen.DEFAULT_SEED + 2)
    pr = datagen.probe_table(npr, nb, seed=datagen.DEFAULT_SEED + 2)
    F = tqp.TableRef([torch.from_numpy(pr["fk"]).to(dev), torch.from_numpy(pr["value"]).to(dev)])
    D = tqp.TableRef([torch.from_numpy(dim["key"]).to(dev), torch.from_numpy(dim["payload"]).to(dev)])
    ctx = tqp.Context(local, 4 << 30)  # (the sort-based group-by of 60M rows sorts 1.4 GB of pairs)
    ctx.set_autotune(True)
    k = 100
    rk = torch.zeros(k, dtype=torch.int64, device=dev)
    riv = torch.zeros(k * 2, dtype=torch.int64, device=dev)
    rng_ = torch.zeros(1, dtype=torch.int64, device=dev)
    rtot = torch.zeros(1, dtype=torch.int64, device=dev)
    rj = torch.zeros(1, dtype=torch.int64, device=dev)
    plan = tqp.make_plan(F, (), D, 0, 0, [3], [("sum", [("col", 1)]), ("count", None)], None, k, 0)
    res = tqp.make_result(None, 0, None, None, rk, riv, None, k, rng_, rtot, rj)

    def join():
        tqp.tqp_run_plan(ctx, plan, res, stream)

    ms = _time_launches(torch, join, max(5, reps // 2))
    ctx.check(stream)
    ctx.set_variant(1)  # the fused probe (L2 reductions), for comparison with the tuned choice
    ms_fused = _time_launches(torch, join, max(5, reps // 2))
    ctx.set_variant(0)  # the radix-partitioned aggregation
    ms_part = _time_launches(torch, join, max(5, reps // 2))
    ctx.set_variant(-1)
    ctx.check(stream)

    # the same build and probe keys, the join materialised as (build, probe) index pairs
    pcap = npr
    bidx = torch.empty(pcap, dtype=torch.int32, device=dev)
    pidx = torch.empty(pcap, dtype=torch.int32, device=dev)
    pcnt = torch.zeros(1, dtype=torch.int64, device=dev)

    def pairs():
        tqp.tqp_hash_join(ctx, D, 0, F, 0, bidx, pidx, pcap, pcnt, stream)

    ms_pairs = _time_launches(torch, pairs, max(5, reps // 2))
    ctx.set_variant(1)  # the sort-based join, for comparison with the tuned choice
    ms_pairs_sort = _time_launches(torch, pairs, max(5, reps // 2))
    ctx.set_variant(0)
    ms_pairs_hash = _time_launches(torch, pairs, max(5, reps // 2))
    ctx.set_variant(-1)
    ctx.check(stream)
    npairs = int(pcnt.item())
    alg_pairs = nb * 4 + npr * 4 + npairs * 8  # build keys, probe keys, the pairs written
    out["hash_join_pairs"] = {
        "workload": "build 1.5M unique int32 keys, probe 60M Zipf(0.5) int32 keys; output (build, probe) int32 "
                    "index pairs, probe index ascending",
        "ms": ms_pairs, "probe_rows_per_s": npr / (ms_pairs / 1e3), "pairs": npairs, "algorithmic_bytes": alg_pairs,
        "achieved_gbs": alg_pairs / (ms_pairs / 1e3) / 1e9,
        "frac_of_measured_hbm": alg_pairs / (ms_pairs / 1e3) / 1e9 / measured_peaks()[0],
        "ms_hash_table": ms_pairs_hash, "ms_sort_based": ms_pairs_sort}
    del bidx, pidx
    # many groups without a join: GROUP BY the 1.5M distinct probe keys, hash vs sort-based aggregation
    G = 1_500_000
    gk = torch.zeros(G, dtype=torch.int64, device=dev)
    giv = torch.zeros(2 * G, dtype=torch.int64, device=dev)
    gng = torch.zeros(1, dtype=torch.int64, device=dev)
    gagg = [("sum", [("col", 1)]), ("count", None)]

    def grp():
        tqp.tqp_groupby_agg(ctx, F, [], [0], gagg, gk, giv, None, G, gng, stream)

    ms_g = _time_launches(torch, grp, max(5, reps // 4))
    ctx.set_variant(1)
    ms_g_sort = _time_launches(torch, grp, max(5, reps // 4))
    ctx.set_variant(0)
    ms_g_hash = _time_launches(torch, grp, max(5, reps // 4))
    ctx.set_variant(-1)
    ctx.check(stream)
    alg_g = npr * 12
    out["groupby_60M_1.5Mgroups"] = {
        "workload": "60M rows (int32 key Zipf(0.5) over 1.5M values, int64 value); GROUP BY key: SUM(value), COUNT; "
                    "keys ascending",
        "ms": ms_g, "rows_per_s": npr / (ms_g / 1e3), "algorithmic_bytes": alg_g,
        "achieved_gbs": alg_g / (ms_g / 1e3) / 1e9,
        "frac_of_measured_hbm": alg_g / (ms_g / 1e3) / 1e9 / measured_peaks()[0],
        "ms_hash": ms_g_hash, "ms_sort_based": ms_g_sort, "groups": int(gng.item())}
    del gk, giv
    alg = npr * 12 + nb * 8
    out["join_group_top100"] = {
        "workload": "build 1.5M unique int32 keys (payload = 150K groups); probe 60M Zipf(0.5) int32 fk + int64 "
                    "value; GROUP BY payload SUM(value), COUNT; top-100 by SUM desc, key asc",
        "ms": ms, "probe_rows_per_s": npr / (ms / 1e3), "algorithmic_bytes": alg,
        "achieved_gbs": alg / (ms / 1e3) / 1e9, "frac_of_measured_hbm": alg / (ms / 1e3) / 1e9 / measured_peaks()[0],
        "ms_radix_partitioned": ms_part, "ms_fused_probe": ms_fused,
        "joined_rows": int(rj.item()), "groups": int(rtot.item())}
    ctx.close()
    out.update(hashed_join_workloads(tqp, torch, dev, local, reps))
    if cpu_seconds > 0:
        ns = 6_000_000
        spec = dict(fact=[pr["fk"][:ns], pr["value"][:ns]], dim=[dim["key"], dim["payload"]], fact_fk=0, dim_key=0,
                    group_cols=[3], aggs=[("sum", [("col", 1)]), ("count", None)], topk=k, topk_agg=0,
                    want_row_ids=False)
        rate, runs = oracle_plan_rate(spec, ns, cpu_seconds)
        out["join_group_top100"]["cpu_baseline"] = {"value": rate, "unit": "probe rows/s", "cores": 1,
                                                    "kind": "oracle",
                                                    "sample": f"first {ns} probe rows with the full build side, "
                                                              f"{runs} runs"}
    return out


def hashed_join_workloads(tqp, torch, dev, local, reps):
    """The join shapes of the dense-key lines over SPARSE build keys (1.5M unique int32 keys scattered over
    [0, 2^31) and Zipf(0.5) probe keys over them), so the build side goes into the hashed open-addressing table
    instead of a direct-mapped one."""
    out = {}
    nb, ngr, npr = 1_500_000, 150_000, 60_000_000
    seed = datagen.DEFAULT_SEED + 2
    dim = datagen.dim_table(nb, ngr, seed=seed, sparse=True)
    pr = datagen.probe_table(npr, nb, seed=seed, sparse=True)
    F = tqp.TableRef([torch.from_numpy(pr["fk"]).to(dev), torch.from_numpy(pr["value"]).to(dev)])
    D = tqp.TableRef([torch.from_numpy(dim["key"]).to(dev), torch.from_numpy(dim["payload"]).to(dev)])
    stream = torch.cuda.current_stream()
    ctx = tqp.Context(local, 1 << 30)
    ctx.set_autotune(True)
    k = 100
    z = lambda m: torch.zeros(m, dtype=torch.int64, device=dev)  # noqa: E731
    rk, riv, rng_, rtot, rj = z(k), z(2 * k), z(1), z(1), z(1)
    plan = tqp.make_plan(F, (), D, 0, 0, [3], [("sum", [("col", 1)]), ("count", None)], None, k, 0)
    res = tqp.make_result(None, 0, None, None, rk, riv, None, k, rng_, rtot, rj)
    run = lambda: tqp.tqp_run_plan(ctx, plan, res, stream)  # noqa: E731
    ms = _time_launches(torch, run, max(5, reps // 2), stream=stream)
    ctx.set_variant(1)
    ms_fused = _time_launches(torch, run, max(5, reps // 2), stream=stream)
    ctx.set_variant(0)
    ms_part = _time_launches(torch, run, max(5, reps // 2), stream=stream)
    ctx.set_variant(-1)
    ctx.check(stream)
    alg = npr * 12 + nb * 8
    peak = measured_peaks()[0]
    out["join_group_top100_hashed"] = {
        "workload": "build 1.5M unique int32 keys scattered over [0, 2^31) (hashed table; payload = 150K groups); "
                    "probe 60M Zipf(0.5) int32 fk + int64 value; GROUP BY payload SUM(value), COUNT; top-100",
        "ms": ms, "probe_rows_per_s": npr / (ms / 1e3), "algorithmic_bytes": alg,
        "achieved_gbs": alg / (ms / 1e3) / 1e9, "frac_of_measured_hbm": alg / (ms / 1e3) / 1e9 / peak,
        "ms_radix_partitioned": ms_part, "ms_fused_probe": ms_fused,
        "joined_rows": int(rj.item()), "groups": int(rtot.item())}
    bidx = torch.empty(npr, dtype=torch.int32, device=dev)
    pidx = torch.empty(npr, dtype=torch.int32, device=dev)
    pcnt = torch.zeros(1, dtype=torch.int64, device=dev)
    pj = lambda: tqp.tqp_hash_join(ctx, D, 0, F, 0, bidx, pidx, npr, pcnt, stream)  # noqa: E731
    ms_pairs = _time_launches(torch, pj, max(5, reps // 2), stream=stream)
    ctx.set_variant(1)
    ms_pairs_sort = _time_launches(torch, pj, max(5, reps // 2), stream=stream)
    ctx.set_variant(0)
    ms_pairs_hash = _time_launches(torch, pj, max(5, reps // 2), stream=stream)
    ctx.set_variant(-1)
    ctx.check(stream)
    npairs = int(pcnt.item())
    alg_pairs = nb * 4 + npr * 4 + npairs * 8
    out["hash_join_pairs_hashed"] = {
        "workload": "build 1.5M unique int32 keys scattered over [0, 2^31) (hashed table), probe 60M Zipf(0.5) int32 "
                    "keys; output (build, probe) int32 index pairs, probe index ascending",
        "ms": ms_pairs, "probe_rows_per_s": npr / (ms_pairs / 1e3), "pairs": npairs, "algorithmic_bytes": alg_pairs,
        "achieved_gbs": alg_pairs / (ms_pairs / 1e3) / 1e9,
        "frac_of_measured_hbm": alg_pairs / (ms_pairs / 1e3) / 1e9 / peak,
        "ms_hash_table": ms_pairs_hash, "ms_sort_based": ms_pairs_sort}
    ctx.close()
    return out


BATCH_PLANS = 512


def batched_plans(tqp, torch, dev, n_plans=BATCH_PLANS, seed=datagen.DEFAULT_SEED + 3):
    """n_plans independent plans (q1 group-by, q6 filter-compact-sum, join-group-top-100 in turn) over tables of
    log-uniform sizes in [10K, 5M] rows.  Every plan reads its own disjoint slice of the generated columns (no
    table is shared, so nothing stays in L2).  Returns (plans, results, buffers, meta)."""
    sizes = datagen.log_uniform_int(seed, 77, n_plans, 10_000, 5_000_000)
    kinds = [i % 3 for i in range(n_plans)]
    scan_rows = int(sum(int(s) for s, k in zip(sizes, kinds) if k != 2))
    probe_rows = int(sum(int(s) for s, k in zip(sizes, kinds) if k == 2))
    # slices start on 16-row boundaries (16-byte aligned for every column type)
    ft = datagen.fact_table(scan_rows + 16 * n_plans, seed=seed, cols=("date", "flag", "status", "quantity", "price", "discount"))
    fcols = {k: torch.from_numpy(v).to(dev) for k, v in ft.items()}
    del ft
    q1_aggs = [("sum", [("col", 3)]), ("sum", [("col", 4)]),
               ("sum", [("col", 4), ("const", 100), ("col", 5), "sub", "mul"]), ("count", None),
               ("avg", [("col", 4)])]
    plans, results, keep = [], [], []
    f0 = 0
    alg_bytes = 0
    for i, (n, kind) in enumerate(zip((int(s) for s in sizes), kinds)):
        z = lambda m, dt=torch.int64: torch.zeros(max(m, 1), dtype=dt, device=dev)  # noqa: E731
        if kind == 0:   # q1: date <= 2450, GROUP BY (flag, status)
            T = tqp.TableRef([fcols[c][f0:f0 + n] for c in ("date", "flag", "status", "quantity", "price",
                                                             "discount")])
            f0 += (n + 15) // 16 * 16
            b = dict(keys=z(64 * 2), iv=z(64 * 5), fv=z(64 * 5, torch.float64), ng=z(1), tot=z(1), nr=z(1))
            plans.append(tqp.make_plan(T, [(0, "le", 2450)], None, 0, 0, [1, 2], q1_aggs))
            results.append(tqp.make_result(None, 0, b["nr"], None, b["keys"], b["iv"], b["fv"], 64, b["ng"],
                                           b["tot"], None))
            alg_bytes += n * 26
        elif kind == 1:  # q6: a 365-day window, discount in [5,7], quantity < 24; SUM(price*discount) + row ids
            T = tqp.TableRef([fcols[c][f0:f0 + n] for c in ("date", "discount", "quantity", "price")])
            f0 += (n + 15) // 16 * 16
            b = dict(ids=z(n, torch.int32), nr=z(1), s=z(1))
            plans.append(tqp.make_plan(T, [(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)],
                                       sum_expr=[("col", 3), ("col", 1), "mul"], emit_row_ids=True))
            results.append(tqp.make_result(b["ids"], n, b["nr"], b["s"]))
            alg_bytes += n * 16 + int(n * 0.02) * 12
        else:            # join: build nb = n/40 unique keys (nb/10 groups), probe n Zipf(0.5) keys, top-100
            nb = max(1000, n // 40)
            dim = datagen.dim_table(nb, max(1, nb // 10), seed=seed + i)
            D = tqp.TableRef([torch.from_numpy(dim["key"]).to(dev), torch.from_numpy(dim["payload"]).to(dev)])
            pr = datagen.probe_table(n, nb, seed=seed + i)
            fk, val = torch.from_numpy(pr["fk"]).to(dev), torch.from_numpy(pr["value"]).to(dev)
            F = tqp.TableRef([fk, val])
            b = dict(keys=z(100), iv=z(200), ng=z(1), tot=z(1), nj=z(1), d=D, fk=fk, val=val)
            plans.append(tqp.make_plan(F, (), D, 0, 0, [3], [("sum", [("col", 1)]), ("count", None)], None, 100, 0))
            results.append(tqp.make_result(None, 0, None, None, b["keys"], b["iv"], None, 100, b["ng"], b["tot"],
                                           b["nj"]))
            alg_bytes += n * 12 + nb * 8
        b["kind"] = kind
        keep.append(b)
    meta = {"scan_rows": scan_rows, "probe_rows": probe_rows, "alg_bytes": alg_bytes}
    return plans, results, keep, meta


def batched_snapshot(torch, keep):
    """The written part of every plan's outputs (counts, sums, groups, row ids), as int64 host tensors."""
    torch.cuda.synchronize()
    out = []
    for b in keep:
        if b["kind"] == 0:
            g = max(int(b["ng"].item()), 0)
            parts = [b["ng"], b["tot"], b["nr"], b["keys"][:2 * g], b["iv"][:5 * g], b["fv"][:5 * g].view(torch.int64)]
        elif b["kind"] == 1:
            k = min(max(int(b["nr"].item()), 0), b["ids"].numel())
            parts = [b["nr"], b["s"], b["ids"][:k].to(torch.int64)]
        else:
            g = max(int(b["ng"].item()), 0)
            parts = [b["ng"], b["tot"], b["nj"], b["keys"][:g], b["iv"][:2 * g]]
        out.append(torch.cat([x.flatten() for x in parts]).cpu())
    return out


def batched_workload(tqp, torch, dev, local, reps, n_plans=BATCH_PLANS):
    """The batched mix: one captured batch (tqp_batch_run) against one tqp_run_plan call per plan."""
    plans, results, keep, meta = batched_plans(tqp, torch, dev, n_plans)
    scan_rows, probe_rows, alg_bytes = meta["scan_rows"], meta["probe_rows"], meta["alg_bytes"]
    stream = torch.cuda.current_stream()
    ctx = tqp.Context(local, 4 << 30)
    ctx.set_autotune(True)  # both arms: launch shapes (and the batch's tile size) picked by timing candidates
    snapshot = lambda: batched_snapshot(torch, keep)  # noqa: E731

    def seq():
        for p, r in zip(plans, results):
            tqp.tqp_run_plan(ctx, p, r, stream)

    def wall(fn, n):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / n * 1e3

    seq_ms = _time_launches(torch, seq, max(3, reps // 4), stream=stream)
    seq_wall = wall(seq, 3)
    ctx.check(stream)
    want = snapshot()
    for b in keep:
        for k in ("keys", "iv", "fv", "ng", "tot", "nr", "ids", "s", "nj"):
            if k in b:
                b[k].fill_(-7)
    batch = tqp.tqp_batch_create(ctx, plans, results)
    run = lambda: tqp.tqp_batch_run(batch, stream)  # noqa: E731
    bat_ms = _time_launches(torch, run, reps, stream=stream)
    bat_wall = wall(run, reps)
    ctx.check(stream)
    got = snapshot()
    identical = all(torch.equal(a, b) for a, b in zip(want, got))
    tqp.tqp_batch_destroy(batch)
    rp = lambda: tqp.tqp_run_plans(ctx, plans, results, stream)  # noqa: E731
    rp_ms = _time_launches(torch, rp, max(3, reps // 4), stream=stream)
    ctx.check(stream)
    ctx.close()
    rows = scan_rows + probe_rows
    return {
        "workload": f"{n_plans} plans (q1 group-by / q6 filter+ids+sum / join+group+top-100 in turn), table sizes "
                    f"log-uniform in [10K, 5M] rows, {rows} rows in all, disjoint slices (no L2 reuse)",
        "batched_graph_ms": bat_ms, "batched_graph_wall_ms": bat_wall,
        "run_plans_ms": rp_ms, "sequential_ms": seq_ms, "sequential_wall_ms": seq_wall,
        "batched_queries_per_s": n_plans / (bat_wall / 1e3), "sequential_queries_per_s": n_plans / (seq_wall / 1e3),
        "speedup_wall": seq_wall / bat_wall, "rows": rows, "batched_rows_per_s": rows / (bat_ms / 1e3),
        "algorithmic_bytes": alg_bytes, "batched_achieved_gbs": alg_bytes / (bat_ms / 1e3) / 1e9,
        "identical_to_sequential": identical,
    }


def q6_windows(k, seed):
    """k filter queries shaped like the headline one, each with its own seeded 365-day window, discount band of
    three values and quantity cutoff."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        d0 = int(rng.integers(0, 2557 - 365))
        disc = int(rng.integers(1, 9))
        qty = int(rng.integers(2, 51))
        out.append([(0, "ge", d0), (0, "lt", d0 + 365), (1, "between", disc - 1, disc + 1), (2, "lt", qty)])
    return out


def shared_scan_workload(tqp, torch, dev, local, table, n, reps):
    """Shared scans on the headline table: K filter queries (count + SUM(price*discount) each) in one
    tqp_filter_shared call against K tqp_filter calls, K = 1, 8, 32; identical outputs checked."""
    ctx = tqp.Context(local, 256 << 20)
    ctx.set_autotune(True)  # the first (warm-up) call of each K picks the launch shape
    stream = torch.cuda.current_stream()
    out = {"workload": f"{n // 1_000_000}M rows (date i32, discount i64, quantity i32, price i64); K queries, each "
                       "a seeded 365-day date window, a three-value discount band and a quantity cutoff; "
                       "count + SUM(price*discount) per query", "by_k": {}}
    for k in (1, 8, 32):
        preds = q6_windows(k, datagen.DEFAULT_SEED + 7)
        qs = [(p, EXPR, torch.zeros(1, dtype=torch.int64, device=dev), torch.zeros(1, dtype=torch.int64, device=dev))
              for p in preds]
        prepared = tqp.ScanQueries(qs)  # marshalled once, as a serving loop would
        shared = _time_launches(torch, lambda: tqp.tqp_filter_shared(ctx, table, prepared, stream), reps,
                                stream=stream)
        got = [(int(c.item()), int(s_.item())) for _, _, c, s_ in qs]
        sep = _time_launches(torch, lambda: [tqp.tqp_filter(ctx, table, p, e, s_, None, 0, c, stream)
                                             for p, e, c, s_ in qs], max(3, reps // 4), stream=stream)
        alone = [(int(c.item()), int(s_.item())) for _, _, c, s_ in qs]
        ctx.check(stream)
        alg = n * 24  # the four staged columns, read once
        out["by_k"][str(k)] = {"ms_shared": shared, "ms_separate": sep, "qps_shared": k / (shared / 1e3),
                               "qps_separate": k / (sep / 1e3), "speedup": sep / shared,
                               "achieved_gbs_shared": alg / (shared / 1e3) / 1e9,
                               "frac_of_measured_hbm": alg / (shared / 1e3) / 1e9 / measured_peaks()[0],
                               "same_as_separate": got == alone}
    ctx.close()
    return out


STR_ROWS = 20_000_000


def string_case_inputs(n, seed=datagen.DEFAULT_SEED + 11):
    """A 24-byte string column (1 to 3 seeded words, 0-padded) and a price column; the query keeps rows whose
    string contains the first two letters of a vocabulary word and whose price is below 5,000,000."""
    s = datagen.string_column(n, seed=seed)
    price = datagen.fact_table(n, seed=seed, cols=["price"])["price"]
    w = datagen.string_vocab(seed)[0][:2].decode()
    preds = [(0, "like", f"%{w}%"), (1, "lt", 5_000_000)]
    return s, price, preds


def string_workload(tqp, torch, dev, local, reps, n=STR_ROWS):
    """LIKE on a string column plus a numeric predicate, COUNT and SUM(price): the pre-pass over the strings,
    then the staged filter over the pass column and the price; a 1M-row prefix checked against the oracle."""
    import oracle
    s, price, preds = string_case_inputs(n)
    T = tqp.TableRef([torch.from_numpy(s).to(dev), torch.from_numpy(price).to(dev)])
    ctx = tqp.Context(local, 256 << 20)
    ctx.set_autotune(True)
    stream = torch.cuda.current_stream()
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    sm = torch.zeros(1, dtype=torch.int64, device=dev)
    expr = [("col", 1)]
    fn = lambda: tqp.tqp_filter(ctx, T, preds, expr, sm, None, 0, cnt, stream)  # noqa: E731
    ms = _time_launches(torch, fn, reps, stream=stream)
    ctx.check(stream)
    m = 1_000_000
    Tm = tqp.TableRef([torch.from_numpy(s[:m]).to(dev), torch.from_numpy(price[:m]).to(dev)])
    tqp.tqp_filter(ctx, Tm, preds, expr, sm, None, 0, cnt, stream)
    ids, want_sum = oracle.filter_rows([s[:m], price[:m]], preds, expr)
    same = int(cnt.item()) == len(ids) and int(sm.item()) == want_sum
    ctx.close()
    alg = n * (24 + 1 + 1 + 8)  # strings, pass byte written and read, price
    return {"workload": f"{n // 1_000_000}M rows: 24-byte strings (1-3 seeded words, 0-padded) LIKE '{preds[0][2]}' "
                        "AND price < 5,000,000; COUNT and SUM(price)",
            "ms": ms, "rows_per_s": n / (ms / 1e3), "algorithmic_bytes": alg,
            "achieved_gbs": alg / (ms / 1e3) / 1e9, "frac_of_measured_hbm": alg / (ms / 1e3) / 1e9 / measured_peaks()[0],
            "kernels": "k_str_prepass (strings -> pass byte), k_filter (pass byte, price)",
            "oracle_equal_1M_prefix": bool(same)}


SERVE_FACT_ROWS = 600_000_000
SERVE_DIM_ROWS = 15_000_000
SERVE_POOL = 512  # result buffer sets, reused round-robin


def serving_workload(tqp, torch, dev, local, seconds=10.0, rate=2000.0,
                     sweep=(2000, 6000, 16000, 32000, 64000, 128000), fifo_max_rate=16000,
                     sweep_seconds=1.0, fact_rows=SERVE_FACT_ROWS, dim_rows=SERVE_DIM_ROWS):
    """Open-loop Poisson arrivals of the three plan shapes over seeded row ranges of a resident fact table
    (the scan-aggregate columns) joined, for the join shape, with a prepared resident dimension; continuous batching
    (tqp_server, 64 plans per batch, 3 batches in flight) against one-at-a-time FIFO (1 plan, 1 in flight)."""
    from datagen import torch_gen
    seed = datagen.DEFAULT_SEED + 4
    t_setup = time.perf_counter()
    names = ("date", "flag", "status", "quantity", "price", "discount", "key")
    fact = torch_gen.fact_table(fact_rows, seed=seed, cols=names, device=dev)
    d = datagen.dim_table(dim_rows, 150_000, seed=seed)
    D = tqp.TableRef([torch.from_numpy(d["key"]).to(dev), torch.from_numpy(d["payload"]).to(dev)])
    del d
    pctx = tqp.Context(local, 2 << 30)
    pdim = tqp.tqp_dim_prepare(pctx, D, 0, [1], max_groups=150_000)
    q1_aggs = [("sum", [("col", 3)]), ("sum", [("col", 4)]),
               ("sum", [("col", 4), ("const", 100), ("col", 5), "sub", "mul"]), ("count", None),
               ("avg", [("col", 4)])]
    q6_preds = [(0, "ge", 731), (0, "lt", 1096), (1, "between", 5, 7), (2, "lt", 24)]
    max_rows = 5_000_000
    pool = []
    for _ in range(SERVE_POOL):
        z = lambda m, dt=torch.int64: torch.zeros(m, dtype=dt, device=dev)  # noqa: E731
        pool.append(dict(ids=z(max_rows, torch.int32), keys=z(128), iv=z(320), fv=z(320, torch.float64), ng=z(1),
                         tot=z(1), nr=z(1), s=z(1), nj=z(1)))
    nq_max = int(max(rate * seconds, max(sweep) * sweep_seconds)) + 1
    sizes = datagen.log_uniform_int(seed, 91, nq_max, 10_000, max_rows)
    offs = datagen.uniform_int(seed, 92, nq_max, 0, (fact_rows - max_rows) // 16, np.int64) * 16
    views = {}

    def query(i):
        kind, n, r0 = i % 3, int(sizes[i]), int(offs[i])
        b = pool[i % SERVE_POOL]
        if kind == 0:
            T = tqp.TableRef([fact[c][r0:r0 + n] for c in names[:6]])
            plan = tqp.make_plan(T, [(0, "le", 2450)], None, 0, 0, [1, 2], q1_aggs)
            res = tqp.make_result(None, 0, b["nr"], None, b["keys"], b["iv"], b["fv"], 64, b["ng"], b["tot"], None)
        elif kind == 1:
            T = tqp.TableRef([fact[c][r0:r0 + n] for c in ("date", "discount", "quantity", "price")])
            plan = tqp.make_plan(T, q6_preds, sum_expr=[("col", 3), ("col", 1), "mul"], emit_row_ids=True)
            res = tqp.make_result(b["ids"], n, b["nr"], b["s"])
        else:
            T = tqp.TableRef([fact["key"][r0:r0 + n], fact["price"][r0:r0 + n]])
            plan = tqp.make_plan(T, (), D, 0, 0, [3], [("sum", [("col", 1)]), ("count", None)], None, 100, 0,
                                 prepared=pdim)
            res = tqp.make_result(None, 0, None, None, b["keys"], b["iv"], None, 100, b["ng"], b["tot"], b["nj"])
        views[i] = T
        return plan, res

    queries = [query(i) for i in range(nq_max)]
    setup_s = time.perf_counter() - t_setup

    # the scan-aggregate query over the whole resident table (600M rows, 15.6 GB of its columns)
    g600 = None
    if fact_rows >= 100_000_000:
        gctx = tqp.Context(local, 256 << 20)
        gctx.set_autotune(True)
        T = tqp.TableRef([fact[c] for c in names[:6]])
        b = pool[0]
        st = torch.cuda.current_stream()
        fn = lambda: tqp.tqp_groupby_agg(gctx, T, [(0, "le", 2450)], [1, 2], q1_aggs, b["keys"], b["iv"],  # noqa
                                         b["fv"], 64, b["ng"], st)
        jit0 = tqp.tqp_jit_stats()["launches"]
        ms = _time_launches(torch, fn, 5, stream=st)
        gctx.check(st)
        jit_launches = tqp.tqp_jit_stats()["launches"] - jit0
        ng = int(b["ng"].item())
        counted = int(b["iv"][:ng * 5].view(ng, 5)[:, 3].sum().item())
        expect = int((fact["date"] <= 2450).sum().item())
        alg = fact_rows * 26
        g600 = {"workload": f"{fact_rows // 1_000_000}M rows (the resident serving table); date<=2450; GROUP BY "
                            "(flag u8, status u8): SUM(qty), SUM(price), SUM(price*(100-disc)), COUNT, AVG(price)",
                "ms": ms, "rows_per_s": fact_rows / (ms / 1e3), "algorithmic_bytes": alg,
                "achieved_gbs": alg / (ms / 1e3) / 1e9, "frac_of_measured_hbm": alg / (ms / 1e3) / 1e9 / measured_peaks()[0],
                "groups": ng, "counts_sum_to_passing_rows": counted == expect,
                "kernel": "compiled for the query's shape at run time" if jit_launches else "generic"}
        gctx.close()
        del T

    def run(max_batch, max_inflight, qps, nq, qlist=None):
        qlist = queries if qlist is None else qlist
        budget = 4 << 30
        ctx = tqp.Context(local, budget + (256 << 20))
        srv = tqp.Server(ctx, max_batch=max_batch, max_inflight=max_inflight, budget_bytes=budget)
        rng = np.random.default_rng(int(qps) * 7 + max_batch)
        arrive = np.cumsum(rng.exponential(1.0 / qps, nq))
        sub_t = np.zeros(nq)
        done = {}
        t0 = time.perf_counter()
        for i in range(nq):
            target = t0 + arrive[i]
            while True:
                now = time.perf_counter()
                if now >= target:
                    break
                if target - now > 3e-4:
                    for c in srv.poll():
                        done[c[0]] = c
            while i >= SERVE_POOL and (i - SERVE_POOL) not in done:  # the result set is still in use
                for c in srv.poll():
                    done[c[0]] = c
            sub_t[i] = time.perf_counter()
            srv.submit(qlist[i][0], qlist[i][1], i)
            if i % 32 == 31:
                for c in srv.poll():
                    done[c[0]] = c
        srv.drain(300.0)
        for c in srv.poll():
            done[c[0]] = c
        srv.close()
        ctx.close()
        lat = np.array([done[i][4] for i in range(nq)])
        end = max(sub_t[i] + done[i][4] for i in range(nq))
        errors = sum(1 for i in range(nq) if done[i][1] != 0)
        return {"offered_qps": qps, "queries": nq, "qps": nq / (end - sub_t[0]),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_batch": float(np.mean([done[i][2] for i in range(nq)])), "errors": errors}

    nq = int(rate * seconds)
    cont = run(64, 3, rate, nq)
    fifo = run(1, 1, rate, nq)
    # the served results of a sample equal the same plans run alone
    actx = tqp.Context(local, 1 << 30)
    same = True
    for i in range(nq - 6, nq):
        b = pool[i % SERVE_POOL]
        before = [t.clone() for t in (b["nr"], b["s"], b["ng"], b["tot"], b["nj"], b["keys"], b["iv"])]
        tqp.tqp_run_plan(actx, queries[i][0], queries[i][1])
        actx.check()
        after = [b["nr"], b["s"], b["ng"], b["tot"], b["nj"], b["keys"], b["iv"]]
        same &= all(torch.equal(x, y) for x, y in zip(before, after))
    actx.close()
    rows = []
    for qps in sweep:
        n_s = int(qps * sweep_seconds)
        row = {"offered_qps": qps, "continuous": run(64, 3, qps, n_s)}
        # one at a time saturates far below the top rates (its queue only grows there)
        row["one_at_a_time"] = run(1, 1, qps, n_s) if qps <= fifo_max_rate else None
        rows.append(row)

    def best(key, limit_ms=10.0):
        ok = [r[key]["qps"] for r in rows
              if r[key] is not None and r[key]["p99_ms"] <= limit_ms and r[key]["errors"] == 0]
        return max(ok) if ok else None

    def saturation(key):
        """The highest completed rate while it still kept up with the offered rate (within 5%)."""
        ok = [r[key]["qps"] for r in rows if r[key] is not None and r[key]["qps"] >= 0.95 * r["offered_qps"]]
        return max(ok) if ok else None

    # full-table filter queries (count + sum over all rows, each its own seeded window): the server's batches
    # pack them into shared scans of up to 32 queries each
    full = None
    if fact_rows >= 100_000_000:
        TF = tqp.TableRef([fact[c] for c in ("date", "discount", "quantity", "price")])
        nfull = 4000
        fq = []
        for i, pr in enumerate(q6_windows(nfull, seed + 5)):
            b = pool[i % SERVE_POOL]
            fq.append((tqp.make_plan(TF, pr, sum_expr=EXPR), tqp.make_result(None, 0, b["nr"], b["s"])))
        frows = []
        for qps in (250, 500, 1000, 2000, 3000, 4000):
            n_s = min(nfull, int(qps * 1.0))
            frows.append({"offered_qps": qps, "continuous_shared": run(64, 2, qps, n_s, fq),
                          "one_at_a_time": run(1, 1, qps, min(n_s, 500), fq) if qps <= 500 else None})
        sat = lambda key: max([r[key]["qps"] for r in frows  # noqa: E731
                               if r[key] is not None and r[key]["qps"] >= 0.95 * r["offered_qps"]
                               and r[key]["errors"] == 0] or [0.0])
        actx = tqp.Context(local, 256 << 20)
        same_f = True
        last = min(nfull, 4000)  # the final sweep point ran queries [0, last): the pool holds the last ones
        for i in range(last - 3, last):
            b = pool[i % SERVE_POOL]
            before = (b["nr"].clone(), b["s"].clone())
            tqp.tqp_run_plan(actx, fq[i][0], fq[i][1])
            actx.check()
            same_f &= torch.equal(before[0], b["nr"]) and torch.equal(before[1], b["s"])
        actx.close()
        full = {"workload": f"filter queries over all {fact_rows // 1_000_000}M rows (date, discount, quantity, "
                            "price: 14.4 GB), each a seeded 365-day window, discount band and quantity cutoff; "
                            "count + SUM(price*discount); open-loop Poisson arrivals",
                "sweep": frows, "saturation_qps": {"continuous_shared": sat("continuous_shared"),
                                                   "one_at_a_time": sat("one_at_a_time")},
                "served_equals_alone_sample": bool(same_f)}
        del TF

    tqp.tqp_dim_destroy(pdim)
    pctx.close()
    return {
        "workload": f"{fact_rows // 1_000_000}M-row resident fact table (scan-aggregate columns, {fact_rows * 30 / 1e9:.0f} GB) "
                    f"+ prepared {dim_rows // 1_000_000}M-row dimension; open-loop Poisson arrivals; each query one of "
                    "q1 group-by / q6 filter+ids+sum / join+group+top-100 over a seeded row range of "
                    "log-uniform [10K, 5M] rows",
        "rate_qps": rate, "seconds": seconds, "continuous_batching": cont, "one_at_a_time": fifo,
        "served_equals_alone_sample": bool(same), "sweep": rows,
        "qps_at_p99_le_10ms": {"continuous": best("continuous"), "one_at_a_time": best("one_at_a_time")},
        "qps_at_p99_le_1ms": {"continuous": best("continuous", 1.0), "one_at_a_time": best("one_at_a_time", 1.0)},
        "saturation_qps": {"continuous": saturation("continuous"), "one_at_a_time": saturation("one_at_a_time")},
        "setup_s": setup_s,
        "full_table_filters": full,
    }, g600


def scan_ceiling(tqp, torch, ctx, table, shape, reps=10, stream=None):
    """Mean ms of tqp_measure_scan_rate (the staged engine with a read-only body) at `shape`, over a burst
    of `reps` back-to-back calls (the host enqueues ahead, so its per-call work is not in the time)."""
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    fn = lambda: tqp.tqp_measure_scan_rate(ctx, table, *shape, out, stream)  # noqa: E731
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def engine_case(args):
    """The staged engine's streaming rate on the headline's predicate columns (date i32, discount i64,
    quantity i32: 16 B/row) for every launch shape: one JSON line per shape."""
    import torch
    import paper_2203_01877_gb300 as tqp
    host = gen_host(0)
    cols = [torch.from_numpy(a).cuda() for a in host[:3]]
    T = tqp.TableRef(cols)
    ctx = tqp.Context(0, 64 << 20)
    bytes_ = sum(c.numel() * c.element_size() for c in cols)
    for tile in (1024, 2048, 4096, 8192):
        for stages in (2, 3, 4):
            for cps in (1, 2):
                try:
                    ms = scan_ceiling(tqp, torch, ctx, T, (tile, stages, cps))
                except tqp.TqpError:
                    continue
                print(json.dumps({"case": "engine", "rows": N_ROWS, "bytes": bytes_, "tile_rows": tile,
                                  "stages": stages, "ctas_per_sm": cps, "ms": ms,
                                  "gbs": bytes_ / (ms / 1e3) / 1e9}), flush=True)
    ctx.close()
    return 0


def l2_red_case(args):
    """The reduction-rate roofline of the joined aggregation: G reductions/s of random 8-byte L2 reductions
    (tqp_measure_l2_red) over table sizes, reductions per row and occupancy; one JSON line per setting."""
    import torch
    import paper_2203_01877_gb300 as tqp
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream()
    rows = args.rows
    table = torch.zeros((96 << 20) // 8, dtype=torch.int64, device=dev)
    for mb in (2.4, 24, 96):
        words = int(mb * (1 << 20)) // 8
        t = table[:words]
        for adds in (1, 2):
            for bps, thr in ((1, 288), (2, 256), (4, 256), (8, 256)):
                fn = lambda: tqp.tqp_measure_l2_red(0, t, rows, adds, bps, thr, st)  # noqa: E731
                ms = _time_launches(torch, fn, 5, stream=st)
                print(json.dumps({"case": "l2red", "table_mb": mb, "adds_per_row": adds, "blocks_per_sm": bps,
                                  "threads": thr, "rows": rows, "ms": ms,
                                  "g_reds_per_s": rows * adds / (ms / 1e3) / 1e9}), flush=True)
    return 0


def profile_case(args):
    """One operator at a profiling size, for ncu: the first call autotunes, the next `--steps` calls run
    inside the NVTX range "tqp_profile" (capture them with --nvtx --nvtx-include "tqp_profile/")."""
    import torch
    import paper_2203_01877_gb300 as tqp
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream()
    ctx = tqp.Context(0, 2 << 30)
    ctx.set_autotune(True)
    if args.variant >= 0:
        ctx.set_variant(args.variant)
    if args.tuning:
        ctx.set_tuning(*[int(x) for x in args.tuning.split(",")])
    n = args.rows
    if args.case == "filter":
        t = datagen.fact_table(n, seed=datagen.DEFAULT_SEED + 1, cols=["date", "discount", "quantity", "price"])
        T = tqp.TableRef([torch.from_numpy(t[c]).to(dev) for c in ("date", "discount", "quantity", "price")])
        ids = torch.empty(n, dtype=torch.int32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        sm = torch.zeros(1, dtype=torch.int64, device=dev)
        fn = lambda: tqp.tqp_filter(ctx, T, PREDS, EXPR, sm, ids, n, cnt, st)  # noqa: E731
    elif args.case == "groupby":
        t = datagen.fact_table(n, seed=datagen.DEFAULT_SEED)
        T = tqp.TableRef([torch.from_numpy(t[c]).to(dev) for c in ("date", "flag", "status", "quantity", "price",
                                                                     "discount")])
        aggs = [("sum", [("col", 3)]), ("sum", [("col", 4)]),
                ("sum", [("col", 4), ("const", 100), ("col", 5), "sub", "mul"]), ("count", None),
                ("avg", [("col", 4)])]
        keys = torch.zeros(128, dtype=torch.int64, device=dev)
        iv = torch.zeros(320, dtype=torch.int64, device=dev)
        fv = torch.zeros(320, dtype=torch.float64, device=dev)
        ng = torch.zeros(1, dtype=torch.int64, device=dev)
        fn = lambda: tqp.tqp_groupby_agg(ctx, T, [(0, "le", 2450)], [1, 2], aggs, keys, iv, fv, 64, ng, st)  # noqa
    elif args.case in ("join", "join_hashed", "pairs", "pairs_hashed"):
        nb, ngr = 1_500_000, 150_000
        sparse = args.case.endswith("_hashed")
        dim = datagen.dim_table(nb, ngr, seed=datagen.DEFAULT_SEED + 2, sparse=sparse)
        pr = datagen.probe_table(n, nb, seed=datagen.DEFAULT_SEED + 2, sparse=sparse)
        F = tqp.TableRef([torch.from_numpy(pr["fk"]).to(dev), torch.from_numpy(pr["value"]).to(dev)])
        D = tqp.TableRef([torch.from_numpy(dim["key"]).to(dev), torch.from_numpy(dim["payload"]).to(dev)])
        z = lambda m: torch.zeros(m, dtype=torch.int64, device=dev)  # noqa: E731
        if args.case.startswith("join"):
            rk, riv, rng_, rtot, rj = z(100), z(200), z(1), z(1), z(1)
            plan = tqp.make_plan(F, (), D, 0, 0, [3], [("sum", [("col", 1)]), ("count", None)], None, 100, 0)
            res = tqp.make_result(None, 0, None, None, rk, riv, None, 100, rng_, rtot, rj)
            fn = lambda: tqp.tqp_run_plan(ctx, plan, res, st)  # noqa: E731
        else:
            bidx = torch.empty(n, dtype=torch.int32, device=dev)
            pidx = torch.empty(n, dtype=torch.int32, device=dev)
            pcnt = z(1)
            fn = lambda: tqp.tqp_hash_join(ctx, D, 0, F, 0, bidx, pidx, n, pcnt, st)  # noqa: E731
    elif args.case == "shared":  # K filter queries in one shared scan
        t = datagen.fact_table(n, seed=datagen.DEFAULT_SEED + 1, cols=["date", "discount", "quantity", "price"])
        T = tqp.TableRef([torch.from_numpy(t[c]).to(dev) for c in ("date", "discount", "quantity", "price")])
        qs = [(p, EXPR, torch.zeros(1, dtype=torch.int64, device=dev), torch.zeros(1, dtype=torch.int64, device=dev))
              for p in q6_windows(args.queries, datagen.DEFAULT_SEED + 7)]
        prepared = tqp.ScanQueries(qs)
        fn = lambda: tqp.tqp_filter_shared(ctx, T, prepared, st)  # noqa: E731
    elif args.case == "strings":  # LIKE on a string column + a numeric predicate
        s, price, preds = string_case_inputs(n)
        T = tqp.TableRef([torch.from_numpy(s).to(dev), torch.from_numpy(price).to(dev)])
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        sm = torch.zeros(1, dtype=torch.int64, device=dev)
        fn = lambda: tqp.tqp_filter(ctx, T, preds, [("col", 1)], sm, None, 0, cnt, st)  # noqa: E731
    else:  # the batched plan mix (512 plans by default)
        plans, results, keep, meta = batched_plans(tqp, torch, dev, n_plans=args.plans)
        batch = tqp.tqp_batch_create(ctx, plans, results)
        fn = lambda: tqp.tqp_batch_run(batch, st)  # noqa: E731
    fn()
    ctx.check(st)
    torch.cuda.nvtx.range_push("tqp_profile")
    for _ in range(args.steps):
        fn()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ctx.check(st)
    print(json.dumps({"case": args.case, "rows": n, "launched_steps": args.steps}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="tqp", choices=["tqp", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="0 skips the CPU baseline")
    ap.add_argument("--rows", type=int, default=N_ROWS, help="smaller cases for profiling only")
    ap.add_argument("--variant", type=int, default=-1, help="profiling: force a join plan's algorithm (0 or 1)")
    ap.add_argument("--no-operators", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving workload")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--queries", type=int, default=32, help="profiling: queries of the shared-scan case")
    ap.add_argument("--tuning", default="", help="profiling: force the scan launch shape, tile,stages,ctas_per_sm")
    ap.add_argument("--plans", type=int, default=BATCH_PLANS, help="profiling: plans of the batch case")
    ap.add_argument("--case", choices=["filter", "groupby", "join", "join_hashed", "pairs", "pairs_hashed", "batch",
                                       "shared", "strings", "l2red", "engine"], default=None,
                    help="profiling: run one operator (first call autotunes; --steps calls in NVTX range tqp_profile)")
    args = ap.parse_args()
    globals()["N_ROWS"] = args.rows
    if args.impl == "reference":
        return run_reference(args)
    if args.case == "l2red":
        return l2_red_case(args)
    if args.case == "engine":
        return engine_case(args)
    if args.case:
        return profile_case(args)

    import torch
    import torch.distributed as dist

    import paper_2203_01877_gb300 as tqp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    dev = torch.device(f"cuda:{local}")

    host = gen_host(rank)
    cols = [torch.from_numpy(a).to(dev) for a in host]
    table = tqp.TableRef(cols)
    ctx = tqp.Context(local, 64 << 20)
    ctx.set_autotune(True)  # the first (warm-up) call picks the launch shape
    ids = torch.empty(N_ROWS, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    s = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        tqp.tqp_filter(ctx, table, PREDS, EXPR, s, ids, N_ROWS, cnt, stream)

    for _ in range(max(3, args.warmup)):
        step()
    ctx.check(stream)
    k = int(cnt.item())

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t_start.record(stream)
        for i in range(args.steps):
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ctx.check(stream)
    total_ms = t_start.elapsed_time(t_end)
    launch_ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    # both filter kernels forced, beside the tuned choice timed above
    variant_ms = {}
    for name, v in (("staged_scan", 0), ("direct", 1)):
        ctx.set_variant(v)
        variant_ms[name] = _time_launches(torch, step, 20, stream=stream)
    ctx.set_variant(-1)
    ctx.check(stream)
    # the staged engine's own ceiling on the staged (predicate) columns: a read-only body, best shape
    ceil_table = tqp.TableRef(cols[:3])
    ceil = min((scan_ceiling(tqp, torch, ctx, ceil_table, sh, 10, stream), sh)
               for sh in ((2048, 3, 2), (2048, 2, 2), (4096, 2, 1)))
    staged_bytes = sum(c.numel() * c.element_size() for c in cols[:3])
    ctx.check(stream)
    if world > 1:
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms_per_step = total_ms / args.steps
    value = N_ROWS * world / (ms_per_step / 1e3)

    # end to end through the public API: pinned host columns -> device -> filter -> results back.
    # The predicate columns are copied to the device each step; the projected
    # price column stays in pinned host memory and the filter reads it in
    # place at the passing rows only (late materialisation over the host link).
    pinned = [torch.from_numpy(a).pin_memory() for a in host]
    dcols = [torch.empty_like(c) for c in cols[:3]]
    dtable = tqp.TableRef(dcols + [pinned[3]], host_ok=True)
    h_cnt = torch.zeros(1, dtype=torch.int64).pin_memory()
    h_sum = torch.zeros(1, dtype=torch.int64).pin_memory()
    h_ids = torch.empty(N_ROWS, dtype=torch.int32).pin_memory()
    e2e_times, d2h = [], 0
    for _ in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for d, p in zip(dcols, pinned[:3]):
            d.copy_(p, non_blocking=True)
        tqp.tqp_filter(ctx, dtable, PREDS, EXPR, s, ids, N_ROWS, cnt, stream)
        h_cnt.copy_(cnt, non_blocking=True)
        h_sum.copy_(s, non_blocking=True)
        torch.cuda.synchronize()
        kk = int(h_cnt.item())
        h_ids[:kk].copy_(ids[:kk])
        e2e_times.append(time.perf_counter() - t0)
        d2h = 16 + 4 * kk
    ctx.check(stream)
    h2d = sum(a.nbytes for a in host[:3]) + 8 * k  # copied columns + the passing rows' prices read in place
    e2e_s = statistics.median(e2e_times[1:]) if len(e2e_times) > 1 else float("nan")

    ops = None
    if rank == 0 and not args.no_operators:
        ops = secondary_workloads(tqp, torch, dev, local, 20, cpu_seconds=min(args.cpu_seconds, 5.0))
        ops["batched_512"] = batched_workload(tqp, torch, dev, local, 20)
        ops["shared_scan_60M"] = shared_scan_workload(tqp, torch, dev, local, table, N_ROWS, 10)
        ops["strings_like_20M"] = string_workload(tqp, torch, dev, local, 10)
        if not args.no_serving:
            ops["serving"], g600 = serving_workload(tqp, torch, dev, local, seconds=args.serve_seconds)
            if g600:
                ops["groupby_600M_6groups"] = g600
    if rank == 0:
        peak, peak_kind = measured_peaks()
        alg = algorithmic_bytes(N_ROWS, k)
        achieved = alg / (launch_ms / 1e3) / 1e9
        cpu = None
        if args.cpu_seconds > 0:
            cores = host_cores()
            cpu_rate, cpu_rows, cpu_runs, _ = oracle_rate(host, args.cpu_seconds, threads=cores)
            one_rate, one_rows, one_runs, _ = oracle_rate(host, args.cpu_seconds, rows_cap=12_000_000)
            cpu = {"value": cpu_rate, "unit": "rows/s", "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                   "sample": f"full {cpu_rows}-row workload, the oracle's row loop over {cores} contiguous row ranges "
                             f"on {cores} threads, {cpu_runs} runs, median of the later half",
                   "one_core": {"value": one_rate, "unit": "rows/s", "cores": 1,
                                "sample": f"first {one_rows} rows, one thread, {one_runs} runs, median of the later "
                                          "half"}}
        line = {
            "metric": "rows/s",
            "value": value,
            "unit": "rows/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "int64",
            "data": "synthetic (seeded counter-based generators)",
            "config": {"workload": WORKLOAD if N_ROWS == 60_000_000 else WORKLOAD.replace("60M", f"{N_ROWS}"),
                       "rows": N_ROWS, "passing_rows": k,
                       "l2": "inputs 1.44 GB > 126 MB L2: no flush between steps"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "kernel": "k_filter_direct" if variant_ms["direct"] < variant_ms["staged_scan"] else "k_filter",
                         "variant_call_ms": variant_ms,
                         "algorithmic_bytes_per_launch": alg, "launch_ms": launch_ms,
                         "engine_ceiling": {"what": "tqp_measure_scan_rate: the staged engine over the three "
                                                    "predicate columns with a read-only body",
                                            "staged_bytes": staged_bytes, "ms": ceil[0],
                                            "gbs": staged_bytes / (ceil[0] / 1e3) / 1e9,
                                            "shape": list(ceil[1])},
                         "traffic": ncu_traffic()},
            "cpu_baseline": cpu,
            "e2e": {"value": N_ROWS / e2e_s, "unit": "rows/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": 2 * args.steps,  # k_filter + k_compact per step
            "clocks": clk.summary(),
            "operators": ops,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

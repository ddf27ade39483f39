#!/usr/bin/env python
"""Throughput of exact balanced-butterfly counting on one GB300 (or N replicas).

One step is the whole hot path over one synthetic graph: bbc_prepare (validation,
degrees, pair-side choice, rank relabelling, the two signed CSR arrays, per-anchor wedge
estimate, work lists) followed by bbc_count with global and per-vertex counts. The
workload is the Chung-Lu power-law graph |U| = 1,000,000, |V| = 200,000, 20,000,000
distinct edges, expected-degree exponent 2.2 on both sides (max 50,000), P(+) = 0.8,
seed 0. The metric is W / step time in wedges per second, where W is the number of
oriented wedges of the graph (the sum over the centre side of C(d, 2)).

  value  device-resident input (edge list already in HBM), as the library sees it
  e2e    the same through host buffers: pinned host edge list copied in, per-vertex
         counts and totals copied out, every step inside the timed region
  roofline  the tile kernel's algorithmic bytes per launch (4 B per wedge visit, two
         visits per wedge with per-vertex counts, plus 20 B per edge) over its average
         launch time, from CUDA events recorded around each launch on its own stream
  cpu_baseline  the CPU oracle on a strided anchor sample of the same graph

--impl reference times the CPU oracle (the only reference implementation of this
method) on the host cores instead. Multi-GPU runs (torchrun) count one replica of the
workload per GPU, with no data-path collective (weak scaling).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "wedges/sec & % HBM roofline; batched graphs/sec vs per-graph launches"
UNIT = "wedges/s"
WORKLOAD = "powerlaw_1m_200k_20m"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_DIR = os.path.join(ROOT, "profiles")
FALLBACK_HBM_GBS = 6800.0


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_barrier(dist) -> None:
    """All ranks meet here (no-op for a single process)."""
    if dist is not None:
        dist.barrier()


def max_over_ranks(ms: float, dist, device) -> float:
    """The largest of the ranks' elapsed times for the same K steps: the job is done when
    the slowest replica is. `device` holds the reduction tensor (cuda for NCCL, cpu for
    gloo)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank_step: float, steps: int, ms: float) -> float:
    """Units processed by all ranks per second of the slowest rank's time (weak scaling:
    every rank counts its own replica of the workload)."""
    return world * units_per_rank_step * steps / (ms / 1e3)


def hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


_CODE_TOKENS = re.compile(r'"(?:\\.|[^"\\\n])*"|\'(?:\\.|[^\'\\\n])*\'|//[^\n]*|/\*.*?\*/|\s+', re.S)


def code_only(text: str) -> str:
    """The source with comments removed and whitespace runs collapsed, so that the digest
    below changes with the code and not with its comments (string literals are kept)."""
    def keep(m):
        t = m.group(0)
        if t.startswith("//") or t.startswith("/*"):
            return " "
        return " " if t.isspace() else t
    return " ".join(_CODE_TOKENS.sub(keep, text).split())


def kernel_source_digest() -> str:
    h = hashlib.sha256()
    for name in ("count.cu", "prep.cu", "bbc_internal.cuh", "graph.cuh"):
        with open(os.path.join(ROOT, "paper_2601_17707_gb300", "csrc", name), encoding="utf-8") as f:
            h.update(code_only(f.read()).encode())
    return h.hexdigest()


def recorded_traffic(workload: str = WORKLOAD):
    """Per-step DRAM bytes of the tile path (the k_tile launch, plus the k_tile_cs launch
    of graphs with centre-split tiles) from the committed ncu summary of this workload
    (profiles/k_tile_<workload>.traffic.json), or None when there is none or the kernel
    source changed since that capture."""
    try:
        with open(os.path.join(TRAFFIC_DIR, f"k_tile_{workload}.traffic.json")) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("source_sha256") != kernel_source_digest():
        return None
    return rec.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in (self.out or "").splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


WORKLOADS = ("powerlaw_1m_200k_20m", "hubs_50k_2m_100m", "uniform_2k_3k")


def make_workload(name: str = WORKLOAD):
    """The bench graph: the 20M-edge power-law graph by default; the 100M-edge heavy-hub
    graph and the 20,000-edge uniform graph are the other single-graph configurations."""
    from paper_2601_17707_gb300 import synth

    if name == "hubs_50k_2m_100m":
        return synth.hubs_50k_2m(seed=0)
    if name == "uniform_2k_3k":
        return synth.uniform_2k_3k(seed=0)
    return synth.powerlaw_1m_200k(seed=0)


def oracle_sample(g, target_s: float):
    """Times the oracle on a strided anchor sample sized for about target_s seconds.
    Every oracle call first builds its adjacency arrays, a fixed cost that one light
    anchor measures; the stride is then sized on the counting time above that cost.
    Returns (wedges per second, wedges visited, seconds, threads, stride)."""
    import oracle

    threads = os.cpu_count() or 1

    def run(stride, offset=0):
        t0 = time.perf_counter()
        _, w = oracle.count_sample(g, stride=stride, offset=offset, threads=threads, per_vertex=True)
        return w, time.perf_counter() - t0

    _, t_fixed = run(g.n_u, offset=g.n_u - 1)
    stride = 8192
    w, dt = run(stride)
    while dt - t_fixed < 0.5 and stride > 1:
        stride = max(1, stride // 8)
        w, dt = run(stride)
    work_s = max(dt - t_fixed, 1e-3)
    stride = max(1, int(stride * work_s / max(target_s - t_fixed, 1.0)))
    w, dt = run(stride)
    return w / dt, w, dt, threads, stride


def bench_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    g = make_workload(args.workload)
    threads = os.cpu_count() or 1
    # size the per-step sample so that warmup + steps stay within a few minutes
    per_step = max(2.0, min(15.0, 150.0 / max(1, args.steps + args.warmup)))
    rate, w, dt, threads, stride = oracle_sample(g, per_step)
    for _ in range(args.warmup):
        oracle.count_sample(g, stride=stride, threads=threads, per_vertex=True)
    times, visited = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, w = oracle.count_sample(g, stride=stride, threads=threads, per_vertex=True)
        times.append(time.perf_counter() - t0)
        visited += w
    total = sum(times)
    value = visited / total
    sample = (f"CPU oracle (bbc_oracle.c, {threads} threads) over every {stride}-th anchor of U "
              f"with per-vertex counts; {visited // max(1, args.steps)} oriented wedges per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": {"workload": args.workload, "n_u": g.n_u, "n_v": g.n_v,
                                        "n_edges": g.n_edges, "seed": 0, "sample_stride": stride},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_motifs(g, u_d, v_d, s_d, W, balanced, unbalanced):
    """The motif counts on the bench graph (pair side as for the butterfly count): the six
    sign classes of Table 7 and balanced (2,3)-bicliques. Per kind: one untimed call (it
    builds the motif work lists), then 3 timed calls; the kernel's device time comes from
    the library's CUDA events. The classes must add up to the butterfly count's totals."""
    from paper_2601_17707_gb300 import bbc

    G = bbc.Graph.prepare(g.n_u, g.n_v, u_d, v_d, s_d)
    out = {}
    try:
        peak, _ = hbm_peak()
        alg_bytes = 4 * W + 20 * g.n_edges        # one wedge pass per call
        for name, kind, k in (("sign_classes", "classes", 2), ("biclique_2_3", "biclique", 3)):
            res = G.count_motif(kind, k=k)
            bbc.profile_start()
            t0 = time.perf_counter()
            for _ in range(3):
                res = G.count_motif(kind, k=k)
            wall_ms = (time.perf_counter() - t0) * 1e3 / 3
            prof = bbc.profile_stop()
            n, ms = prof.get("k_tile_motif", (0, 0.0))
            kern_ms = ms / max(1, n)
            out[name] = {"counts": list(res), "kernel_ms": kern_ms, "call_ms": wall_ms,
                         "wedges_per_s": W / (kern_ms / 1e3) if kern_ms else None,
                         "roofline_frac": (alg_bytes / (kern_ms / 1e3) / 1e9) / peak if kern_ms else None}
        cl = out["sign_classes"]["counts"]
        out["classes_consistent"] = (sum(cl[:4]) == balanced and cl[4] + cl[5] == unbalanced)
    finally:
        G.free()
    return out


def bench_dynamic_batch(g, n_updates, seed):
    """A batch of edge updates on the bench graph (a third each: sign flips and deletions
    of present edges, insertions of absent pairs): bbc_count_delta's time against
    re-preparing and recounting the updated graph, and the two results compared."""
    import torch

    from paper_2601_17707_gb300 import bbc

    rng = np.random.default_rng(seed)
    keys = g.u.astype(np.int64) * g.n_v + g.v.astype(np.int64)      # sorted, distinct
    k3 = n_updates // 3
    pick = rng.choice(keys.shape[0], size=2 * k3, replace=False)
    flip, dele = pick[:k3], pick[k3:]
    ins = []
    while len(ins) < n_updates - 2 * k3:
        cand = int(rng.integers(0, g.n_u)) * g.n_v + int(rng.integers(0, g.n_v))
        j = np.searchsorted(keys, cand)
        if (j >= keys.shape[0] or keys[j] != cand) and cand not in ins:
            ins.append(cand)
    ins = np.array(ins, dtype=np.int64)
    uk = np.concatenate([keys[flip], keys[dele], ins])
    u = (uk // g.n_v).astype(np.int32)
    v = (uk % g.n_v).astype(np.int32)
    s = np.concatenate([-g.sign[flip], np.zeros(k3, np.int8),
                        np.where(rng.random(ins.shape[0]) < 0.8, 1, -1)]).astype(np.int8)
    # the updated edge list
    keep = np.ones(keys.shape[0], dtype=bool)
    keep[dele] = False
    sign2 = g.sign.copy()
    sign2[flip] = -sign2[flip]
    u2 = np.concatenate([g.u[keep], (ins // g.n_v).astype(np.int32)])
    v2 = np.concatenate([g.v[keep], (ins % g.n_v).astype(np.int32)])
    s2 = np.concatenate([sign2[keep], s[2 * k3:]]).astype(np.int8)
    dev = torch.device("cuda")
    u_d, v_d, s_d = (torch.from_numpy(x).to(dev) for x in (u, v, s))
    G = bbc.Graph.prepare(g.n_u, g.n_v, torch.from_numpy(g.u).to(dev), torch.from_numpy(g.v).to(dev),
                          torch.from_numpy(g.sign).to(dev))
    try:
        b0, ub0 = G.count()[:2]
        G.count_delta(u_d, v_d, s_d)
        times = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d = G.count_delta(u_d, v_d, s_d)
            times.append((time.perf_counter() - t0) * 1e3)
    finally:
        G.free()
    u2d, v2d, s2d = (torch.from_numpy(x).to(dev) for x in (u2, v2, s2))
    recount = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = bbc.Graph.prepare(g.n_u, g.n_v, u2d, v2d, s2d)
        b1, ub1 = G2.count()[:2]
        recount.append((time.perf_counter() - t0) * 1e3)
        G2.free()
    return {"updates": int(n_updates), "delta_ms": float(np.median(times)),
            "prepare_and_count_ms": float(np.median(recount)),
            "delta": list(d), "exact": (b1 - b0, ub1 - ub0) == tuple(d),
            "timing": "host wall clock around each call (both synchronise), median"}


def bench_dynamic(g, sizes=(10, 100, 1000)):
    return [bench_dynamic_batch(g, n, seed=7 + i) for i, n in enumerate(sizes)]


def tile_path_time(prof):
    """(launches, total ms) of the tile path in a per-kernel profile: the k_tile launches,
    with the k_tile_cs launches (the centre passes of centre-split tiles, one after each
    per-vertex k_tile launch of such a graph) added to their time."""
    n, ms = prof.get("k_tile", (0, 0.0))
    return n, ms + prof.get("k_tile_cs", (0, 0.0))[1]


def per_kernel_roofline(work, prof, passes, peak):
    """{kernel: achieved GB/s and fraction of `peak`} from the work behind each path
    (wedges and pair-side edges of its anchors; 4 B per wedge visit, `passes` visits per
    wedge, 20 B per edge) and its CUDA-event time per launch (the tile path's time is
    k_tile's plus k_tile_cs's)."""
    out = {}
    for k, (items, wedges, edges) in work.items():
        n, ms = tile_path_time(prof) if k == "k_tile" else prof.get(k, (0, 0.0))
        if not n or not items:
            continue
        alg = 4 * passes * wedges + 20 * edges
        gbs = alg / (ms / n / 1e3) / 1e9
        out[k] = {"items": items, "wedges": wedges, "ms_per_launch": ms / n,
                  "algorithmic_bytes": alg, "achieved_gbs": gbs, "frac": gbs / peak}
    return out


def bench_batched(args, dev):
    """The batched workload: 4,096 Chung-Lu graphs counted by one replay of a captured CUDA
    graph (autotuned) against per-graph launches of the single-graph path. Every member's
    count is compared with the oracle-written golden."""
    import torch

    from paper_2601_17707_gb300 import bbc, synth

    t0 = time.perf_counter()
    specs = synth.batch_specs(4096, seed=0)
    gs = synth.batch_graphs(specs)
    gen_s = time.perf_counter() - t0
    G = [bbc.Graph.from_synthetic(g) for g in gs]
    W = sum(h.info().wedges for h in G)
    E = sum(g.n_edges for g in gs)
    t0 = time.perf_counter()
    tuned = bbc.autotune_batch(G)
    tune_s = time.perf_counter() - t0
    ref = bbc.count_batch(G)                 # builds and caches the plan for the tuned choice
    for _ in range(2):
        bbc.count_batch(G)
    torch.cuda.synchronize(dev)
    reps = max(3, args.steps)
    t0 = time.perf_counter()
    for _ in range(reps):
        got = bbc.count_batch(G)
    t_batch = (time.perf_counter() - t0) / reps
    consistent = got == ref
    gold = read_batch_golden()
    exact = (gold == got) if gold is not None else None
    # per-kernel device times of one batch (launched directly while profiling) and the
    # work behind each path, from the tuned lists the plan used
    bbc.profile_start()
    bbc.count_batch(G)
    prof = bbc.profile_stop()
    work = {}
    for h in G:
        for k, t in h.work().items():
            a = work.setdefault(k, [0, 0, 0])
            for i in range(3):
                a[i] += t[i]
    peak, _ = hbm_peak()
    kernels = per_kernel_roofline({k: tuple(v) for k, v in work.items()}, prof, 1, peak)
    # per-graph launches on one stream with one sync at the end: the plain kernel
    # (static one-block-per-anchor schedule) and, for context, the work-queue kernel
    totals = torch.empty(2 * len(G), dtype=torch.int64, device=dev)

    def per_graph(tuning):
        for i, h in enumerate(G):
            h.count_async(totals[2 * i:2 * i + 2], tuning=tuning)
        torch.cuda.synchronize(dev)
        best = 1e30
        for _ in range(2):
            t0 = time.perf_counter()
            for i, h in enumerate(G):
                h.count_async(totals[2 * i:2 * i + 2], tuning=tuning)
            torch.cuda.synchronize(dev)
            best = min(best, time.perf_counter() - t0)
        single = totals.view(-1, 2)[:, 0].cpu().numpy().view(np.uint64).tolist()
        return best, [int(x) for x in single] == ref

    plain = bbc.default_tuning()
    plain.plain = 1
    t_per, ok1 = per_graph(plain)
    t_per_q, ok2 = per_graph(None)
    consistent = consistent and ok1 and ok2
    for h in G:
        h.free()
    return {"workload": "batch_4096_chung_lu", "graphs": len(G), "edges": E, "wedges": W,
            "graphs_per_s": len(G) / t_batch, "wedges_per_s": W / t_batch,
            "ms_per_batch": 1e3 * t_batch,
            "per_graph_plain_graphs_per_s": len(G) / t_per, "per_graph_plain_ms": 1e3 * t_per,
            "speedup_vs_per_graph_plain": t_per / t_batch,
            "per_graph_queue_graphs_per_s": len(G) / t_per_q, "per_graph_queue_ms": 1e3 * t_per_q,
            "speedup_vs_per_graph_queue": t_per_q / t_batch,
            "counts_identical": bool(consistent), "exact": exact,
            "exact_against": "tests/golden/batch_4096_chung_lu.txt (CPU oracle), every member",
            "tuning": tuned.as_dict(), "autotune_s": tune_s, "kernels": kernels,
            "timing": f"host wall clock around bbc_count_batch (replay + D2H + sync), mean of "
                      f"{reps}; per-graph: bbc_count_async per graph on one stream, one sync "
                      "(plain = static one-block-per-anchor kernel; queue = work-queue kernel)",
            "generation_s": gen_s}, (gs, gold)


def bench_serving(args, pool):
    """Poisson arrivals at several offered rates; 99% of requests from the batch pool,
    1% large (|U| = 200,000, |V| = 100,000, 5M edges); 8 GB device budget. Every ticket is
    compared with the oracle-written golden of its graph; per rate the record also gives
    the device time of the counting ticks (busy fraction), the preparation time, the large
    requests' wedges and times, and the latency of the small requests alone."""
    from paper_2601_17707_gb300 import bbc, synth

    gs, gold = pool
    large = synth.large_serving_graph(seed=0)
    lg = read_golden("serve_large_200k_100k_5m")
    large_want = int(lg["balanced"]) if lg is not None else None
    # one large request alone: its reservation against the device memory it reached (the
    # library pool's high-water mark, preparation temporaries and tick buffers included)
    srv = bbc.Server(8 << 30)
    warm = srv.submit(gs[0])
    srv.wait(warm, timeout_s=60.0)
    used0, _ = bbc.memory_usage(reset_high=True)
    t = srv.submit(large)
    got_large = srv.wait(t, timeout_s=600.0)
    _, high = bbc.memory_usage()
    q = srv.request_info(t)
    srv.close()
    alone = {"wedges": q["wedges"], "reserved_gb": q["reserved_bytes"] / 1e9,
             "measured_peak_gb": (high - used0) / 1e9, "latency_ms": q["latency_us"] / 1e3,
             "prepare_ms": q["prepare_us"] / 1e3, "count_ms": q["count_us"] / 1e3,
             "ticks": q["ticks"], "tick_gpu_ms": q["tick_gpu_us"] / 1e3,
             "exact": got_large == large_want if large_want is not None else None}
    rng = np.random.default_rng(0)
    out = []
    for rate in args.serve_rates:
        n = int(min(args.serve_max_requests, max(200, rate * args.serve_seconds)))
        srv = bbc.Server(8 << 30)
        gaps = rng.exponential(1.0 / rate, size=n)
        picks = rng.integers(0, len(gs), size=n)
        is_large = rng.random(n) < 0.01
        tickets = []
        t_start = time.perf_counter()
        t_next = t_start
        for k in range(n):
            t_next += gaps[k]
            while time.perf_counter() < t_next:
                pass
            g = large if is_large[k] else gs[picks[k]]
            tickets.append(srv.submit(g))
        got = [srv.wait(t, timeout_s=600.0) for t in tickets]
        wall = time.perf_counter() - t_start
        st = srv.stats()
        c = srv.counters()
        infos = [srv.request_info(t) for t in tickets]
        srv.close()
        want = [large_want if is_large[k] else (gold[picks[k]] if gold is not None else None)
                for k in range(n)]
        exact = None if any(w is None for w in want) else got == want
        small_lat = sorted(q["latency_us"] for q, L in zip(infos, is_large) if not L)
        big = [q for q, L in zip(infos, is_large) if L]

        def pct(a, q):
            return a[min(len(a) - 1, int(q * (len(a) - 1) + 0.5))] / 1e3 if a else None

        out.append({
            "offered_graphs_per_s": rate, "requests": n, "large": int(is_large.sum()),
            "graphs_per_s": n / wall, "p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3,
            "mean_ms": st["mean_us"] / 1e3, "exact": exact,
            "small_p50_ms": pct(small_lat, 0.5), "small_p99_ms": pct(small_lat, 0.99),
            "ticks": c["ticks"], "tick_gpu_ms": c["tick_gpu_us"] / 1e3,
            "tick_wall_ms": c["tick_wall_us"] / 1e3, "prep_wall_ms": c["prep_wall_us"] / 1e3,
            "gpu_busy_frac": c["tick_gpu_us"] / (wall * 1e6),
            "tick_thread_busy_frac": c["tick_wall_us"] / (wall * 1e6),
            "mean_tick_ms": c["tick_wall_us"] / 1e3 / max(1, c["ticks"]),
            "peak_reserved_gb": c["peak_reserved_bytes"] / 1e9, "max_queued": c["max_queued"],
            "admitted_after_wait": c["admitted_after_wait"],
            "large_requests": [{"wedges": q["wedges"], "latency_ms": q["latency_us"] / 1e3,
                                "queued_ms": q["queued_us"] / 1e3, "prepare_ms": q["prepare_us"] / 1e3,
                                "count_ms": q["count_us"] / 1e3, "ticks": q["ticks"],
                                "tick_gpu_ms": q["tick_gpu_us"] / 1e3} for q in big[:3]],
        })
    return {"budget_gb": 8, "latency": "submit to completion, library clock",
            "exact_against": "tests/golden (CPU oracle): batch members and the 5M-edge request",
            "large_request_alone": alone, "rates": out}


GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")
GOLDEN_NAME = {"powerlaw_1m_200k_20m": "powerlaw_1m_200k_20m", "hubs_50k_2m_100m": "hubs_50k_2m_100m",
               "uniform_2k_3k": "uniform_2k_3k_20k"}


def read_golden(workload: str):
    """The oracle-written totals and per-vertex digests of a workload (tests/golden/), or
    None when there is no such file."""
    path = os.path.join(GOLDEN_DIR, f"full_{GOLDEN_NAME.get(workload, workload)}.txt")
    if not os.path.exists(path):
        return None
    out = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            out[k] = v
    return out


def read_batch_golden():
    """Per member of the 4,096-graph batch, its oracle-written balanced total (or None)."""
    path = os.path.join(GOLDEN_DIR, "batch_4096_chung_lu.txt")
    if not os.path.exists(path):
        return None
    rows = []
    with open(path) as f:
        for line in f:
            t = line.split()
            if t and t[0] == "g":
                rows.append(int(t[5]))
    return rows


def u64_digest(t) -> str:
    """SHA-256 of a per-vertex result (int64 CUDA tensor holding uint64 values) as
    little-endian uint64, the layout of the golden digests."""
    a = t.cpu().numpy().view(np.uint64)
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<u8").tobytes()).hexdigest()


def single_graph(args, workload, steps, warmup, dev, dist, world, with_e2e):
    """One single-graph configuration: `steps` timed steps of bbc_prepare + bbc_count with
    per-vertex counts on device-resident input (the production launch path: no per-kernel
    events, the side streams live), then a separate pass with per-kernel CUDA events for
    the roofline figures, a count-only pass, and optionally the same step through host
    buffers. The last timed step's totals and per-vertex digests are compared with the
    oracle-written golden."""
    import torch

    from paper_2601_17707_gb300 import bbc

    g = make_workload(workload)
    u_h = torch.from_numpy(g.u).pin_memory()
    v_h = torch.from_numpy(g.v).pin_memory()
    s_h = torch.from_numpy(g.sign).pin_memory()
    u_d, v_d, s_d = u_h.to(dev), v_h.to(dev), s_h.to(dev)
    per_u = torch.empty(g.n_u, dtype=torch.int64, device=dev)
    per_v = torch.empty(g.n_v, dtype=torch.int64, device=dev)
    per_u_h = torch.empty(g.n_u, dtype=torch.int64).pin_memory()
    per_v_h = torch.empty(g.n_v, dtype=torch.int64).pin_memory()
    totals = torch.empty(2, dtype=torch.int64, device=dev)
    totals_h = torch.empty(2, dtype=torch.int64).pin_memory()
    stream = torch.cuda.current_stream(dev)

    G0 = bbc.Graph.prepare(g.n_u, g.n_v, u_d, v_d, s_d)
    info = G0.info()
    work0 = G0.work()
    # count-only tile kernel: global totals, no per-vertex pass
    G0.count_async(totals)
    bbc.profile_start()
    for _ in range(3):
        G0.count_async(totals)
    prof_co = bbc.profile_stop()
    G0.free()
    W = info.wedges

    def step_device():
        G = bbc.Graph.prepare(g.n_u, g.n_v, u_d, v_d, s_d)
        G.count_async(totals, per_u, per_v)
        G.free()

    def step_host():
        # the public call with host buffers: H2D of the edge list inside bbc_prepare
        G = bbc.Graph.prepare(g.n_u, g.n_v, u_h.numpy(), v_h.numpy(), s_h.numpy())
        G.count_async(totals, per_u, per_v)
        per_u_h.copy_(per_u, non_blocking=True)
        per_v_h.copy_(per_v, non_blocking=True)
        totals_h.copy_(totals, non_blocking=True)
        torch.cuda.synchronize(dev)
        G.free()

    # inputs smaller than L2 (129 MB): write a 256 MB buffer before every timed step,
    # outside the events; larger inputs evict themselves
    input_bytes = g.n_edges * 9
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if input_bytes < (160 << 20) else None
    l2_note = (f"inputs larger than L2: {input_bytes / 1e6:.0f} MB edge list and the CSR per step"
               if flush is None else "L2 flushed (256 MB written) before every timed step, outside the events")

    def timed(fn, k):
        rank_barrier(dist)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if flush is None:
            e0.record(stream)
            for _ in range(k):
                fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
        else:
            ms = 0.0
            for _ in range(k):
                flush.fill_(1)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms += e0.elapsed_time(e1)
        rank_barrier(dist)
        return max_over_ranks(ms, dist, dev)

    for _ in range(warmup):
        step_device()
    torch.cuda.synchronize(dev)
    launches0 = bbc.launch_count()
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        ms = timed(step_device, steps)
    launches = bbc.launch_count() - launches0
    # what the timed steps computed, against the oracle-written golden
    b_last, ub_last = [int(x) for x in totals.cpu().numpy().view(np.uint64)]
    gold = read_golden(workload)
    check = {"balanced": b_last, "unbalanced": ub_last}
    if gold is not None:
        check["per_u_sha256_equal"] = u64_digest(per_u) == gold["per_u_sha256"]
        check["per_v_sha256_equal"] = u64_digest(per_v) == gold["per_v_sha256"]
        check["exact"] = (b_last == int(gold["balanced"]) and ub_last == int(gold["unbalanced"])
                          and check["per_u_sha256_equal"] and check["per_v_sha256_equal"])
        check["against"] = f"tests/golden/full_{GOLDEN_NAME.get(workload, workload)}.txt (CPU oracle)"
    else:
        check["exact"] = None

    # per-kernel device times: a separate pass with CUDA events around every counting
    # kernel (profiling serialises the side streams, so it is not the timed pass)
    prof_steps = max(1, min(steps, 5))
    bbc.profile_start()
    for _ in range(prof_steps):
        step_device()
    torch.cuda.synchronize(dev)
    prof = bbc.profile_stop()

    e2e = None
    if with_e2e:
        for _ in range(max(1, warmup // 2)):
            step_host()
        ms_e2e = timed(step_host, steps)
        e2e = {"value": whole_job_rate(world, W, steps, ms_e2e), "unit": UNIT,
               "h2d_bytes_per_step": g.n_edges * (4 + 4 + 1),
               "d2h_bytes_per_step": (g.n_u + g.n_v) * 8 + 16, "ms_per_step": ms_e2e / steps}

    peak, peak_kind = hbm_peak()
    roof = None
    tile_launches, tile_ms = prof.get("k_tile", (0, 0.0))
    # graphs with centre-split tiles finish their centre pass in a second launch per step
    # (k_tile_cs): the tile path is both
    cs_launches, cs_ms = prof.get("k_tile_cs", (0, 0.0))
    if tile_launches:
        alg_bytes = 4 * 2 * W + 20 * g.n_edges   # per launch (one launch per step)
        path_ms = tile_path_time(prof)[1] / tile_launches
        achieved = alg_bytes / (path_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": recorded_traffic(workload),
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s", "kernel": "k_tile + k_tile_cs" if cs_launches else "k_tile",
                "kernel_ms_per_launch": path_ms,
                "algorithmic_bytes_per_launch": alg_bytes}
        if cs_launches:
            roof["k_tile_ms_per_launch"] = tile_ms / tile_launches
            roof["k_tile_cs_ms_per_launch"] = cs_ms / cs_launches
    co = None
    n_co, ms_co = prof_co.get("k_tile", (0, 0.0))
    if n_co:
        alg_co = 4 * W + 20 * g.n_edges
        ach = alg_co / (ms_co / n_co / 1e3) / 1e9
        co = {"kernel_ms_per_launch": ms_co / n_co, "algorithmic_bytes_per_launch": alg_co,
              "achieved": ach, "frac": ach / peak}
    return {
        "g": g, "u_d": u_d, "v_d": v_d, "s_d": s_d, "W": W, "info": info, "ms": ms,
        "value": whole_job_rate(world, W, steps, ms), "ms_per_step": ms / steps, "steps": steps,
        "warmup": warmup, "launches": launches, "clocks": clk.summary(), "check": check,
        "roofline": roof, "count_only": co, "kernel_profile": prof,
        "kernels": per_kernel_roofline(work0, prof, 2, peak), "e2e": e2e, "l2": l2_note,
        "config": {"workload": workload, "n_u": g.n_u, "n_v": g.n_v, "n_edges": g.n_edges,
                   "wedges": W, "pair_side": "V" if info.side == 1 else "U", "seed": 0,
                   "per_vertex": True, "step": "bbc_prepare + bbc_count (global + per-vertex)",
                   "l2": l2_note},
    }


def bench_gpu(args):
    import torch

    from paper_2601_17707_gb300 import _build, bbc

    world, rank, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    _build.build()
    bbc.load()
    dev = torch.device("cuda", local)

    main = single_graph(args, args.workload, args.steps, args.warmup, dev, dist, world,
                        with_e2e=not args.no_e2e)
    g, W = main["g"], main["W"]

    # the other single-graph configurations, each with its own roofline and check
    others = {}
    if not args.no_other_configs and world == 1:
        for wl in WORKLOADS:
            if wl == args.workload:
                continue
            r = single_graph(args, wl, 5 if wl == "hubs_50k_2m_100m" else 20, 3, dev, None, 1,
                             with_e2e=False)
            others[wl] = {k: r[k] for k in ("value", "ms_per_step", "steps", "warmup", "check",
                                            "roofline", "count_only", "kernels", "clocks", "config")}
            others[wl]["unit"] = UNIT
            del r

    motifs = dynamic = None
    if not args.no_motifs:
        motifs = bench_motifs(g, main["u_d"], main["v_d"], main["s_d"], W,
                              main["check"]["balanced"], main["check"]["unbalanced"])
        dynamic = bench_dynamic(g)

    batched = serving = None
    if not args.no_batched:
        batched, pool = bench_batched(args, dev)
        if not args.no_serve:
            serving = bench_serving(args, pool)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, w, dt, threads, stride = oracle_sample(g, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"every {stride}-th anchor of U with per-vertex counts: {w} oriented "
                         f"wedges in {dt:.1f} s"}

    if rank == 0:
        config = dict(main["config"])
        config["parallelism"] = f"replicas x{world}"
        config["balanced"] = main["check"]["balanced"]
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": config,
            "exact": main["check"]["exact"], "check": main["check"],
            "timing": "value: CUDA events around the timed steps on the production launch path "
                      "(no per-kernel events); roofline: a separate pass with CUDA events around "
                      "every counting kernel",
            "roofline": main["roofline"], "count_only": main["count_only"], "cpu_baseline": cpu,
            "e2e": main["e2e"], "clocks": main["clocks"], "gpu_launches": main["launches"],
            "kernel_profile": main["kernel_profile"], "kernels": main["kernels"],
            "configs": others, "motifs": motifs, "dynamic": dynamic, "batched": batched,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=WORKLOADS, default=WORKLOAD,
                    help="the single-graph configuration (the batch and serving legs are fixed)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-batched", action="store_true", help="skip the 4,096-graph batch")
    ap.add_argument("--no-motifs", action="store_true",
                    help="skip the sign-class / (2,3) counts and the update-batch delta")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving sweep")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the other two single-graph configurations")
    ap.add_argument("--serve-rates", type=float, nargs="+",
                    default=[100, 300, 1000, 3000, 10000, 20000])
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-max-requests", type=int, default=3000)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_gpu(args)


if __name__ == "__main__":
    main()

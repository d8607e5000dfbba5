"""Benchmark of the NSSG hot path on GB300.

One step = one pass of the whole path over one synthetic workload: ingest, exact kNN
graph, candidate pools, SSG prune, reverse-neighbour merge, navigating-node connectivity
(the build, Alg. 3), then Search-on-Graph (Alg. 1) for every query and the brute-force
ground truth with recall@10 (Sec. 5.2).

Workload (default): 1,000,000 x 128 integer-valued vectors shaped like SIFT1M (synthetic,
seeded), K = 200, L = 100, R = 50, alpha = 60 degrees, 10 navigating nodes, 10,000
queries; L_search is the smallest value of a sweep whose recall@10 reaches 0.95.

Prints one JSON line.  `value` is build seconds per million points (lower is better);
search QPS at recall@10 >= 0.95 is reported beside it.  Under torchrun every rank builds
its own replica (no collective on the data path) and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "NSSG build s/1M pts & QPS@recall@10=0.95, mixed-prec vs plain FP32 path"
LS_SWEEP = [10, 12, 16, 20, 24, 32, 40, 48, 64, 80, 100, 128, 160, 200, 256, 320, 400, 512, 768,
            1024]
NOMINAL_SM = 152
FP32_LANES_PER_SM = 128


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained", d["bf16_tflops"]),
                "sm_max_mhz": d.get("sm_max_mhz", 2070.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0, "source": "fallback"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(values, ws):
    """Element-wise max over ranks of a list of floats (identity for one rank)."""
    if ws == 1:
        return list(values)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(values, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.cpu().tolist()


def aggregate(step_ms, points_per_rank, ws):
    """Whole-job build time per million points: the slowest rank's mean step time over the
    points all ranks built (replicas: every rank builds its own index)."""
    worst = reduce_max([float(np.mean(step_ms))], ws)[0]
    total_points = points_per_rank * ws
    return worst / 1000.0 / (total_points / 1e6), worst


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples (the JSON line carries their summary); SSG_BENCH_OUT picks the folder
        out = os.environ.get("SSG_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_gpu{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1].split()[0]))
                    mx.append(float(parts[2].split()[0]))
                except ValueError:
                    continue
                for nm, v in zip(names[1:], parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(busy)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# the files holding each kernel's device code and its launch (the column order decides the
# tensor-core kNN's traffic); host-only headers are left out
KNN_SOURCES = ("knn_tc.cu", "knn_order.cu", "knn_select.cuh", "common.cuh", "tc_common.cuh")
SEARCH_SOURCES = ("search.cu", "graph_dev.cuh", "common.cuh")


def kernel_source_hash(files=KNN_SOURCES):
    h = hashlib.sha256()
    for f in files:
        p = os.path.join(ROOT, "paper_1907_06146_gb300", "csrc", f)
        if os.path.exists(p):
            with open(p, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str, workload: str, files=KNN_SOURCES):
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(f"{kernel}:{workload}")
    if not e or e.get("source_hash") != kernel_source_hash(files):
        return None
    return e.get("dram_bytes_per_launch")


def make_workload(name: str, n: int | None, rank: int):
    from paper_1907_06146_gb300 import synth
    kw = {}
    if n is not None:
        kw["n"] = n
    if name == "sift_like":
        return synth.sift_like(seed=synth.SEED_SIFT + rank, **kw)
    if name == "small":
        return synth.small(seed=synth.SEED_SMALL + rank, **kw)
    if name == "gist_like":
        return synth.gist_like(seed=synth.SEED_GIST + rank, **kw)
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on a bounded sample of the same workload.
# ---------------------------------------------------------------------------------------
def oracle_sample_seconds_per_million(w, n_nodes: int, seed: int):
    """Times the oracle's kNN rows (for each sampled node and for the neighbours whose rows
    its pool reads), pools and prunes of n_nodes seeded random nodes, and extrapolates to
    seconds per million points.  The reverse merge and connectivity are not in the sample."""
    import oracle
    rng = np.random.default_rng(seed)
    nodes = np.sort(rng.choice(w.n, size=n_nodes, replace=False)).astype(np.int64)
    t0 = time.perf_counter()
    ids, _ = oracle.knn_rows(w.base, w.K, rows=nodes)
    t1 = time.perf_counter()
    # rows the pool walk reads: the node's own row and those of its neighbours up to the
    # point where the pool reaches L (with K >= L only the first neighbour's row)
    need = []
    for r in range(n_nodes):
        cnt = 0
        for t in range(w.K):
            need.append(int(ids[r, t]))
            cnt += 1 + w.K
            if cnt >= w.L:
                break
    need = np.unique(np.asarray(need, np.int64))
    need = need[~np.isin(need, nodes)]
    t2 = time.perf_counter()
    nb_ids, _ = oracle.knn_rows(w.base, w.K, rows=need)
    t3 = time.perf_counter()
    knn = np.zeros((w.n, w.K), np.int32)
    knn[nodes] = ids
    knn[need] = nb_ids
    t4 = time.perf_counter()
    pid, _, pl = oracle.pool(w.base, knn, w.L, rows=nodes)
    oracle.prune(w.base, pid, pl, w.R, w.alpha, nodes=nodes)
    t5 = time.perf_counter()
    knn_rows = n_nodes + need.size
    per_row = ((t1 - t0) + (t3 - t2)) / knn_rows
    per_node = (t5 - t4) / n_nodes
    return (per_row + per_node) * 1e6, {"knn_rows": int(knn_rows), "nodes": n_nodes,
                                        "sec": (t1 - t0) + (t3 - t2) + (t5 - t4)}


def oracle_edge_seconds_per_million(w, n_sub: int = 10_000, seed: int = 77):
    """The oracle's reverse merge and connectivity per point: the oracle builds the graph of
    the first n_sub points (exact kNN, pools, prune, untimed), then its reverse merge and
    connectivity from w.n_nav navigating nodes are timed and scaled to 1M points (both
    stages are linear in the number of points)."""
    import oracle
    from paper_1907_06146_gb300 import synth
    sub = np.ascontiguousarray(w.base[:n_sub])
    ids, _ = oracle.knn_rows(sub, w.K)
    pid, _, pl = oracle.pool(sub, ids, w.L)
    adj0, deg0 = oracle.prune(sub, pid, pl, w.R, w.alpha)
    nav = synth.nav_ids(n_sub, w.n_nav, seed)
    t0 = time.perf_counter()
    adj1, deg1 = oracle.reverse(sub, adj0, deg0, w.alpha)
    t1 = time.perf_counter()
    oracle.connect(sub, adj1, deg1, nav)
    t2 = time.perf_counter()
    return (t2 - t0) / n_sub * 1e6, {"reverse_s": t1 - t0, "connect_s": t2 - t1, "points": n_sub}


def cpu_baseline_line(w, nodes: int, nodes_1core: int, seed: int):
    """The oracle on the host cores: kNN rows, pools and prunes of a seeded node sample plus
    the reverse merge and connectivity of a 10,000-point build, on all cores and on one."""
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    v, info = oracle_sample_seconds_per_million(w, nodes, seed)
    e, einfo = oracle_edge_seconds_per_million(w)
    oracle.set_threads(1)
    try:
        v1, info1 = oracle_sample_seconds_per_million(w, nodes_1core, seed + 1)
        e1, _ = oracle_edge_seconds_per_million(w)
    finally:
        oracle.set_threads(cores)
    return {"value": v + e, "unit": "s/1M pts", "cores": cores, "kind": "oracle",
            "value_1core": v1 + e1,
            "parts_s_per_1M": {"knn_pool_prune": v, "reverse_connect": e,
                               "knn_pool_prune_1core": v1, "reverse_connect_1core": e1},
            "sample": f"{nodes} seeded random nodes ({nodes_1core} on one core): their exact kNN "
                      f"rows and those of the neighbours their pools read ({info['knn_rows']} "
                      f"rows of {w.n}x{w.d}), pools and prunes, per node; plus the reverse merge "
                      f"and connectivity of the oracle's own graph of the first "
                      f"{einfo['points']} points, per point; both scaled to 1M points"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = make_workload(args.workload, args.n, 0)
    cores = oracle.max_threads()
    # the reverse merge and connectivity per point, from the oracle's own 10,000-point build
    edge, einfo = oracle_edge_seconds_per_million(w)
    per_step = []
    for s in range(args.warmup + args.steps):
        v, info = oracle_sample_seconds_per_million(w, args.ref_nodes, 1000 + s)
        if s >= args.warmup:
            per_step.append(v + edge)
    value = float(np.mean(per_step))
    sample = (f"per step: oracle kNN rows + pools + prunes of {args.ref_nodes} seeded random "
              f"nodes of the {w.n}x{w.d} workload, per node; plus (measured once) the reverse "
              f"merge and connectivity of the oracle's own graph of the first {einfo['points']} "
              f"points, per point; scaled to 1M points")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/1M pts",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{w.name} n={w.n} d={w.d} K={w.K} L={w.L} R={w.R} "
                                   f"alpha={w.alpha} nav={w.n_nav} queries={w.queries.shape[0]}"},
            "cpu_baseline": {"value": value, "unit": "s/1M pts", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "s/1M pts", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(ssg, g, base, w, seconds: float, rate: float, seed: int = 190706145,
                recall: bool = True):
    """Open-loop Poisson stream of requests against a continuous-batching server: batch
    sizes log-uniform in [1, 4096], k in {1, 10, 100}, L_search uniform in [k, 512]; each
    request's queries are a contiguous block of the query set (a view, so submitting costs
    no gather).  Returns latency percentiles, throughput and recall@10 of the requests with
    k >= 10."""
    import threading
    import time as _t

    rng = np.random.default_rng(seed)
    srv = ssg.Server(g, base, n_streams=4, max_batch=8192, mem_budget_bytes=256 << 20)
    nq_all = w.queries.shape[0]
    reqs = []
    t = 0.0
    while t < seconds:
        t += rng.exponential(1.0 / rate)
        nq = min(int(np.exp(rng.uniform(0.0, np.log(4096.0)))), nq_all)
        k = int(rng.choice([1, 10, 100]))
        ls = int(rng.integers(k, 513))
        s0 = int(rng.integers(0, nq_all - nq + 1))
        reqs.append((t, np.arange(s0, s0 + nq), k, ls))
    tickets = [None] * len(reqs)
    results = [None] * len(reqs)
    done = threading.Event()

    def waiter():
        for i in range(len(reqs)):
            while tickets[i] is None:
                _t.sleep(0.0002)
            results[i] = srv.wait(tickets[i])
        done.set()

    th = threading.Thread(target=waiter)
    th.start()
    t0 = _t.perf_counter()
    for i, (ta, rows, k, ls) in enumerate(reqs):
        now = _t.perf_counter() - t0
        if ta > now:
            _t.sleep(ta - now)
        tickets[i] = srv.submit(w.queries[rows[0]:rows[-1] + 1], k, ls)
    submit_s = _t.perf_counter() - t0
    done.wait()
    wall = _t.perf_counter() - t0
    th.join()
    st = srv.stats()
    srv.close()
    lat = np.array([r[2] for r in results])
    total_q = int(sum(len(r[1]) for r in reqs))
    rec = None
    if recall:
        # recall@10 of the k >= 10 requests, first 10 ids against brute force
        import torch
        sel = [i for i, r in enumerate(reqs) if r[2] >= 10]
        rows = np.concatenate([reqs[i][1] for i in sel])
        found = np.concatenate([results[i][0][:, :10] for i in sel])
        truth, _ = ssg.knn_query(base, torch.from_numpy(w.queries[rows]).cuda(), 10)
        hits = ssg.recall_hits(torch.from_numpy(np.ascontiguousarray(found)).cuda(), truth, 10)
        rec = hits / (10.0 * len(rows))
    return {"requests": len(reqs), "queries": total_q, "offered_rate_req_s": rate,
            "achieved_submit_rate_req_s": len(reqs) / submit_s,
            "seconds": wall, "qps": total_q / wall, "latency_ms_p50": float(np.percentile(lat, 50)),
            "latency_ms_p99": float(np.percentile(lat, 99)),
            "recall@10_k>=10": rec, "batches": st["batches"],
            "max_batches_in_flight": st["max_batches_in_flight"],
            "max_queries_in_flight": st["max_queries_in_flight"],
            "mix": "Poisson arrivals; batch 1..4096 log-uniform; k in {1,10,100}; "
                   "L_search uniform in [k, 512]"}


def run_serving_curve(ssg, g, base, w, seconds: float, rates):
    """The serving run at each offered rate (requests per second): achieved QPS, p50 and p99
    latency; the saturation point is the largest achieved QPS.  Recall is scored at the
    first rate (a query's result does not depend on the load)."""
    pts = []
    for i, r in enumerate(rates):
        p = run_serving(ssg, g, base, w, seconds, r, seed=190706145 + i, recall=(i == 0))
        pts.append({k: p[k] for k in ("offered_rate_req_s", "achieved_submit_rate_req_s", "qps",
                                      "latency_ms_p50", "latency_ms_p99", "requests", "queries",
                                      "max_batches_in_flight", "recall@10_k>=10")})
    best = max(pts, key=lambda p: p["qps"])
    return {"points": pts, "saturation_qps": best["qps"],
            "saturation_at_offered_req_s": best["offered_rate_req_s"],
            "seconds_per_point": seconds,
            "mix": "Poisson arrivals; batch 1..4096 log-uniform; k in {1,10,100}; "
                   "L_search uniform in [k, 512]; 4 batch slots"}


def run_float_arm(ssg, n, d, K, L, R, ls=64, seed=190706144, w=None, label=None):
    """One float index built through the certified bf16 path and through the plain fp32
    path (fp32 kNN GEMM, fp32 warp prune): build times, whether the edge sets are identical,
    and recall@10 at one L_search on the workload's queries.  Default data: a 16-centre
    Gaussian mixture shaped like the many-index batch (the recipe of synth.batched_index)."""
    import torch
    from paper_1907_06146_gb300 import synth
    if w is None:
        w = synth.small(n=n, d=d, nq=1000, seed=seed)
    n, d = w.base.shape
    base = torch.from_numpy(w.base).cuda()
    q = torch.from_numpy(w.queries).cuda()
    nq = w.queries.shape[0]
    nav = synth.nav_ids(n, 10, seed)
    truth, _ = ssg.knn_query(base, q, 10)
    out = {"workload": (label or "16-centre Gaussian mixture") +
                       f" n={n} d={d} (float32) K={K} L={L} R={R} alpha=60 nav=10"}
    graphs = {}
    for arm, kw in (("bf16", {"prec": "auto"}), ("fp32", {"prec": "fp32", "gram_prec": "fp32"})):
        g = ssg.build(base, K, L, R, 60.0, nav=nav, **kw)  # warm-up
        del g
        g = ssg.build(base, K, L, R, 60.0, nav=nav, **kw)
        ids, _ = g.search(base, q, 10, ls)
        st = g.stats
        out[arm] = {"build_s_per_1M": st["ms_total"] / 1e3 * 1e6 / n, "ms_total": st["ms_total"],
                    "ms_knn": st["ms_knn"], "ms_knn_gemm": st["ms_knn_gemm"],
                    "ms_knn_certify": st["ms_knn_certify"],
                    "gemm_prec_used": st["gemm_prec_used"],
                    "knn_candidates": st["knn_candidates"],
                    "knn_rows_not_certified_by_first_pass": st["n_knn_fallback_rows"],
                    "knn_bf16_pairs": st["knn_bf16_pairs"],
                    "stages_ms": {k: st[k] for k in ("ms_pool", "ms_prune", "ms_reverse",
                                                     "ms_connect")},
                    "recall@10": ssg.recall_hits(ids, truth, 10) / (10.0 * nq), "L_search": ls}
        graphs[arm] = g
    out["edge_sets_identical"] = bool(torch.equal(graphs["bf16"].adj, graphs["fp32"].adj)
                                      and torch.equal(graphs["bf16"].deg, graphs["fp32"].deg))
    out["bf16_over_fp32_speedup"] = out["fp32"]["ms_total"] / out["bf16"]["ms_total"]
    return out


def run_serve_deep(ssg, n, tiles, seconds, rate, target):
    """The 96-d L2-normalised workload at n points: built with Alg. 4's search-based pools
    over `tiles` tiles (no O(n^2) kNN graph), its recall@10 sweep, and the serving run on
    it.  Returns build time, stage times, the sweep and the serving figures."""
    import torch
    from paper_1907_06146_gb300 import synth
    t0 = time.perf_counter()
    w = synth.deep_like(n=n, nq=10_000)
    gen_s = time.perf_counter() - t0
    base = torch.from_numpy(w.base).cuda()
    queries = torch.from_numpy(w.queries).cuda()
    nq = w.queries.shape[0]
    truth, _ = ssg.knn_query(base, queries, 10)
    g = ssg.build(base, w.K, w.L, w.R, w.alpha, n_nav=w.n_nav, pool_tiles=tiles)
    del g
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = ssg.build(base, w.K, w.L, w.R, w.alpha, n_nav=w.n_nav, pool_tiles=tiles)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    sweep, at = [], None
    for ls in LS_SWEEP:
        ids, _ = g.search(base, queries, 10, ls)
        r = ssg.recall_hits(ids, truth, 10) / (nq * 10.0)
        sweep.append((ls, r))
        if r >= target:
            ts = []
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                g.search(base, queries, 10, ls)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            at = {"L_search": ls, "recall@10": r, "qps": nq / (min(ts) / 1e3)}
            break
    serving = run_serving(ssg, g, base, w, seconds, rate) if seconds > 0 else None
    out = {"workload": f"deep_like n={n} d=96 (2,000-Gaussian mixture, L2-normalised)",
           "K": w.K, "L": w.L, "R": w.R, "alpha": w.alpha, "pool_tiles": tiles,
           "host_generation_s": gen_s, "build_s": build_s,
           "stages_ms": {k: g.stats[k] for k in ("ms_knn", "ms_knn_gemm", "ms_pool", "ms_prune",
                                                  "ms_reverse", "ms_connect", "ms_total")},
           "n_repair": g.stats["n_repair"], "avg_out_degree": float(g.deg.float().mean().item()),
           "sweep": sweep, "at_target": at, "serving": serving}
    del g
    return out


def run_batched(ssg, count, n_streams):
    """Independent indices (float Gaussian mixtures, shapes from synth.batched_specs) built
    by ssg_build_batched and one by one; wall-clock seconds with the device synchronised."""
    import torch
    from paper_1907_06146_gb300 import synth
    specs = synth.batched_specs(count)
    data = [torch.from_numpy(synth.batched_index(sp).base).cuda() for sp in specs]
    Ks = [sp["K"] for sp in specs]
    Ls = [sp["L"] for sp in specs]
    points = sum(sp["n"] for sp in specs)
    warm = ssg.build_batched(data[-2:], Ks[-2:], Ls[-2:], 32, 60.0, n_streams=2)
    del warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gs = ssg.build_batched(data, Ks, Ls, 32, 60.0, n_streams=n_streams)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    degs = [int(g.deg.sum().item()) for g in gs]
    # the plain fp32 batch (fp32 kNN GEMM and prune); how many adjacency rows equal the
    # mixed-precision batch's (certified: all of them)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gm = ssg.build_batched(data, Ks, Ls, 32, 60.0, n_streams=n_streams, prec="fp32")
    torch.cuda.synchronize()
    t_fp32 = time.perf_counter() - t0
    rows_same = 0
    for ge, gx in zip(gs, gm):
        rows_same += int(((ge.adj == gx.adj).all(dim=1) & (ge.deg == gx.deg)).sum().item())
    del gs, gm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    same = True
    for b, K, L, dg in zip(data, Ks, Ls, degs):
        g = ssg.build(b, K, L, 32, 60.0)
        same = same and int(g.deg.sum().item()) == dg
        del g
    torch.cuda.synchronize()
    t_one = time.perf_counter() - t0
    return {"indices": count, "points": points, "streams": n_streams,
            "batched_s": t_batch, "one_by_one_s": t_one, "speedup": t_one / t_batch,
            "batched_s_per_1M_pts": t_batch * 1e6 / points,
            "degree_sums_equal": same,
            "fp32_batched_s": t_fp32,
            "mixed_over_fp32_batched_speedup": t_fp32 / t_batch,
            "rows_equal_fp32_frac": rows_same / points,
            "shapes": "n log-uniform 10k-500k, d in {64,96,128,256}, L in {100,200}, K=100, "
                      "R=32, alpha=60; 16-centre float mixtures"}


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
def run_gpu(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1907_06146_gb300 import ssg, synth
    ssg.lib()

    w = make_workload(args.workload, args.n, rank)
    nav = synth.nav_ids(w.n, w.n_nav, synth.SEED_DEEP + rank)
    base = torch.from_numpy(w.base).cuda()
    queries = torch.from_numpy(w.queries).cuda()
    nq = w.queries.shape[0]
    stream = torch.cuda.current_stream()

    def step(ls):
        g = ssg.build(base, w.K, w.L, w.R, w.alpha, nav=nav, prec=args.prec,
                      tune_table=args.tune_table)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ids, _ = g.search(base, queries, 10, ls)
        e1.record(stream)
        truth, _ = ssg.knn_query(base, queries, 10)
        e2.record(stream)
        hits = ssg.recall_hits(ids, truth, 10)
        torch.cuda.synchronize()
        return g, ids, e0.elapsed_time(e1), e1.elapsed_time(e2), hits / (nq * 10.0)

    # calibration: smallest L_search of the sweep with recall@10 >= 0.95
    g = ssg.build(base, w.K, w.L, w.R, w.alpha, nav=nav, prec=args.prec)
    truth, _ = ssg.knn_query(base, queries, 10)
    ls_used, rec_used = LS_SWEEP[-1], None
    sweep = []
    for ls in LS_SWEEP:
        ids, _ = g.search(base, queries, 10, ls)
        r = ssg.recall_hits(ids, truth, 10) / (nq * 10.0)
        sweep.append((ls, r))
        if r >= args.target_recall:
            ls_used, rec_used = ls, r
            break
    # the search's work at that L_search (untimed): algorithmic bytes per query
    _, _, work = ssg.search_work(base, g.adj, g.deg, g.nav, queries, 10, ls_used)
    row_b = g.stats["search_row_bytes"]  # 1: the graph searches a byte copy of the rows
    search_bytes = (work["adjacency_entries"] * 4 + work["expansions"] * 4
                    + work["distances"] * w.d * row_b + nq * w.d * 4)
    del g

    for _ in range(args.warmup):
        step(ls_used)

    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ssg.launch_count()
    build_ms, search_ms, gt_ms, recalls, stats = [], [], [], [], []
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        g, ids, s_ms, gt, rec = step(ls_used)
        build_ms.append(g.stats["ms_total"])
        stats.append(g.stats)
        search_ms.append(s_ms)
        gt_ms.append(gt)
        recalls.append(rec)
        del g
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t_wall0
    launches = ssg.launch_count() - launches0
    clk = clocks.stop()

    value, worst_build_ms = aggregate(build_ms, w.n, ws)
    worst_search_ms = reduce_max([float(np.mean(search_ms))], ws)[0]
    qps = nq * ws / (worst_search_ms / 1000.0)

    # end to end through the host-buffer entry point: H2D of the base and D2H of the graph
    # inside the timed region
    pinned = torch.from_numpy(w.base).pin_memory()
    host_base = pinned.numpy()
    adj_pin = torch.empty((w.n, w.R), dtype=torch.int32).pin_memory().numpy()
    deg_pin = torch.empty((w.n,), dtype=torch.int32).pin_memory().numpy()
    e2e_ms = []
    for s in range(1 + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g, adj_h, deg_h = ssg.build_host(host_base, w.K, w.L, w.R, w.alpha, nav=nav, prec=args.prec,
                                         adj_out=adj_pin, deg_out=deg_pin)
        t1 = time.perf_counter()
        del g
        if s > 0:
            e2e_ms.append((t1 - t0) * 1000.0)
    e2e_value, _ = aggregate(e2e_ms, w.n, ws)

    serving = None
    if rank == 0 and args.serve_seconds > 0:
        g_srv = ssg.build(base, w.K, w.L, w.R, w.alpha, nav=nav, prec=args.prec)
        rates = [float(r) for r in args.serve_rates.split(",")]
        serving = run_serving_curve(ssg, g_srv, base, w, args.serve_seconds, rates)
        del g_srv

    float_arm = None
    if rank == 0 and args.float_n > 0:
        float_arm = run_float_arm(ssg, args.float_n, args.float_d, 100, 200, 32)

    wide_arm = None
    if rank == 0 and args.wide_n > 0 and w.name != "gist_like":
        # the 960-d GIST-shaped data (SURVEY config 3's shape) at a size both paths finish
        gw = synth.gist_like(n=args.wide_n, nq=1000)
        wide_arm = run_float_arm(ssg, 0, 0, gw.K, gw.L, gw.R, ls=64, w=gw,
                                 label="GIST-shaped softplus mixture, values in [0, 1],")

    # the optional arms run by default on the SIFT-shaped headline workload
    headline = w.name == "sift_like"
    if args.alg4_tiles is None:
        args.alg4_tiles = 128 if headline else 0
    if args.batched is None:
        args.batched = 16 if headline else 0
    if args.ablations is None:
        args.ablations = headline
    alg4 = None
    if rank == 0 and args.alg4_tiles > 0:
        # Alg. 4: pools searched on the fly over the cluster-ordered tiles, no kNN graph
        g4 = ssg.build(base, w.K, w.L, w.R, w.alpha, nav=nav, prec=args.prec,
                       pool_tiles=args.alg4_tiles)
        g4 = ssg.build(base, w.K, w.L, w.R, w.alpha, nav=nav, prec=args.prec,
                       pool_tiles=args.alg4_tiles)
        sweep4 = []
        for ls in LS_SWEEP:
            ids4, _ = g4.search(base, queries, 10, ls)
            r4 = ssg.recall_hits(ids4, truth, 10) / (nq * 10.0)
            sweep4.append((ls, r4))
            if r4 >= args.target_recall:
                break
        alg4 = {"pool_tiles": args.alg4_tiles, "build_s_per_1M": g4.stats["ms_total"] / 1e3 * 1e6 / w.n,
                "stages_ms": {k: g4.stats[k] for k in ("ms_knn", "ms_pool", "ms_prune", "ms_reverse",
                                                       "ms_connect", "ms_total")},
                "sweep": sweep4, "n_repair": g4.stats["n_repair"],
                "knn_graph_bytes_not_stored": int(w.n * w.K * 8)}
        del g4

    ablations = None
    if rank == 0 and args.ablations:
        from paper_1907_06146_gb300 import ablations as abl
        ablations = abl.run_all(ssg, synth, w)

    serving_deep = None
    if rank == 0 and args.serve_deep > 0:
        serving_deep = run_serve_deep(ssg, args.serve_deep, args.serve_deep_tiles,
                                      args.serve_seconds, args.serve_rate, args.target_recall)

    batched = None
    if rank == 0 and args.batched > 0:
        batched = run_batched(ssg, args.batched, args.batched_streams)

    # the plain FP32 path on the same input, once (untimed in value): its build time, the
    # recall of its graph at the same L_search, and whether its edge set equals this one's
    fp32_arm = None
    if rank == 0 and args.fp32_arm and args.prec != "fp32":
        g_mp = ssg.build(base, w.K, w.L, w.R, w.alpha, nav=nav, prec=args.prec)
        g32 = ssg.build(base, w.K, w.L, w.R, w.alpha, nav=nav, prec="fp32")
        ids32, _ = g32.search(base, queries, 10, ls_used)
        rec32 = ssg.recall_hits(ids32, truth, 10) / (nq * 10.0)
        same = bool(torch.equal(g32.deg, g_mp.deg) and torch.equal(g32.adj, g_mp.adj))
        fp32_arm = {"build_s_per_1M": g32.stats["ms_total"] / 1000.0 * 1e6 / w.n,
                    "ms_knn": g32.stats["ms_knn"], "recall@10": rec32, "L_search": ls_used,
                    "edge_sets_identical": same,
                    "mixed_over_fp32_speedup": g32.stats["ms_total"] / float(np.mean(build_ms))}
        del g32, g_mp, ids32

    # roofline of the dominant kernel: the distance GEMM + top-K selection
    peaks = load_peaks()
    gemm_ms = float(np.mean([s["ms_knn_gemm"] for s in stats]))
    flops = 2.0 * w.n * (w.n - 1) * w.d
    used_prec = stats[0]["gemm_prec_used"]
    if used_prec == 1:
        kname = "knn_select_bf16_tc"
        peak = peaks["bf16_tflops_sustained"]
        bound, peak_note = "tensor", f"bf16 dense, {peaks['source']} sustained"
    else:
        kname = "knn_select_fp32"
        peak = NOMINAL_SM * FP32_LANES_PER_SM * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
        bound, peak_note = "alu", "fp32 FMA: 152 SMs x 128 lanes x 2 flop x max SM clock"
    achieved = flops / (gemm_ms / 1000.0) / 1e12
    traffic = committed_traffic(kname, w.name)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_line(w, args.cpu_nodes, args.cpu_nodes_1core, 4242)

    if rank != 0:
        return
    st0 = stats[-1]
    line = {
        "metric": METRIC, "value": value, "unit": "s/1M pts", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": wall * 1000.0 / args.steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if used_prec == 1 else "f32", "data": "synthetic",
        "config": {"workload": f"{w.name} n={w.n} d={w.d} K={w.K} L={w.L} R={w.R} "
                               f"alpha={w.alpha} nav={w.n_nav} queries={nq}",
                   "l2": f"inputs larger than L2 (base {w.base.nbytes // 2**20} MiB)",
                   "gemm_prec": args.prec,
                   "tune_table": args.tune_table,
                   "parallelism": f"replicas x{ws}"},
        "search": {"qps": qps, "recall@10": float(np.mean(recalls)), "L_search": ls_used,
                   "k": 10, "ms": float(np.mean(search_ms)), "sweep": sweep,
                   "work_per_query": {k2: v / nq for k2, v in work.items()},
                   "roofline": {"bound": "hbm", "achieved": search_bytes / (np.mean(search_ms) / 1e3) / 1e9,
                                "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                "frac": search_bytes / (np.mean(search_ms) / 1e3) / 1e9 / peaks["hbm_gbs"],
                                "traffic": committed_traffic("k_search", w.name, SEARCH_SOURCES),
                                "kernel": "k_search",
                                "algorithmic": "per query: 4 B per adjacency entry read and per "
                                               f"expansion (degree), d x {row_b} B per distance "
                                               "(the rows the search reads), d x 4 B query"}},
        "stages_ms": {k: float(np.mean([s[k] for s in stats])) for k in
                      ("ms_ingest", "ms_knn", "ms_knn_gemm", "ms_pool", "ms_prune", "ms_reverse",
                       "ms_connect", "ms_total")},
        "ground_truth_ms": float(np.mean(gt_ms)),
        "serving": serving,
        "serving_deep": serving_deep,
        "fp32_path": fp32_arm,
        "float_mixed": float_arm,
        "wide_mixed": wide_arm,
        "batched": batched,
        "ablations": ablations,
        "alg4": alg4,
        "counters": {k: st0[k] for k in ("n_repair", "n_angle_fp64", "n_order_fp64",
                                         "n_knn_fallback_rows", "max_indegree", "exact_mode",
                                         "knn_candidates", "knn_bf16_pairs")},
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": kname,
                     "peak_source": peak_note, "algorithmic": "2 n (n-1) d flop per launch"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "s/1M pts", "h2d_bytes_per_step": int(w.base.nbytes),
                "d2h_bytes_per_step": int(w.n * w.R * 4 + w.n * 4)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "worst_rank_build_ms": worst_build_ms,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sift_like", choices=["sift_like", "small", "gist_like"])
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--prec", default="auto", choices=["auto", "fp32", "bf16"])
    ap.add_argument("--target-recall", type=float, default=0.95)
    ap.add_argument("--tune-table", default=None,
                    help="launch-parameter file passed to every timed build (ssg_build_opts."
                         "tune_table)")
    ap.add_argument("--ref-nodes", type=int, default=128,
                    help="nodes the reference arm (the oracle) samples per step")
    ap.add_argument("--cpu-nodes", type=int, default=2000,
                    help="nodes the cpu_baseline samples on all host cores")
    ap.add_argument("--cpu-nodes-1core", type=int, default=48,
                    help="nodes the cpu_baseline samples on one host core")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched", type=int, default=None,
                    help="also build this many independent indices (log-uniform 10k-500k points, "
                         "d in {64,96,128,256}), batched and one by one (default: 16 on the "
                         "SIFT-shaped workload, else 0)")
    ap.add_argument("--batched-streams", type=int, default=8)
    ap.add_argument("--alg4-tiles", type=int, default=None,
                    help="also build with Alg. 4's search-based pools over this many tiles "
                         "(default: 128 on the SIFT-shaped workload, else 0)")
    ap.add_argument("--ablations", dest="ablations", action="store_true", default=None,
                    help="also run the alpha sweep, exact-SSG overlap and edge-time scaling "
                         "(default on the SIFT-shaped workload)")
    ap.add_argument("--no-ablations", dest="ablations", action="store_false")
    ap.add_argument("--no-fp32-arm", dest="fp32_arm", action="store_false",
                    help="skip the one plain-FP32 build reported beside the mixed-precision path")
    ap.add_argument("--serve-seconds", type=float, default=1.5,
                    help="length of each serving run of the curve (0 = skip)")
    ap.add_argument("--serve-rates", default="200,1000,2000,4000,8000",
                    help="offered request rates of the serving curve (requests per second)")
    ap.add_argument("--serve-rate", type=float, default=200.0,
                    help="requests per second offered to the 10M serving case (--serve-deep)")
    ap.add_argument("--float-n", type=int, default=200_000,
                    help="points of the float index built through both precisions (0 = skip)")
    ap.add_argument("--float-d", type=int, default=128)
    ap.add_argument("--wide-n", type=int, default=200_000,
                    help="points of the 960-d GIST-shaped index built through both precisions "
                         "(0 = skip)")
    ap.add_argument("--serve-deep", type=int, default=0,
                    help="also build the 96-d L2-normalised workload at this many points with "
                         "search-based pools and serve it (10000000: the 10M serving case)")
    ap.add_argument("--serve-deep-tiles", type=int, default=256,
                    help="tiles each node's pool is searched over for --serve-deep")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

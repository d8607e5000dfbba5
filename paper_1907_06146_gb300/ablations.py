"""Ablations on synthetic data, restating the paper's studies for this library.

* alpha_sweep: the angle alpha against out-degree, build time and search speed at
  recall@10 >= 0.95 (the paper's alpha study, Sec. 5.4).
* exact_vs_nssg: the exact SSG (Alg. 2 on the complete graph) against the NSSG built by
  Alg. 3 on the same points: how many edges they share (the paper's comparison of the two
  graphs, Sec. 4.1 / appendix).
* pool_variant: the pool loop as printed against the own-row-first reading (the node's
  whole kNN row first), built and searched on the same points.
* edge_scaling: time of the edge stages (pools, prune, reverse merge, connectivity) and of
  the kNN graph against n (the paper's scaling of index construction, Sec. 5.5).

Every function runs on the GPU through the library; no CPU reference is involved.
"""
import math
import time

import numpy as np

LS_SWEEP = (10, 12, 16, 20, 24, 32, 40, 48, 64, 96, 128)


def _qps_at(ssg, g, base, queries, truth, target=0.95):
    import torch
    nq = queries.shape[0]
    for ls in LS_SWEEP:
        ids, _ = g.search(base, queries, 10, ls)
        rec = ssg.recall_hits(ids, truth, 10) / (nq * 10.0)
        if rec >= target:
            ts = []
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                g.search(base, queries, 10, ls)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return ls, rec, nq / (min(ts) / 1e3)
    return None, rec, None


def alpha_sweep(ssg, w, n=200_000, nq=2_000, alphas=(30.0, 40.0, 50.0, 60.0, 70.0, 80.0)):
    """Build the first n points of workload w at each alpha; search its first nq queries."""
    import torch
    base = torch.from_numpy(np.ascontiguousarray(w.base[:n])).cuda()
    queries = torch.from_numpy(np.ascontiguousarray(w.queries[:nq])).cuda()
    truth, _ = ssg.knn_query(base, queries, 10)
    out = []
    for a in alphas:
        try:
            g = ssg.build(base, w.K, w.L, w.R, a, n_nav=w.n_nav)
        except ssg.SSGError as e:
            # a small alpha can fill every reached node's R slots before connectivity is
            # repaired; the build then stops (the reading taken for that case)
            out.append({"alpha": a, "error": str(e)})
            continue
        deg = g.deg.float()
        ls, rec, qps = _qps_at(ssg, g, base, queries, truth)
        out.append({"alpha": a, "avg_out_degree": float(deg.mean().item()),
                    "max_out_degree": int(deg.max().item()), "build_ms": g.stats["ms_total"],
                    "edge_ms": g.stats["ms_total"] - g.stats["ms_knn"],
                    "L_search_at_0.95": ls, "recall": rec, "qps": qps})
        del g
    return {"n": n, "queries": nq, "K": w.K, "L": w.L, "R": w.R, "points": out}


def exact_vs_nssg(ssg, synth, n=700, d=32, alpha=60.0, seed=7001):
    """Edges of the exact SSG (every other point a candidate, sorted by distance, the angle
    rule with no degree cap below 128) against the NSSG (K = 20, L = 100, R = 128)."""
    import torch
    w = synth.small(n=n, d=d, nq=0, seed=seed)
    base = torch.from_numpy(w.base).cuda()
    ids, _ = ssg.knn(base, n - 1)
    plen = torch.full((n,), n - 1, dtype=torch.int32, device="cuda")
    adj_e, deg_e = ssg.prune(base, ids, plen, 128, alpha)
    g = ssg.build(base, 20, 100, 128, alpha, n_nav=3)
    ae, de = adj_e.cpu().numpy(), deg_e.cpu().numpy()
    an, dn = g.adj.cpu().numpy(), g.deg.cpu().numpy()
    ee = {(i, int(j)) for i in range(n) for j in ae[i, :de[i]]}
    en = {(i, int(j)) for i in range(n) for j in an[i, :dn[i]]}
    both = len(ee & en)
    return {"n": n, "d": d, "alpha": alpha, "exact_edges": len(ee), "nssg_edges": len(en),
            "shared": both, "exact_covered": both / max(1, len(ee)),
            "nssg_in_exact": both / max(1, len(en)),
            "exact_nodes_at_cap_128": int((de >= 128).sum())}


def pool_variant(ssg, w, n=200_000, nq=2_000):
    """Alg. 3's pool loop as printed against the own-row-first reading (the node's whole kNN
    row, then its neighbours' rows): build time, out-degree and search at recall 0.95."""
    import torch
    base = torch.from_numpy(np.ascontiguousarray(w.base[:n])).cuda()
    queries = torch.from_numpy(np.ascontiguousarray(w.queries[:nq])).cuda()
    truth, _ = ssg.knn_query(base, queries, 10)
    out = {}
    for name, own in (("as_printed", False), ("own_row_first", True)):
        g = ssg.build(base, w.K, w.L, w.R, w.alpha, n_nav=w.n_nav, pool_own_row_first=own)
        del g
        g = ssg.build(base, w.K, w.L, w.R, w.alpha, n_nav=w.n_nav, pool_own_row_first=own)
        ls, rec, qps = _qps_at(ssg, g, base, queries, truth)
        out[name] = {"build_ms": g.stats["ms_total"], "pool_ms": g.stats["ms_pool"],
                     "avg_out_degree": float(g.deg.float().mean().item()),
                     "L_search_at_0.95": ls, "recall": rec, "qps": qps}
        del g
    return {"n": n, "queries": nq, "K": w.K, "L": w.L, "R": w.R, "variants": out}


def edge_scaling(ssg, w, ns=(62_500, 125_000, 250_000, 500_000, 1_000_000)):
    """kNN-graph and edge-stage times of builds on the first n points."""
    import torch
    out = []
    for n in ns:
        if n > w.n:
            break
        base = torch.from_numpy(np.ascontiguousarray(w.base[:n])).cuda()
        g = ssg.build(base, w.K, w.L, w.R, w.alpha, n_nav=w.n_nav)
        del g
        g = ssg.build(base, w.K, w.L, w.R, w.alpha, n_nav=w.n_nav)
        st = g.stats
        edge = st["ms_pool"] + st["ms_prune"] + st["ms_reverse"] + st["ms_connect"]
        out.append({"n": n, "knn_ms": st["ms_knn"], "edge_ms": edge, "total_ms": st["ms_total"]})
        del g, base
    if len(out) >= 2:
        a, b = out[0], out[-1]
        slope = math.log(b["edge_ms"] / a["edge_ms"]) / math.log(b["n"] / a["n"])
        kslope = math.log(b["knn_ms"] / a["knn_ms"]) / math.log(b["n"] / a["n"])
    else:
        slope = kslope = None
    return {"points": out, "edge_time_exponent": slope, "knn_time_exponent": kslope}


def run_all(ssg, synth, w):
    t0 = time.perf_counter()
    res = {"alpha_sweep": alpha_sweep(ssg, w),
           "exact_vs_nssg": exact_vs_nssg(ssg, synth),
           "pool_variant": pool_variant(ssg, w),
           "edge_scaling": edge_scaling(ssg, w)}
    res["seconds"] = time.perf_counter() - t0
    return res

"""Batched serving workload, autotuner and measurement (beyond the paper).

Workload: `n_queries` BFS / SSSP / personalized-PageRank queries (one third
each, PPR with `ppr_iters` iterations) from uniform-random sources with
out-arcs, over `n_graphs` directed R-MAT graphs whose scales are drawn
unevenly from [scale_lo, scale_hi] (small graphs are more frequent: scale =
lo + floor((hi - lo + 1) * u^2)).

Autotuner: times candidate team / bin configurations (cluster size, the arc
count from which a graph's queries get a cluster team, the warp and CTA
degree bins) on a calibration subset of the queries and keeps the fastest.
Every timed run is the library's persistent launch replayed from its
captured CUDA graph; this module only arranges calls and reduces results.
"""
from __future__ import annotations

import itertools
import time

import numpy as np

APPS = ("bfs", "sssp", "ppr")


def make_workload(n_graphs=64, n_queries=512, scale_lo=14, scale_hi=20, edgefactor=16, ppr_iters=20, seed=1):
    import graphgen
    rng = np.random.default_rng(seed)
    u = rng.random(n_graphs)
    scales = np.minimum(scale_lo + np.floor((scale_hi - scale_lo + 1) * u * u).astype(int), scale_hi)
    graphs = []
    for i, s in enumerate(scales):
        g = graphgen.rmat(int(s), edgefactor, seed=1000 + i)
        graphgen.add_weights(g, seed=2000 + i)
        graphs.append(g)
    queries = []
    pools = [graphgen.sources(g, min(g.n, 64), seed=3000 + i) for i, g in enumerate(graphs)]
    for q in range(n_queries):
        gi = int(rng.integers(0, n_graphs))
        src = int(pools[gi][int(rng.integers(0, len(pools[gi])))])
        queries.append((gi, APPS[q % 3], src, ppr_iters if APPS[q % 3] == "ppr" else 0))
    return graphs, queries, scales


def _run(gg, handles, queries, cfg, reps=3, warm=1):
    b = gg.gg_batch_create(handles, [gg.make_query(gi, app, s, it) for gi, app, s, it in queries], **cfg)
    try:
        for _ in range(warm):
            gg.gg_batch_run(b)
        times = [gg.gg_batch_run(b) for _ in range(reps)]
        st = gg.gg_batch_query_stats(b, len(queries))
        return b, times, st
    except Exception:
        gg.gg_batch_free(b)
        raise


def candidates(scale_hi=20, edgefactor=16):
    """Team sizes (threads per CTA x CTAs per cluster), the graph size from
    which a query gets a cluster team, and the degree bins."""
    out = []
    for threads in (256, 1024):
        for warp_deg, cta_deg in ((8, 256), (32, 1024)):
            out.append(dict(cluster=1, warp_deg=warp_deg, cta_deg=cta_deg, big_arcs=1 << 62, threads=threads))
            for cluster, big_scale in itertools.product((8, 16), (scale_hi - 3, scale_hi - 1)):
                out.append(dict(cluster=cluster, warp_deg=warp_deg, cta_deg=cta_deg,
                                big_arcs=edgefactor << big_scale, threads=threads, small_first=4))
    return out


def autotune(gg, handles, queries, cands, calib=128, seed=5):
    """Fastest candidate on a calibration subset; returns (best, table)."""
    rng = np.random.default_rng(seed)
    sub = [queries[i] for i in sorted(rng.choice(len(queries), min(calib, len(queries)), replace=False))]
    table = []
    for cfg in cands:
        try:
            b, times, _ = _run(gg, handles, sub, cfg, reps=2, warm=1)
        except gg.GGError as e:   # e.g. a cluster size the device cannot place
            table.append({**{k: int(v) for k, v in cfg.items()}, "ms": None, "error": str(e)[:80]})
            continue
        gg.gg_batch_free(b)
        table.append({**{k: int(v) for k, v in cfg.items()}, "ms": round(min(times), 3)})
    best = min((r for r in table if r["ms"] is not None), key=lambda r: r["ms"])
    return {k: best[k] for k in ("cluster", "warp_deg", "cta_deg", "big_arcs", "threads", "small_first")
            if k in best}, table


def measure(gg, graphs, queries, scales, tune=True, reps=5, ppr_iters=20):
    """Load the graphs, autotune, serve every query `reps` times; returns the
    JSON-ready summary (makespan, GTEPS, latency percentiles)."""
    t0 = time.perf_counter()
    handles = [gg.gg_load_csr(g.n, g.m, g.rowptr, g.colidx, g.weights, gg.GG_DIRECTED) for g in graphs]
    t_load = time.perf_counter() - t0
    try:
        cands = candidates()
        if tune:
            best, table = autotune(gg, handles, queries, cands)
        else:
            best, table = cands[0], []
        b, times, st = _run(gg, handles, queries, best, reps=reps, warm=1)
        gg.gg_batch_free(b)
    finally:
        for h in handles:
            gg.gg_free_graph(h)
    ms = float(np.median(times))
    arcs = int(st["arcs"].sum())
    lat = st["latency_ns"].astype(np.float64) / 1e6
    svc = st["service_ns"].astype(np.float64) / 1e6
    by_app = {}
    for app in APPS:
        sel = np.array([q[1] == app for q in queries])
        by_app[app] = {"queries": int(sel.sum()), "latency_p50_ms": round(float(np.percentile(lat[sel], 50)), 3),
                       "latency_p99_ms": round(float(np.percentile(lat[sel], 99)), 3),
                       "arcs": int(st["arcs"][sel].sum())}
    return {
        "workload": f"{len(queries)} queries (BFS, SSSP, personalized PageRank {ppr_iters} iterations, "
                    f"one third each) over {len(graphs)} R-MAT graphs of scales {int(min(scales))}-"
                    f"{int(max(scales))} (ef 16, weights 1..255)",
        "graphs_by_scale": {int(s): int((scales == s).sum()) for s in sorted(set(scales.tolist()))},
        "total_arcs_in_graphs": int(sum(g.m for g in graphs)),
        "config": best, "autotune": sorted((r for r in table if r["ms"] is not None), key=lambda r: r["ms"])[:6],
        "autotune_candidates": len(table),
        "makespan_ms": round(ms, 3), "makespan_ms_runs": [round(t, 3) for t in times],
        "gteps": round(arcs / (ms * 1e-3) / 1e9, 3), "arcs_traversed": arcs,
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3), "p99": round(float(np.percentile(lat, 99)), 3),
                       "max": round(float(lat.max()), 3)},
        "service_ms": {"p50": round(float(np.percentile(svc, 50)), 3), "p99": round(float(np.percentile(svc, 99)), 3)},
        "by_app": by_app, "cuda_graph": True, "load_s": round(t_load, 2),
    }


def main():
    import argparse
    import json

    from . import gg
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=64)
    ap.add_argument("--queries", type=int, default=512)
    ap.add_argument("--no-tune", action="store_true")
    a = ap.parse_args()
    graphs, queries, scales = make_workload(a.graphs, a.queries)
    print(json.dumps(measure(gg, graphs, queries, scales, tune=not a.no_tune)))


if __name__ == "__main__":
    main()

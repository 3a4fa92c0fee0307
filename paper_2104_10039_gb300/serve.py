"""Batched serving workload, autotuner and measurement (beyond the paper).

Workload: `n_queries` BFS / SSSP / personalized-PageRank queries (one third
each, PPR with `ppr_iters` iterations) from uniform-random sources with
out-arcs, over `n_graphs` directed R-MAT graphs whose scales are drawn
unevenly from [scale_lo, scale_hi] (small graphs are more frequent: scale =
lo + floor((hi - lo + 1) * u^2)).

Autotuner: first the team shape (threads per CTA, cluster size, the arc
count from which a graph's queries get a cluster team, small-first
clusters) on a calibration subset of the queries, then, for every graph
scale, the warp and CTA degree bins on that scale's queries; each query
then runs with its graph scale's bins.
Every timed run is the library's persistent launch replayed from its
captured CUDA graph; this module only arranges calls and reduces results.
The measurement also runs the tuned batch under each claim order (most
estimated work first, least first, traversals before personalized
PageRank) and two unbatched baselines of the same queries, one after
another: each query alone in its own launch, and BFS / SSSP through the
library's per-graph engine (gg_run, exact).
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


def _run(gg, handles, queries, cfg, reps=3, warm=1, bins=None):
    """Create the batch (queries: (graph, app, source, iters); bins: per-query
    (warp_deg, cta_deg) or None), run warm-up and timed launches."""
    qs = [gg.make_query(gi, app, s, it, warp_deg=bins[i][0] if bins else 0, cta_deg=bins[i][1] if bins else 0)
          for i, (gi, app, s, it) in enumerate(queries)]
    b = gg.gg_batch_create(handles, qs, **cfg)
    try:
        for _ in range(warm):
            gg.gg_batch_run(b)
        times = [gg.gg_batch_run(b) for _ in range(reps)]
        st = gg.gg_batch_query_stats(b, len(queries))
        return b, times, st
    except Exception:
        gg.gg_batch_free(b)
        raise


BIN_CANDIDATES = ((8, 256), (16, 1024), (32, 1024), (64, 4096))


def team_candidates(scale_hi=20, edgefactor=16):
    """Team shapes: threads per CTA, CTAs per cluster, the graph size from
    which a query gets a cluster team, and small-first clusters."""
    out = []
    for threads in (256, 1024):
        out.append(dict(cluster=1, warp_deg=32, cta_deg=1024, big_arcs=1 << 62, threads=threads, small_first=0))
        for cluster, big_scale in itertools.product((8, 16), (scale_hi - 3, scale_hi - 1)):
            out.append(dict(cluster=cluster, warp_deg=32, cta_deg=1024, big_arcs=edgefactor << big_scale,
                            threads=threads, small_first=4))
    return out


def _timed(gg, handles, queries, cfg, bins=None):
    try:
        b, times, _ = _run(gg, handles, queries, cfg, reps=2, warm=1, bins=bins)
    except gg.GGError as e:   # e.g. a cluster size the device cannot place
        return None, str(e)[:80]
    gg.gg_batch_free(b)
    return round(min(times), 3), None


def autotune(gg, handles, queries, graph_scales, calib=128, per_scale=48, seed=5):
    """(1) the team shape on a calibration subset of the queries with the
    default bins; (2) for every graph scale, the degree bins on that scale's
    queries under the chosen team shape. Returns (config, bins by scale,
    tables)."""
    rng = np.random.default_rng(seed)
    sub = [queries[i] for i in sorted(rng.choice(len(queries), min(calib, len(queries)), replace=False))]
    teams = []
    for cfg in team_candidates():
        ms, err = _timed(gg, handles, sub, cfg)
        teams.append({**{k: int(v) for k, v in cfg.items()}, "ms": ms, **({"error": err} if err else {})})
    best = min((r for r in teams if r["ms"] is not None), key=lambda r: r["ms"])
    cfg = {k: best[k] for k in ("cluster", "warp_deg", "cta_deg", "big_arcs", "threads", "small_first")}
    bins_by_scale, bin_table = {}, []
    for sc in sorted(set(graph_scales)):
        qs = [q for q in queries if graph_scales[q[0]] == sc][:per_scale]
        if not qs:
            continue
        row = {"scale": int(sc), "queries": len(qs)}
        for wd, cd in BIN_CANDIDATES:
            ms, _ = _timed(gg, handles, qs, cfg, bins=[(wd, cd)] * len(qs))
            row[f"{wd}/{cd}"] = ms
        bins_by_scale[int(sc)] = min(BIN_CANDIDATES, key=lambda b: row[f"{b[0]}/{b[1]}"] or float("inf"))
        bin_table.append(row)
    return cfg, bins_by_scale, {"teams": sorted((r for r in teams if r["ms"] is not None), key=lambda r: r["ms"])[:6],
                                "team_candidates": len(teams), "bins_by_scale_ms": bin_table}


def _latency_summary(lat, queries):
    """p50 / p99 latency (ms) over all queries and per application."""
    lat = np.asarray(lat, np.float64)
    out = {"p50": round(float(np.percentile(lat, 50)), 3), "p99": round(float(np.percentile(lat, 99)), 3),
           "max": round(float(lat.max()), 3)}
    for app in APPS:
        sel = np.array([q[1] == app for q in queries])
        if sel.any():
            out[f"{app}_p50"] = round(float(np.percentile(lat[sel], 50)), 3)
            out[f"{app}_p99"] = round(float(np.percentile(lat[sel], 99)), 3)
    return out


def unbatched(gg, handles, queries, cfg, bins):
    """Baseline without batching: every query alone in its own persistent
    launch (the same kernel and team shape), launched one after another.
    Returns each query's device time (ms, replayed launch)."""
    times = []
    for i, (gi, app, s, it) in enumerate(queries):
        b, t, _ = _run(gg, handles, [(gi, app, s, it)], cfg, reps=1, warm=1, bins=[bins[i]])
        gg.gg_batch_free(b)
        times.append(t[0])
    return np.asarray(times)


def engine_baseline(gg, handles, queries, single_times):
    """Baseline through the library's per-graph engine: each BFS / SSSP query
    as an exact gg_run to its fixed point (push / pull direction switch), one
    after another; personalized PageRank has no gg_run form, so those
    queries keep their single-query launch time. Returns device ms per query."""
    times = np.array(single_times, np.float64)
    for i, (gi, app, s, it) in enumerate(queries):
        if app == "ppr":
            continue
        p = gg.make_params(max_iters=1 << 20, source=s, flags=gg.GG_TIMING)
        gg.gg_run(handles[gi], app, 1.0, "exact", p)   # warm
        gg.gg_run(handles[gi], app, 1.0, "exact", p)
        times[i] = gg.stats(handles[gi]).ms_run
    return times


ORDERS = {"most_work_first": 0, "least_work_first": 1, "traversals_first": 2}


def measure(gg, graphs, queries, scales, tune=True, reps=5, ppr_iters=20, baseline=True):
    """Load the graphs, autotune, serve every query `reps` times; returns the
    JSON-ready summary (makespan, GTEPS, latency percentiles)."""
    t0 = time.perf_counter()
    handles = [gg.gg_load_csr(g.n, g.m, g.rowptr, g.colidx, g.weights, gg.GG_DIRECTED) for g in graphs]
    t_load = time.perf_counter() - t0
    try:
        if tune:
            cfg, bins_by_scale, table = autotune(gg, handles, queries, scales)
        else:
            cfg, bins_by_scale, table = team_candidates()[0], {}, {}
        bins = [bins_by_scale.get(int(scales[gi]), (cfg["warp_deg"], cfg["cta_deg"])) for gi, _, _, _ in queries]
        b, times, st = _run(gg, handles, queries, cfg, reps=reps, warm=1, bins=bins)
        gg.gg_batch_free(b)
        by_order = {}
        for name, o in ORDERS.items():
            bo, to, sto = _run(gg, handles, queries, {**cfg, "order": o}, reps=3, warm=1, bins=bins)
            gg.gg_batch_free(bo)
            by_order[name] = {"makespan_ms": round(float(np.median(to)), 3),
                              "latency_ms": _latency_summary(sto["latency_ns"].astype(np.float64) / 1e6, queries)}
        base = None
        if baseline:
            single = unbatched(gg, handles, queries, cfg, bins)
            engine = engine_baseline(gg, handles, queries, single)
            base = {}
            for name, t in (("one_launch_per_query", single), ("gg_run_per_query", engine)):
                base[name] = {"makespan_ms": round(float(t.sum()), 3),
                              "latency_ms": _latency_summary(np.cumsum(t), queries),
                              "gteps": round(float(st["arcs"].sum()) / (float(t.sum()) * 1e-3) / 1e9, 3)}
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
        "config": cfg, "bins_by_scale": {str(k): list(v) for k, v in bins_by_scale.items()}, "autotune": table,
        "makespan_ms": round(ms, 3), "makespan_ms_runs": [round(t, 3) for t in times],
        "gteps": round(arcs / (ms * 1e-3) / 1e9, 3), "arcs_traversed": arcs,
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3), "p99": round(float(np.percentile(lat, 99)), 3),
                       "max": round(float(lat.max()), 3)},
        "service_ms": {"p50": round(float(np.percentile(svc, 50)), 3), "p99": round(float(np.percentile(svc, 99)), 3)},
        "by_app": by_app, "cuda_graph": True, "load_s": round(t_load, 2),
        "by_order": by_order,
        **({"baseline": {**base, "note": "the same queries unbatched, run one after another; latency = "
                                            "completion time in workload order"},
            "speedup": {k: round(v["makespan_ms"] / ms, 3) for k, v in base.items()}} if base else {}),
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

#!/usr/bin/env python
"""Bench of the GraphGuess hot path on one GB300 (or N replicas).

One step = one pass over every step of the hot path on the directed R-MAT
scale-24 workload (16 777 216 vertices, 268 435 456 arcs, weights in
[1, 255]):
  load the CSR already resident in HBM and build the in-edge view (gg_load_csr),
  exact PageRank (20 iterations) and exact SSSP (the baselines of Sec. 5),
  then for every sample ratio sigma in {0.1, 0.3, 0.5, 0.7, 0.9}: PageRank
  and SSSP under adaptive correction (alpha 4, theta 0.05), each re-sampling
  its edges (Sec. 3.4) and running the approximate gathers, corrections,
  push frontier and change statistics.

value = GTEPS = arcs gathered by all runs of the step (the size of every
iteration's edge set) / step time, summed over ranks. e2e = the same with the
CSR in pinned host memory (host-to-device copies inside the step) and every
run's vertex values copied back to the host.

The same step on directed R-MAT scale 22 (4 194 304 vertices, 67 108 864
arcs) is reported under "rmat22"; the parameter sweep, the 16-source SSSP
table and the learned scorer's training traces use that graph (and scale 12).

--impl reference times the CPU oracle (the reference arm of this repository)
on a bounded sample of the workload, described in its line.
"""
from __future__ import annotations

import argparse
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

SCALE = 24
SECONDARY_SCALE = 22
EDGEFACTOR = 16
GRAPH_SEED, WEIGHT_SEED, SOURCE_SEED, SAMPLE_SEED = 1, 7, 2, 1
SIGMAS = (0.1, 0.3, 0.5, 0.7, 0.9)
ALPHA, THETA, PR_ITERS, DAMPING = 4, 0.05, 20, 0.85
MAX_ITERS_MIN = 1 << 20
METRIC = "GTEPS & HBM-roofline fraction; time-to-accuracy vs exact, same GB300"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=SCALE, help="R-MAT scale (the workload is 24)")
    ap.add_argument("--no-secondary", action="store_true", help="skip the R-MAT 22 step and its tables")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-scale24", action="store_true")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(ms_local, units_local, world, device="cpu"):
    """Whole-job figures of one timed region: the slowest rank's time and the
    units all ranks processed (torch.distributed; NCCL on GPUs, gloo on CPU)."""
    if world == 1:
        return ms_local, units_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def workload(scale):
    import graphgen
    g = graphgen.rmat(scale, EDGEFACTOR, seed=GRAPH_SEED)
    graphgen.add_weights(g, seed=WEIGHT_SEED)
    source = int(graphgen.sources(g, 1, seed=SOURCE_SEED)[0])
    return g, source


def workload_config(scale, n, m, source, world):
    """The workload both arms name (the reference arm times a bounded sample
    of it, described in its cpu_baseline)."""
    return {"workload": f"rmat{scale}-ef{EDGEFACTOR}-directed: load + exact PageRank/SSSP + "
                        f"adaptive-correction PageRank/SSSP at sigma {list(SIGMAS)}",
            "vertices": n, "arcs": m, "alpha": ALPHA, "theta": THETA,
            "pagerank_iters": PR_ITERS, "damping": DAMPING, "sssp_source": source,
            "sssp_iters": "exact run to its fixed point; adaptive runs the same count",
            "runs_per_step": len(run_list(source)), "parallelism": f"replicas x{world}",
            "l2": f"inputs larger than L2 ({4 * m / 1e6:.0f} MB of arcs + {4 * m / 1e6:.0f} MB of weights per load)"}


def run_list(source):
    runs = [("pagerank", 1.0, "exact"), ("sssp", 1.0, "exact")]
    for s in SIGMAS:
        runs += [("pagerank", s, "adaptive"), ("sssp", s, "adaptive")]
    return runs


def params(gg, app, source, timing=True, iters=None, theta=THETA, extra_flags=0):
    """PageRank runs PR_ITERS iterations. The exact SSSP run goes to its fixed
    point; the adaptive SSSP runs get the same number of iterations as the
    exact one (the paper compares executions of equal iteration counts,
    Sec. 5)."""
    flags = (gg.GG_TIMING if timing else 0) | extra_flags
    if app == "pagerank":
        return gg.make_params(alpha=ALPHA, theta=theta, max_iters=iters or PR_ITERS, damping=DAMPING,
                              seed=SAMPLE_SEED, flags=flags)
    return gg.make_params(alpha=ALPHA, theta=theta, max_iters=iters or MAX_ITERS_MIN, source=source,
                          seed=SAMPLE_SEED, flags=flags)


# --------------------------------------------------------- algorithmic bytes --
# Bytes an iteration must move by the method's definition (the gathered value
# vector is read from L2 and counted once per vertex). n = vertices, e = arcs of the
# iteration's edge set, m = all arcs.
def gather_bytes(app, n, e):
    if app == "pagerank":        # sources 4e; row ptr, rank, degree, rank', contrib' 20n; contrib 4n
        return 4 * e + 24 * n
    return 8 * e + 16 * n         # sources + weights 8e; row ptr, value, value', gathered value 16n


def correct_bytes(app, n, m):
    """A correction over all m arcs: sources (and weights) read, flags
    written (and read: the min applications keep some), per-vertex state;
    rebuilding the packed list is not part of it."""
    if app == "pagerank":        # sources 4m; flags m/8; row ptr, rank, degree, rank', contrib', contrib, acc 28n
        return 4 * m + m // 8 + 28 * n
    return 8 * m + m // 4 + 20 * n


def clocks_sampler():
    """nvidia-smi sampling of SM clocks and throttle reasons, started before and
    stopped after the timed region."""
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                              "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None
    lines = []
    t = threading.Thread(target=lambda: lines.extend(p.stdout), daemon=True)
    t.start()
    return p, t, lines


def clocks_summary(handle, device):
    if handle is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p, t, lines = handle
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    t.join(timeout=5)
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9 or f[0] != str(device):
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for name, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "samples": len(sm), "reasons": sorted(reasons)}


def peak_hbm():
    try:
        with open(PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def recorded_traffic(cls, algorithmic_bytes):
    """DRAM bytes per launch of a kernel class: the committed ncu capture's
    traffic / algorithmic-bytes ratio times this launch's algorithmic bytes,
    if the capture was taken on the current tile-engine sources."""
    from paper_2104_10039_gb300 import profile_traffic
    try:
        with open(TRAFFIC) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("kernel_hash") != profile_traffic.kernel_hash():
        return None
    c = t.get("classes", {}).get(cls)
    return int(c["ratio"] * algorithmic_bytes) if c else None


# ------------------------------------------------------------------ our arm --
def bench_ours(a, rank, world, local):
    import torch
    from paper_2104_10039_gb300 import build
    build.build()
    from paper_2104_10039_gb300 import gg  # noqa: F401  (fails loudly without libgg.so)

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    g, source = workload(a.scale)
    out, collected = measure(g, source, a.scale, a.steps, a.warmup, rank, world, local, e2e=True, clocks=True)
    if rank != 0:
        return None
    return out, g, source, collected


def measure(g, source, scale, steps, warmup, rank, world, local, e2e=True, clocks=True):
    """Time `steps` executions of the step on graph g (after `warmup`): device
    time with the CSR resident in HBM, then (e2e) the same with the CSR in
    pinned host memory and every run's values copied back. Returns the JSON
    fields of the line and the per-run statistics of the last timed step."""
    import torch
    from paper_2104_10039_gb300 import gg

    n, m = g.n, g.m
    d_rowptr = torch.from_numpy(g.rowptr).cuda()
    d_colidx = torch.from_numpy(g.colidx).cuda()
    d_w = torch.from_numpy(g.weights.view(np.int32)).cuda()
    h_rowptr = torch.from_numpy(g.rowptr).pin_memory()
    h_colidx = torch.from_numpy(g.colidx).pin_memory()
    h_w = torch.from_numpy(g.weights.view(np.int32)).pin_memory()
    out_host = torch.empty(n, dtype=torch.int32).pin_memory()
    runs = run_list(source)
    stream = torch.cuda.current_stream()

    def step(e2e=False, collect=None):
        if e2e:
            h = gg.gg_load_csr(n, m, h_rowptr, h_colidx, h_w, gg.GG_DIRECTED)
        else:
            h = gg.gg_load_csr(n, m, d_rowptr, d_colidx, d_w, gg.GG_DIRECTED | gg.GG_DEVICE_PTRS)
        arcs = 0
        launches = gg.stats(h).kernels_load
        per = {"load_ms": gg.stats(h).ms_load, "exact_equivalent_arcs": 0}
        sssp_iters = None
        try:
            for app, sigma, policy in runs:
                iters = sssp_iters if (app == "sssp" and policy != "exact") else None
                gg.gg_run(h, app, sigma, policy, params(gg, app, source, iters=iters))
                st = gg.stats(h)
                if app == "sssp" and policy == "exact":
                    sssp_iters = st.iterations
                arcs += st.arcs_processed
                per["exact_equivalent_arcs"] += st.iterations * m
                launches += st.kernels_launched
                if e2e:
                    gg.gg_result(h, gg.GG_RESULT_VALUES, out_host, 4 * n)
                if collect is not None:
                    collect.append((app, sigma, policy, st, gg.result_array(h, gg.GG_RESULT_ITER_STATS)))
        finally:
            gg.gg_free_graph(h)
        return arcs, launches, per

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(warmup):
        step()
    # ---- timed region: device-resident inputs ------------------------------
    clk = clocks_sampler() if (rank == 0 and clocks) else None
    collected = []
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    arcs_total, launches_total, eq_total = 0, 0, 0
    for k in range(steps):
        arcs, launches, per = step(collect=collected if k == steps - 1 else None)
        arcs_total += arcs
        launches_total += launches
        eq_total += per["exact_equivalent_arcs"]
    ev1.record(stream)
    barrier()
    clk_sum = clocks_summary(clk, local) if clk is not None else None
    ms, arcs_all = aggregate(ev0.elapsed_time(ev1), arcs_total, world, "cuda")
    value = arcs_all / (ms * 1e-3) / 1e9
    _, eq_all = aggregate(ev0.elapsed_time(ev1), eq_total, world, "cuda")

    # ---- end to end: host buffers, copies inside ---------------------------
    e_value = None
    if e2e:
        step(e2e=True)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e_arcs = 0
        for _ in range(steps):
            e_arcs += step(e2e=True)[0]
        e1.record(stream)
        barrier()
        e_ms, e_arcs_all = aggregate(e0.elapsed_time(e1), e_arcs, world, "cuda")
        e_value = e_arcs_all / (e_ms * 1e-3) / 1e9
    del d_rowptr, d_colidx, d_w, h_rowptr, h_colidx, h_w, out_host
    torch.cuda.empty_cache()

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "GTEPS", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": round(ms / steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/u32",
        "data": "synthetic (seeded R-MAT; the paper's datasets are not available)",
        "config": workload_config(scale, n, m, source, world),
        "roofline": roofline(collected, n, m),
    }
    if e2e:
        out["e2e"] = {"value": round(e_value, 3), "unit": "GTEPS",
                      "h2d_bytes_per_step": int(4 * (n + 1) + 8 * m),
                      "d2h_bytes_per_step": int(4 * n * len(runs))}
    out["gpu_launches"] = int(launches_total)
    out["exact_equivalent_gteps"] = round(eq_all / (ms * 1e-3) / 1e9, 3)
    if clocks:
        out["clocks"] = clk_sum
    return out, collected


def roofline(collected, n, m):
    """Roofline of the kernel class (application, gather / correction / push)
    with the most device time in the last timed step: algorithmic bytes per
    launch / average CUDA-event launch time, against the measured HBM peak."""
    classes = {}
    for app, sigma, policy, st, it in collected:
        for cls, ms_c, n_c in (("gather", st.ms_gather, st.n_gather), ("correct", st.ms_correct, st.n_correct),
                               ("push", st.ms_push, st.n_push)):
            c = classes.setdefault((app, cls), [0.0, 0, 0.0])
            c[0] += ms_c
            c[1] += n_c
        for row in it:
            mode = int(row["mode"]) & ~0x400   # a pull that read frontier sources only (GG_ITER_FILTER)
            if mode in (0, 1):    # pull gathers (push iterations carry the GG_ITER_PUSH bit)
                classes[(app, "gather")][2] += gather_bytes(app, n, int(row["arcs"]))
            elif mode == 2:
                classes[(app, "correct")][2] += correct_bytes(app, n, m)
    cands = [k for k in classes if classes[k][2] > 0 and classes[k][1]]
    if not cands:
        return None
    dom = max(cands, key=lambda k: classes[k][0])
    peak, peak_kind = peak_hbm()
    avg_s = classes[dom][0] * 1e-3 / classes[dom][1]
    bytes_per = classes[dom][2] / classes[dom][1]
    achieved = bytes_per / avg_s / 1e9
    name = KERNEL_NAMES.get(dom, KERNEL_NAMES.get(dom[1], "")).format(a=dom[0])
    return {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_kind,
            "traffic": recorded_traffic(f"{dom[0]}/{dom[1]}", bytes_per),
            "algorithmic_bytes_per_launch": int(bytes_per),
            "avg_launch_ms": round(classes[dom][0] / classes[dom][1], 4),
            "ms_last_step": {f"{k[0]}/{k[1]}": round(v[0], 3) for k, v in classes.items()}}


KERNEL_NAMES = {("pagerank", "gather"): "k_hub_values + k_pull_arcs<PR> + k_long_rows<PR> + k_pr_apply",
                ("pagerank", "correct"): ("k_hub_values + k_pull_arcs<PR> (values kept) + k_long_rows + k_carries "
                                          "+ k_prc_flags + k_pr_apply"),
                "gather": "k_pull_arcs<{a}> + k_long_rows<{a}> + k_min_apply<{a}>",
                "correct": ("k_pull_arcs<{a}> (values kept) + k_long_rows + k_carries + k_minc_flags<{a}> "
                            "+ k_min_apply<{a}>"),
                "push": "k_push<{a}> + k_append_frontier"}


def accuracy_table(g, source, collected, full=True):
    """Time to accuracy (Sec. 4.2 metrics, target error <= 1 %): for the exact
    run and for adaptive correction over sigma x theta, the fewest iterations T
    whose result is within 1 % of the reference (the exact run at its full
    iteration count) and the device time of that run; plus the accuracy of
    every adaptive run of the timed step. full=False searches the plain
    adaptive policy only, up to the exact run's iteration count."""
    from paper_2104_10039_gb300 import gg, metrics
    h = gg.gg_load_csr(g.n, g.m, g.rowptr, g.colidx, g.weights, gg.GG_DIRECTED)
    target = 0.01
    try:
        def run(app, sigma, policy, iters, theta=THETA, flags=0):
            gg.gg_run(h, app, sigma, policy, params(gg, app, source, timing=False, iters=iters, theta=theta,
                                                    extra_flags=flags))
            return gg.values(h, app), gg.stats(h)

        def error(app, vals, ref):
            if app == "pagerank":
                return metrics.top_k_error(vals, ref, 100)
            return metrics.stretch_error(vals, ref, source)["error"]

        ref, full_iters = {}, {}
        for app in ("pagerank", "sssp"):
            v, st = run(app, 1.0, "exact", None)
            ref[app], full_iters[app] = v, st.iterations
        timed = []
        for app, sigma, policy, st, _ in collected:
            if policy == "exact":
                continue
            vals, _ = run(app, sigma, policy, full_iters[app])
            err = error(app, vals, ref[app])
            timed.append({"app": app, "sigma": sigma, "theta": THETA, "iters": st.iterations,
                          "ms": round(st.ms_run, 3), "error": round(err, 5),
                          "accuracy_pct": round(metrics.accuracy(err), 3)})

        def first_within(app, sigma, policy, theta, t_max, flags=0, alpha=ALPHA, ratio=0.5):
            """Fewest iterations whose result is within the target (the error of
            an adaptive run is not monotone in T: it dips after corrections)."""
            for t in range(1, t_max + 1):
                gg.gg_run(h, app, sigma, policy, gg.make_params(
                    alpha=alpha, theta=theta, max_iters=t, damping=DAMPING, source=source, seed=SAMPLE_SEED,
                    flags=flags, trigger_ratio=ratio))
                if error(app, gg.values(h, app), ref[app]) <= target:
                    return {"iters": t, "ms": round(gg.stats(h).ms_run, 3)}
            return None

        tta = {}
        for app in ("pagerank", "sssp"):
            ex = first_within(app, 1.0, "exact", THETA, full_iters[app])
            best = None
            # (policy, theta, flags, alpha, trigger ratio)
            variants = [("adaptive", 0.05, 0, 4, 0), ("adaptive", 0.005, 0, 4, 0), ("adaptive", 0.05, 0, 2, 0),
                        ("triggered", 0.05, 0, 8, 0.3), ("triggered", 0.005, 0, 8, 0.1)]
            if not full:
                variants = variants[:1]
            elif app == "pagerank":   # the share influence and renormalisation flags
                variants += [("adaptive", 0.05, gg.GG_RENORM, 4, 0), ("adaptive", 0.05, gg.GG_RENORM, 2, 0),
                             ("adaptive", 0.0005, gg.GG_INFL_SHARE | gg.GG_RENORM, 4, 0),
                             ("triggered", 0.0005, gg.GG_INFL_SHARE | gg.GG_RENORM, 8, 0.3)]
            for policy, theta, fl, alpha, ratio in variants:
                for sigma in (0.5, 0.9):
                    r = first_within(app, sigma, policy, theta, (2 if full else 1) * full_iters[app], fl, alpha,
                                     ratio)
                    if r and (best is None or r["ms"] < best["ms"]):
                        best = {"policy": policy, "sigma": sigma, "theta": theta, "alpha": alpha,
                                **({"trigger_ratio": ratio} if policy == "triggered" else {}),
                                "flags": [n for n, b in (("GG_INFL_SHARE", gg.GG_INFL_SHARE),
                                                         ("GG_RENORM", gg.GG_RENORM)) if fl & b], **r}
            if best and ex:
                best["speedup_vs_exact"] = round(ex["ms"] / best["ms"], 3)
            tta[app] = {"exact": ex, "adaptive_best": best}
    finally:
        gg.gg_free_graph(h)
    return {"target_error": target, "metric": {"pagerank": "top-100 error", "sssp": "mean stretch error"},
            "reference_iters": full_iters, "time_to_target": tta, "timed_runs": timed}


def sweep_table(g, source, thetas=(0.05, 0.2, 0.5, 0.8), alphas=(2, 4, 8)):
    """The scope's parameter sweep: adaptive correction over sigma x theta x
    alpha for PageRank (20 iterations) and SSSP (the exact run's iteration
    count); device time of each run and its error against the exact result
    (top-100 / mean stretch). Rows: [sigma, theta, alpha, ms, error]."""
    from paper_2104_10039_gb300 import gg, metrics
    h = gg.gg_load_csr(g.n, g.m, g.rowptr, g.colidx, g.weights, gg.GG_DIRECTED)
    out = {}
    try:
        for app in ("pagerank", "sssp"):
            gg.gg_run(h, app, 1.0, "exact", params(gg, app, source, timing=False))
            ref, iters, ex_ms = gg.values(h, app), gg.stats(h).iterations, gg.stats(h).ms_run
            rows = []
            for sigma in SIGMAS:
                for theta in thetas:
                    for alpha in alphas:
                        p = gg.make_params(alpha=alpha, theta=theta, max_iters=iters, damping=DAMPING, source=source,
                                           seed=SAMPLE_SEED)
                        gg.gg_run(h, app, sigma, "adaptive", p)
                        v = gg.values(h, app)
                        err = (metrics.top_k_error(v, ref, 100) if app == "pagerank"
                               else metrics.stretch_error(v, ref, source)["error"])
                        rows.append([sigma, theta, alpha, round(gg.stats(h).ms_run, 3), round(err, 4)])
            out[app] = {"exact": {"iters": iters, "ms": round(ex_ms, 3)}, "metric": "top-100 error"
                        if app == "pagerank" else "mean stretch error",
                        "columns": ["sigma", "theta", "alpha", "ms", "error"], "rows": rows}
    finally:
        gg.gg_free_graph(h)
    return out


def sssp_sources(g, k=16, sigma=0.5):
    """SSSP from 16 random sources with out-arcs (seed 2): exact and adaptive
    (alpha 4, theta 0.05, the exact run's iteration count) device time and the
    adaptive run's mean-stretch error; means over the sources."""
    import graphgen
    from paper_2104_10039_gb300 import gg, metrics
    srcs = graphgen.sources(g, k, seed=SOURCE_SEED)
    h = gg.gg_load_csr(g.n, g.m, g.rowptr, g.colidx, g.weights, gg.GG_DIRECTED)
    ex, ad, err = [], [], []
    try:
        for s in srcs:
            s = int(s)
            gg.gg_run(h, "sssp", 1.0, "exact", params(gg, "sssp", s, timing=False))
            ref, iters = gg.values(h, "sssp"), gg.stats(h).iterations
            ex.append(gg.stats(h).ms_run)
            gg.gg_run(h, "sssp", sigma, "adaptive", params(gg, "sssp", s, timing=False, iters=iters))
            ad.append(gg.stats(h).ms_run)
            err.append(metrics.stretch_error(gg.values(h, "sssp"), ref, s)["error"])
    finally:
        gg.gg_free_graph(h)
    return {"sources": len(srcs), "sigma": sigma, "exact_ms_mean": round(float(np.mean(ex)), 3),
            "adaptive_ms_mean": round(float(np.mean(ad)), 3), "stretch_error_mean": round(float(np.mean(err)), 4),
            "stretch_error_max": round(float(np.max(err)), 4)}


def scale24_section():
    """The scope's configuration 3: BFS, SSSP and CC on the symmetrised
    R-MAT scale-24 graph and the Erdos-Renyi graph of the same size (268 M
    arcs each), exact and adaptive correction at sigma 0.3 (alpha 4, theta
    0.05), each to its fixed point: device time, arcs, GTEPS and the adaptive
    run's error (mean stretch; CC relative component-count error)."""
    import graphgen
    from paper_2104_10039_gb300 import gg, metrics
    out = {}
    for name in ("rmat24", "er24"):
        g = (graphgen.rmat(24, 16, seed=1, symmetric=True) if name == "rmat24"
             else graphgen.erdos_renyi(1 << 24, avg_degree=16, seed=1, symmetric=True))
        graphgen.add_weights(g, seed=WEIGHT_SEED)
        s = int(graphgen.sources(g, 1, seed=SOURCE_SEED)[0])
        h = gg.gg_load_csr(g.n, g.m, g.rowptr, g.colidx, g.weights, gg.GG_SYMMETRIC)
        res = {"vertices": g.n, "arcs": g.m, "load_ms": round(gg.stats(h).ms_load, 3)}
        try:
            for app in ("bfs", "sssp", "cc"):
                row = {}
                for policy, sigma in (("exact", 1.0), ("adaptive", 0.3)):
                    p = gg.make_params(alpha=ALPHA, theta=THETA, max_iters=MAX_ITERS_MIN, source=s, seed=SAMPLE_SEED)
                    gg.gg_run(h, app, sigma, policy, p)   # warm (and the sample)
                    gg.gg_run(h, app, sigma, policy, p)
                    st = gg.stats(h)
                    row[policy] = {"ms": round(st.ms_run, 3), "iterations": st.iterations,
                                   "arcs": int(st.arcs_processed),
                                   "gteps": round(st.arcs_processed / (st.ms_run * 1e-3) / 1e9, 2)}
                    if policy == "exact":
                        ref = gg.values(h, app)
                    else:
                        v = gg.values(h, app)
                        row[policy]["error"] = round(metrics.wcc_relative_error(v, ref)["error"] if app == "cc"
                                                     else metrics.stretch_error(v, ref, s)["error"], 5)
                res[app] = row
        finally:
            gg.gg_free_graph(h)
        out[name] = res
    return out


def learned_section(g, source, train_graphs):
    """Learned correction (beyond the paper): the scorer is trained on the
    traces of plain adaptive runs on R-MAT scale 12 and scale 22 (the
    workloads' small and mid-size graphs), then GG_POLICY_LEARNED is compared
    with plain adaptive correction on graph g (device time and error at equal
    iteration counts, time to 1 %)."""
    import torch

    import graphgen
    from paper_2104_10039_gb300 import gg, learned_eval
    g12 = graphgen.add_weights(graphgen.rmat(12, EDGEFACTOR, seed=GRAPH_SEED), seed=WEIGHT_SEED)
    s12 = int(graphgen.sources(g12, 1, seed=SOURCE_SEED)[0])
    X, Y = learned_eval.collect_traces(gg, torch, [(g12, s12)] + list(train_graphs))
    P, tr = learned_eval.train(gg, torch, X, Y)
    del X, Y
    torch.cuda.empty_cache()
    return {"evaluated_on": f"rmat{int(np.log2(g.n))} directed", "trained_on": "rmat12 + rmat22 directed traces",
            "training": tr, "alpha": learned_eval.ALPHA, "theta": learned_eval.THETA,
            "results": learned_eval.compare(gg, g, source, P, sigmas=(0.5, 0.9))}


# ------------------------------------------------------------- oracle (CPU) --
def cpu_sample(g, iters=PR_ITERS, nthreads=0):
    """The oracle as it stands on the host cores: one adaptive-correction
    PageRank run (sigma 0.5) over the workload graph, in-edge build and
    sampling included (nthreads 0: every core)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.run(g.n, g.rowptr, g.colidx, app="pagerank", policy="adaptive", sigma=0.5,
                   seed=SAMPLE_SEED, alpha=ALPHA, theta=THETA, max_iters=iters, damping=DAMPING,
                   nthreads=nthreads)
    dt = time.perf_counter() - t0
    return float(r["iter_arcs"].sum()), dt


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else os.cpu_count()


def bench_reference(a, rank, world):
    """The reference arm: the CPU oracle as it stands on the host cores. Its
    in-edge build alone takes about 20 s at scale 24, so each step is a
    bounded sample: one adaptive-correction PageRank run on directed R-MAT
    scale SECONDARY_SCALE (the same generator and parameters, a quarter of
    the workload's vertices and arcs), in-edge build and sampling included."""
    if rank != 0:
        return None
    g_full_n, g_full_m = 1 << a.scale, EDGEFACTOR << a.scale
    sample_scale = min(a.scale, SECONDARY_SCALE)
    g, source = workload(sample_scale)
    if a.scale != sample_scale:
        source = workload_source(a.scale)
    for _ in range(a.warmup):
        cpu_sample(g)
    arcs, secs = 0.0, 0.0
    for _ in range(a.steps):
        x, dt = cpu_sample(g)
        arcs += x
        secs += dt
    v = arcs / secs / 1e9
    sample = (f"each step: one adaptive-correction PageRank run (sigma 0.5, alpha {ALPHA}, theta {THETA}, "
              f"{PR_ITERS} iterations) on directed rmat{sample_scale} (ef {EDGEFACTOR}, same generator), in-edge "
              f"build and sampling included; value = its arcs / its time")
    return {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GTEPS",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": round(1e3 * secs / a.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded R-MAT)",
            "config": workload_config(a.scale, g_full_n, g_full_m, source, world),
            "reference_step": {"runs_per_step": 1, "app": "pagerank", "policy": "adaptive", "sigma": 0.5,
                               "iterations": PR_ITERS, "graph": f"rmat{sample_scale}-ef{EDGEFACTOR}-directed",
                               "vertices": g.n, "arcs": g.m},
            "cpu_baseline": {"value": round(v, 4), "unit": "GTEPS", "cores": omp_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 4), "unit": "GTEPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def workload_source(scale):
    """The workload's SSSP source (the reference line names the same
    configuration as ours); the graph itself is dropped."""
    return workload(scale)[1]


def main():
    a = parse()
    rank, world, local = dist_info()
    if a.impl == "reference":
        out = bench_reference(a, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    res = bench_ours(a, rank, world, local)
    if res is None:
        return
    out, g, source, collected = res
    g2 = s2 = None
    if not a.no_secondary and a.scale != SECONDARY_SCALE:
        g2, s2 = workload(SECONDARY_SCALE)
        sec, coll2 = measure(g2, s2, SECONDARY_SCALE, min(a.steps, 10), 3, rank, 1, local, e2e=False, clocks=False)
        out["rmat22"] = {k: sec[k] for k in ("value", "unit", "ms_per_step", "steps", "roofline",
                                             "exact_equivalent_gteps", "config")}
    if not a.no_accuracy:
        out["time_to_accuracy"] = accuracy_table(g, source, collected, full=(g2 is None))
        if g2 is not None:
            out["rmat22"]["time_to_accuracy"] = accuracy_table(g2, s2, coll2)
        out["learned_correction"] = learned_section(g, source, [(g2, s2)] if g2 is not None else [])
        gs, ss = (g2, s2) if g2 is not None else (g, source)
        out["sweep"] = sweep_table(gs, ss)
        out["sssp_16_sources"] = sssp_sources(gs)
    if not a.no_scale24:
        out["scale24_symmetric"] = scale24_section()
    if not a.no_serving:
        from paper_2104_10039_gb300 import gg, serve
        graphs, queries, scales = serve.make_workload()
        out["serving"] = serve.measure(gg, graphs, queries, scales)
    if not a.no_cpu_baseline and world == 1:
        arcs, secs = cpu_sample(g)
        out["cpu_baseline"] = {"value": round(arcs / secs / 1e9, 4), "unit": "GTEPS",
                               "cores": omp_threads(), "kind": "oracle",
                               "sample": f"one adaptive-correction PageRank run (sigma 0.5, {PR_ITERS} "
                                         f"iterations) on the workload graph, in-edge build and sampling "
                                         f"included, {secs:.1f} s"}
        g1 = g2 if g2 is not None else g
        arcs1, secs1 = cpu_sample(g1, iters=3, nthreads=1)
        out["cpu_baseline"]["single_thread"] = {
            "value": round(arcs1 / secs1 / 1e9, 4), "unit": "GTEPS", "cores": 1,
            "sample": f"the same run cut to 3 iterations on one thread on rmat{int(np.log2(g1.n))}, {secs1:.1f} s"}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

"""Learned correction end to end (beyond the paper): record traces at every
full correction of plain adaptive runs, train the scorer on the GPU, then run
GG_POLICY_LEARNED against plain adaptive correction on a target graph and
compare device time and error at equal iteration counts, and the time to a
target error.

Everything on the data runs in libgg (traces, training, scoring, runs);
this module arranges the calls and evaluates results on the host.

    python -m paper_2104_10039_gb300.learned_eval --scale 24

prints one JSON object (trained on R-MAT scale 12 and 22 traces, evaluated
on directed R-MAT of the given scale).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import metrics, scorer

ALPHA, THETA, SIGMA, DAMPING, PR_ITERS = 4, 0.05, 0.5, 0.85, 20
SAMPLE_SEED = 1
LABEL_TOL = 1e-3


def _params(gg, app, source, iters, policy_kw=None, alpha=ALPHA, theta=THETA):
    kw = dict(alpha=alpha, theta=theta, max_iters=iters, damping=DAMPING, seed=SAMPLE_SEED, source=source)
    kw.update(policy_kw or {})
    return gg.make_params(**kw)


def collect_traces(gg, torch, graphs, apps=("pagerank", "sssp"), sigma=SIGMA, alpha=ALPHA, theta=THETA,
                   label_tol=LABEL_TOL):
    """Feature / label rows of every full correction of plain adaptive runs of
    `apps` on each (graph, source); returns device tensors (X [rows, 8], Y)."""
    xs, ys = [], []
    for g, source in graphs:
        h = gg.gg_load_csr(g.n, g.m, g.rowptr, g.colidx, g.weights, gg.GG_DIRECTED)
        try:
            for app in apps:
                iters = PR_ITERS if app == "pagerank" else 1 << 20
                cap = (iters // (alpha + 1) + 2) * g.n if app == "pagerank" else 64 * g.n
                fx = torch.empty((cap, 8), dtype=torch.float32, device="cuda")
                fy = torch.empty(cap, dtype=torch.uint8, device="cuda")
                gg.gg_set_trace(h, fx, fy, cap, label_tol)
                gg.gg_run(h, app, sigma, "adaptive", _params(gg, app, source, iters, alpha=alpha, theta=theta))
                rows = gg.stats(h).trace_rows
                gg.gg_set_trace(h, None, None, 0, 0.0)
                xs.append(fx[:rows].clone())
                ys.append(fy[:rows].clone())
                del fx, fy
        finally:
            gg.gg_free_graph(h)
    return torch.cat(xs), torch.cat(ys)


def train(gg, torch, X, Y, steps=3000, lr=0.2, batch=128, seed=0):
    """Minibatch SGD over a fixed permutation of the rows; returns the
    parameters (host float32) and the loss curve."""
    rows = int(X.shape[0])
    P = torch.from_numpy(scorer.init_params(seed)).cuda()
    losses = torch.empty(steps, device="cuda")
    t0 = time.perf_counter()
    gg.gg_mlp_train(X, Y, rows, P, batch, steps, lr, scorer.coprime_stride(rows), 0, losses=losses)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    L = losses.cpu().numpy()
    return P.cpu().numpy(), {"rows": rows, "positive_frac": float(Y.float().mean().item()), "steps": steps,
                             "batch": batch, "lr": lr, "seconds": round(dt, 3),
                             "loss_first": float(L[:20].mean()), "loss_last": float(L[-100:].mean())}


def _error(app, vals, ref, source):
    if app == "pagerank":
        return metrics.top_k_error(vals, ref, 100)
    return metrics.stretch_error(vals, ref, source)["error"]


# (label, policy, fallback fraction, selection cost): plain adaptive correction;
# learned without fallback; falling back above half the arcs; and cost-aware
# selections (the threshold rises by `cost` per bit of the in-degree, so hub
# rows need stronger scores)
POLICIES = (("adaptive", "adaptive", 1.0, 0.0), ("learned", "learned", 1.0, 0.0),
            ("learned_fallback_0.5", "learned", 0.5, 0.0), ("learned_cost_0.1", "learned", 1.0, 0.1),
            ("learned_cost_0.3", "learned", 1.0, 0.3))


def compare(gg, g, source, P, apps=("pagerank", "sssp"), sigmas=(0.5, 0.9), select_logit=0.0, target=0.01):
    """Plain adaptive vs learned correction (without fallback, falling back
    to the full correction when the selection holds more than half the arcs,
    and with cost-aware selections) on g: per app and sigma, device time and
    error at the exact run's iteration count, and the time to reach `target`
    error (fewest iterations; searched only where plain adaptive correction
    reaches it, the accuracy both arms are compared at)."""
    h = gg.gg_load_csr(g.n, g.m, g.rowptr, g.colidx, g.weights, gg.GG_DIRECTED)
    out = {}
    try:
        gg.gg_set_scorer(h, P)
        for app in apps:
            gg.gg_run(h, app, 1.0, "exact", _params(gg, app, source, PR_ITERS if app == "pagerank" else 1 << 20))
            ref = gg.values(h, app)
            full_iters = gg.stats(h).iterations
            ex_ms = gg.stats(h).ms_run
            res = {"exact": {"iters": full_iters, "ms": round(ex_ms, 3)}}

            def run(policy, sigma, iters, frac, cost):
                gg.gg_run(h, app, sigma, policy, _params(gg, app, source, iters,
                                                         {"select_logit": select_logit, "fallback_frac": frac,
                                                          "select_cost": cost}))
                st = gg.stats(h)
                return gg.values(h, app), st

            for sigma in sigmas:
                row = {}
                for label, policy, frac, cost in POLICIES:
                    run(policy, sigma, full_iters, frac, cost)   # warm
                    vals, st = run(policy, sigma, full_iters, frac, cost)
                    it = gg.result_array(h, gg.GG_RESULT_ITER_STATS)
                    lm = (it["mode"] & gg.GG_ITER_LEARNED) != 0
                    row[label] = {"ms": round(st.ms_run, 3), "error": round(_error(app, vals, ref, source), 5),
                                   "corrections": st.corrections, "learned_corrections": st.learned_corrections,
                                   "selected_frac": round(float(it["selected"][lm].mean() / g.n), 4) if lm.any()
                                   else None,
                                   "selected_arc_frac": round(float(it["arcs"][lm].mean() / max(g.m, 1)), 4)
                                   if lm.any() else None}
                    ttt = None
                    if label == "adaptive" or row["adaptive"]["time_to_target"] is not None:
                        for t in range(1, 2 * full_iters + 1):
                            v, s2 = run(policy, sigma, t, frac, cost)
                            if _error(app, v, ref, source) <= target:
                                ttt = {"iters": t, "ms": round(s2.ms_run, 3)}
                                break
                    row[label]["time_to_target"] = ttt
                for label, _, _, _ in POLICIES[1:]:
                    a, b = row["adaptive"]["time_to_target"], row[label]["time_to_target"]
                    row[label]["speedup_at_target"] = round(a["ms"] / b["ms"], 3) if a and b else None
                    row[label]["speedup_equal_iters"] = round(row["adaptive"]["ms"] / row[label]["ms"], 3)
                res[f"sigma_{sigma}"] = row
            out[app] = res
    finally:
        gg.gg_free_graph(h)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=24)
    ap.add_argument("--steps", type=int, default=3000)
    args = ap.parse_args()
    import torch

    import graphgen
    from . import gg

    def graph(scale):
        g = graphgen.add_weights(graphgen.rmat(scale, 16, seed=1), seed=7)
        return g, int(graphgen.sources(g, 1, seed=2)[0])

    t0 = time.perf_counter()
    X, Y = collect_traces(gg, torch, [graph(12), graph(22)])
    P, tr = train(gg, torch, X, Y, steps=args.steps)
    del X, Y
    g, s = graph(args.scale)
    res = compare(gg, g, s, P)
    print(json.dumps({"workload": f"rmat{args.scale} directed, ef16, weights 1..255", "vertices": g.n, "arcs": g.m,
                      "trained_on": "traces of adaptive runs (alpha 4, theta 0.05, sigma 0.5) on R-MAT 12 and 22",
                      "training": tr, "alpha": ALPHA, "theta": THETA, "target_error": 0.01, "results": res,
                      "wall_s": round(time.perf_counter() - t0, 1)}))


if __name__ == "__main__":
    main()

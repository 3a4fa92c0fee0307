"""Run one GraphGuess case through the C ABI, for profilers (ncu) and quick
timing: builds the seeded R-MAT graph, loads it, runs the requested
application / policy and prints the library's statistics.

Example (the correction kernels of SSSP at scale 22, every iteration a
correction):

    python -m paper_2104_10039_gb300.profile_case --app sssp --policy adaptive \
        --alpha 0 --iters 3 --scale 22 --force-pull
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--app", default="pagerank", choices=["pagerank", "sssp", "bfs", "cc"])
    ap.add_argument("--policy", default="adaptive", choices=["exact", "sp", "sms", "adaptive"])
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--edgefactor", type=int, default=16)
    ap.add_argument("--symmetric", action="store_true")
    ap.add_argument("--sigma", type=float, default=0.5)
    ap.add_argument("--alpha", type=int, default=4)
    ap.add_argument("--theta", type=float, default=0.05)
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--force-pull", action="store_true")
    ap.add_argument("--timing", action="store_true")
    ap.add_argument("--pull-filter", action="store_true",
                    help="min applications: pulls read frontier sources only (GG_PULL_FILTER)")
    a = ap.parse_args(argv)

    import graphgen
    from paper_2104_10039_gb300 import build
    build.build()
    from paper_2104_10039_gb300 import gg

    g = graphgen.rmat(a.scale, a.edgefactor, seed=1, symmetric=a.symmetric)
    graphgen.add_weights(g, seed=7)
    src = int(graphgen.sources(g, 1, seed=2)[0])
    h = gg.gg_load_csr(g.n, g.m, g.rowptr, g.colidx, g.weights,
                       gg.GG_SYMMETRIC if a.symmetric else gg.GG_DIRECTED)
    try:
        flags = (gg.GG_FORCE_PULL if a.force_pull else 0) | (gg.GG_TIMING if a.timing else 0)
        flags |= gg.GG_PULL_FILTER if a.pull_filter else 0
        for _ in range(a.repeat):
            gg.gg_run(h, a.app, a.sigma, a.policy,
                      gg.make_params(alpha=a.alpha, theta=a.theta, max_iters=a.iters, source=src,
                                     seed=1, flags=flags))
            st = gg.stats(h)
        print(json.dumps({f: getattr(st, f) for f, _ in gg.gg_stats._fields_}))
    finally:
        gg.gg_free_graph(h)


if __name__ == "__main__":
    main()

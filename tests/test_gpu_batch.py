"""GPU parity of batched serving (beyond the paper): BFS / SSSP /
personalized-PageRank queries over several graphs of uneven size in one
persistent launch (replayed from a captured CUDA graph), under team and
degree-bin configurations that exercise every path (single CTAs, cluster
teams of 2 / 4 / 8, thread / warp / CTA bins).

Bars: BFS levels and SSSP distances bit-exact against the oracle's exact
runs; personalized PageRank within 1e-5 relative L1 of the FP64 oracle."""
import numpy as np
import pytest

import graphgen
import oracle
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gg():
    return gc.lib()


def _graphs():
    gs = [graphgen.rmat(12, seed=3), graphgen.rmat(9, edgefactor=5, seed=4), graphgen.rmat(11, seed=5),
          graphgen.erdos_renyi(3001, avg_degree=7, seed=2, symmetric=False),
          graphgen.from_arcs(7, [(0, 1), (0, 1), (1, 1), (2, 0), (6, 3), (3, 6), (5, 0)]),
          graphgen.rmat(10, edgefactor=24, seed=6)]
    for g in gs:
        graphgen.add_weights(g, seed=11)
    return gs


def _queries(gg, gs, n_q, seed):
    rng = np.random.default_rng(seed)
    qs = []
    for i in range(n_q):
        gi = int(rng.integers(0, len(gs)))
        app = ("bfs", "sssp", "ppr")[i % 3]
        src = int(rng.integers(0, gs[gi].n))
        iters = int(rng.choice([0, 1, 7, 20])) if app == "ppr" else 0
        qs.append((gi, app, src, iters))
    qs.append((4, "sssp", 4, 0))          # a source without out-arcs
    qs.append((0, "ppr", 0, 3))
    return qs


def _oracle(g, app, src, iters):
    if app == "ppr":
        return oracle.run(g.n, g.rowptr, g.colidx, app="ppr", source=src, max_iters=iters, nthreads=0)["values"]
    return oracle.run(g.n, g.rowptr, g.colidx, g.weights, app=app, source=src, max_iters=1 << 20,
                      nthreads=0)["values"]


@pytest.mark.parametrize("cluster,warp_deg,cta_deg,big_arcs,threads,small_first", [
    (1, 32, 1024, 0, 256, 0), (4, 8, 64, 20000, 256, 0), (8, 2, 16, 0, 512, 0), (2, 1, 1, 40000, 1024, 1),
    (4, 1000000, 1000000, 0, 256, 0), (8, 16, 128, 30000, 1024, 0), (4, 8, 64, 30000, 512, 2)])
def test_batch_matches_oracle(gg, cluster, warp_deg, cta_deg, big_arcs, threads, small_first):
    gs = _graphs()
    hs = [gc.load(gg, g) for g in gs]
    b = None
    try:
        qs = _queries(gg, gs, 40, seed=cluster * 7 + warp_deg)
        b = gg.gg_batch_create(hs, [gg.make_query(gi, app, s, it) for gi, app, s, it in qs], cluster=cluster,
                               warp_deg=warp_deg, cta_deg=cta_deg, big_arcs=big_arcs, threads=threads,
                               small_first=small_first)
        for rep in range(2):          # first run captures the graph, the second replays it
            gg.gg_batch_run(b)
            st = gg.gg_batch_query_stats(b, len(qs))
            for q, (gi, app, s, it) in enumerate(qs):
                g = gs[gi]
                got = gg.gg_batch_result(b, q, g.n, app)
                want = _oracle(g, app, s, it)
                if app == "ppr":
                    assert gc.rel_l1(got, want) <= 1e-5, (q, gi, s, it)
                else:
                    assert np.array_equal(got, want), (q, gi, app, s)
                big = cluster > 1 and g.m >= big_arcs
                assert st["team"][q] == (cluster if big else 1)
                assert st["latency_ns"][q] >= st["service_ns"][q] > 0
    finally:
        if b:
            gg.gg_batch_free(b)
        for h in hs:
            gg.gg_free_graph(h)


def test_batch_errors(gg):
    g = graphgen.rmat(6, seed=1)          # no weights
    h = gc.load(gg, g)
    try:
        for q, kw in (((0, "sssp", 0), {}), ((1, "bfs", 0), {}), ((0, "bfs", g.n), {}), ((0, "cc", 0), {}),
                      ((0, "bfs", 0), {"cluster": 3}), ((0, "bfs", 0), {"warp_deg": 8, "cta_deg": 4}),
                      ((0, "bfs", 0), {"threads": 128})):
            with pytest.raises(gg.GGError) as e:
                gg.gg_batch_create([h], [gg.make_query(*q)], **kw)
            assert e.value.status == gg.GG_ERR_INVALID_ARG
    finally:
        gg.gg_free_graph(h)


def test_batch_per_query_bins(gg):
    """Queries of one batch with different degree bins (as the autotuner sets
    them per graph scale)."""
    gs = _graphs()
    hs = [gc.load(gg, g) for g in gs]
    b = None
    try:
        qs = _queries(gg, gs, 30, seed=99)
        rng = np.random.default_rng(4)
        bins = [((1, 1), (2, 16), (8, 256), (32, 1024), (0, 0))[int(rng.integers(0, 5))] for _ in qs]
        b = gg.gg_batch_create(hs, [gg.make_query(gi, app, s, it, warp_deg=bn[0], cta_deg=bn[1]) for (gi, app, s, it), bn in zip(qs, bins)],
                               cluster=4, big_arcs=30000, threads=512, small_first=2)
        gg.gg_batch_run(b)
        for q, (gi, app, s, it) in enumerate(qs):
            g = gs[gi]
            got = gg.gg_batch_result(b, q, g.n, app)
            want = _oracle(g, app, s, it)
            if app == "ppr":
                assert gc.rel_l1(got, want) <= 1e-5, (q, bins[q])
            else:
                assert np.array_equal(got, want), (q, app, bins[q])
        with pytest.raises(gg.GGError):
            gg.gg_batch_create(hs, [gg.make_query(0, "bfs", 0, 0, 0.85, 8, 4)])
    finally:
        if b:
            gg.gg_batch_free(b)
        for h in hs:
            gg.gg_free_graph(h)

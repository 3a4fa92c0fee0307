"""GPU parity at the workloads' full sizes, in the configuration bench.py
times: the directed R-MAT scale-24 graph (16 777 216 vertices, 268 435 456
arcs) for PageRank and SSSP, R-MAT scale 22 (67 108 864 directed arcs), and
the symmetrised R-MAT scale-24 and Erdos-Renyi graphs (268 435 456 arcs) for
BFS, SSSP and CC at sample ratio 0.3. The oracle runs on every host core
(its results do not depend on the thread count).

Bars as in test_gpu_parity: bit-exact for the in-edge build, the sampled
flags and the integer applications (values and post-correction flags);
PageRank within 1e-5 relative L1, through mask replay when it corrects.
"""
import os

import numpy as np
import pytest

import graphgen
import oracle
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu

ALPHA, THETA, PR_ITERS = 4, 0.05, 20
BIG = 1 << 20


@pytest.fixture(scope="module")
def gg():
    return gc.lib()


@pytest.fixture(scope="module")
def rmat24():
    g = graphgen.rmat(24, 16, seed=1)
    graphgen.add_weights(g, seed=7)
    return g, int(graphgen.sources(g, 1, seed=2)[0])


def test_rmat24_directed_build_and_sampler(gg, rmat24):
    """In-edge build and sampled flags of the 268 M-arc directed graph, every
    element (Sec. 2.1 in-edges sorted by source, Sec. 3.4 sampling)."""
    g, _ = rmat24
    h = gc.load(gg, g, device_ptrs=True)
    try:
        ip, isrc, iw, pos = oracle.csc_from_csr(g.n, g.rowptr, g.colidx, g.weights)
        assert np.array_equal(gg.result_array(h, gg.GG_RESULT_CSC_PTR), ip)
        assert np.array_equal(gg.result_array(h, gg.GG_RESULT_CSC_SRC), isrc)
        assert np.array_equal(gg.result_array(h, gg.GG_RESULT_CSC_W), iw)
        gg.gg_sample_edges(h, 0.3, 1)
        assert np.array_equal(gg.mask_bits(h, g.m), oracle.sample_mask(g.n, ip, isrc, 0.3, 1))
    finally:
        gg.gg_free_graph(h)


def test_rmat24_directed_pagerank(gg, rmat24):
    """PageRank on the directed scale-24 graph: exact within 1e-5 relative L1
    of the FP64 oracle; adaptive correction (alpha 4, theta 0.05) at sigma 0.1
    and 0.5 through mask replay, as bench.py runs it."""
    g, _ = rmat24
    h = gc.load(gg, g)
    try:
        got, _, _ = gc.gpu_run(gg, h, g, "pagerank", "exact", T=PR_ITERS)
        ref = oracle.run(g.n, g.rowptr, g.colidx, app="pagerank", policy="exact", max_iters=PR_ITERS,
                         nthreads=0)
        assert gc.rel_l1(got, ref["values"]) <= 1e-5
        del ref
        for sigma in (0.1, 0.5):
            vals, ref, st = gc.pagerank_with_replay(gg, h, g, "adaptive", sigma, ALPHA, THETA, PR_ITERS, seed=1)
            assert ref["replay_violations"] == 0, ref["replay_max_margin"]
            assert ref["replay_mismatch"] <= g.m // 10000
            assert gc.rel_l1(vals, ref["values"]) <= 1e-5
            assert st.corrections == 4
    finally:
        gg.gg_free_graph(h)


def test_rmat24_directed_sssp_bit_exact(gg, rmat24):
    """SSSP on the directed scale-24 graph: exact, and adaptive correction at
    sigma 0.5 and 0.1 cut at the exact run's iteration count (bench.py's
    protocol) and run to its own fixed point; values and flags bit-exact."""
    g, s = rmat24
    h = gc.load(gg, g)
    try:
        got, _, st = gc.gpu_run(gg, h, g, "sssp", "exact", T=BIG, source=s)
        ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", policy="exact", max_iters=BIG,
                         source=s, nthreads=0)
        assert np.array_equal(got, ref["values"])
        assert st.iterations == ref["iterations"]
        t_exact = st.iterations
        for sigma, T in ((0.5, t_exact), (0.1, t_exact), (0.5, BIG)):
            got, mask, st = gc.gpu_run(gg, h, g, "sssp", "adaptive", sigma=sigma, alpha=ALPHA, theta=THETA,
                                       T=T, source=s, seed=1)
            ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", policy="adaptive", sigma=sigma,
                             seed=1, alpha=ALPHA, theta=THETA, max_iters=T, source=s, nthreads=0)
            assert np.array_equal(got, ref["values"]), (sigma, T)
            assert np.array_equal(mask, ref["mask"]), (sigma, T)
            assert st.iterations == ref["iterations"]
    finally:
        gg.gg_free_graph(h)


@pytest.fixture(scope="module")
def rmat22():
    g = graphgen.rmat(22, 16, seed=1)
    graphgen.add_weights(g, seed=7)
    return g, int(graphgen.sources(g, 1, seed=2)[0])


def test_rmat22_csc_and_sampler(gg, rmat22):
    g, _ = rmat22
    h = gc.load(gg, g, device_ptrs=True)
    try:
        ip, isrc, iw, pos = oracle.csc_from_csr(g.n, g.rowptr, g.colidx, g.weights)
        assert np.array_equal(gg.result_array(h, gg.GG_RESULT_CSC_PTR), ip)
        assert np.array_equal(gg.result_array(h, gg.GG_RESULT_CSC_SRC), isrc)
        assert np.array_equal(gg.result_array(h, gg.GG_RESULT_CSC_W), iw)
        o2i = gg.result_array(h, gg.GG_RESULT_OUT_TO_IN)
        sample = np.random.default_rng(0).integers(0, g.m, 100000)
        assert np.array_equal(pos[o2i[sample]], sample)
        gg.gg_sample_edges(h, 0.5, 1)
        want = oracle.sample_mask(g.n, ip, isrc, 0.5, 1)
        assert np.array_equal(gg.mask_bits(h, g.m), want)
        cs = np.concatenate([[0], np.cumsum(want.astype(np.int64))])
        assert np.array_equal(gg.result_array(h, gg.GG_RESULT_SPARSE_PTR), cs[ip])
    finally:
        gg.gg_free_graph(h)


def test_rmat22_pagerank_exact_and_adaptive(gg, rmat22):
    g, _ = rmat22
    h = gc.load(gg, g)
    try:
        got, _, _ = gc.gpu_run(gg, h, g, "pagerank", "exact", T=PR_ITERS)
        ref = oracle.run(g.n, g.rowptr, g.colidx, app="pagerank", policy="exact", max_iters=PR_ITERS,
                         nthreads=0)
        assert gc.rel_l1(got, ref["values"]) <= 1e-5
        for sigma in (0.1, 0.5):
            vals, ref, st = gc.pagerank_with_replay(gg, h, g, "adaptive", sigma, ALPHA, THETA, PR_ITERS, seed=1)
            assert ref["replay_violations"] == 0, ref["replay_max_margin"]
            assert ref["replay_mismatch"] <= g.m // 10000
            assert gc.rel_l1(vals, ref["values"]) <= 1e-5
            assert st.corrections == 4
    finally:
        gg.gg_free_graph(h)


def test_rmat22_sssp_bit_exact(gg, rmat22):
    g, s = rmat22
    h = gc.load(gg, g)
    try:
        for policy, sigma in (("exact", 1.0), ("adaptive", 0.5), ("adaptive", 0.1)):
            got, mask, st = gc.gpu_run(gg, h, g, "sssp", policy, sigma=sigma, alpha=ALPHA, theta=THETA,
                                       T=BIG, source=s, seed=1)
            ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", policy=policy, sigma=sigma,
                             seed=1, alpha=ALPHA, theta=THETA, max_iters=BIG, source=s, nthreads=0)
            assert np.array_equal(got, ref["values"]), policy
            if mask is not None:
                assert np.array_equal(mask, ref["mask"]), policy
            assert st.iterations == ref["iterations"]
    finally:
        gg.gg_free_graph(h)


@pytest.fixture(scope="module", params=["rmat24", "er24"])
def sym24(request):
    if request.param == "rmat24":
        g = graphgen.rmat(24, 16, seed=1, symmetric=True)
    else:
        g = graphgen.erdos_renyi(1 << 24, avg_degree=16, seed=1, symmetric=True)
    graphgen.add_weights(g, seed=7)
    return g, int(graphgen.sources(g, 1, seed=2)[0])


@pytest.mark.parametrize("app", ["bfs", "sssp", "cc"])
def test_scale24_symmetric_bit_exact(gg, sym24, app):
    g, s = sym24
    h = gc.load(gg, g)
    try:
        got, mask, st = gc.gpu_run(gg, h, g, app, "adaptive", sigma=0.3, alpha=ALPHA, theta=THETA,
                                   T=BIG, source=s, seed=1)
        ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights if app == "sssp" else None, app=app,
                         policy="adaptive", sigma=0.3, seed=1, alpha=ALPHA, theta=THETA, max_iters=BIG,
                         source=s, symmetric=True, nthreads=0)
        assert np.array_equal(got, ref["values"])
        assert np.array_equal(mask, ref["mask"])
        assert st.iterations == ref["iterations"]
    finally:
        gg.gg_free_graph(h)


def test_rmat22_learned_and_triggered_sssp_bit_exact(gg, rmat22):
    """The learned correction (a scorer whose selection is decided exactly:
    logit = bfloat16(sqrt(in-degree)/64) - t) and the triggered policy at the
    bench's size, against the oracle."""
    from paper_2104_10039_gb300 import scorer
    g, s = rmat22
    lo, hi = (float(oracle.bf16(np.float32(np.sqrt(np.float32(k)) / np.float32(64)))) for k in (40, 41))
    P = np.zeros(scorer.N_PARAM, np.float32)
    P[scorer.OFF_W1] = P[scorer.OFF_W2] = P[scorer.OFF_W3] = 1.0
    P[scorer.OFF_B3] = -(lo + hi) / 2
    h = gc.load(gg, g)
    try:
        gg.gg_set_scorer(h, P)
        p = gg.make_params(alpha=ALPHA, theta=THETA, max_iters=BIG, source=s, seed=1)
        gg.gg_run(h, "sssp", 0.3, "learned", p)
        got, mask = gg.values(h, "sssp"), gg.mask_bits(h, g.m)
        assert gg.stats(h).learned_corrections >= 1
        ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", policy="learned", mlp=P, sigma=0.3,
                         seed=1, alpha=ALPHA, theta=THETA, source=s, max_iters=BIG, nthreads=0)
        assert np.array_equal(got, ref["values"]) and np.array_equal(mask, ref["mask"])
        p = gg.make_params(alpha=8, theta=THETA, max_iters=BIG, source=s, seed=1, trigger_ratio=0.2)
        gg.gg_run(h, "sssp", 0.3, "triggered", p)
        ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", policy="triggered", sigma=0.3, seed=1,
                         alpha=8, theta=THETA, trigger_ratio=0.2, source=s, max_iters=BIG, nthreads=0)
        assert np.array_equal(gg.values(h, "sssp"), ref["values"])
        assert np.array_equal(gg.mask_bits(h, g.m), ref["mask"])
    finally:
        gg.gg_free_graph(h)


def test_serving_workload_sample(gg):
    """Queries of the serving workload (64 R-MAT graphs, scales 14-20) in the
    configuration its autotuner picks on GB300, against the oracle: the
    largest graphs' queries (cluster teams) and a few small ones."""
    from paper_2104_10039_gb300 import serve
    graphs, queries, scales = serve.make_workload()
    order = sorted(range(len(queries)), key=lambda q: -graphs[queries[q][0]].m)
    pick = order[:9] + order[-3:]
    used = sorted({queries[q][0] for q in pick})
    remap = {gi: i for i, gi in enumerate(used)}
    hs = [gc.load(gg, graphs[gi]) for gi in used]
    b = None
    try:
        qs = [queries[q] for q in pick]
        b = gg.gg_batch_create(hs, [gg.make_query(remap[gi], app, src, it) for gi, app, src, it in qs], cluster=8,
                               warp_deg=32, cta_deg=1024, big_arcs=1 << 21, threads=1024, small_first=4)
        gg.gg_batch_run(b)
        for q, (gi, app, src, it) in enumerate(qs):
            g = graphs[gi]
            got = gg.gg_batch_result(b, q, g.n, app)
            if app == "ppr":
                want = oracle.run(g.n, g.rowptr, g.colidx, app="ppr", source=src, max_iters=it, nthreads=0)["values"]
                assert gc.rel_l1(got, want) <= 1e-5, (q, gi)
            else:
                want = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app=app, source=src, max_iters=BIG,
                                  nthreads=0)["values"]
                assert np.array_equal(got, want), (q, gi, app)
    finally:
        if b:
            gg.gg_batch_free(b)
        for h in hs:
            gg.gg_free_graph(h)

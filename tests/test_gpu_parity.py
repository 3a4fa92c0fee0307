"""GPU parity: every step of the hot path through the C ABI against the
oracle, element by element, on seeded inputs that span several tiles and a
ragged tail, plus the edge cases (empty graphs, isolated vertices, single
vertex, duplicates, self-loops).

Bars: bit-exact for the in-edge build, the sampled flags, the packed active
edges and every integer application (values and post-correction flags);
PageRank within 1e-5 relative L1 of the FP64 oracle (exact mode, SP, and the
correcting policies through mask replay).
"""
import numpy as np
import pytest

import graphgen
import oracle
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu

PR_TOL = 1e-5


@pytest.fixture(scope="module")
def gg():
    return gc.lib()


def _graphs():
    gs = [graphgen.rmat(12, seed=1),                       # 4096 vertices, 65536 arcs, 272 tiles
          graphgen.rmat(9, edgefactor=5, seed=3),
          graphgen.erdos_renyi(3001, avg_degree=7, seed=2, symmetric=False),
          graphgen.from_arcs(7, [(0, 1), (0, 1), (1, 1), (2, 0), (6, 3), (3, 6), (5, 0)]),
          graphgen.from_arcs(1, [(0, 0)]),
          graphgen.from_arcs(5, [])]
    for g in gs:
        graphgen.add_weights(g, seed=11)
    return gs


def _sym_graphs():
    gs = [graphgen.rmat(12, seed=1, symmetric=True),
          graphgen.erdos_renyi(5000, avg_degree=6, seed=4, symmetric=True),
          graphgen.from_arcs(10, [(i, j) for i in range(5) for j in range(5) if i != j] +
                             [(i, j) for i in range(5, 10) for j in range(5, 10) if i != j] +
                             [(4, 5), (5, 4)], symmetric=True)]
    for g in gs:
        graphgen.add_weights(g, seed=11)
    return gs


# ------------------------------------------------------ a1: in-edge build --

@pytest.mark.parametrize("device_ptrs", [False, True])
def test_csc_build_bit_exact(gg, device_ptrs):
    for g in _graphs() + _sym_graphs():
        h = gc.load(gg, g, device_ptrs=device_ptrs)
        try:
            ip, isrc, iw, pos = oracle.csc_from_csr(g.n, g.rowptr, g.colidx, g.weights)
            assert np.array_equal(gg.result_array(h, gg.GG_RESULT_CSC_PTR), ip)
            assert np.array_equal(gg.result_array(h, gg.GG_RESULT_CSC_SRC), isrc)
            assert np.array_equal(gg.result_array(h, gg.GG_RESULT_CSC_W), iw)
            o2i = gg.result_array(h, gg.GG_RESULT_OUT_TO_IN)
            assert np.array_equal(pos[o2i], np.arange(g.m))
        finally:
            gg.gg_free_graph(h)


# ----------------------------------------------------------- a2: sampling --

@pytest.mark.parametrize("sigma", [0.1, 0.5, 0.97, 1.0])
def test_sampler_bit_exact(gg, sigma):
    for g in _graphs() + _sym_graphs():
        h = gc.load(gg, g)
        try:
            gg.gg_sample_edges(h, sigma, 1234567)
            ip, isrc, iw, _ = oracle.csc_from_csr(g.n, g.rowptr, g.colidx, g.weights)
            want = oracle.sample_mask(g.n, ip, isrc, sigma, 1234567, symmetric=g.symmetric)
            got = gg.mask_bits(h, g.m)
            assert np.array_equal(got, want)
            # packed active in-edges: same rows, same order
            sp_ptr = gg.result_array(h, gg.GG_RESULT_SPARSE_PTR)
            sp_src = gg.result_array(h, gg.GG_RESULT_SPARSE_SRC)
            cs = np.concatenate([[0], np.cumsum(want.astype(np.int64))])
            assert np.array_equal(sp_ptr, cs[ip])
            assert np.array_equal(sp_src, isrc[want.astype(bool)])
        finally:
            gg.gg_free_graph(h)


def _check_packed(gg, h, g, mask):
    """The library's packed active in-edges equal the packing of `mask`."""
    ip, isrc, _, _ = oracle.csc_from_csr(g.n, g.rowptr, g.colidx, g.weights)
    sp_ptr = gg.result_array(h, gg.GG_RESULT_SPARSE_PTR)
    sp_src = gg.result_array(h, gg.GG_RESULT_SPARSE_SRC)
    cs = np.concatenate([[0], np.cumsum(mask.astype(np.int64))])
    assert np.array_equal(sp_ptr, cs[ip])
    assert np.array_equal(sp_src, isrc[mask.astype(bool)])


@pytest.mark.parametrize("app", ["pagerank", "sssp"])
def test_packed_list_built_when_needed(gg, app):
    """The packed list after a correction (or a sampling) is built when a
    gather or a result needs it: runs that end on a correction, or whose
    approximate iterations all push, still give the packing of the final flags
    and the right active-arc count."""
    g = graphgen.rmat(12, seed=1)
    graphgen.add_weights(g, seed=11)
    s = int(graphgen.sources(g, 1, seed=2)[0])
    h = gc.load(gg, g)
    try:
        for T, flags in ((3, 0), (6, 0), (7, 8), (11, 4)):   # 8: GG_FORCE_PUSH, 4: GG_FORCE_PULL
            if app == "pagerank" and flags:
                continue
            p = gg.make_params(alpha=2, theta=0.05, max_iters=T, source=s, seed=13, flags=flags)
            gg.gg_run(h, app, 0.5, "gg", p)
            mask = gg.mask_bits(h, g.m)
            _check_packed(gg, h, g, mask)
            it = gg.result_array(h, gg.GG_RESULT_ITER_STATS)
            corr = np.flatnonzero((it["mode"] & 3) == 2)
            if len(corr):
                assert int(it["active_after"][corr[-1]]) == int(mask.sum()), (T, flags)
        gg.gg_sample_edges(h, 0.3, 77)
        _check_packed(gg, h, g, gg.mask_bits(h, g.m))
    finally:
        gg.gg_free_graph(h)


# ------------------------------------------------------------- pagerank --

@pytest.mark.parametrize("T", [1, 3, 20])
def test_pagerank_exact(gg, T):
    for g in _graphs():
        h = gc.load(gg, g)
        try:
            got, _, st = gc.gpu_run(gg, h, g, "pagerank", "exact", T=T)
            ref = oracle.run(g.n, g.rowptr, g.colidx, app="pagerank", policy="exact", max_iters=T)
            assert gc.rel_l1(got, ref["values"]) <= PR_TOL
            assert st.iterations == T and st.arcs_processed == T * g.m
        finally:
            gg.gg_free_graph(h)


@pytest.mark.parametrize("sigma", [0.1, 0.5, 0.9])
def test_pagerank_sp_exact_flags(gg, sigma):
    for g in _graphs()[:3]:
        h = gc.load(gg, g)
        try:
            got, mask, _ = gc.gpu_run(gg, h, g, "pagerank", "sp", sigma=sigma, T=20, seed=5)
            ref = oracle.run(g.n, g.rowptr, g.colidx, app="pagerank", policy="sp", sigma=sigma,
                             seed=5, max_iters=20)
            assert np.array_equal(mask, ref["mask"])
            assert gc.rel_l1(got, ref["values"]) <= PR_TOL
        finally:
            gg.gg_free_graph(h)


@pytest.mark.parametrize("policy,alpha,theta,sigma", [
    ("gg", 4, 0.05, 0.5), ("gg", 2, 0.3, 0.3), ("gg", 0, 0.5, 0.5), ("gg", 1, 0.8, 0.7),
    ("sms", 3, 0.1, 0.5), ("sms", 0, 0.05, 0.2), ("gg", 3, -0.5, 0.4)])
def test_pagerank_corrections_with_mask_replay(gg, policy, alpha, theta, sigma):
    for g in _graphs()[:4]:
        h = gc.load(gg, g)
        try:
            vals, ref, st = gc.pagerank_with_replay(gg, h, g, policy, sigma, alpha, theta, 20, seed=9)
            assert ref["replay_violations"] == 0, ref["replay_max_margin"]
            assert ref["replay_mismatch"] <= max(2, g.m // 10000)
            assert gc.rel_l1(vals, ref["values"]) <= PR_TOL
            assert st.corrections == len(gc.correction_indices(policy, alpha, 20))
        finally:
            gg.gg_free_graph(h)


def test_pagerank_deterministic(gg):
    g = graphgen.rmat(12, seed=1)
    h = gc.load(gg, g)
    try:
        a, ma, _ = gc.gpu_run(gg, h, g, "pagerank", "gg", sigma=0.5, alpha=2, theta=0.05, seed=3)
        b, mb, _ = gc.gpu_run(gg, h, g, "pagerank", "gg", sigma=0.5, alpha=2, theta=0.05, seed=3)
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)) and np.array_equal(ma, mb)
    finally:
        gg.gg_free_graph(h)


# ----------------------------------------------------- min applications --

MIN_CASES = [("exact", 4, 0.05, 1.0), ("sp", 4, 0.05, 0.3), ("sms", 2, 0.2, 0.5),
             ("gg", 3, 0.05, 0.3), ("gg", 1, 0.5, 0.5), ("gg", 0, 0.2, 0.4), ("gg", 2, -0.1, 0.3),
             ("gg", 2, 1.5, 0.6)]


# auto, GG_FORCE_PULL, GG_FORCE_PUSH, pull reading frontier sources only (GG_PULL_FILTER)
DIR_FLAGS = [0, 4, 8, 4 | 128]


@pytest.mark.parametrize("flags", DIR_FLAGS)
@pytest.mark.parametrize("app", ["sssp", "bfs"])
def test_traversal_bit_exact(gg, app, flags):
    for g in _graphs():
        h = gc.load(gg, g)
        try:
            srcs = graphgen.sources(g, 2, seed=2) if g.m else np.array([0])
            for policy, alpha, theta, sigma in MIN_CASES:
                for s in srcs:
                    got, mask, st = gc.gpu_run(gg, h, g, app, policy, sigma=sigma, alpha=alpha,
                                               theta=theta, T=100000, source=int(s), seed=7,
                                               flags=flags)
                    ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app=app, policy=policy,
                                     sigma=sigma, seed=7, alpha=alpha, theta=theta,
                                     max_iters=100000, source=int(s))
                    assert np.array_equal(got, ref["values"]), (g.name, policy, alpha, theta)
                    if mask is not None:
                        assert np.array_equal(mask, ref["mask"]), (g.name, policy, alpha, theta)
                    assert st.iterations == ref["iterations"]
                    assert st.corrections == ref["corrections"]
        finally:
            gg.gg_free_graph(h)


@pytest.mark.parametrize("flags", DIR_FLAGS)
def test_cc_bit_exact(gg, flags):
    for g in _sym_graphs():
        h = gc.load(gg, g)
        try:
            for policy, alpha, theta, sigma in MIN_CASES:
                got, mask, st = gc.gpu_run(gg, h, g, "cc", policy, sigma=sigma, alpha=alpha,
                                           theta=theta, T=100000, seed=7, flags=flags)
                ref = oracle.run(g.n, g.rowptr, g.colidx, app="cc", policy=policy, sigma=sigma,
                                 seed=7, alpha=alpha, theta=theta, max_iters=100000, symmetric=True)
                assert np.array_equal(got, ref["values"]), (g.name, policy)
                if mask is not None:
                    assert np.array_equal(mask, ref["mask"]), (g.name, policy)
                assert st.iterations == ref["iterations"]
        finally:
            gg.gg_free_graph(h)


@pytest.mark.parametrize("app", ["sssp", "bfs", "cc"])
def test_filtered_pull_marks_its_gathers(gg, app):
    """GG_PULL_FILTER: every pull gather reads frontier sources only (mode bit
    GG_ITER_FILTER), corrections never do; values, flags and per-iteration
    change counts equal the unfiltered pull's and the oracle's."""
    g = graphgen.rmat(14, seed=5, symmetric=app == "cc")
    graphgen.add_weights(g, seed=11)
    s = int(graphgen.sources(g, 1, seed=2)[0]) if app != "cc" else 0
    h = gc.load(gg, g)
    try:
        runs = {}
        for fl in (4 | 128, 4):
            p = gg.make_params(alpha=2, theta=0.05, max_iters=100000, source=s, seed=9, flags=fl)
            gg.gg_run(h, app, 0.4, "gg", p)
            runs[fl] = (gg.values(h, app), gg.mask_bits(h, g.m), gg.result_array(h, gg.GG_RESULT_ITER_STATS))
        ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app=app, policy="gg", sigma=0.4, seed=9, alpha=2,
                         theta=0.05, max_iters=100000, source=s, symmetric=app == "cc")
        for fl, (vals, mask, it) in runs.items():
            assert np.array_equal(vals, ref["values"]), fl
            assert np.array_equal(mask, ref["mask"]), fl
            kinds = it["mode"] & 3
            filt = (it["mode"] & gg.GG_ITER_FILTER) != 0
            if fl & 128:
                assert np.all(filt[kinds < 2]) and not np.any(filt[kinds == 2])
                assert np.any(kinds == 2) and np.any(kinds < 2)
            else:
                assert not np.any(filt)
        a, b = runs[4 | 128][2], runs[4][2]
        assert np.array_equal(a["changed"], b["changed"]) and np.array_equal(a["arcs"], b["arcs"])
    finally:
        gg.gg_free_graph(h)


def test_est_strict_and_iteration_cap(gg):
    g = graphgen.add_weights(graphgen.rmat(10, seed=8), seed=3)
    s = int(graphgen.sources(g, 1, seed=2)[0])
    h = gc.load(gg, g)
    try:
        for T in (1, 2, 5):
            got, mask, _ = gc.gpu_run(gg, h, g, "sssp", "gg", sigma=0.3, alpha=1, theta=0.1, T=T,
                                      source=s, seed=4, flags=gg.GG_EST_STRICT)
            ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", policy="gg",
                             sigma=0.3, seed=4, alpha=1, theta=0.1, max_iters=T, source=s,
                             flags=oracle.EST_STRICT)
            assert np.array_equal(got, ref["values"]) and np.array_equal(mask, ref["mask"])
    finally:
        gg.gg_free_graph(h)


# ------------------------------------------------------------- errors --

def test_errors_are_statuses(gg):
    g = graphgen.rmat(6, seed=1)
    bad = g.rowptr.copy()
    bad[5], bad[6] = bad[6] + 1, bad[5]
    with pytest.raises(gg.GGError) as e:
        gg.gg_load_csr(g.n, g.m, bad, g.colidx)
    assert e.value.status == gg.GG_ERR_BAD_GRAPH
    badc = g.colidx.copy()
    badc[3] = g.n
    with pytest.raises(gg.GGError) as e:
        gg.gg_load_csr(g.n, g.m, g.rowptr, badc)
    assert e.value.status == gg.GG_ERR_BAD_GRAPH
    with pytest.raises(gg.GGError) as e:
        gg.gg_load_csr(0, 0, g.rowptr, g.colidx)
    assert e.value.status == gg.GG_ERR_INVALID_ARG
    h = gc.load(gg, g)
    try:
        with pytest.raises(gg.GGError) as e:
            gg.gg_result(h, gg.GG_RESULT_VALUES, np.empty(g.n, np.float32), 4 * g.n)
        assert e.value.status == gg.GG_ERR_STATE
        with pytest.raises(gg.GGError) as e:
            gg.gg_run(h, "sssp", 0.5, "gg", gg.make_params())   # no weights
        assert e.value.status == gg.GG_ERR_INVALID_ARG
        with pytest.raises(gg.GGError) as e:
            gg.gg_run(h, "bfs", 0.5, "gg", gg.make_params(source=g.n))
        assert e.value.status == gg.GG_ERR_INVALID_ARG
        with pytest.raises(gg.GGError) as e:
            gg.gg_sample_edges(h, 0.0, 1)
        assert e.value.status == gg.GG_ERR_INVALID_ARG
        with pytest.raises(gg.GGError) as e:
            gg.gg_run(h, "pagerank", 1.5, "gg", gg.make_params())
        assert e.value.status == gg.GG_ERR_INVALID_ARG
        gg.gg_run(h, "pagerank", 0.5, "gg", gg.make_params(max_iters=3))
        with pytest.raises(gg.GGError) as e:
            gg.gg_result(h, gg.GG_RESULT_VALUES, np.empty(2, np.float32), 8)
        assert e.value.status == gg.GG_ERR_INVALID_ARG
    finally:
        gg.gg_free_graph(h)


@pytest.mark.parametrize("flags", [32, 64, 96])   # GG_INFL_SHARE, GG_RENORM, both
@pytest.mark.parametrize("policy,alpha,theta,sigma", [("sp", 4, 0.05, 0.5), ("gg", 2, 0.01, 0.4),
                                                       ("gg", 0, 0.1, 0.3), ("sms", 3, 0.02, 0.6)])
def test_pagerank_share_and_renorm_variants(gg, flags, policy, alpha, theta, sigma):
    for g in _graphs()[:4]:
        h = gc.load(gg, g)
        try:
            masks = []
            for c in gc.correction_indices(policy, alpha, 20):
                _, mk, _ = gc.gpu_run(gg, h, g, "pagerank", policy, sigma, alpha, theta, T=c + 1, seed=9,
                                      flags=flags)
                masks.append(mk)
            vals, _, _ = gc.gpu_run(gg, h, g, "pagerank", policy, sigma, alpha, theta, T=20, seed=9,
                                    flags=flags)
            ref = oracle.run(g.n, g.rowptr, g.colidx, app="pagerank", policy=policy, sigma=sigma, seed=9,
                             alpha=alpha, theta=theta, max_iters=20, flags=flags, replay_masks=masks,
                             replay_tol=1e-5, nthreads=0)
            assert ref["replay_violations"] == 0, ref["replay_max_margin"]
            assert gc.rel_l1(vals, ref["values"]) <= PR_TOL
        finally:
            gg.gg_free_graph(h)

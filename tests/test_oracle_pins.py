"""Pins of the oracle against facts fixed outside it: published known-answer
values, textbook algorithms on tiny graphs, closed forms, the paper's special
cases and invariants that hold exactly. CPU only."""
import os

import numpy as np
import pytest

import graphgen
import oracle
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_hex(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def _small_graphs(weighted=False, symmetric=False):
    gs = []
    for seed in (1, 2, 3):
        g = graphgen.rmat(5, edgefactor=4, seed=seed, symmetric=symmetric)
        gs.append(g)
        g2 = graphgen.erdos_renyi(48, avg_degree=3, seed=seed, symmetric=symmetric)
        gs.append(g2)
    if weighted:
        for g in gs:
            graphgen.add_weights(g, seed=11)
    return gs


# ---------------------------------------------------------------- sampler --

def test_splitmix64_known_answers():
    gamma = 0x9E3779B97F4A7C15
    want = [int(r[0], 16) for r in _golden_hex("splitmix64_seed0.txt")]
    got = [oracle.splitmix64((k * gamma) & 0xFFFFFFFFFFFFFFFF) for k in range(3)]
    assert got == want


def test_sampling_key_layout_pinned_by_known_answer():
    # h(0) = 0xe220a839..., so the flag of the all-zero key flips between
    # sigma = 0.8833 and 0.8834; seed XOR (src<<32 | dst) must reach it.
    top = 0xE220A839 / 2**32
    lo, hi = top - 1e-6, top + 1e-6
    assert not oracle.arc_sampled(0, 0, lo, 0)
    assert oracle.arc_sampled(0, 0, hi, 0)
    for src, dst in [(1, 2), (7, 0), (0, 9), (123456, 654321)]:
        seed = (src << 32) | dst
        assert not oracle.arc_sampled(src, dst, lo, seed)
        assert oracle.arc_sampled(src, dst, hi, seed)
        # symmetric keying orders the pair (min, max)
        assert oracle.arc_sampled(dst, src, hi, seed, symmetric=True) == \
            oracle.arc_sampled(min(src, dst), max(src, dst), hi, seed, symmetric=True)


def test_sampling_fraction_nesting_and_symmetry():
    g = graphgen.rmat(12, seed=1)
    in_ptr, in_src, _, _ = oracle.csc_from_csr(g.n, g.rowptr, g.colidx)
    m = g.m
    prev = None
    for sigma in (0.1, 0.3, 0.5, 0.7, 0.9, 1.0):
        mask = oracle.sample_mask(g.n, in_ptr, in_src, sigma, seed=99)
        k = int(mask.sum())
        sd = np.sqrt(m * sigma * (1 - sigma))
        assert abs(k - sigma * m) <= 5 * sd + 1e-9, (sigma, k)
        if prev is not None:               # a larger sigma keeps every arc
            assert np.all(mask >= prev)
        prev = mask
    assert prev.all()
    gs = graphgen.rmat(10, seed=3, symmetric=True)
    ip, isrc, _, _ = oracle.csc_from_csr(gs.n, gs.rowptr, gs.colidx)
    mk = oracle.sample_mask(gs.n, ip, isrc, 0.5, seed=5, symmetric=True)
    dst = np.repeat(np.arange(gs.n), np.diff(ip))
    flags = {}
    for s, d, f in zip(isrc, dst, mk):
        key = (min(s, d), max(s, d))
        assert flags.setdefault(key, f) == f


# -------------------------------------------------------------- transpose --

def test_csc_matches_stable_sort():
    for g in _small_graphs(weighted=True) + [graphgen.rmat(12, seed=1)]:
        in_ptr, in_src, in_w, pos = oracle.csc_from_csr(g.n, g.rowptr, g.colidx, g.weights)
        src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
        order = np.argsort(g.colidx, kind="stable")
        assert np.array_equal(in_src, src[order])
        assert np.array_equal(pos, order)
        if g.weights is not None:
            assert np.array_equal(in_w, g.weights[order])
        assert np.array_equal(in_ptr, np.concatenate([[0], np.cumsum(np.bincount(g.colidx, minlength=g.n))]))
        for u in range(min(g.n, 200)):
            row = in_src[in_ptr[u]:in_ptr[u + 1]]
            assert np.all(np.diff(row) >= 0)


# --------------------------------------------------------------- schedule --

def test_schedules():
    A, X, C = oracle.MODE_APPROX, oracle.MODE_ACCURATE, oracle.MODE_CORRECTION
    assert [oracle.iteration_mode("adaptive", 2, i) for i in range(9)] == [A, A, C] * 3
    assert [oracle.iteration_mode("adaptive", 0, i) for i in range(4)] == [C] * 4
    assert [oracle.iteration_mode("sms", 3, i) for i in range(7)] == [A, A, A, C, X, X, X]
    assert [oracle.iteration_mode("sp", 3, i) for i in range(5)] == [A] * 5
    assert [oracle.iteration_mode("exact", 3, i) for i in range(5)] == [X] * 5


# -------------------------------------------------------------- pagerank --

@pytest.mark.parametrize("T", [1, 2, 7, 20])
def test_pagerank_exact_matches_dense_power_iteration(T):
    for g in _small_graphs():
        r = oracle.run(g.n, g.rowptr, g.colidx, app="pagerank", policy="exact", max_iters=T)
        ref = brute.pagerank_dense(g, 0.85, T)
        assert np.abs(r["values"] - ref).sum() / np.abs(ref).sum() < 1e-13


def test_pagerank_uniform_rank_invariant():
    n = 37
    cycle = graphgen.from_arcs(n, [(i, (i + 1) % n) for i in range(n)])
    complete = graphgen.from_arcs(9, [(i, j) for i in range(9) for j in range(9) if i != j])
    for g in (cycle, complete):
        for T in (1, 5, 20):
            r = oracle.run(g.n, g.rowptr, g.colidx, app="pagerank", max_iters=T)
            assert np.allclose(r["values"], 1.0 / g.n, rtol=1e-14, atol=0)


def test_pagerank_star_and_path_closed_forms():
    d = float(np.float32(0.85))
    n = 11
    star = graphgen.from_arcs(n, [(i, 0) for i in range(1, n)])
    base = (1 - d) / n
    for T in (1, 2, 3, 10):
        v = oracle.run(n, star.rowptr, star.colidx, max_iters=T)["values"]
        assert np.allclose(v[1:], base, rtol=1e-14)
        hub = base + d * (n - 1) * (1.0 / n if T == 1 else base)
        assert v[0] == pytest.approx(hub, rel=1e-14)
    n = 9
    path = graphgen.from_arcs(n, [(i, i + 1) for i in range(n - 1)])
    base = (1 - d) / n
    for T in (1, 3, 8, 15):
        v = oracle.run(n, path.rowptr, path.colidx, max_iters=T)["values"]
        for k in range(n):
            if T <= k:
                want = base * (1 - d ** T) / (1 - d) + d ** T / n
            else:
                want = base * (1 - d ** (k + 1)) / (1 - d)
            assert v[k] == pytest.approx(want, rel=1e-13), (T, k)


def test_pagerank_influence_hand_example():
    # Vertex 3 has in-arcs from 0 and 1. Vertex 0 has out-degree 3 and vertex
    # 1 out-degree 1, so at iteration 0 (ranks 1/N) the contributions in CSC
    # order are c and 3c: influence 1 for 0->3, 3c/(c+3c) = 0.75 for 1->3.
    arcs = [(0, 3), (0, 4), (0, 5), (1, 3), (2, 0)]
    g = graphgen.from_arcs(6, arcs)
    in_ptr, in_src, _, _ = oracle.csc_from_csr(g.n, g.rowptr, g.colidx)
    k03 = in_ptr[3] + list(in_src[in_ptr[3]:in_ptr[4]]).index(0)
    k13 = in_ptr[3] + list(in_src[in_ptr[3]:in_ptr[4]]).index(1)
    for theta, want13 in ((0.8, 0), (0.74, 1)):
        r = oracle.run(g.n, g.rowptr, g.colidx, policy="sms", alpha=0, theta=theta,
                       max_iters=1, sigma=0.5, seed=3)
        assert r["mask"][k03] == 1 and r["mask"][k13] == want13
    # Reversed ids: the heavy source comes first, the light one gets
    # influence c/(3c+c) = 0.25.
    arcs = [(1, 3), (1, 4), (1, 5), (0, 3), (2, 1)]
    g = graphgen.from_arcs(6, arcs)
    in_ptr, in_src, _, _ = oracle.csc_from_csr(g.n, g.rowptr, g.colidx)
    k03 = in_ptr[3] + list(in_src[in_ptr[3]:in_ptr[4]]).index(0)
    k13 = in_ptr[3] + list(in_src[in_ptr[3]:in_ptr[4]]).index(1)
    for theta, want13 in ((0.26, 0), (0.24, 1)):
        r = oracle.run(g.n, g.rowptr, g.colidx, policy="sms", alpha=0, theta=theta, max_iters=1)
        assert r["mask"][k03] == 1 and r["mask"][k13] == want13


def test_pagerank_approximate_is_below_exact():
    for g in _small_graphs() + [graphgen.rmat(10, seed=4)]:
        ex = oracle.run(g.n, g.rowptr, g.colidx, max_iters=12)["values"]
        for policy in ("sp", "sms", "gg"):
            ap = oracle.run(g.n, g.rowptr, g.colidx, policy=policy, sigma=0.4, seed=8,
                            alpha=3, theta=0.3, max_iters=12)["values"]
            assert np.all(ap <= ex * (1 + 1e-12))


# --------------------------------------------------------- min applications --

def test_sssp_bfs_exact_match_textbook():
    for g in _small_graphs(weighted=True):
        srcs = graphgen.sources(g, 3, seed=2)
        for s in srcs:
            r = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", source=int(s),
                           max_iters=1000)
            assert np.array_equal(r["values"], brute.dijkstra(g, int(s)))
            r = oracle.run(g.n, g.rowptr, g.colidx, app="bfs", source=int(s), max_iters=1000)
            assert np.array_equal(r["values"], brute.bfs_levels(g, int(s)))


def test_cc_exact_matches_union_find():
    for g in _small_graphs(symmetric=True):
        r = oracle.run(g.n, g.rowptr, g.colidx, app="cc", max_iters=1000, symmetric=True)
        assert np.array_equal(r["values"], brute.cc_min_labels(g))


def test_min_app_approximations_are_upper_bounds_of_real_paths():
    for g in _small_graphs(weighted=True):
        s = int(graphgen.sources(g, 1, seed=2)[0])
        exact = brute.dijkstra(g, s).astype(np.int64)
        arcs = brute.arcs_of(g)
        for policy in ("sp", "gg", "sms"):
            r = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", policy=policy,
                           sigma=0.3, seed=4, alpha=2, theta=0.2, source=s, max_iters=1000)
            v = r["values"].astype(np.int64)
            assert np.all(v >= exact)
            # every finite value other than the source's is realised by an
            # arc from a vertex whose value plus the weight is at most it
            ok = np.zeros(g.n, bool)
            ok[s] = v[s] == 0
            for a, b, w in arcs:
                if v[a] != brute.INF and v[b] != brute.INF and v[a] + w <= v[b]:
                    ok[b] = True
            assert np.all(ok | (v == brute.INF))
    for g in _small_graphs(symmetric=True):
        exact = brute.cc_min_labels(g)
        r = oracle.run(g.n, g.rowptr, g.colidx, app="cc", policy="sp", sigma=0.3, seed=4,
                       max_iters=1000, symmetric=True)
        lab = r["values"]
        assert np.all(lab >= exact)
        assert np.all(exact[lab] == exact)     # label is a vertex of the same component


# ----------------------------------------------------------- special cases --

@pytest.mark.parametrize("app", ["pagerank", "sssp", "bfs"])
def test_special_cases_reduce_to_exact(app):
    for g in _small_graphs(weighted=True):
        s = int(graphgen.sources(g, 1, seed=2)[0])
        T = 12 if app == "pagerank" else 1000
        kw = dict(app=app, source=s, max_iters=T)
        ex = oracle.run(g.n, g.rowptr, g.colidx, g.weights, **kw)["values"]
        same = [
            oracle.run(g.n, g.rowptr, g.colidx, g.weights, policy="sp", sigma=1.0, **kw),
            oracle.run(g.n, g.rowptr, g.colidx, g.weights, policy="sms", alpha=0, sigma=0.3, **kw),
            oracle.run(g.n, g.rowptr, g.colidx, g.weights, policy="gg", alpha=0, sigma=0.3, **kw),
        ]
        for r in same:
            assert np.array_equal(r["values"], ex)


def test_negative_theta_reactivates_every_arc():
    g = graphgen.rmat(9, seed=5)
    r = oracle.run(g.n, g.rowptr, g.colidx, policy="gg", sigma=0.2, alpha=2, theta=-1e-3,
                   max_iters=3)
    assert r["corrections"] == 1 and r["mask"].all()


def test_dumbbell_bridge_restored_by_correction():
    # Two 5-cliques {0..4} and {5..9} joined by the bridge 4-5 (Fig. 1b).
    arcs = [(i, j) for i in range(5) for j in range(5) if i != j]
    arcs += [(i, j) for i in range(5, 10) for j in range(5, 10) if i != j]
    arcs += [(4, 5), (5, 4)]
    g = graphgen.from_arcs(10, arcs, symmetric=True)
    def split_in_two(s):
        # bridge dropped, and the sampled arcs still connect each clique
        kept = [(a, b) for a, b in arcs if oracle.arc_sampled(a, b, 0.5, s, symmetric=True)]
        lab = brute.cc_min_labels(graphgen.from_arcs(10, kept))
        return lab.tolist() == [0] * 5 + [5] * 5

    seed = next(s for s in range(1000) if split_in_two(s))
    sp = oracle.run(g.n, g.rowptr, g.colidx, app="cc", policy="sp", sigma=0.5, seed=seed,
                    symmetric=True, max_iters=100)
    assert len(set(sp["values"].tolist())) == 2
    gg = oracle.run(g.n, g.rowptr, g.colidx, app="cc", policy="gg", sigma=0.5, seed=seed,
                    alpha=2, theta=0.5, symmetric=True, max_iters=100)
    assert set(gg["values"].tolist()) == {0}


# ------------------------------------------------------------- mask replay --

def test_mask_replay_of_own_masks_and_planted_flip():
    g = graphgen.rmat(10, seed=6)
    kw = dict(policy="gg", sigma=0.5, seed=2, alpha=2, theta=0.1)
    masks = []
    for k in range(3):
        masks.append(oracle.run(g.n, g.rowptr, g.colidx, max_iters=3 * (k + 1), **kw)["mask"])
    ref = oracle.run(g.n, g.rowptr, g.colidx, max_iters=9, **kw)
    rep = oracle.run(g.n, g.rowptr, g.colidx, max_iters=9, replay_masks=masks, **kw)
    assert rep["replay_mismatch"] == 0 and np.array_equal(rep["values"], ref["values"])
    bad = [m.copy() for m in masks]
    first_active = int(np.flatnonzero(bad[0])[0])   # a first in-arc: influence 1
    bad[0][first_active] ^= 1
    rep = oracle.run(g.n, g.rowptr, g.colidx, max_iters=9, replay_masks=bad, **kw)
    assert rep["replay_mismatch"] >= 1 and rep["replay_violations"] >= 1


def _csc_index(g, src, dst):
    in_ptr, in_src, _, _ = oracle.csc_from_csr(g.n, g.rowptr, g.colidx)
    row = list(in_src[in_ptr[dst]:in_ptr[dst + 1]])
    return int(in_ptr[dst] + row.index(src))


def test_sssp_influence_hand_example():
    # Source 0; after iteration 0, dist = 5, 1, 1 at vertices 1, 2, 3. In the
    # correction (iteration 1) vertex 4 sees, in source order, candidates
    # 10 (first: influence 1), 8 (lowers 10: influence 0.2) and 9 (lowers
    # nothing: 0). Arc 5->4 comes from an unreached vertex: no candidate.
    arcs = [(0, 1, 5), (0, 2, 1), (0, 3, 1), (1, 4, 5), (2, 4, 7), (3, 4, 8), (5, 4, 1)]
    g = graphgen.from_arcs(6, [(a, b) for a, b, _ in arcs], weights=[w for _, _, w in arcs])
    k14, k24, k34, k54 = (_csc_index(g, s, 4) for s in (1, 2, 3, 5))
    for theta, want in ((0.15, [1, 1, 0]), (0.25, [1, 0, 0]), (-0.5, [1, 1, 1])):
        r = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", policy="sms", alpha=1,
                       theta=theta, sigma=1.0, source=0, max_iters=2)
        assert [r["mask"][k] for k in (k14, k24, k34)] == want
        assert r["mask"][k54] == 1                 # unevaluated arc keeps its flag
    r = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", policy="sms", alpha=1,
                   theta=0.15, sigma=1.0, source=0, max_iters=2, flags=oracle.EST_STRICT)
    assert r["mask"][k54] == 0
    assert r["values"].tolist()[:5] == [0, 5, 1, 1, 8]


def test_cc_influence_is_binary():
    # Iteration 0 gives labels 3, 1, 2 to vertices 4, 5, 6 (neighbours of 3,
    # 1, 2). In the correction vertex 9 sees candidates 3 (first), 1 (lowers
    # the running label: influence 1, not 2/3) and 2 (lowers nothing).
    pairs = [(3, 4), (1, 5), (2, 6), (4, 9), (5, 9), (6, 9)]
    arcs = pairs + [(b, a) for a, b in pairs]
    g = graphgen.from_arcs(10, arcs, symmetric=True)
    k = [_csc_index(g, s, 9) for s in (4, 5, 6)]
    r = oracle.run(g.n, g.rowptr, g.colidx, app="cc", policy="sms", alpha=1, theta=0.7,
                   sigma=1.0, max_iters=2, symmetric=True)
    assert [r["mask"][x] for x in k] == [1, 1, 0]


def test_influence_share_is_order_free():
    # Contributions c (source of out-degree 3) and 3c (out-degree 1) into
    # vertex 3: shares 1/4 and 3/4 whichever source id comes first.
    for arcs, light, heavy in (([(0, 3), (0, 4), (0, 5), (1, 3), (2, 0)], 0, 1),
                               ([(1, 3), (1, 4), (1, 5), (0, 3), (2, 1)], 1, 0)):
        g = graphgen.from_arcs(6, arcs)
        kl, kh = _csc_index(g, light, 3), _csc_index(g, heavy, 3)
        for theta, want in ((0.5, (0, 1)), (0.2, (1, 1)), (0.8, (0, 0))):
            r = oracle.run(g.n, g.rowptr, g.colidx, policy="sms", alpha=0, theta=theta, max_iters=1,
                           flags=oracle.INFL_SHARE)
            assert (r["mask"][kl], r["mask"][kh]) == want


def test_renormalised_sp_equals_pagerank_of_the_sampled_subgraph():
    for g in _small_graphs() + [graphgen.rmat(8, seed=9)]:
        sigma, seed = 0.5, 21
        kept = [(s, d) for s, d, _ in brute.arcs_of(g) if oracle.arc_sampled(s, d, sigma, seed)]
        sub = graphgen.from_arcs(g.n, kept)
        for T in (1, 5, 12):
            r = oracle.run(g.n, g.rowptr, g.colidx, policy="sp", sigma=sigma, seed=seed, max_iters=T,
                           flags=oracle.RENORM)
            ref = brute.pagerank_dense(sub, 0.85, T)
            assert np.abs(r["values"] - ref).sum() / np.abs(ref).sum() < 1e-13


# ------------------------------------------------ triggered corrections --

def _broom():
    # BFS levels of sizes 1, 8, 4, 2, 1 from vertex 0: iteration i of a run
    # on all arcs changes exactly the vertices of level i + 1.
    arcs = [(0, v) for v in range(1, 9)] + [(1, 9), (2, 10), (3, 11), (4, 12), (9, 13), (10, 14),
                                             (13, 15)]
    return graphgen.from_arcs(16, arcs)


@pytest.mark.parametrize("ratio,alpha,modes", [
    # changed per iteration 8, 4, 2, 1, 0: 4 <= 0.5 * 8 triggers after the
    # second; the next window starts at 1 and triggers when it reaches 0
    (0.5, 10, "AACAAC"),
    (0.4, 10, "AAACAC"),     # 2 <= 0.4 * 8 after the third
    (0.0, 3, "AAACAC"),      # only the window length (3), then the quiet iteration
    (0.0, 2, "AACAAC"),
    (2.0, 10, "ACACAC"),     # a ratio >= 1 triggers after every approximate iteration
])
def test_triggered_schedule_hand_example(ratio, alpha, modes):
    g = _broom()
    r = oracle.run(g.n, g.rowptr, g.colidx, app="bfs", policy="triggered", sigma=1.0, alpha=alpha,
                   trigger_ratio=ratio, source=0, max_iters=50)
    code = {oracle.MODE_APPROX: "A", oracle.MODE_CORRECTION: "C"}
    assert "".join(code[int(x)] for x in r["iter_mode"]) == modes
    assert list(r["iter_changed"]) == [8, 4, 2, 1, 0, 0]
    assert np.array_equal(r["values"], brute.bfs_levels(g, 0))


def _trigger_rule_holds(r, alpha, ratio, pagerank):
    """Every mode of the run follows the triggered rule from the run's own
    per-iteration change statistics."""
    A, C = oracle.MODE_APPROX, oracle.MODE_CORRECTION
    modes = [int(x) for x in r["iter_mode"]]
    stat = r["iter_sum_delta"] if pagerank else r["iter_changed"]
    ratio = float(np.float32(ratio))
    want_c = alpha == 0
    window, first = 0, 0.0
    for i, md in enumerate(modes):
        assert md == (C if want_c else A), (i, modes)
        if md == C:
            window, want_c = 0, alpha == 0
        else:
            window += 1
            if window == 1:
                first = float(stat[i])
            want_c = window >= alpha or float(stat[i]) <= ratio * first


@pytest.mark.parametrize("app", ["pagerank", "sssp", "bfs", "cc"])
def test_triggered_schedule_follows_its_rule(app):
    sym = app == "cc"
    for g in _small_graphs(weighted=True, symmetric=sym) + [graphgen.rmat(9, seed=3, symmetric=sym)]:
        if g.weights is None:
            graphgen.add_weights(g, seed=11)
        s = int(graphgen.sources(g, 1, seed=2)[0])
        for alpha, ratio in ((4, 0.5), (6, 0.2), (1, 0.0), (0, 0.5)):
            r = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app=app, policy="triggered", sigma=0.4,
                           seed=3, alpha=alpha, theta=0.1, trigger_ratio=ratio, source=s,
                           max_iters=15 if app == "pagerank" else 1000, symmetric=sym)
            _trigger_rule_holds(r, alpha, ratio, app == "pagerank")


def test_triggered_special_cases_reduce_to_adaptive():
    for g in _small_graphs(weighted=True):
        s = int(graphgen.sources(g, 1, seed=2)[0])
        for app, T in (("pagerank", 12), ("sssp", 1000), ("bfs", 1000)):
            kw = dict(app=app, source=s, max_iters=T, sigma=0.3, seed=5, theta=0.1)
            for alpha_gg, alpha_tr, ratio in ((0, 0, 0.5), (1, 1, 0.0), (1, 5, 1.0), (1, 3, 7.0)):
                gg = oracle.run(g.n, g.rowptr, g.colidx, g.weights, policy="gg", alpha=alpha_gg, **kw)
                tr = oracle.run(g.n, g.rowptr, g.colidx, g.weights, policy="triggered", alpha=alpha_tr,
                                trigger_ratio=ratio, **kw)
                assert np.array_equal(tr["values"], gg["values"]), (app, alpha_tr, ratio)
                assert np.array_equal(tr["mask"], gg["mask"])


def test_triggered_min_apps_reach_the_exact_fixed_point():
    for g in _small_graphs(weighted=True):
        s = int(graphgen.sources(g, 1, seed=2)[0])
        r = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", policy="triggered", sigma=0.3,
                       seed=6, alpha=5, theta=0.3, trigger_ratio=0.3, source=s, max_iters=1000)
        assert np.array_equal(r["values"], brute.dijkstra(g, s))
    for g in _small_graphs(symmetric=True):
        r = oracle.run(g.n, g.rowptr, g.colidx, app="cc", policy="triggered", sigma=0.3, seed=6,
                       alpha=5, theta=0.3, trigger_ratio=0.3, max_iters=1000, symmetric=True)
        assert np.array_equal(r["values"], brute.cc_min_labels(g))


def test_replayed_modes_reproduce_the_run():
    g = graphgen.rmat(8, seed=4)
    for policy, alpha in (("gg", 3), ("sms", 4), ("triggered", 5)):
        r = oracle.run(g.n, g.rowptr, g.colidx, policy=policy, sigma=0.4, seed=2, alpha=alpha,
                       theta=0.05, trigger_ratio=0.5, max_iters=14)
        rr = oracle.run(g.n, g.rowptr, g.colidx, policy="triggered", sigma=0.4, seed=2, alpha=1,
                        theta=0.05, trigger_ratio=0.0, max_iters=14, replay_modes=r["iter_mode"])
        assert np.array_equal(rr["iter_mode"], r["iter_mode"])
        assert np.array_equal(rr["values"], r["values"]) and np.array_equal(rr["mask"], r["mask"])


# ------------------------------------------------- personalized PageRank --

def test_ppr_matches_dense_power_iteration():
    for g in _small_graphs()[:4]:
        for s in (0, g.n - 1):
            for T in (1, 3, 12):
                r = oracle.run(g.n, g.rowptr, g.colidx, app="ppr", source=s, max_iters=T)
                ref = brute.ppr_dense(g, 0.85, T, s)
                assert np.abs(r["values"] - ref).sum() <= 1e-13 * max(np.abs(ref).sum(), 1e-300)


def test_ppr_path_closed_form():
    g = graphgen.from_arcs(4, [(0, 1), (1, 2), (2, 3)])
    d = float(np.float32(0.85))
    r = oracle.run(g.n, g.rowptr, g.colidx, app="ppr", source=0, max_iters=2)
    assert np.allclose(r["values"], [1 - d, d * (1 - d), d * d, 0.0], rtol=0, atol=1e-15)
    # T = 3 puts d^3 on vertex 3, which has no out-arcs: that mass leaves
    # (no dangling redistribution), so T = 4 holds d^3 (1-d) there
    r = oracle.run(g.n, g.rowptr, g.colidx, app="ppr", source=0, max_iters=3)
    assert np.allclose(r["values"], [1 - d, d * (1 - d), d * d * (1 - d), d ** 3], rtol=0, atol=1e-15)
    r = oracle.run(g.n, g.rowptr, g.colidx, app="ppr", source=0, max_iters=4)
    assert np.allclose(r["values"], [1 - d, d * (1 - d), d * d * (1 - d), d ** 3 * (1 - d)], rtol=0, atol=1e-15)


def test_ppr_averaged_over_sources_is_pagerank():
    # rank_t is linear in the restart and starting vectors: the mean of the
    # personalized vectors over every source is the global PageRank
    g = graphgen.rmat(6, edgefactor=4, seed=2)
    for T in (1, 4, 10):
        mean = np.zeros(g.n)
        for s in range(g.n):
            mean += oracle.run(g.n, g.rowptr, g.colidx, app="ppr", source=s, max_iters=T)["values"]
        mean /= g.n
        pr = oracle.run(g.n, g.rowptr, g.colidx, app="pagerank", max_iters=T)["values"]
        assert np.abs(mean - pr).sum() <= 1e-13


# ------------------------------------- GraphGuess PageRank, exact rationals --

@pytest.mark.parametrize("policy,variant", [("gg", 0), ("sms", 0), ("gg", oracle.RENORM),
                                            ("gg", oracle.INFL_SHARE), ("sms", oracle.RENORM | oracle.INFL_SHARE)])
def test_graphguess_pagerank_matches_rational_replica(policy, variant):
    # Approximate iterations after a correction depend on the flags the
    # correction chose; a replica in exact rational arithmetic (a different
    # program: sorted arc list, fractions, dense passes) pins the oracle's
    # values and flags through several corrections.
    rng = np.random.default_rng(5)
    checked = 0
    for trial in range(12):
        n = int(rng.integers(3, 9))
        m = int(rng.integers(n, 3 * n))
        arcs = [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(m)]
        g = graphgen.from_arcs(n, arcs)
        sigma, seed = (0.4, 0.7)[trial % 2], 30 + trial
        init = {e: int(oracle.arc_sampled(s, d, sigma, seed)) for e, (s, d, _) in enumerate(brute.arcs_of(g))}
        for alpha, theta, iters in ((1, 0.3071, 7), (2, 0.1193, 9), (0, 0.5517, 4)):
            want, want_flags, margin = brute.graphguess_pagerank_rational(
                g, 0.85, iters, init, alpha, theta, policy,
                renorm=bool(variant & oracle.RENORM), share=bool(variant & oracle.INFL_SHARE))
            if margin is not None and margin < 1e-9:
                continue   # an influence within rounding of theta: FP64 may decide it either way
            r = oracle.run(g.n, g.rowptr, g.colidx, policy=policy, sigma=sigma, seed=seed, alpha=alpha,
                           theta=theta, max_iters=iters, flags=variant)
            assert np.abs(r["values"] - want).sum() <= 1e-13 * np.abs(want).sum(), (trial, alpha)
            assert np.array_equal(np.asarray(r["mask"], np.uint8), want_flags), (trial, alpha)
            checked += 1
    assert checked >= 30


@pytest.mark.parametrize("app", ["sssp", "bfs", "cc"])
def test_graphguess_min_apps_match_replica(app):
    # Values and flags of the min applications through corrections under the
    # GG, SMS and SP schedules, against a replica with unbounded integers and
    # exact-fraction influence.
    rng = np.random.default_rng(11)
    checked = 0
    for trial in range(16):
        n = int(rng.integers(3, 12))
        m = int(rng.integers(n, 4 * n))
        arcs = [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(m)]
        g = graphgen.from_arcs(n, arcs, symmetric=(app == "cc"))
        w = rng.integers(1, 256, g.m).astype(np.uint32)
        if app == "cc":
            w = np.ones(g.m, np.uint32)
        g.weights = w
        sigma, seed = (0.3, 0.6, 0.9)[trial % 3], 70 + trial
        src = int(rng.integers(0, n))
        init = {e: int(oracle.arc_sampled(s, d, sigma, seed, symmetric=g.symmetric))
                for e, (s, d, _) in enumerate(brute.arcs_of(g))}
        for policy, alpha, theta, strict in (("gg", 1, 0.05, False), ("gg", 2, 0.2, False), ("gg", 0, 0.5, True),
                                             ("sms", 2, 0.125, False), ("sp", 0, 0.05, False)):
            # to the fixed point, and cut after 2 and 4 iterations (the states
            # on the way depend on the schedule; the fixed point does not)
            for iters in (200, 2, 4):
                want, want_flags = brute.graphguess_min_replica(g, app, src, iters, init, alpha, theta, policy, strict)
                r = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app=app, policy=policy, sigma=sigma, seed=seed,
                               alpha=alpha, theta=theta, max_iters=iters, source=src, symmetric=g.symmetric,
                               flags=oracle.EST_STRICT if strict else 0)
                assert np.array_equal(r["values"], want), (trial, policy, alpha, iters)
                assert np.array_equal(np.asarray(r["mask"], np.uint8), want_flags), (trial, policy, alpha, iters)
                checked += 1
    assert checked == 240

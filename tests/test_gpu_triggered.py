"""GPU parity of the statistics-triggered correction policy
(GG_POLICY_TRIGGERED): corrections follow the approximate iteration whose
change statistic falls to trigger_ratio x the window's first, or the alpha-th
approximate iteration of the window.

SSSP / BFS / CC decide on the exact count of changed vertices, so values,
flags and the whole iteration schedule are bit-exact against the oracle.
PageRank decides on sum |old-new| in fixed point (2^-40) over FP32 ranks:
the test checks that the GPU's schedule follows the rule on its own
statistics, that those statistics match the FP64 oracle's, and that the
oracle, replaying the GPU's schedule and post-correction flags, lands
within 1e-5 relative L1 of the GPU's ranks.
"""
import numpy as np
import pytest

import graphgen
import oracle
from tests import gpu_common as gc
from tests.test_gpu_parity import _graphs, _sym_graphs

pytestmark = pytest.mark.gpu

PR_TOL = 1e-5
FX = 2.0 ** -40
CASES = [(4, 0.5), (8, 0.1), (1, 0.0), (0, 0.5), (30, 0.3)]


@pytest.fixture(scope="module")
def gg():
    return gc.lib()


def _modes(gg, h):
    return gg.result_array(h, gg.GG_RESULT_ITER_STATS)


@pytest.mark.parametrize("flags", [0, 4])   # auto pull/push, GG_FORCE_PULL
@pytest.mark.parametrize("app", ["sssp", "bfs", "cc"])
def test_triggered_min_apps_bit_exact(gg, app, flags):
    graphs = _sym_graphs() if app == "cc" else _graphs()
    for g in graphs:
        h = gc.load(gg, g)
        try:
            srcs = graphgen.sources(g, 2, seed=5) if (g.m and app != "cc") else np.array([0])
            for alpha, ratio in CASES:
                for s in srcs:
                    got, mask, st = gc.gpu_run(gg, h, g, app, "triggered", sigma=0.4, alpha=alpha,
                                               theta=0.2, T=100000, source=int(s), seed=3, flags=flags,
                                               trigger_ratio=ratio)
                    it = _modes(gg, h)
                    ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app=app, policy="triggered",
                                     sigma=0.4, seed=3, alpha=alpha, theta=0.2, trigger_ratio=ratio,
                                     max_iters=100000, source=int(s), symmetric=app == "cc")
                    case = (g.name, alpha, ratio, int(s))
                    assert np.array_equal(got, ref["values"]), case
                    assert np.array_equal(mask, ref["mask"]), case
                    assert st.iterations == ref["iterations"] and st.corrections == ref["corrections"]
                    assert np.array_equal(it["mode"] & 3, ref["iter_mode"].astype(np.uint32)), case
                    assert np.array_equal(it["changed"], ref["iter_changed"].astype(np.uint64)), case
        finally:
            gg.gg_free_graph(h)


def _check_rule(modes, stat, alpha, ratio):
    ratio = float(np.float32(ratio))
    want_c, window, first = alpha == 0, 0, 0.0
    for i, md in enumerate(modes):
        assert md == (2 if want_c else 0), (i, list(modes))
        if md == 2:
            window, want_c = 0, alpha == 0
        else:
            window += 1
            if window == 1:
                first = float(stat[i])
            want_c = window >= alpha or float(stat[i]) <= ratio * first


@pytest.mark.parametrize("flags", [0, 64, 32])   # plain, GG_RENORM, GG_INFL_SHARE
@pytest.mark.parametrize("alpha,ratio,theta,sigma", [(6, 0.5, 0.01, 0.4), (10, 0.2, 0.05, 0.5),
                                                     (3, 0.0, 0.02, 0.3), (0, 0.5, 0.1, 0.3)])
def test_triggered_pagerank_schedule_and_replay(gg, flags, alpha, ratio, theta, sigma):
    T = 20
    for g in _graphs()[:4]:
        h = gc.load(gg, g)
        try:
            vals, _, st = gc.gpu_run(gg, h, g, "pagerank", "triggered", sigma, alpha, theta, T=T, seed=9,
                                     flags=flags, trigger_ratio=ratio)
            it = _modes(gg, h)
            modes = (it["mode"] & 3).astype(np.int64)
            _check_rule(modes, it["sum_delta"].astype(np.float64), alpha, ratio)
            assert st.corrections == int((modes == 2).sum())
            # the schedule is deterministic: a shorter run stops at each correction
            masks = []
            for c in np.flatnonzero(modes == 2):
                _, mk, _ = gc.gpu_run(gg, h, g, "pagerank", "triggered", sigma, alpha, theta, T=int(c) + 1,
                                      seed=9, flags=flags, trigger_ratio=ratio)
                masks.append(mk)
            ref = oracle.run(g.n, g.rowptr, g.colidx, app="pagerank", policy="triggered", sigma=sigma,
                             seed=9, alpha=alpha, theta=theta, max_iters=T, flags=flags,
                             trigger_ratio=ratio, replay_modes=modes, replay_masks=masks,
                             replay_tol=1e-5, nthreads=0)
            assert ref["replay_violations"] == 0, ref["replay_max_margin"]
            assert gc.rel_l1(vals, ref["values"]) <= PR_TOL
            sd = it["sum_delta"].astype(np.float64) * FX
            tol = 3e-5 * max(float(np.abs(ref["values"]).sum()), 1e-30) + g.n * FX
            assert np.all(np.abs(sd - ref["iter_sum_delta"]) <= tol), (sd, ref["iter_sum_delta"])
        finally:
            gg.gg_free_graph(h)


def test_triggered_rejects_bad_ratio(gg):
    g = graphgen.rmat(6, seed=1)
    h = gc.load(gg, g)
    try:
        for bad in (-0.5, float("nan"), float("inf")):
            with pytest.raises(gg.GGError) as e:
                gg.gg_run(h, "pagerank", 0.5, "triggered", gg.make_params(trigger_ratio=bad))
            assert e.value.status == gg.GG_ERR_INVALID_ARG
        gg.gg_run(h, "pagerank", 0.5, "gg", gg.make_params(trigger_ratio=-1.0))   # ignored elsewhere
    finally:
        gg.gg_free_graph(h)

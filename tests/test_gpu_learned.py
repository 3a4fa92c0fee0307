"""GPU parity of the learned correction (beyond the paper): the scorer's
tensor-core forward and its training kernel against the oracle's FP64
restatement, the traces (features and labels) the library records at full
corrections, and whole GG_POLICY_LEARNED runs.

Bars. Scorer logits: |gpu - oracle| <= 2e-3 (1 + |logit|) (FP32 accumulation
order and an occasional bfloat16 rounding of a hidden value that falls the
other way). Gradient: relative L2 error <= 5e-3. Traces of SSSP / BFS / CC:
bit-exact features and labels. Runs: the oracle adopts the GPU's selections
(checking that each differing one lies within 0.05 of the threshold) and,
for PageRank, its post-correction flags; then integer applications must be
bit-exact and PageRank within 1e-5 relative L1.
"""
import numpy as np
import pytest

import graphgen
import oracle
from paper_2104_10039_gb300 import scorer
from tests import gpu_common as gc
from tests.test_gpu_parity import _graphs, _sym_graphs

pytestmark = pytest.mark.gpu

PR_TOL = 1e-5
SEL_TOL = 0.05


@pytest.fixture(scope="module")
def gg():
    return gc.lib()


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def _rand_params(seed):
    rng = np.random.default_rng(seed)
    P = scorer.init_params(seed)
    P[scorer.OFF_B1:scorer.OFF_W2] = rng.normal(0, 0.2, 64)
    P[scorer.OFF_B2:scorer.OFF_W3] = rng.normal(0, 0.2, 64)
    P[scorer.OFF_B3] = 0.1
    return P


def _features(rows, seed):
    rng = np.random.default_rng(seed)
    x = np.empty((rows, 8), np.float32)
    x[:, 0:2] = np.sqrt(rng.integers(0, 5000, (rows, 2))) / 64
    x[:, 2:5] = rng.exponential(1.0, (rows, 3)) * (rng.random((rows, 3)) < 0.7)
    x[:, 5] = rng.random(rows)
    x[:, 6] = rng.integers(0, 30, rows) / 64
    x[:, 7] = rng.integers(0, 4, rows)
    return x


@pytest.mark.parametrize("rows", [1, 15, 16, 1003, 70001])
def test_scorer_logits_match_oracle(gg, torch, rows):
    for seed in (1, 2):
        P = _rand_params(seed)
        x = _features(rows, seed)
        dx, dp = torch.from_numpy(x).cuda(), torch.from_numpy(P).cuda()
        out = torch.full((rows,), float("nan"), device="cuda")
        gg.gg_mlp_score(dx, rows, dp, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        want = oracle.mlp_forward(P, x)
        assert np.all(np.abs(got - want) <= 2e-3 * (1 + np.abs(want))), np.max(np.abs(got - want))


def test_scorer_single_path_is_exact(gg, torch):
    P = np.zeros(scorer.N_PARAM, np.float32)
    P[scorer.OFF_W1] = P[scorer.OFF_W2] = P[scorer.OFF_W3] = 1.0
    P[scorer.OFF_B1] = -1.5
    P[scorer.OFF_B2] = 0.25
    P[scorer.OFF_B3] = 0.5
    x = _features(999, 3)
    x[:, 0] = np.random.default_rng(3).normal(2, 2, 999)
    dx, dp = torch.from_numpy(x).cuda(), torch.from_numpy(P).cuda()
    out = torch.empty(999, device="cuda")
    gg.gg_mlp_score(dx, 999, dp, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().astype(np.float64), oracle.mlp_forward(P, x))


def test_training_gradient_loss_and_update(gg, torch):
    rows = 300
    x = _features(rows, 5)
    y = (np.random.default_rng(5).random(rows) < 0.4).astype(np.uint8)
    P = _rand_params(6)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    for batch in (128, 37, 300, 1000):   # one block, a partial block, several blocks (rows wrap around)
        dp = torch.from_numpy(P.copy()).cuda()
        grad = torch.empty(scorer.N_PARAM, device="cuda")
        loss = torch.empty(1, device="cuda")
        gg.gg_mlp_train(dx, dy, rows, dp, batch, 1, 0.5, 1, 7, losses=loss, grad_last=grad)
        torch.cuda.synchronize()
        want, want_loss = oracle.mlp_grad(P, x, y, idx=(7 + np.arange(batch)) % rows)
        got = grad.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - want) <= 5e-3 * np.linalg.norm(want)
        assert abs(float(loss.cpu()[0]) - want_loss) <= 1e-4 * want_loss
        # the update is P - lr * grad, in FP32
        assert np.array_equal(dp.cpu().numpy(), (P - np.float32(0.5) * grad.cpu().numpy()).astype(np.float32))


def test_training_is_deterministic_and_lowers_the_loss(gg, torch):
    rows = 4096
    x = _features(rows, 8)
    # a learnable rule: label = in-degree feature above its median
    y = (x[:, 0] > np.median(x[:, 0])).astype(np.uint8)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    outs = []
    for _ in range(2):
        dp = torch.from_numpy(scorer.init_params(9)).cuda()
        losses = torch.empty(400, device="cuda")
        gg.gg_mlp_train(dx, dy, rows, dp, 128, 400, 0.5, scorer.coprime_stride(rows), 0, losses=losses)
        torch.cuda.synchronize()
        outs.append((dp.cpu().numpy(), losses.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    L = outs[0][1]
    assert L[-50:].mean() < 0.5 * L[:10].mean()


def _trace(gg, torch, g, app, T, sigma=0.5, alpha=2, theta=0.1, s=0, label_tol=1e-3):
    h = gc.load(gg, g)
    try:
        cap = (T // (alpha + 1) + 1) * g.n
        fx = torch.zeros((cap, 8), device="cuda")
        fy = torch.zeros(cap, dtype=torch.uint8, device="cuda")
        gg.gg_set_trace(h, fx, fy, cap, label_tol)
        gc.gpu_run(gg, h, g, app, "gg", sigma=sigma, alpha=alpha, theta=theta, T=T, source=s, seed=3,
                   flags=gg.GG_FORCE_PULL if app != "pagerank" else 0)
        rows = gg.stats(h).trace_rows
        return fx[:rows].cpu().numpy(), fy[:rows].cpu().numpy()
    finally:
        gg.gg_free_graph(h)


@pytest.mark.parametrize("app", ["sssp", "bfs", "cc"])
def test_trace_min_apps_bit_exact(gg, torch, app):
    graphs = _sym_graphs() if app == "cc" else _graphs()[:3]
    for g in graphs:
        s = int(graphgen.sources(g, 1, seed=2)[0]) if app != "cc" else 0
        X, Y = _trace(gg, torch, g, app, T=100000, s=s)
        ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app=app, policy="gg", sigma=0.5, seed=3, alpha=2,
                         theta=0.1, source=s, max_iters=100000, symmetric=app == "cc", trace_cap=len(X) + g.n)
        assert len(X) == len(ref["trace_x"]) > 0
        assert np.array_equal(X, ref["trace_x"]) and np.array_equal(Y, ref["trace_y"])


@pytest.mark.parametrize("app", ["sssp", "bfs"])
def test_trace_consecutive_corrections(gg, torch, app):
    """alpha 0: every iteration is a correction, so each one's features read
    the flags (active in-degrees) that the previous correction left."""
    g = _graphs()[0]
    s = int(graphgen.sources(g, 1, seed=2)[0])
    X, Y = _trace(gg, torch, g, app, T=6, alpha=0, s=s)
    ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app=app, policy="gg", sigma=0.5, seed=3, alpha=0,
                     theta=0.1, source=s, max_iters=6, trace_cap=len(X) + g.n)
    assert len(X) == len(ref["trace_x"]) > g.n
    assert np.array_equal(X, ref["trace_x"]) and np.array_equal(Y, ref["trace_y"])


def test_trace_push_frontier_keeps_the_change_features(gg, torch):
    g = _graphs()[0]
    s = int(graphgen.sources(g, 1, seed=2)[0])
    h = gc.load(gg, g)
    try:
        cap = 40 * g.n
        fx = torch.zeros((cap, 8), device="cuda")
        fy = torch.zeros(cap, dtype=torch.uint8, device="cuda")
        gg.gg_set_trace(h, fx, fy, cap, 0.0)
        gc.gpu_run(gg, h, g, "sssp", "gg", sigma=0.5, alpha=2, theta=0.1, T=100000, source=s, seed=3,
                   flags=gg.GG_FORCE_PUSH)
        rows = gg.stats(h).trace_rows
        X = fx[:rows].cpu().numpy()
    finally:
        gg.gg_free_graph(h)
    ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", policy="gg", sigma=0.5, seed=3, alpha=2,
                     theta=0.1, source=s, max_iters=100000, trace_cap=cap)
    assert np.array_equal(X, ref["trace_x"])


def test_trace_pagerank(gg, torch):
    g = _graphs()[0]
    X, Y = _trace(gg, torch, g, "pagerank", T=12, label_tol=1e-3)
    ref = oracle.run(g.n, g.rowptr, g.colidx, policy="gg", sigma=0.5, seed=3, alpha=2, theta=0.1, max_iters=12,
                     trace_cap=len(X) + g.n, label_tol=1e-3)
    R = ref["trace_x"]
    assert X.shape == R.shape and X.shape[0] > 0
    exact_cols = [0, 1, 6, 7]
    assert np.array_equal(X[:, exact_cols], R[:, exact_cols])
    # active fraction: the GPU flags come from FP32 influence, so compare where
    # the masks agree (the first correction only uses sampled flags)
    assert np.array_equal(X[:g.n, 5], R[:g.n, 5])
    assert np.allclose(X[:, 2:5], R[:, 2:5], rtol=2e-4, atol=1e-5)
    agree = np.mean(X[:, 5] == R[:, 5])
    assert agree > 0.999
    assert np.mean(Y == ref["trace_y"]) > 0.995


def _indeg_scorer(d):
    lo, hi = (float(oracle.bf16(np.float32(np.sqrt(np.float32(k)) / np.float32(64)))) for k in (d, d + 1))
    P = np.zeros(scorer.N_PARAM, np.float32)
    P[scorer.OFF_W1] = P[scorer.OFF_W2] = P[scorer.OFF_W3] = 1.0
    P[scorer.OFF_B3] = -(lo + hi) / 2
    return P


def _gpu_learned(gg, h, g, app, P, T, alpha, theta, sigma, s, flags=0, tau=0.0, frac=1.0, cost=0.0):
    gg.gg_set_scorer(h, P)
    p = gg.make_params(alpha=alpha, theta=theta, max_iters=T, source=s, seed=5, flags=flags, select_logit=tau,
                       fallback_frac=frac, select_cost=cost)
    gg.gg_run(h, app, sigma, "learned", p)
    return gg.values(h, app), gg.mask_bits(h, g.m), gg.stats(h), gg.result_array(h, gg.GG_RESULT_ITER_STATS)


@pytest.mark.parametrize("app", ["sssp", "bfs", "cc"])
@pytest.mark.parametrize("flags", [0, 4, 8, 4 | 128])   # auto, pull, push, pull of frontier sources only
def test_learned_min_apps_bit_exact(gg, app, flags):
    graphs = _sym_graphs() if app == "cc" else _graphs()
    for g in graphs:
        h = gc.load(gg, g)
        try:
            s = int(graphgen.sources(g, 1, seed=2)[0]) if (app != "cc" and g.m) else 0
            for d, frac in ((4, 1.0), (0, 0.3), (20, -1.0)):
                P = _indeg_scorer(d)
                vals, mask, st, it = _gpu_learned(gg, h, g, app, P, 100000, 2, 0.2, 0.4, s, flags, 0.0, frac)
                ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app=app, policy="learned", mlp=P, sigma=0.4,
                                 seed=5, alpha=2, theta=0.2, source=s, max_iters=100000, fallback_frac=frac,
                                 symmetric=app == "cc")
                case = (g.name, d, frac, flags)
                assert np.array_equal(vals, ref["values"]), case
                assert np.array_equal(mask, ref["mask"]), case
                assert st.iterations == ref["iterations"] and st.corrections == ref["corrections"], case
                sel = np.where((it["mode"] & gg.GG_ITER_LEARNED) != 0, it["selected"].astype(np.int64), -1)
                assert np.array_equal(sel, ref["iter_selected"]), case
                assert np.array_equal(it["changed"], ref["iter_changed"].astype(np.uint64)), case
        finally:
            gg.gg_free_graph(h)


@pytest.mark.parametrize("app", ["sssp", "bfs"])
def test_learned_selection_cost_bit_exact(gg, app):
    """Cost-aware selection (select_cost: the threshold rises with the bit
    length of the in-degree) with a scorer whose decisions are exact: values,
    flags and the selected counts equal the oracle's."""
    for g in _graphs():
        h = gc.load(gg, g)
        try:
            s = int(graphgen.sources(g, 1, seed=2)[0]) if g.m else 0
            for d, tau, cost in ((4, 0.0, 2.0 ** -7), (1, -0.02, 2.0 ** -9)):
                P = _indeg_scorer(d)
                vals, mask, st, it = _gpu_learned(gg, h, g, app, P, 100000, 2, 0.2, 0.4, s, 0, tau, 1.0, cost)
                ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app=app, policy="learned", mlp=P, sigma=0.4,
                                 seed=5, alpha=2, theta=0.2, source=s, max_iters=100000, select_logit=tau,
                                 select_cost=cost)
                case = (g.name, d, tau, cost)
                assert np.array_equal(vals, ref["values"]), case
                assert np.array_equal(mask, ref["mask"]), case
                sel = np.where((it["mode"] & gg.GG_ITER_LEARNED) != 0, it["selected"].astype(np.int64), -1)
                assert np.array_equal(sel, ref["iter_selected"]), case
        finally:
            gg.gg_free_graph(h)


def _replayed_selections(gg, h, g, app, P, T, alpha, theta, sigma, s, tau, flags=0):
    """The GPU's selection and post-correction flags at each learned
    correction, from runs stopped right after it (the runs are deterministic)."""
    _, _, _, it = _gpu_learned(gg, h, g, app, P, T, alpha, theta, sigma, s, flags, tau)
    sels, masks = [], []
    for c in np.flatnonzero((it["mode"] & 3) == 2):
        _, mk, _, it_c = _gpu_learned(gg, h, g, app, P, int(c) + 1, alpha, theta, sigma, s, flags, tau)
        masks.append(mk)
        if it_c["mode"][c] & gg.GG_ITER_LEARNED:
            sels.append((gg.result_array(h, gg.GG_RESULT_SCORES) > np.float32(tau)).astype(np.uint8))
    return sels, masks


@pytest.mark.parametrize("flags", [0, 64])   # plain, GG_RENORM
def test_learned_pagerank_with_replay(gg, flags):
    T, alpha, theta, sigma = 16, 3, 0.02, 0.4
    for g in _graphs()[:3]:
        h = gc.load(gg, g)
        try:
            for P, tau in ((_indeg_scorer(12), 0.0), (_rand_params(4), None)):
                if tau is None:   # a threshold near the median of the first scoring
                    _gpu_learned(gg, h, g, "pagerank", P, alpha + 1, alpha, theta, sigma, 0, flags, 0.0)
                    tau = float(np.median(gg.result_array(h, gg.GG_RESULT_SCORES)))
                vals, _, st, it = _gpu_learned(gg, h, g, "pagerank", P, T, alpha, theta, sigma, 0, flags, tau)
                assert st.learned_corrections >= 1
                sels, masks = _replayed_selections(gg, h, g, "pagerank", P, T, alpha, theta, sigma, 0, tau, flags)
                ref = oracle.run(g.n, g.rowptr, g.colidx, app="pagerank", policy="learned", mlp=P, sigma=sigma,
                                 seed=5, alpha=alpha, theta=theta, max_iters=T, flags=flags, select_logit=tau,
                                 replay_select=sels, replay_select_tol=SEL_TOL, replay_masks=masks,
                                 replay_tol=1e-5, nthreads=0)
                assert ref["select_violations"] == 0, ref["select_max_margin"]
                assert ref["replay_violations"] == 0, ref["replay_max_margin"]
                assert gc.rel_l1(vals, ref["values"]) <= PR_TOL
        finally:
            gg.gg_free_graph(h)


def test_learned_min_app_random_scorer_with_replay(gg):
    g = _graphs()[0]
    s = int(graphgen.sources(g, 1, seed=2)[0])
    h = gc.load(gg, g)
    try:
        P = _rand_params(11)
        _gpu_learned(gg, h, g, "sssp", P, 3, 2, 0.2, 0.4, s, 4, 0.0)
        tau = float(np.median(gg.result_array(h, gg.GG_RESULT_SCORES)))
        vals, mask, st, _ = _gpu_learned(gg, h, g, "sssp", P, 100000, 2, 0.2, 0.4, s, 4, tau)
        sels, _ = _replayed_selections(gg, h, g, "sssp", P, 100000, 2, 0.2, 0.4, s, tau, 4)
        ref = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", policy="learned", mlp=P, sigma=0.4, seed=5,
                         alpha=2, theta=0.2, source=s, max_iters=100000, select_logit=tau, replay_select=sels,
                         replay_select_tol=SEL_TOL)
        assert ref["select_violations"] == 0, ref["select_max_margin"]
        assert np.array_equal(vals, ref["values"]) and np.array_equal(mask, ref["mask"])
    finally:
        gg.gg_free_graph(h)


def test_learned_errors(gg, torch):
    g = graphgen.rmat(6, seed=1)
    h = gc.load(gg, g)
    try:
        with pytest.raises(gg.GGError) as e:
            gg.gg_run(h, "pagerank", 0.5, "learned", gg.make_params())
        assert e.value.status == gg.GG_ERR_STATE
        with pytest.raises(ValueError):
            gg.gg_set_scorer(h, np.zeros(10, np.float32))
        x = torch.zeros((4, 8), device="cuda")
        y = torch.zeros(4, dtype=torch.uint8, device="cuda")
        p = torch.zeros(scorer.N_PARAM, device="cuda")
        with pytest.raises(gg.GGError) as e:
            gg.gg_mlp_train(x, y, 4, p, 16385, 1, 0.1, 1)
        assert e.value.status == gg.GG_ERR_INVALID_ARG
        with pytest.raises(gg.GGError) as e:
            gg.gg_mlp_train(x, y, 4, p, 4, 1, 0.1, 4)
        assert e.value.status == gg.GG_ERR_INVALID_ARG
    finally:
        gg.gg_free_graph(h)

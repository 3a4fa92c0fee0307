"""Pins of the oracle's learned correction (beyond the paper): the bfloat16
rounding, the scorer's forward pass and gradient, the features recorded in
traces, and the selection semantics (corrected vertices re-gather all
in-edges; the others keep value and flags)."""
from fractions import Fraction

import numpy as np
import pytest

import graphgen
import oracle
from paper_2104_10039_gb300 import scorer
from tests import brute


def _bf16_brute(x: float) -> float:
    """Nearest bfloat16 (8 significant bits) to the float32 x, ties to even,
    by exact rational arithmetic."""
    if x == 0.0:
        return x
    f = Fraction(float(np.float32(x)))
    sign = -1 if f < 0 else 1
    f = abs(f)
    e = 0
    while f >= 2:
        f /= 2
        e += 1
    while f < 1:
        f *= 2
        e -= 1
    e = max(e, -126)                      # subnormal grid below 2^-126
    ulp = Fraction(2) ** (e - 7)
    q, r = divmod(abs(Fraction(float(np.float32(x)))), ulp)
    if r > ulp / 2 or (r == ulp / 2 and q % 2 == 1):
        q += 1
    return float(sign * q * ulp)


def test_bf16_rounding_known_values_and_brute_force():
    cases = {1.0: 1.0, 1 + 2 ** -8: 1.0, 1 + 3 * 2 ** -8: 1 + 2 ** -6, 1 + 2 ** -8 + 2 ** -20: 1 + 2 ** -7,
             -1 - 3 * 2 ** -8: -1 - 2 ** -6, 3.0: 3.0, 2.0 ** -130: 2.0 ** -130}
    for x, want in cases.items():
        assert float(oracle.bf16(np.float32(x))) == want, x
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.normal(0, 1, 300), rng.normal(0, 1e-30, 20), rng.normal(0, 1e20, 20)])
    got = oracle.bf16(xs.astype(np.float32))
    for x, g in zip(xs.astype(np.float32), got):
        assert float(g) == _bf16_brute(float(x))


def _zero_params():
    return np.zeros(scorer.N_PARAM, np.float32)


def test_scorer_closed_form_single_path():
    # hidden unit 0 = relu(x0), second-layer unit 0 = relu(h0), logit = h2_0 + b3
    P = _zero_params()
    P[scorer.OFF_W1 + 0] = 1.0
    P[scorer.OFF_W2 + 0] = 1.0
    P[scorer.OFF_W3 + 0] = 1.0
    P[scorer.OFF_B3] = 0.5
    x = np.zeros((4, 8), np.float32)
    x[:, 0] = [1.0 + 3 * 2 ** -8, -2.0, 0.0, 100.25]
    x[:, 1:] = 7.0                                   # ignored by the zero weights
    got = oracle.mlp_forward(P, x)
    want = [1 + 2 ** -6 + 0.5, 0.5, 0.5, 100.0 + 0.5]   # 100.25 rounds to 100 in bfloat16
    assert np.array_equal(got, want)
    # biases are applied before the ReLU, in FP32
    P[scorer.OFF_B1 + 0] = -1.5
    P[scorer.OFF_B2 + 0] = 0.25
    got = oracle.mlp_forward(P, x)
    # 100 - 1.5 = 98.5 (a bfloat16 value); 98.5 + 0.25 = 98.75 lies halfway
    # between the bfloat16 neighbours 98.5 and 99 and rounds to the even 99
    assert np.array_equal(got, [0.5 + 0.25, 0.5 + 0.25, 0.5 + 0.25, 99.0 + 0.5])


def test_scorer_matches_dense_layers_without_rounding():
    rng = np.random.default_rng(5)
    P = scorer.init_params(2)
    P[scorer.OFF_B1:scorer.OFF_W2] = rng.normal(0, 0.1, 64)
    P[scorer.OFF_B2:scorer.OFF_W3] = rng.normal(0, 0.1, 64)
    x = rng.normal(0, 1, (50, 8)).astype(np.float32)
    W1 = P[:512].reshape(64, 8).astype(np.float64)
    W2 = P[576:4672].reshape(64, 64).astype(np.float64)
    h1 = np.maximum(x @ W1.T + P[512:576], 0)
    h2 = np.maximum(h1 @ W2.T + P[4672:4736], 0)
    z = h2 @ P[4736:4800].astype(np.float64) + np.float64(P[4800])
    assert np.allclose(oracle.mlp_forward(P, x, round_bf16=False), z, rtol=1e-12, atol=1e-12)
    # bfloat16 rounding moves the logits by a few parts in a thousand at most
    zr = oracle.mlp_forward(P, x)
    assert np.max(np.abs(zr - z)) < 0.02 * max(1.0, np.max(np.abs(z)))


def test_scorer_gradient_matches_finite_differences():
    rng = np.random.default_rng(7)
    P = scorer.init_params(4)
    P[scorer.OFF_B1:scorer.OFF_W2] = 0.05
    P[scorer.OFF_B2:scorer.OFF_W3] = 0.05
    x = rng.normal(0, 1, (12, 8)).astype(np.float32)
    y = (rng.random(12) < 0.5).astype(np.uint8)
    g, loss = oracle.mlp_grad(P, x, y, round_bf16=False)

    def loss_of(Q):
        z = oracle.mlp_forward(Q, x, round_bf16=False)
        return float(np.mean(np.maximum(z, 0) - z * y + np.log1p(np.exp(-np.abs(z)))))

    assert abs(loss - loss_of(P)) < 1e-12
    idx = np.concatenate([rng.choice(512, 12, replace=False), 512 + rng.choice(64, 6, replace=False),
                          576 + rng.choice(4096, 20, replace=False), 4672 + rng.choice(64, 6, replace=False),
                          4736 + rng.choice(64, 8, replace=False), [4800]])
    h = 1e-3
    for i in idx:
        Qp, Qm = P.copy(), P.copy()
        Qp[i] += np.float32(h)
        Qm[i] -= np.float32(h)
        fd = (loss_of(Qp) - loss_of(Qm)) / (float(Qp[i]) - float(Qm[i]))
        assert abs(fd - g[i]) <= 1e-4 * abs(g[i]) + 1e-7, (int(i), fd, g[i])


def _broom():
    arcs = [(0, v) for v in range(1, 9)] + [(1, 9), (2, 10), (3, 11), (4, 12), (9, 13), (10, 14), (13, 15)]
    return graphgen.from_arcs(16, arcs)


def test_trace_features_and_labels_by_hand():
    # BFS from 0 over every arc, a correction at iteration 2 (alpha 2): the
    # two executed iterations changed levels 1 and 2; the correction changes
    # level 3 (vertices 13, 14), which are its label-1 rows.
    g = _broom()
    r = oracle.run(g.n, g.rowptr, g.colidx, app="bfs", policy="gg", sigma=1.0, alpha=2, source=0,
                   max_iters=3, trace_cap=64)
    X, Y = r["trace_x"], r["trace_y"]
    assert X.shape == (16, 8)
    indeg = np.diff(oracle.csc_from_csr(g.n, g.rowptr, g.colidx)[0])
    outdeg = np.diff(g.rowptr)
    assert np.array_equal(X[:, 0], np.sqrt(indeg.astype(np.float32)) / np.float32(64))
    assert np.array_equal(X[:, 1], np.sqrt(outdeg.astype(np.float32)) / np.float32(64))
    lvl = brute.bfs_levels(g, 0)
    assert np.array_equal(X[:, 2], (lvl == 2).astype(np.float32))   # changed in iteration 1
    assert np.array_equal(X[:, 3], (lvl == 1).astype(np.float32))   # changed in iteration 0
    assert np.array_equal(X[:, 4], np.zeros(16, np.float32))
    assert np.array_equal(X[:, 5], np.ones(16, np.float32))         # sigma 1: every in-edge active
    assert np.all(X[:, 6] == np.float32(2 / 64)) and np.all(X[:, 7] == 2.0)
    assert np.array_equal(Y, (lvl == 3).astype(np.uint8))


def test_trace_pagerank_changes_and_labels():
    g = graphgen.rmat(6, edgefactor=4, seed=3)
    T = 5                                   # corrections at iterations 2 and 5 (alpha 2)
    r = oracle.run(g.n, g.rowptr, g.colidx, policy="gg", sigma=1.0, alpha=2, max_iters=T, trace_cap=10 * g.n,
                   label_tol=1e-3)
    X, Y = r["trace_x"], r["trace_y"]
    assert X.shape == (g.n, 8)              # the correction at iteration 5 lies past T
    ranks = [brute.pagerank_dense(g, 0.85, t) for t in range(4)]
    # sigma 1 makes every approximate iteration exact; change = n * |r_t - r_{t-1}|
    for col, t in ((2, 2), (3, 1)):
        want = g.n * np.abs(ranks[t] - ranks[t - 1])
        assert np.allclose(X[:, col], want, rtol=1e-6, atol=1e-12)
    assert np.all(X[:, 4] == 0)
    want_y = np.abs(ranks[3] - ranks[2]) > 1e-3 * np.abs(ranks[3])
    assert np.array_equal(Y.astype(bool), want_y)


def _indeg_threshold(d):
    """A logit offset between the bfloat16 features of in-degrees d and d+1."""
    lo, hi = (float(oracle.bf16(np.float32(np.sqrt(np.float32(k)) / np.float32(64)))) for k in (d, d + 1))
    assert lo < hi
    return (lo + hi) / 2


def _select_indeg_params(t):
    """A scorer whose logit is bfloat16(sqrt(in-degree)/64) - t."""
    P = _zero_params()
    P[scorer.OFF_W1 + 0] = 1.0
    P[scorer.OFF_W2 + 0] = 1.0
    P[scorer.OFF_W3 + 0] = 1.0
    P[scorer.OFF_B3] = -t
    return P


@pytest.mark.parametrize("app", ["pagerank", "sssp"])
def test_learned_correction_touches_only_selected_rows(app):
    g = graphgen.add_weights(graphgen.rmat(7, edgefactor=6, seed=2), seed=5)
    s = int(graphgen.sources(g, 1, seed=2)[0])
    alpha, sigma, theta = 2, 0.4, 0.1
    P = _select_indeg_params(_indeg_threshold(6))          # in-degree > 6 is selected
    kw = dict(app=app, sigma=sigma, seed=3, alpha=alpha, theta=theta, source=s)
    before = oracle.run(g.n, g.rowptr, g.colidx, g.weights, policy="gg", max_iters=alpha, **kw)
    full = oracle.run(g.n, g.rowptr, g.colidx, g.weights, policy="gg", max_iters=alpha + 1, **kw)
    lr = oracle.run(g.n, g.rowptr, g.colidx, g.weights, policy="learned", mlp=P, max_iters=alpha + 1, **kw)
    ip = oracle.csc_from_csr(g.n, g.rowptr, g.colidx)[0]
    indeg = np.diff(ip)
    sel = indeg > 6
    assert lr["iter_selected"][alpha] == int(sel.sum()) > 0
    feat = oracle.bf16(np.sqrt(indeg.astype(np.float32)) / np.float32(64)).astype(np.float64)
    assert np.array_equal(lr["logits"], feat - np.float64(np.float32(_indeg_threshold(6))))
    # selected rows: the full correction's value and flags; others: unchanged
    assert np.array_equal(lr["values"][sel], full["values"][sel])
    assert np.array_equal(lr["values"][~sel], before["values"][~sel])
    arc_sel = np.repeat(sel, indeg)
    assert np.array_equal(lr["mask"][arc_sel], full["mask"][arc_sel])
    assert np.array_equal(lr["mask"][~arc_sel], before["mask"][~arc_sel])


def test_learned_special_cases():
    g = graphgen.add_weights(graphgen.rmat(8, seed=6), seed=5)
    s = int(graphgen.sources(g, 1, seed=2)[0])
    P = scorer.init_params(1)
    for app, T in (("pagerank", 14), ("sssp", 1000)):
        kw = dict(app=app, sigma=0.3, seed=3, alpha=3, theta=0.1, source=s, max_iters=T)
        gg = oracle.run(g.n, g.rowptr, g.colidx, g.weights, policy="gg", **kw)
        every = oracle.run(g.n, g.rowptr, g.colidx, g.weights, policy="learned", mlp=P, select_logit=-np.inf,
                           **kw)
        fallback = oracle.run(g.n, g.rowptr, g.colidx, g.weights, policy="learned", mlp=P, fallback_frac=-1.0,
                              **kw)
        for r in (every, fallback):
            assert np.array_equal(r["values"], gg["values"]) and np.array_equal(r["mask"], gg["mask"])
        assert np.all(fallback["iter_selected"] == -1)
    # nothing selected: the learned correction is an identity step and makes
    # the next correction full; dropping the identity steps gives the same run
    kw = dict(app="pagerank", sigma=0.3, seed=3, theta=0.05)
    none = oracle.run(g.n, g.rowptr, g.colidx, policy="learned", mlp=P, select_logit=np.inf, max_iters=16,
                      alpha=3, **kw)
    modes = list(none["iter_mode"])
    ident = [i for i in range(16) if none["iter_selected"][i] == 0]
    assert ident == [3, 11]                 # corrections at 3, 7, 11, 15: learned, full, learned, full
    kept = [md for i, md in enumerate(modes) if i not in ident]
    ref = oracle.run(g.n, g.rowptr, g.colidx, policy="triggered", alpha=1, max_iters=len(kept),
                     replay_modes=kept, **kw)
    assert np.array_equal(none["values"], ref["values"]) and np.array_equal(none["mask"], ref["mask"])


def test_learned_min_app_terminates_at_exact_fixed_point():
    for g in [graphgen.add_weights(graphgen.rmat(8, seed=k), seed=5) for k in (1, 2)]:
        s = int(graphgen.sources(g, 1, seed=2)[0])
        for t in (-np.inf, 0.0, 0.03, np.inf):
            P = _select_indeg_params(0.03 if np.isfinite(t) else 0.0)
            r = oracle.run(g.n, g.rowptr, g.colidx, g.weights, app="sssp", policy="learned", mlp=P,
                           select_logit=t if not np.isfinite(t) else 0.0, sigma=0.3, seed=4, alpha=2, theta=0.3,
                           source=s, max_iters=10000)
            assert np.array_equal(r["values"], brute.dijkstra(g, s))
            assert r["iterations"] < 10000


def _bitlen(d):
    d = np.asarray(d, np.int64)
    out = np.zeros(d.shape, np.int64)
    x = d.copy()
    while np.any(x > 0):
        out += x > 0
        x >>= 1
    return out


def test_learned_selection_cost():
    """select_cost (beyond the paper): a vertex with in-degree d is selected
    when its logit exceeds fmaf(select_cost, bit length of d, select_logit).
    Cost 0 is the plain threshold; a cost no logit can reach selects only rows
    without in-edges, which corrects nothing, so the run equals selecting none;
    in between, the count selected at a learned correction is the number of
    logits above each vertex's own threshold."""
    g = graphgen.add_weights(graphgen.rmat(8, seed=6), seed=5)
    s = int(graphgen.sources(g, 1, seed=2)[0])
    P = scorer.init_params(1)
    indeg = np.bincount(g.colidx, minlength=g.n)
    for app, T in (("pagerank", 14), ("sssp", 1000)):
        kw = dict(app=app, sigma=0.3, seed=3, alpha=3, theta=0.1, source=s, max_iters=T, policy="learned", mlp=P)
        plain = oracle.run(g.n, g.rowptr, g.colidx, g.weights, select_logit=0.1, **kw)
        zero = oracle.run(g.n, g.rowptr, g.colidx, g.weights, select_logit=0.1, select_cost=0.0, **kw)
        for key in ("values", "mask", "iter_selected"):
            assert np.array_equal(plain[key], zero[key]), (app, key)
        none = oracle.run(g.n, g.rowptr, g.colidx, g.weights, select_logit=np.inf, **kw)
        huge = oracle.run(g.n, g.rowptr, g.colidx, g.weights, select_logit=0.0, select_cost=1e30, **kw)
        assert np.array_equal(none["values"], huge["values"]) and np.array_equal(none["mask"], huge["mask"])
        mid = oracle.run(g.n, g.rowptr, g.colidx, g.weights, select_logit=0.05, select_cost=0.01, **kw)
        learned_its = [i for i, c in enumerate(mid["iter_selected"]) if c >= 0]
        assert learned_its, app
        thr = np.float32(np.float64(np.float32(0.01)) * _bitlen(indeg) + np.float64(np.float32(0.05)))
        want = int(np.sum(mid["logits"] > thr.astype(np.float64)))
        assert mid["iter_selected"][learned_its[-1]] == want, app
        # the cost lowers the selection below the plain one at the same logit threshold
        flat = oracle.run(g.n, g.rowptr, g.colidx, g.weights, select_logit=0.05, **kw)
        assert int(np.sum(flat["logits"] > np.float32(0.05))) >= want

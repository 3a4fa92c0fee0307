"""The seeded input generator: known answers of its random stream, exact
sizes, determinism and the structure the workloads need."""
import os

import numpy as np

import graphgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    for r in rows:
        v = [int(x, 16) for x in r]
        assert graphgen.philox4x32_10(v[:4], v[4:6]) == v[6:10]


def test_rmat_sizes_determinism_and_sorted_rows():
    g = graphgen.rmat(12, seed=1)
    assert g.n == 4096 and g.m == 65536 and g.rowptr[-1] == g.m
    h = graphgen.rmat(12, seed=1)
    assert np.array_equal(g.rowptr, h.rowptr) and np.array_equal(g.colidx, h.colidx)
    assert not np.array_equal(graphgen.rmat(12, seed=2).colidx, g.colidx)
    for v in range(0, g.n, 7):
        row = g.colidx[g.rowptr[v]:g.rowptr[v + 1]]
        assert np.all(np.diff(row) >= 0)
    indeg = np.bincount(g.colidx, minlength=g.n)
    assert indeg.max() > 20 * indeg.mean()        # power-law skew


def test_symmetric_graphs_and_weights():
    for g in (graphgen.rmat(10, seed=3, symmetric=True),
              graphgen.erdos_renyi(1000, avg_degree=16, seed=3, symmetric=True)):
        graphgen.add_weights(g, seed=7)
        src = np.repeat(np.arange(g.n), np.diff(g.rowptr))
        fwd = sorted(zip(src.tolist(), g.colidx.tolist(), g.weights.tolist()))
        bwd = sorted(zip(g.colidx.tolist(), src.tolist(), g.weights.tolist()))
        assert fwd == bwd
        assert g.weights.min() >= 1 and g.weights.max() <= 255


def test_sources_have_out_arcs():
    g = graphgen.rmat(12, seed=1)
    s = graphgen.sources(g, 16, seed=2)
    assert len(s) == 16 and len(set(s.tolist())) == 16
    assert np.all(np.diff(g.rowptr)[s] > 0)


def test_top_k_tie_break_matches_full_sort():
    from paper_2104_10039_gb300 import metrics
    rng = np.random.default_rng(0)
    for _ in range(200):
        n = int(rng.integers(1, 300))
        v = rng.integers(0, 20, n).astype(float)
        k = int(rng.integers(0, n + 3))
        ref = np.lexsort((np.arange(n), -v))[:min(k, n)]
        assert np.array_equal(metrics.top_k(v, k), ref)
    assert metrics.top_k_error(np.array([3.0, 2, 1, 0]), np.array([0.0, 1, 2, 3]), 2) == 1.0

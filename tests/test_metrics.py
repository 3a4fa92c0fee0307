"""Host-side accuracy metrics of Sec. 4.2 on hand-made examples (CPU)."""
import numpy as np

from paper_2104_10039_gb300 import metrics

U = metrics.UNREACHED


def test_top_k_orders_by_value_then_id():
    v = np.array([0.5, 0.9, 0.5, 0.1, 0.9, 0.5])
    assert metrics.top_k(v, 3).tolist() == [1, 4, 0]
    assert metrics.top_k(v, 4).tolist() == [1, 4, 0, 2]
    assert metrics.top_k(v, 10).tolist() == [1, 4, 0, 2, 5, 3]
    assert metrics.top_k(v, 0).tolist() == []


def test_top_k_matches_a_full_sort():
    rng = np.random.default_rng(3)
    for _ in range(20):
        v = rng.integers(0, 8, 200).astype(np.float64)   # many ties
        k = int(rng.integers(1, 60))
        want = sorted(range(200), key=lambda i: (-v[i], i))[:k]
        assert metrics.top_k(v, k).tolist() == want


def test_top_k_error_is_the_fraction_missing_from_the_exact_set():
    exact = np.array([9.0, 8, 7, 6, 5, 4])
    approx = np.array([9.0, 8, 1, 6, 5, 7])   # top-3 {0, 1, 5} vs {0, 1, 2}
    assert metrics.top_k_error(approx, exact, 3) == 1 / 3
    assert metrics.top_k_error(exact, exact, 3) == 0.0
    assert metrics.accuracy(metrics.top_k_error(approx, exact, 3)) == (1 - 1 / 3) * 100


def test_stretch_error_skips_the_source_and_counts_unreached_as_failures():
    exact = np.array([0, 2, 4, U, 5], np.uint32)   # source 0; vertex 3 unreachable
    approx = np.array([0, 3, 4, U, U], np.uint32)  # 1: stretch 1.5; 2: 1; 4: left unreached
    r = metrics.stretch_error(approx, exact, 0)
    assert r["reachable"] == 3 and r["unreached"] == 1
    assert abs(r["error"] - (0.5 + 0.0 + 1.0) / 3) < 1e-15
    assert abs(r["mean_stretch"] - 1.25) < 1e-15
    assert metrics.stretch_error(exact, exact, 0)["error"] == 0.0


def test_wcc_relative_error_and_mislabelled_fraction():
    exact = np.array([0, 0, 0, 3, 3, 5])          # 3 components
    approx = np.array([0, 0, 2, 3, 3, 5])         # vertex 2 split off: 4 components
    r = metrics.wcc_relative_error(approx, exact)
    assert r["components_exact"] == 3 and r["components_approx"] == 4
    assert abs(r["error"] - 1 / 3) < 1e-15
    assert abs(r["mislabelled"] - 1 / 6) < 1e-15

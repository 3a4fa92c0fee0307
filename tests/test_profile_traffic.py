"""The key under which ncu traffic ratios are stored follows the tile
engine's code, not its comments or layout (CPU)."""
from paper_2104_10039_gb300 import profile_traffic as pt


def test_code_key_ignores_comments_and_layout():
    a = "int f(int x) {\n    return x + 1;   // add one\n}\n/* block\n comment */"
    b = "int f(int x) { return x + 1; }"
    c = "int f(int x) { return x + 2; }"
    assert pt._code(a) == pt._code(b)
    assert pt._code(b) != pt._code(c)


def test_algorithmic_bytes_model():
    n, m = 1000, 16000
    assert pt.gather_bytes("pagerank", n, m) == 4 * m + 24 * n
    assert pt.gather_bytes("sssp", n, m) == 8 * m + 16 * n
    assert pt.correct_bytes("pagerank", n, m, 5000) == 4 * m + 4 * 5000 + m // 8 + 28 * n
    assert pt.correct_bytes("sssp", n, m, 5000) == 8 * m + 8 * 5000 + m // 4 + 20 * n


def test_bench_uses_the_same_per_unit_model():
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    for app in ("pagerank", "sssp"):
        assert bench.gather_bytes(app, 1000, 16000) == pt.gather_bytes(app, 1000, 16000)
        assert bench.correct_bytes(app, 1000, 16000, 5000) == pt.correct_bytes(app, 1000, 16000, 5000)

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
    assert pt.correct_bytes("pagerank", n, m) == 4 * m + m // 8 + 28 * n
    assert pt.correct_bytes("sssp", n, m) == 8 * m + m // 4 + 20 * n


def test_bench_uses_the_same_per_unit_model():
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    for app in ("pagerank", "sssp"):
        assert bench.gather_bytes(app, 1000, 16000) == pt.gather_bytes(app, 1000, 16000)
        assert bench.correct_bytes(app, 1000, 16000) == pt.correct_bytes(app, 1000, 16000)


def test_class_window_picks_the_last_sequence(tmp_path):
    """The launch-list reader sums a class's last launch sequence: a gather
    and a correction each end at their apply pass, and begin at k_hub_values
    when it precedes the arcs pass."""
    names = ["k_validate(int)", "k_pull_arcs<0, 4, 1>(PullArgs)", "k_long_rows<0>(PullArgs)", "k_pr_apply(PullArgs)",
             "k_pull_arcs<0, 4, 1>(PullArgs)", "k_long_rows<0>(PullArgs)", "k_carries<0>(PullArgs)",
             "k_prc_flags(PullArgs)", "k_pr_apply(PullArgs)", "k_scan_reduce(int)", "k_pack_arcs<0>(int)",
             "k_hub_values(PullArgs)", "k_pull_arcs<0, 4, 1>(PullArgs)", "k_long_rows<0>(PullArgs)",
             "k_pr_apply(PullArgs)"]
    hdr = ["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"]
    lines = [",".join(f'"{h}"' for h in hdr)]
    for i, nm in enumerate(names):
        lines.append(f'"{i}","{nm}","dram__bytes_read.sum","Mbyte","{i + 1}"')
        lines.append(f'"{i}","{nm}","dram__bytes_write.sum","Kbyte","{1000 * (i + 1)}"')
        lines.append(f'"{i}","{nm}","gpu__time_duration.sum","us","{i}"')
    p = tmp_path / "l.csv"
    p.write_text("==PROF== noise\n" + "\n".join(lines) + "\n")
    launches = pt._launches(str(p))
    assert len(launches) == len(names) and launches[3][1] == 8e6 and launches[3][2] == 3e3
    g = pt.class_window(launches, "gather")
    assert [x[0] for x in g] == names[11:15]   # with the hub values written before it
    c = pt.class_window(launches, "correct")
    assert [x[0] for x in c] == names[4:9]
    assert sum(x[1] for x in c) == sum(2e6 * (i + 1) for i in range(4, 9))

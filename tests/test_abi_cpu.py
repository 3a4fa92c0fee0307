"""CPU-side checks of the C ABI: libgg.so builds for sm_103a, loads, and
exports every entry point include/gg.h declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "gg.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gg_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2104_10039_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert {"gg_load_csr", "gg_sample_edges", "gg_run", "gg_result"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_binding_marshals_without_gpu():
    from paper_2104_10039_gb300 import gg
    assert gg.gg_last_error() == ""
    p = gg.make_params(alpha=3, theta=0.25, max_iters=7, seed=2**64 - 1)
    assert (p.alpha, p.max_iters, p.seed) == (3, 7, 2**64 - 1)
    assert abs(p.trigger_ratio - 0.5) < 1e-7 and p.select_logit == 0.0 and p.fallback_frac == 1.0


def test_binding_layouts_match_the_header():
    """Sizes and field offsets of the binding's structs against gg.h, as a C
    compiler lays them out."""
    import subprocess
    import tempfile
    from paper_2104_10039_gb300 import gg
    structs = {"gg_params": gg.gg_params, "gg_stats": gg.gg_stats, "gg_query": gg.gg_query,
               "gg_batch_config": gg.gg_batch_config, "gg_query_stats": gg.gg_query_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gg.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append('printf("gg_iter_stats %zu\\n", sizeof(gg_iter_stats));')
    for fname in gg.ITER_STATS_DTYPE.names:
        lines.append(f'printf("gg_iter_stats.{fname} %zu\\n", offsetof(gg_iter_stats, {fname}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        with open(src, "w") as f:
            f.write("\n".join(lines))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = dict(ln.split() for ln in subprocess.run([exe], capture_output=True, text=True,
                                                          check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(out[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)
    assert int(out["gg_iter_stats"]) == gg.ITER_STATS_DTYPE.itemsize
    for fname in gg.ITER_STATS_DTYPE.names:
        assert int(out[f"gg_iter_stats.{fname}"]) == gg.ITER_STATS_DTYPE.fields[fname][1], fname


def test_noalloc_limit_matches_the_header():
    """The binding's copy of GG_NOALLOC_MAX_ITEMS is the header's #define."""
    from paper_2104_10039_gb300 import gg
    with open(os.path.join(ROOT, "include", "gg.h")) as f:
        m = re.search(r"#define\s+GG_NOALLOC_MAX_ITEMS\s+\((\d+)u\s*<<\s*(\d+)\)", f.read())
    assert m, "GG_NOALLOC_MAX_ITEMS not found in gg.h"
    assert int(m.group(1)) << int(m.group(2)) == gg.GG_NOALLOC_MAX_ITEMS

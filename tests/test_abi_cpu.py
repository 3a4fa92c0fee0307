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
    assert ctypes.sizeof(gg.gg_params) == 40
    assert gg.ITER_STATS_DTYPE.itemsize == 40

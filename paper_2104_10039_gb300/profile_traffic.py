"""DRAM traffic of the pull kernels from ncu launch lists, for bench.py's
roofline line.

Each launch list is one case run by ``profile_case`` under ``ncu`` with the
one-pass metrics dram__bytes_read.sum, dram__bytes_write.sum and
gpu__time_duration.sum on every launch (``--csv --log-file``). This tool
finds the class's last launch sequence in the list (a gather: k_pull_arcs,
k_long_rows and the apply pass; a correction: k_pull_arcs, k_long_rows,
k_carries, the flag pass and the apply pass; for PageRank each preceded by
k_hub_values), sums its DRAM bytes and records them next to the
case's algorithmic bytes (the same per-unit model bench.py uses), together
with a hash of the kernel sources, in profiles/traffic.json. bench.py scales
the traffic to its own launches by their algorithmic bytes (traffic grows
with the arcs and vertices a launch processes) and reports null when the
kernel sources changed since.

    python -m paper_2104_10039_gb300.profile_traffic CLASS CSV N M [CLASS CSV N M ...]

CLASS is app/gather or app/correct; N, M the case's vertices and arcs (a
gather of the full list, a correction).
"""
from __future__ import annotations

import csv
import hashlib
import json
import os
import re
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
# the pull kernels (gathers and corrections of every application)
KERNEL_FILES = ("gg_pull.cu",)


def _code(text: str) -> str:
    """Source text without comments and with whitespace runs collapsed, so
    that the hash follows the code and not its commentary."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_hash() -> str:
    """Hash of the measured kernels' device code: their files plus the
    constants and the argument struct they are compiled with (comments and
    layout ignored)."""
    h = hashlib.sha256()
    for f in KERNEL_FILES:
        with open(os.path.join(CSRC, f)) as fh:
            h.update(_code(fh.read()).encode())
    with open(os.path.join(CSRC, "gg_internal.cuh")) as fh:
        text = fh.read()
    for pat in (r"constexpr int kThreads.*?constexpr uint32_t kInf[^\n]*", r"constexpr int kHubCodes[^\n]*",
                r"struct PullArgs \{.*?\n\};"):
        m = re.search(pat, text, re.S)
        h.update(_code(m.group(0) if m else "").encode())
    return h.hexdigest()[:16]


def gather_bytes(app, n, e):
    if app == "pagerank":
        return 4 * e + 24 * n
    return 8 * e + 16 * n


def correct_bytes(app, n, m):
    """A correction over all m arcs: sources (and weights) read, flags
    written (and read: the min applications keep some), per-vertex state;
    rebuilding the packed list is not part of it."""
    if app == "pagerank":        # sources 4m; flags m/8; row ptr, rank, degree, rank', contrib', contrib, acc 28n
        return 4 * m + m // 8 + 28 * n
    return 8 * m + m // 4 + 20 * n


def _launches(path: str) -> list:
    """[(kernel name, dram bytes, ns)] in launch order from an ncu --csv log."""
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "ns": 1, "nsecond": 1, "us": 1e3,
             "usecond": 1e3, "ms": 1e6, "msecond": 1e6}
    out, hdr = {}, None
    with open(path) as f:
        for r in csv.reader(f):
            if not r:
                continue
            if r[0] == "ID":
                hdr = r
                continue
            if hdr is None:
                continue
            d = dict(zip(hdr, r))
            rec = out.setdefault(int(d["ID"]), [d["Kernel Name"], 0.0, 0.0])
            v = float(d["Metric Value"].replace(",", "")) * scale[d["Metric Unit"]]
            if d["Metric Name"] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                rec[1] += v
            elif d["Metric Name"] == "gpu__time_duration.sum":
                rec[2] += v
    return [tuple(out[k]) for k in sorted(out)]


def _is(name: str, kernel: str) -> bool:
    return re.search(r"\b%s\b" % kernel, name) is not None


def class_window(launches: list, kind: str) -> list:
    """The last launch sequence of a gather (kind 'gather') or a correction
    ('correct') in the list."""
    found = None
    for i, (name, _, _) in enumerate(launches):
        if not _is(name, "k_pull_arcs") or i + 2 >= len(launches) or not _is(launches[i + 1][0], "k_long_rows"):
            continue
        corr = _is(launches[i + 2][0], "k_carries")
        if corr != (kind == "correct"):
            continue
        first = i - 1 if i > 0 and _is(launches[i - 1][0], "k_hub_values") else i
        for j in range(i + 2, len(launches)):
            if _is(launches[j][0], r"k_(pr|min)_apply"):
                found = launches[first:j + 1]
                break
    if found is None:
        raise SystemExit(f"no {kind} launch sequence in the list")
    return found


def main(argv):
    if len(argv) % 4 or not argv:
        raise SystemExit(__doc__)
    rec = {"kernel_hash": kernel_hash(), "classes": {}}
    for i in range(0, len(argv), 4):
        cls, path, n, m = argv[i], argv[i + 1], int(argv[i + 2]), int(argv[i + 3])
        app, kind = cls.split("/")
        algo = gather_bytes(app, n, m) if kind == "gather" else correct_bytes(app, n, m)
        win = class_window(_launches(path), kind)
        dram = sum(x[1] for x in win)
        rec["classes"][cls] = {"dram_bytes": int(dram), "algorithmic_bytes": int(algo),
                               "ratio": round(dram / algo, 4), "us": round(sum(x[2] for x in win) / 1e3, 1),
                               "kernels": [re.sub(r"\(.*", "", x[0]) for x in win],
                               "capture": os.path.basename(path), "vertices": n, "arcs": m}
    with open(TRAFFIC, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec, indent=1))


if __name__ == "__main__":
    main(sys.argv[1:])

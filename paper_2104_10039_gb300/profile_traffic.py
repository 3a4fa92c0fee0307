"""DRAM traffic of the pull kernels from ncu captures, for bench.py's
roofline line.

Each capture is one case run by ``profile_case`` under ``ncu`` (one launch
of each kernel of a class: the gather, or the two correction launches). This
tool reads the captures' raw pages (``ncu -i <rep> --page raw --csv``), sums
dram__bytes_read.sum + dram__bytes_write.sum over the class's launches, and
records that traffic next to the case's algorithmic bytes (the same per-unit
model bench.py uses), together with a hash of the tile-engine sources, in
profiles/traffic.json. bench.py scales the traffic to its own launches by
their algorithmic bytes (traffic grows with the arcs and vertices a launch
processes) and reports null when the kernel sources changed since.

    python -m paper_2104_10039_gb300.profile_traffic CLASS REP N M E_NEW [CLASS REP N M E_NEW ...]

CLASS is app/gather or app/correct; N, M the case's vertices and arcs;
E_NEW the arcs active after a correction (0 for a gather of all M arcs).
"""
from __future__ import annotations

import csv
import hashlib
import json
import os
import re
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
# the pull kernels (gathers and corrections of every application) and the
# tile count kernel a correction ends with
KERNEL_FILES = ("gg_pull.cu", "gg_sample.cu")


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
    for pat in (r"constexpr int kThreads.*?constexpr uint32_t kInf[^\n]*", r"struct PullArgs \{.*?\n\};"):
        m = re.search(pat, text, re.S)
        h.update(_code(m.group(0) if m else "").encode())
    return h.hexdigest()[:16]


def gather_bytes(app, n, e):
    if app == "pagerank":
        return 4 * e + 24 * n
    return 8 * e + 16 * n


def correct_bytes(app, n, m, e_new):
    if app == "pagerank":
        return 4 * m + 4 * e_new + m // 8 + 28 * n
    return 8 * m + 8 * e_new + m // 4 + 20 * n


def dram_bytes(rep: str) -> tuple:
    out = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True, text=True,
                         check=True).stdout
    rows = list(csv.reader(out.splitlines()))
    hdr, units = rows[0], rows[1]
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    total, names = 0.0, []
    for r in rows[2:]:
        for key in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            i = hdr.index(key)
            total += float(r[i].replace(",", "")) * scale[units[i]]
        names.append(r[hdr.index("Kernel Name")])
    return total, names


def main(argv):
    if len(argv) % 5 or not argv:
        raise SystemExit(__doc__)
    rec = {"kernel_hash": kernel_hash(), "classes": {}}
    for i in range(0, len(argv), 5):
        cls, rep, n, m, e_new = argv[i], argv[i + 1], int(argv[i + 2]), int(argv[i + 3]), int(argv[i + 4])
        app, kind = cls.split("/")
        algo = gather_bytes(app, n, m) if kind == "gather" else correct_bytes(app, n, m, e_new)
        dram, names = dram_bytes(rep)
        rec["classes"][cls] = {"dram_bytes": int(dram), "algorithmic_bytes": int(algo),
                               "ratio": round(dram / algo, 4), "kernels": names,
                               "capture": os.path.basename(rep), "vertices": n, "arcs": m}
    with open(TRAFFIC, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec, indent=1))


if __name__ == "__main__":
    main(sys.argv[1:])

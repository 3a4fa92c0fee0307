"""Seeded synthetic graph inputs (R-MAT, Erdos-Renyi, weights, sources).

This module is the one piece shared by the oracle side and the CUDA side of
the tests: it builds the input graphs and holds none of GraphGuess's own
arithmetic. The generator code is plain C (``graphgen.c``), compiled on first
use with gcc into ``libgraphgen.so`` next to this file.

Workload recipe (synthetic stand-ins for the paper's Wikipedia, LiveJournal,
Twitter and Friendster graphs, Sec. 4.1):

* R-MAT (Chakrabarti-Zhan-Faloutsos 2004), a=0.57 b=0.19 c=0.19 d=0.05, no
  noise, seeded bijective relabelling of vertex ids, self-loops and
  duplicates kept. Directed: ``2**scale * edgefactor`` arcs. Symmetric:
  ``2**scale * edgefactor / 2`` pairs, both directions stored.
* Erdos-Renyi multigraph with uniform endpoints, matched average degree.
* Weights uniform in [1, 255], keyed on the unordered pair.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so (gcc, OpenMP) if stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.graphgen_rmat_csr.restype = ctypes.c_int64
        lib.graphgen_rmat_csr.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                          ctypes.c_int, ctypes.c_int, i32p, i32p]
        lib.graphgen_er_csr.restype = ctypes.c_int64
        lib.graphgen_er_csr.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                        ctypes.c_int, i32p, i32p]
        lib.graphgen_weights.restype = ctypes.c_int
        lib.graphgen_weights.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_uint64,
                                         ctypes.c_uint32, ctypes.c_uint32, u32p]
        lib.graphgen_sources.restype = ctypes.c_int
        lib.graphgen_sources.argtypes = [ctypes.c_int32, i32p, ctypes.c_uint64, ctypes.c_int, i32p]
        lib.graphgen_philox.restype = None
        lib.graphgen_philox.argtypes = [u32p, u32p, u32p]
        _lib = lib
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


@dataclass
class Graph:
    """A CSR graph: rowptr int32[n+1], colidx int32[m] (out-arcs, rows sorted
    by destination), optional weights uint32[m]."""
    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    weights: Optional[np.ndarray] = None
    symmetric: bool = False
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.colidx.shape[0])


def rmat(scale: int, edgefactor: int = 16, seed: int = 1, symmetric: bool = False,
         a: float = 0.57, b: float = 0.19, c: float = 0.19, permute: bool = True) -> Graph:
    """R-MAT graph with 2**scale vertices and 2**scale*edgefactor arcs."""
    n = 1 << scale
    m = n * edgefactor
    npairs = m // 2 if symmetric else m
    rowptr = np.empty(n + 1, np.int32)
    colidx = np.empty(max(m, 1), np.int32)
    got = _load().graphgen_rmat_csr(scale, npairs, a, b, c, seed, int(symmetric), int(permute),
                                    _p(rowptr, ctypes.c_int32), _p(colidx, ctypes.c_int32))
    if got != m:
        raise RuntimeError(f"graphgen_rmat_csr failed ({got})")
    return Graph(n, rowptr, colidx[:m], None, symmetric,
                 f"rmat{scale}-ef{edgefactor}-{'sym' if symmetric else 'dir'}-s{seed}")


def erdos_renyi(n: int, avg_degree: int = 16, seed: int = 1, symmetric: bool = True) -> Graph:
    """Uniform-endpoint multigraph on n vertices with n*avg_degree arcs."""
    m = n * avg_degree
    npairs = m // 2 if symmetric else m
    rowptr = np.empty(n + 1, np.int32)
    colidx = np.empty(max(m, 1), np.int32)
    got = _load().graphgen_er_csr(n, npairs, seed, int(symmetric),
                                  _p(rowptr, ctypes.c_int32), _p(colidx, ctypes.c_int32))
    if got != m:
        raise RuntimeError(f"graphgen_er_csr failed ({got})")
    return Graph(n, rowptr, colidx[:m], None, symmetric,
                 f"er{n}-d{avg_degree}-{'sym' if symmetric else 'dir'}-s{seed}")


def add_weights(g: Graph, seed: int = 7, lo: int = 1, hi: int = 255) -> Graph:
    """Attach uint32 weights uniform in [lo, hi] (keyed on the unordered pair)."""
    w = np.empty(max(g.m, 1), np.uint32)
    rc = _load().graphgen_weights(g.n, _p(g.rowptr, ctypes.c_int32), _p(g.colidx, ctypes.c_int32),
                                  seed, lo, hi, _p(w, ctypes.c_uint32))
    if rc != 0:
        raise RuntimeError("graphgen_weights failed")
    g.weights = w[:g.m]
    return g


def sources(g: Graph, k: int = 16, seed: int = 2) -> np.ndarray:
    """k distinct uniform-random vertices with out-degree > 0."""
    out = np.empty(max(k, 1), np.int32)
    got = _load().graphgen_sources(g.n, _p(g.rowptr, ctypes.c_int32), seed, k,
                                   _p(out, ctypes.c_int32))
    return out[:got].copy()


def philox4x32_10(ctr, key) -> list:
    """The generator's random stream, exposed for its known-answer test."""
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    o = np.empty(4, np.uint32)
    _load().graphgen_philox(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(o, ctypes.c_uint32))
    return [int(x) for x in o]


def from_arcs(n: int, arcs, weights=None, symmetric: bool = False, name: str = "") -> Graph:
    """Small hand-built graph from a list of (src, dst) arcs (kept in the
    given multiplicity; rows sorted by destination, stable for duplicates)."""
    arcs = list(arcs)
    src = np.array([a for a, _ in arcs], np.int64)
    dst = np.array([b for _, b in arcs], np.int64)
    order = np.lexsort((dst, src)) if len(arcs) else np.zeros(0, np.int64)
    rowptr = np.zeros(n + 1, np.int32)
    if len(arcs):
        np.add.at(rowptr, src + 1, 1)
    rowptr = np.cumsum(rowptr, dtype=np.int64).astype(np.int32)
    colidx = dst[order].astype(np.int32)
    w = None
    if weights is not None:
        w = np.asarray(weights, np.uint32)[order]
    return Graph(n, rowptr, colidx, w, symmetric, name)

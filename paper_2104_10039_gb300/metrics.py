"""Accuracy metrics of Sec. 4.2 (host-side evaluation of results already
copied out of the library): top-K error for PageRank, stretch error for
SSSP / BFS, relative error for WCC, and accuracy = (1 - error) * 100.

Readings where the paper is brief:
* top-K: the K vertices with the largest values, ties broken by smaller id;
  error = fraction of the approximate top-K that is not in the exact top-K.
* stretch: per vertex approx / exact over vertices the exact run reaches
  (source excluded, exact distance > 0); a vertex the approximate run leaves
  unreached counts as a full failure (error 1); error = mean(stretch - 1).
* WCC relative error: |#components(approx) - #components(exact)| /
  #components(exact); the fraction of vertices whose label differs is also
  reported.
"""
from __future__ import annotations

import numpy as np

UNREACHED = 0xFFFFFFFF


def top_k(values: np.ndarray, k: int) -> np.ndarray:
    """Ids of the k largest values (value descending, id ascending), in O(n):
    everything above the k-th largest value, then the smallest ids equal to it."""
    v = np.asarray(values, np.float64)
    n = v.shape[0]
    k = min(k, n)
    if k == 0:
        return np.zeros(0, np.int64)
    thr = np.partition(v, n - k)[n - k]
    above = np.flatnonzero(v > thr)
    equal = np.flatnonzero(v == thr)[: k - above.shape[0]]
    ids = np.concatenate([above, equal])
    order = np.lexsort((ids, -v[ids]))
    return ids[order]


def top_k_error(approx: np.ndarray, exact: np.ndarray, k: int = 100) -> float:
    a = set(top_k(approx, k).tolist())
    e = set(top_k(exact, k).tolist())
    return len(a - e) / max(len(a), 1)


def stretch_error(approx: np.ndarray, exact: np.ndarray, source: int) -> dict:
    approx = np.asarray(approx, np.uint64)
    exact = np.asarray(exact, np.uint64)
    sel = (exact != UNREACHED) & (exact > 0)
    sel[source] = False
    n = int(sel.sum())
    if n == 0:
        return {"error": 0.0, "mean_stretch": 1.0, "unreached": 0, "reachable": 0}
    a = approx[sel]
    e = exact[sel].astype(np.float64)
    reached = a != UNREACHED
    stretch = np.where(reached, a.astype(np.float64) / e, np.nan)
    per_vertex = np.where(reached, stretch - 1.0, 1.0)
    return {"error": float(per_vertex.mean()),
            "mean_stretch": float(np.nanmean(stretch)) if reached.any() else float("inf"),
            "unreached": int((~reached).sum()), "reachable": n}


def wcc_relative_error(approx_labels: np.ndarray, exact_labels: np.ndarray) -> dict:
    ca = len(np.unique(approx_labels))
    ce = len(np.unique(exact_labels))
    return {"error": abs(ca - ce) / max(ce, 1), "components_approx": ca, "components_exact": ce,
            "mislabelled": float(np.mean(np.asarray(approx_labels) != np.asarray(exact_labels)))}


def accuracy(error: float) -> float:
    return (1.0 - error) * 100.0

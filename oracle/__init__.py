"""GraphGuess oracle - TEST INFRASTRUCTURE ONLY.

A plain CPU restatement of GraphGuess (arXiv 2104.10039) used to judge the
CUDA library: the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import it; the product path never does. It shares no
code with the CUDA library (``paper_2104_10039_gb300``) and neither imports
the other. PageRank runs in FP64, the min applications in exact integers.

The arithmetic lives in ``gg_oracle.c`` (compiled with gcc on first use);
this module only marshals arguments. Each function cites the part of the
paper it restates:

* ``csc_from_csr``   - in-edge view for pull-based gathering (Sec. 3.1).
* ``sample_mask``    - uniform sparsification with ratio sigma (Sec. 3.4).
* ``iteration_mode`` - approximate window alpha, corrections, SP and SMS
                       schedules (Sec. 3.4, Sec. 5.2).
* ``run``            - the vertex program of Alg. 1 / Alg. 2 (GG-Gather with
                       edge influence, GG-Apply, GG-VStatus, GG-EStatus) under
                       the accurate / approximate modes of Sec. 3.3.

The paper prints no worked numeric example of approximate-mode PageRank
after a correction (its influence figures are missing); that part is pinned
against a replica in exact rational arithmetic on tiny graphs (the tests'
brute-force module), and the GPU's FP32 flags are judged by mask replay.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gg_oracle.c")
_LIB = os.path.join(_HERE, "libggoracle.so")
_lib = None

PAGERANK, SSSP, BFS, CC, PPR = 0, 1, 2, 3, 4
APPS = {"pagerank": PAGERANK, "pr": PAGERANK, "sssp": SSSP, "bfs": BFS, "cc": CC, "ppr": PPR}
EXACT, NONE, STATIC_SWITCH, ADAPTIVE, TRIGGERED, LEARNED = 0, 1, 2, 3, 4, 5
POLICIES = {"exact": EXACT, "none": NONE, "sp": NONE, "static_switch": STATIC_SWITCH,
            "sms": STATIC_SWITCH, "adaptive": ADAPTIVE, "gg": ADAPTIVE, "triggered": TRIGGERED,
            "learned": LEARNED}
MLP_NPARAM = 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1   # W1, b1, W2, b2, w3, b3
MODE_APPROX, MODE_ACCURATE, MODE_CORRECTION = 0, 1, 2
STOP_QUIESCE, EST_STRICT, INFL_SHARE, RENORM = 1, 2, 32, 64
INF = 0xFFFFFFFF


class _Params(ctypes.Structure):
    _fields_ = [("app", ctypes.c_int32), ("policy", ctypes.c_int32),
                ("sample_ratio", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("alpha", ctypes.c_uint32), ("theta", ctypes.c_double),
                ("max_iters", ctypes.c_uint32), ("damping", ctypes.c_double),
                ("epsilon", ctypes.c_double), ("source", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("symmetric", ctypes.c_int32),
                ("nthreads", ctypes.c_int32),
                ("replay_masks", ctypes.POINTER(ctypes.c_uint8)),
                ("n_replay", ctypes.c_int32), ("replay_tol", ctypes.c_double),
                ("trigger_ratio", ctypes.c_double), ("replay_modes", ctypes.POINTER(ctypes.c_int8)),
                ("mlp", ctypes.POINTER(ctypes.c_float)), ("select_logit", ctypes.c_double),
                ("fallback_frac", ctypes.c_double), ("replay_select", ctypes.POINTER(ctypes.c_uint8)),
                ("n_replay_select", ctypes.c_int32), ("replay_select_tol", ctypes.c_double),
                ("trace_x", ctypes.POINTER(ctypes.c_float)), ("trace_y", ctypes.POINTER(ctypes.c_uint8)),
                ("trace_cap", ctypes.c_int64), ("label_tol", ctypes.c_double), ("select_cost", ctypes.c_float)]


class _Out(ctypes.Structure):
    _fields_ = [("pr_values", ctypes.POINTER(ctypes.c_double)),
                ("int_values", ctypes.POINTER(ctypes.c_uint32)),
                ("mask", ctypes.POINTER(ctypes.c_uint8)),
                ("iter_arcs", ctypes.POINTER(ctypes.c_int64)),
                ("iter_mode", ctypes.POINTER(ctypes.c_int32)),
                ("iter_changed", ctypes.POINTER(ctypes.c_int64)),
                ("iter_sum_delta", ctypes.POINTER(ctypes.c_double)),
                ("iter_selected", ctypes.POINTER(ctypes.c_int64)),
                ("logits", ctypes.POINTER(ctypes.c_double)),
                ("iterations", ctypes.c_int32), ("corrections", ctypes.c_int32),
                ("replay_mismatch", ctypes.c_int64), ("replay_max_margin", ctypes.c_double),
                ("replay_violations", ctypes.c_int64), ("select_mismatch", ctypes.c_int64),
                ("select_violations", ctypes.c_int64), ("select_max_margin", ctypes.c_double),
                ("trace_rows", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile gg_oracle.c into libggoracle.so (gcc -O2, OpenMP) if stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32p, u32p = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint32)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.orc_splitmix64.restype = ctypes.c_uint64
        lib.orc_splitmix64.argtypes = [ctypes.c_uint64]
        lib.orc_arc_sampled.restype = ctypes.c_int
        lib.orc_arc_sampled.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_uint64]
        lib.orc_csc_from_csr.restype = ctypes.c_int
        lib.orc_csc_from_csr.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, u32p,
                                         i32p, i32p, u32p, i32p]
        lib.orc_sample_mask.restype = None
        lib.orc_sample_mask.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_uint64, u8p]
        lib.orc_iteration_mode.restype = ctypes.c_int
        lib.orc_iteration_mode.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32]
        f32p, f64p = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)
        lib.orc_bf16.restype = ctypes.c_float
        lib.orc_bf16.argtypes = [ctypes.c_float]
        lib.orc_mlp_forward.restype = None
        lib.orc_mlp_forward.argtypes = [f32p, f32p, ctypes.c_int64, ctypes.c_int, f64p]
        lib.orc_mlp_grad.restype = ctypes.c_double
        lib.orc_mlp_grad.argtypes = [f32p, f32p, u8p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                                     ctypes.c_int, f64p]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_run.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, u32p,
                                ctypes.POINTER(_Params), ctypes.POINTER(_Out)]
        _lib = lib
    return _lib


def _p(a: Optional[np.ndarray], ct):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ct))


def splitmix64(state: int) -> int:
    """SplitMix64 output for one state (the sampling hash's mixer)."""
    return int(_load().orc_splitmix64(ctypes.c_uint64(state & 0xFFFFFFFFFFFFFFFF)))


def arc_sampled(src: int, dst: int, sigma: float, seed: int, symmetric: bool = False) -> bool:
    """Initial active flag of arc src->dst (Sec. 3.4)."""
    return bool(_load().orc_arc_sampled(src, dst, int(symmetric), sigma, seed))


def csc_from_csr(n, rowptr, colidx, weights=None):
    """In-edge (CSC) view: (in_ptr, in_src, in_w, csr_pos); in-rows list their
    sources in ascending order (Sec. 3.1's pull model gathers over them)."""
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    colidx = np.ascontiguousarray(colidx, np.int32)
    m = colidx.shape[0]
    w = None if weights is None else np.ascontiguousarray(weights, np.uint32)
    in_ptr = np.empty(n + 1, np.int32)
    in_src = np.empty(max(m, 1), np.int32)
    in_w = np.empty(max(m, 1), np.uint32)
    pos = np.empty(max(m, 1), np.int32)
    rc = _load().orc_csc_from_csr(n, m, _p(rowptr, ctypes.c_int32), _p(colidx, ctypes.c_int32),
                                  _p(w, ctypes.c_uint32), _p(in_ptr, ctypes.c_int32),
                                  _p(in_src, ctypes.c_int32), _p(in_w, ctypes.c_uint32),
                                  _p(pos, ctypes.c_int32))
    if rc != 0:
        raise ValueError("bad graph")
    return in_ptr, in_src[:m], in_w[:m], pos[:m]


def sample_mask(n, in_ptr, in_src, sigma, seed, symmetric=False) -> np.ndarray:
    """uint8 flag per CSC arc after sparsification with ratio sigma (Sec. 3.4)."""
    in_ptr = np.ascontiguousarray(in_ptr, np.int32)
    in_src = np.ascontiguousarray(in_src, np.int32)
    mask = np.empty(max(in_src.shape[0], 1), np.uint8)
    _load().orc_sample_mask(n, _p(in_ptr, ctypes.c_int32), _p(in_src, ctypes.c_int32),
                            int(symmetric), sigma, seed, _p(mask, ctypes.c_uint8))
    return mask[:in_src.shape[0]]


def iteration_mode(policy, alpha: int, i: int) -> int:
    """MODE_APPROX / MODE_ACCURATE / MODE_CORRECTION of iteration i."""
    pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
    return int(_load().orc_iteration_mode(pol, alpha, i))


def run(n, rowptr, colidx, weights=None, *, app="pagerank", policy="exact", sigma=1.0,
        seed=0, alpha=4, theta=0.05, max_iters=20, damping=0.85, epsilon=0.0, source=0,
        flags=0, symmetric=False, nthreads=1, replay_masks=None, replay_tol=1e-5,
        trigger_ratio=0.5, replay_modes=None, mlp=None, select_logit=0.0, fallback_frac=1.0,
        replay_select=None, replay_select_tol=0.05, trace_cap=0, label_tol=1e-3, select_cost=0.0):
    """Run one GraphGuess execution on the CPU; returns a dict with ``values``
    (float64 for PageRank, uint32 otherwise), the final CSC-order ``mask`` and
    per-iteration statistics. ``damping`` and ``theta`` are given as the float32
    values the CUDA library receives. ``replay_masks`` (list of uint8[m] CSC
    masks, one per correction) makes the run adopt those flags after checking
    that every decision it disagrees with lies within ``replay_tol`` of theta.
    ``policy="triggered"`` corrects after the approximate iteration whose change
    statistic (changed vertices; sum |old-new| for PageRank) is at most
    ``trigger_ratio`` times the window's first, or after ``alpha`` approximate
    iterations. ``replay_modes`` (int per iteration, MODE_*) makes the run
    follow the given modes instead of its policy's (iterations past the given
    ones are approximate). ``policy="learned"`` scores every vertex with the
    MLP ``mlp`` (MLP_NPARAM float32) at each correction and corrects only
    those with a logit above ``select_logit`` (plus ``select_cost`` times the bit
    length of the vertex's in-degree, as one fused float operation);
    ``replay_select`` (uint8[n] per
    learned correction) adopts the given selections after checking that every
    differing one lies within ``replay_select_tol`` of the threshold.
    ``trace_cap`` > 0 records features / labels of every vertex at each full
    correction (``trace_x``, ``trace_y``)."""
    a = APPS[app] if isinstance(app, str) else int(app)
    pol = POLICIES[policy] if isinstance(policy, str) else int(policy)
    rowptr = np.ascontiguousarray(rowptr, np.int32)
    colidx = np.ascontiguousarray(colidx, np.int32)
    m = int(colidx.shape[0])
    w = None if weights is None else np.ascontiguousarray(weights, np.uint32)
    rep = None
    n_rep = 0
    if replay_masks is not None and len(replay_masks):
        rep = np.ascontiguousarray(np.stack([np.asarray(x, np.uint8) for x in replay_masks]))
        n_rep = rep.shape[0]
    modes = None
    if replay_modes is not None:
        modes = np.full(max(max_iters, 1), 0, np.int8)
        modes[:len(replay_modes)] = np.asarray(replay_modes, np.int8)
    mlp_a = None if mlp is None else np.ascontiguousarray(mlp, np.float32)
    if mlp_a is not None and mlp_a.shape[0] != MLP_NPARAM:
        raise ValueError("mlp must hold %d parameters" % MLP_NPARAM)
    rsel = None
    n_rsel = 0
    if replay_select is not None and len(replay_select):
        rsel = np.ascontiguousarray(np.stack([np.asarray(x, np.uint8) for x in replay_select]))
        n_rsel = rsel.shape[0]
    tx = np.zeros((max(trace_cap, 1), 8), np.float32) if trace_cap > 0 else None
    ty = np.zeros(max(trace_cap, 1), np.uint8) if trace_cap > 0 else None
    prm = _Params(a, pol, float(sigma), seed & 0xFFFFFFFFFFFFFFFF, alpha,
                  float(np.float32(theta)), max_iters, float(np.float32(damping)),
                  float(np.float32(epsilon)), source, flags, int(symmetric), nthreads,
                  _p(rep, ctypes.c_uint8), n_rep, replay_tol, float(np.float32(trigger_ratio)),
                  _p(modes, ctypes.c_int8), _p(mlp_a, ctypes.c_float), float(select_logit),
                  float(fallback_frac), _p(rsel, ctypes.c_uint8), n_rsel, float(replay_select_tol),
                  _p(tx, ctypes.c_float), _p(ty, ctypes.c_uint8), int(trace_cap), float(label_tol),
                  float(np.float32(select_cost)))
    T = max(max_iters, 1)
    pr = np.empty(n, np.float64) if a in (PAGERANK, PPR) else None
    iv = np.empty(n, np.uint32) if a not in (PAGERANK, PPR) else None
    mask = np.empty(max(m, 1), np.uint8)
    it_arcs = np.zeros(T, np.int64)
    it_mode = np.full(T, -1, np.int32)
    it_changed = np.zeros(T, np.int64)
    it_sum = np.zeros(T, np.float64)
    it_sel = np.full(T, -1, np.int64)
    logits = np.full(n, np.nan, np.float64)
    out = _Out(_p(pr, ctypes.c_double), _p(iv, ctypes.c_uint32), _p(mask, ctypes.c_uint8),
               _p(it_arcs, ctypes.c_int64), _p(it_mode, ctypes.c_int32),
               _p(it_changed, ctypes.c_int64), _p(it_sum, ctypes.c_double), _p(it_sel, ctypes.c_int64),
               _p(logits, ctypes.c_double), 0, 0, 0, 0.0, 0, 0, 0, 0.0, 0)
    rc = _load().orc_run(n, m, _p(rowptr, ctypes.c_int32), _p(colidx, ctypes.c_int32),
                         _p(w, ctypes.c_uint32), ctypes.byref(prm), ctypes.byref(out))
    if rc != 0:
        raise ValueError("oracle rejected its arguments")
    it = out.iterations
    return {
        "values": pr if a in (PAGERANK, PPR) else iv,
        "mask": mask[:m],
        "iterations": it,
        "corrections": out.corrections,
        "iter_arcs": it_arcs[:it],
        "iter_mode": it_mode[:it],
        "iter_changed": it_changed[:it],
        "iter_sum_delta": it_sum[:it],
        "iter_selected": it_sel[:it],
        "logits": logits,
        "select_mismatch": out.select_mismatch,
        "select_violations": out.select_violations,
        "select_max_margin": out.select_max_margin,
        "trace_x": tx[:out.trace_rows] if tx is not None else None,
        "trace_y": ty[:out.trace_rows] if ty is not None else None,
        "replay_mismatch": out.replay_mismatch,
        "replay_max_margin": out.replay_max_margin,
        "replay_violations": out.replay_violations,
    }


# ------------------------------------------------------------------ scorer --

def bf16(x) -> np.ndarray:
    """float32 values rounded to bfloat16 (nearest, ties to even), as float32."""
    x = np.asarray(x, np.float32)
    lib = _load()
    return np.array([lib.orc_bf16(float(v)) for v in x.ravel()], np.float32).reshape(x.shape)


def mlp_forward(params, x, round_bf16=True) -> np.ndarray:
    """Logits (float64) of the feature rows x[rows, 8] under the scorer's
    arithmetic (bfloat16 weights and layer inputs, exact sums)."""
    P = np.ascontiguousarray(params, np.float32)
    X = np.ascontiguousarray(x, np.float32).reshape(-1, 8)
    out = np.empty(X.shape[0], np.float64)
    _load().orc_mlp_forward(_p(P, ctypes.c_float), _p(X, ctypes.c_float), X.shape[0], int(round_bf16),
                            _p(out, ctypes.c_double))
    return out


def mlp_grad(params, x, y, idx=None, round_bf16=True):
    """(gradient float64[MLP_NPARAM], mean logistic loss) over rows idx."""
    P = np.ascontiguousarray(params, np.float32)
    X = np.ascontiguousarray(x, np.float32).reshape(-1, 8)
    Y = np.ascontiguousarray(y, np.uint8)
    I = np.arange(X.shape[0], dtype=np.int64) if idx is None else np.ascontiguousarray(idx, np.int64)
    g = np.empty(MLP_NPARAM, np.float64)
    loss = _load().orc_mlp_grad(_p(P, ctypes.c_float), _p(X, ctypes.c_float), _p(Y, ctypes.c_uint8),
                                _p(I, ctypes.c_int64), I.shape[0], int(round_bf16), _p(g, ctypes.c_double))
    return g, float(loss)


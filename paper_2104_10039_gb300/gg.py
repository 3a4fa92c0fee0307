"""Python binding of libgg.so (include/gg.h): the same entry points, argument
marshalling only. Every step of the computation runs in the library's CUDA
kernels; there is no Python or CPU fallback. Importing this module raises if
libgg.so has not been built (``python -m paper_2104_10039_gb300.build``).

Array arguments are numpy arrays (host) or any object with ``data_ptr()``
(e.g. a CUDA torch tensor, device memory) or plain integer addresses.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libgg.so is not built ({LIB_PATH}); run "
                      "`python -m paper_2104_10039_gb300.build` (needs nvcc)")

_lib = ctypes.CDLL(LIB_PATH)

# ---- enums and flags (gg.h) ---------------------------------------------
GG_OK, GG_ERR_INVALID_ARG, GG_ERR_BAD_GRAPH, GG_ERR_OOM, GG_ERR_CUDA, GG_ERR_STATE, \
    GG_ERR_TIMEOUT, GG_ERR_UNSUPPORTED = range(8)
GG_APP_PAGERANK, GG_APP_SSSP, GG_APP_BFS, GG_APP_CC, GG_APP_PPR = range(5)
GG_POLICY_EXACT, GG_POLICY_NONE, GG_POLICY_STATIC_SWITCH, GG_POLICY_ADAPTIVE, GG_POLICY_TRIGGERED, \
    GG_POLICY_LEARNED = range(6)
(GG_RESULT_VALUES, GG_RESULT_MASK, GG_RESULT_STATS, GG_RESULT_ITER_STATS, GG_RESULT_CSC_PTR,
 GG_RESULT_CSC_SRC, GG_RESULT_CSC_W, GG_RESULT_SPARSE_PTR, GG_RESULT_SPARSE_SRC,
 GG_RESULT_OUT_TO_IN, GG_RESULT_SCORES) = range(11)
GG_DIRECTED, GG_SYMMETRIC, GG_DEVICE_PTRS = 0, 1, 2
GG_STOP_QUIESCE, GG_EST_STRICT, GG_FORCE_PULL, GG_FORCE_PUSH, GG_TIMING = 1, 2, 4, 8, 16
GG_INFL_SHARE, GG_RENORM, GG_PULL_FILTER = 32, 64, 128
GG_INF = 0xFFFFFFFF
GG_ITER_PUSH = 0x100
GG_ITER_LEARNED = 0x200
GG_ITER_FILTER = 0x400

APPS = {"pagerank": GG_APP_PAGERANK, "pr": GG_APP_PAGERANK, "sssp": GG_APP_SSSP,
        "bfs": GG_APP_BFS, "cc": GG_APP_CC, "ppr": GG_APP_PPR}
POLICIES = {"exact": GG_POLICY_EXACT, "none": GG_POLICY_NONE, "sp": GG_POLICY_NONE,
            "static_switch": GG_POLICY_STATIC_SWITCH, "sms": GG_POLICY_STATIC_SWITCH,
            "adaptive": GG_POLICY_ADAPTIVE, "gg": GG_POLICY_ADAPTIVE,
            "triggered": GG_POLICY_TRIGGERED, "learned": GG_POLICY_LEARNED}


class gg_params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_uint32), ("theta", ctypes.c_float),
                ("max_iters", ctypes.c_uint32), ("damping", ctypes.c_float),
                ("epsilon", ctypes.c_float), ("source", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("trigger_ratio", ctypes.c_float), ("select_logit", ctypes.c_float),
                ("fallback_frac", ctypes.c_float), ("select_cost", ctypes.c_float)]


class gg_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_uint32), ("corrections", ctypes.c_uint32),
                ("push_iterations", ctypes.c_uint32), ("pull_iterations", ctypes.c_uint32),
                ("arcs_processed", ctypes.c_uint64), ("active_arcs", ctypes.c_uint64),
                ("changed_last", ctypes.c_uint64), ("device_error", ctypes.c_uint32),
                ("kernels_load", ctypes.c_uint32), ("ms_load", ctypes.c_float),
                ("ms_sample", ctypes.c_float), ("ms_run", ctypes.c_float),
                ("ms_gather", ctypes.c_float), ("ms_correct", ctypes.c_float),
                ("ms_push", ctypes.c_float), ("n_gather", ctypes.c_uint32),
                ("n_correct", ctypes.c_uint32), ("n_push", ctypes.c_uint32),
                ("kernels_launched", ctypes.c_uint32), ("learned_corrections", ctypes.c_uint32),
                ("trace_rows", ctypes.c_uint64)]


ITER_STATS_DTYPE = np.dtype([("mode", np.uint32), ("max_delta_bits", np.uint32),
                             ("arcs", np.uint64), ("changed", np.uint64),
                             ("sum_delta", np.uint64), ("active_after", np.uint64),
                             ("selected", np.uint64)])

_vp = ctypes.c_void_p
_lib.gg_load_csr.restype = ctypes.c_int
_lib.gg_load_csr.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.c_int64, _vp, _vp, _vp,
                             ctypes.c_uint32]
_lib.gg_sample_edges.restype = ctypes.c_int
_lib.gg_sample_edges.argtypes = [_vp, ctypes.c_double, ctypes.c_uint64]
_lib.gg_run.restype = ctypes.c_int
_lib.gg_run.argtypes = [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(gg_params)]
_lib.gg_result.restype = ctypes.c_int
_lib.gg_result.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int]
_lib.gg_result_size.restype = ctypes.c_size_t
_lib.gg_result_size.argtypes = [_vp, ctypes.c_int]
_lib.gg_set_stream.restype = ctypes.c_int
_lib.gg_set_stream.argtypes = [_vp, _vp]
_lib.gg_free_graph.restype = None
_lib.gg_free_graph.argtypes = [_vp]
_lib.gg_last_error.restype = ctypes.c_char_p
_lib.gg_last_error.argtypes = []
_lib.gg_sample_csc_noalloc.restype = ctypes.c_int
_lib.gg_sample_csc_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int64, _vp, _vp, ctypes.c_double,
                                       ctypes.c_uint64, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
GG_NOALLOC_MAX_ITEMS = 1 << 24
_lib.gg_set_scorer.restype = ctypes.c_int
_lib.gg_set_scorer.argtypes = [_vp, _vp]
_lib.gg_set_trace.restype = ctypes.c_int
_lib.gg_set_trace.argtypes = [_vp, _vp, _vp, ctypes.c_uint64, ctypes.c_float]
_lib.gg_mlp_score.restype = ctypes.c_int
_lib.gg_mlp_score.argtypes = [_vp, ctypes.c_uint64, _vp, _vp, _vp]
_lib.gg_mlp_train.restype = ctypes.c_int
_lib.gg_mlp_train.argtypes = [_vp, _vp, ctypes.c_uint64, _vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_float,
                              ctypes.c_uint64, ctypes.c_uint64, _vp, _vp, _vp]
GG_MLP_NPARAM = 4801


class GGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where} failed with status {status}: {gg_last_error()}")


def _check(status: int, where: str):
    if status != GG_OK:
        raise GGError(status, where)


def _addr(x) -> Optional[int]:
    """Address of a buffer: numpy array, object with data_ptr(), int or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    return int(x)


def gg_last_error() -> str:
    msg = _lib.gg_last_error()
    return msg.decode() if msg else ""


def gg_load_csr(n: int, m: int, rowptr, colidx, weights=None, gflags: int = GG_DIRECTED) -> int:
    """Load a CSR graph; returns the opaque handle (an integer)."""
    h = _vp()
    _check(_lib.gg_load_csr(ctypes.byref(h), n, m, _addr(rowptr), _addr(colidx), _addr(weights),
                            gflags), "gg_load_csr")
    return h.value


def gg_sample_edges(g: int, sample_ratio: float, seed: int):
    _check(_lib.gg_sample_edges(g, sample_ratio, seed & 0xFFFFFFFFFFFFFFFF), "gg_sample_edges")


def make_params(alpha=4, theta=0.05, max_iters=20, damping=0.85, epsilon=0.0, source=0, seed=0,
                flags=0, trigger_ratio=0.5, select_logit=0.0, fallback_frac=1.0, select_cost=0.0) -> gg_params:
    return gg_params(alpha, theta, max_iters, damping, epsilon, source,
                     seed & 0xFFFFFFFFFFFFFFFF, flags, trigger_ratio, select_logit, fallback_frac, select_cost)


def gg_run(g: int, app, sample_ratio: float, policy, params: gg_params):
    a = APPS[app] if isinstance(app, str) else int(app)
    p = POLICIES[policy] if isinstance(policy, str) else int(policy)
    _check(_lib.gg_run(g, a, sample_ratio, p, ctypes.byref(params)), "gg_run")


GG_RESULT_SIZE_ERROR = (1 << 64) - 1


def gg_result_size(g: int, kind: int) -> int:
    n = int(_lib.gg_result_size(g, kind))
    if n == GG_RESULT_SIZE_ERROR:
        raise GGError(GG_ERR_CUDA, "gg_result_size")
    return n


def gg_result(g: int, kind: int, dst, nbytes: int, dst_is_device: bool = False):
    _check(_lib.gg_result(g, kind, _addr(dst), nbytes, int(dst_is_device)), "gg_result")


def gg_set_stream(g: int, stream):
    """stream: a cudaStream_t value, e.g. torch.cuda.current_stream().cuda_stream."""
    _check(_lib.gg_set_stream(g, stream), "gg_set_stream")


def gg_free_graph(g: int):
    _lib.gg_free_graph(g)


def gg_sample_csc_noalloc(n: int, m: int, in_ptr, in_src, sample_ratio: float, seed: int,
                          symmetric: bool, mask, sp_ptr, sp_src, sp_nnz, stream=None):
    """Sampling of caller-owned device arrays without any device allocation
    (see gg.h); every array argument is device memory."""
    _check(_lib.gg_sample_csc_noalloc(n, m, _addr(in_ptr), _addr(in_src), sample_ratio,
                                      seed & 0xFFFFFFFFFFFFFFFF, int(symmetric), _addr(mask),
                                      _addr(sp_ptr), _addr(sp_src), _addr(sp_nnz),
                                      None if stream is None else int(stream)),
           "gg_sample_csc_noalloc")


# ---- convenience wrappers (still only marshalling) -----------------------
_RESULT_DTYPES = {GG_RESULT_MASK: np.uint32, GG_RESULT_CSC_PTR: np.int32,
                  GG_RESULT_CSC_SRC: np.int32, GG_RESULT_CSC_W: np.uint32,
                  GG_RESULT_SPARSE_PTR: np.int32, GG_RESULT_SPARSE_SRC: np.int32,
                  GG_RESULT_OUT_TO_IN: np.int32, GG_RESULT_SCORES: np.float32}


def result_array(g: int, kind: int, dtype=None) -> np.ndarray:
    """Copy a result into a new host numpy array."""
    nbytes = gg_result_size(g, kind)
    if kind == GG_RESULT_ITER_STATS:
        out = np.empty(nbytes // ITER_STATS_DTYPE.itemsize, ITER_STATS_DTYPE)
    else:
        dt = np.dtype(dtype or _RESULT_DTYPES.get(kind, np.uint32))
        out = np.empty(nbytes // dt.itemsize, dt)
    if nbytes:
        gg_result(g, kind, out, nbytes)
    return out


def values(g: int, app) -> np.ndarray:
    a = APPS[app] if isinstance(app, str) else int(app)
    return result_array(g, GG_RESULT_VALUES, np.float32 if a == GG_APP_PAGERANK else np.uint32)


def stats(g: int) -> gg_stats:
    s = gg_stats()
    gg_result(g, GG_RESULT_STATS, ctypes.addressof(s), ctypes.sizeof(s))
    return s


def mask_bits(g: int, m: int) -> np.ndarray:
    """Edge flags as a uint8 array over the m CSC arcs."""
    words = result_array(g, GG_RESULT_MASK)
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")
    return bits[:m].astype(np.uint8)


def gg_set_scorer(g: int, params: np.ndarray):
    """Scorer parameters (host float32[GG_MLP_NPARAM]) for GG_POLICY_LEARNED."""
    P = np.ascontiguousarray(params, np.float32)
    if P.shape != (GG_MLP_NPARAM,):
        raise ValueError(f"params must hold {GG_MLP_NPARAM} float32 values")
    _check(_lib.gg_set_scorer(g, P.ctypes.data), "gg_set_scorer")


def gg_set_trace(g: int, features, labels, cap_rows: int, label_tol: float = 1e-3):
    """Record training rows into device buffers features[cap_rows][8] (float32)
    and labels[cap_rows] (uint8); features=None stops recording."""
    _check(_lib.gg_set_trace(g, _addr(features), _addr(labels), int(cap_rows), float(label_tol)),
           "gg_set_trace")


def gg_mlp_score(features, rows: int, params, logits, stream=None):
    """Logits of device feature rows (float32[rows][8]) into device logits[rows]."""
    _check(_lib.gg_mlp_score(_addr(features), int(rows), _addr(params), _addr(logits), _addr(stream)),
           "gg_mlp_score")


def gg_mlp_train(features, labels, rows: int, params, batch: int, steps: int, lr: float, stride: int,
                 start: int = 0, losses=None, grad_last=None, stream=None):
    """Minibatch SGD on the scorer's device parameters (updated in place)."""
    _check(_lib.gg_mlp_train(_addr(features), _addr(labels), int(rows), _addr(params), int(batch), int(steps),
                             float(lr), int(stride), int(start), _addr(losses), _addr(grad_last), _addr(stream)),
           "gg_mlp_train")


# ------------------------------------------------------- batched serving --
class gg_query(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_int32), ("app", ctypes.c_int32), ("source", ctypes.c_int32),
                ("iters", ctypes.c_uint32), ("damping", ctypes.c_float), ("warp_deg", ctypes.c_int32),
                ("cta_deg", ctypes.c_int32)]


class gg_batch_config(ctypes.Structure):
    _fields_ = [("cluster", ctypes.c_int32), ("warp_deg", ctypes.c_int32), ("cta_deg", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("big_arcs", ctypes.c_int64), ("small_first", ctypes.c_int32),
                ("order", ctypes.c_int32)]


class gg_query_stats(ctypes.Structure):
    _fields_ = [("latency_ns", ctypes.c_uint64), ("service_ns", ctypes.c_uint64), ("arcs", ctypes.c_uint64),
                ("iterations", ctypes.c_uint32), ("team", ctypes.c_uint32)]


_lib.gg_batch_create.restype = ctypes.c_int
_lib.gg_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(gg_query), ctypes.c_int32,
                                 ctypes.POINTER(gg_batch_config), ctypes.POINTER(_vp)]
_lib.gg_batch_run.restype = ctypes.c_int
_lib.gg_batch_run.argtypes = [_vp, ctypes.POINTER(ctypes.c_float)]
_lib.gg_batch_query_stats.restype = ctypes.c_int
_lib.gg_batch_query_stats.argtypes = [_vp, ctypes.POINTER(gg_query_stats), ctypes.c_int32]
_lib.gg_batch_result.restype = ctypes.c_int
_lib.gg_batch_result.argtypes = [_vp, ctypes.c_int32, _vp, ctypes.c_size_t]
_lib.gg_batch_free.restype = None
_lib.gg_batch_free.argtypes = [_vp]


def make_query(graph: int, app, source: int, iters: int = 20, damping: float = 0.85, warp_deg: int = 0,
               cta_deg: int = 0) -> gg_query:
    a = APPS[app] if isinstance(app, str) else int(app)
    return gg_query(graph, a, source, iters, damping, warp_deg, cta_deg)


GG_ORDER_MOST_WORK, GG_ORDER_LEAST_WORK, GG_ORDER_TRAVERSALS_FIRST = 0, 1, 2


def gg_batch_create(graphs, queries, cluster=4, warp_deg=32, cta_deg=1024, big_arcs=1 << 22, threads=256,
                    small_first=0, order=GG_ORDER_MOST_WORK) -> int:
    """Plan a batch over loaded graph handles; returns the batch handle."""
    ga = (_vp * len(graphs))(*graphs)
    qa = (gg_query * len(queries))(*queries)
    cfg = gg_batch_config(cluster, warp_deg, cta_deg, threads, big_arcs, small_first, order)
    h = _vp()
    _check(_lib.gg_batch_create(ga, len(graphs), qa, len(queries), ctypes.byref(cfg), ctypes.byref(h)),
           "gg_batch_create")
    return h.value


def gg_batch_run(b: int) -> float:
    """Serve every query; returns the launch's device time in ms."""
    ms = ctypes.c_float(0.0)
    _check(_lib.gg_batch_run(b, ctypes.byref(ms)), "gg_batch_run")
    return ms.value


def gg_batch_query_stats(b: int, n: int) -> np.ndarray:
    out = (gg_query_stats * n)()
    _check(_lib.gg_batch_query_stats(b, out, n), "gg_batch_query_stats")
    return np.array([(s.latency_ns, s.service_ns, s.arcs, s.iterations, s.team) for s in out],
                    dtype=[("latency_ns", np.uint64), ("service_ns", np.uint64), ("arcs", np.uint64),
                           ("iterations", np.uint32), ("team", np.uint32)])


def gg_batch_result(b: int, q: int, n: int, app) -> np.ndarray:
    a = APPS[app] if isinstance(app, str) else int(app)
    out = np.empty(n, np.float32 if a == GG_APP_PPR else np.uint32)
    _check(_lib.gg_batch_result(b, q, out.ctypes.data, out.nbytes), "gg_batch_result")
    return out


def gg_batch_free(b: int):
    _lib.gg_batch_free(b)

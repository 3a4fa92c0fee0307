/*
 * gg.h - C ABI of libgg.so, a GB300 (sm_103a) implementation of GraphGuess
 * (Ramezani, Kandemir, Sivasubramaniam, "GraphGuess: Approximate Graph
 * Processing System with Adaptive Correction", arXiv 2104.10039).
 *
 * The problem (Sec. 3): run a vertex program over an unchanged graph whose
 * edges carry one active flag each (Sec. 3.3), starting from a sampled
 * fraction sigma of active edges (Sec. 3.4), with approximate iterations
 * (active in-edges only) and periodic correction iterations (all in-edges,
 * edge influence recomputed, flags reset to influence > theta), trading
 * accuracy for time.
 *
 * Conventions shared by every entry point
 *  - Every call returns a gg_status; nothing aborts the process. On failure
 *    gg_last_error() returns a message (thread-local, valid until the next
 *    call on the same thread).
 *  - Pointers are host pointers unless a flag or argument says device.
 *  - All device work is enqueued on the graph's stream (gg_set_stream,
 *    default: the legacy default stream). Only gg_result and gg_run of the
 *    min applications synchronise it.
 *  - Indices are int32 (n < 2^31, m < 2^31). Vertex values of SSSP, BFS and
 *    CC are uint32 with GG_INF = 0xFFFFFFFF meaning "unreached".
 *  - The library owns all device memory it allocates; it is released by
 *    gg_free_graph.
 *  - No kernel of the library waits on another block or another launch, so
 *    no call can hang on the device; GG_ERR_TIMEOUT stays reserved in the
 *    status enum and is not returned.
 */
#ifndef GG_H
#define GG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GG_OK = 0,
    GG_ERR_INVALID_ARG = 1,   /* null pointer, size or parameter out of range */
    GG_ERR_BAD_GRAPH = 2,     /* CSR not monotone, rowptr[0] != 0, rowptr[n] != m, colidx out of range */
    GG_ERR_OOM = 3,           /* a device allocation failed */
    GG_ERR_CUDA = 4,          /* a CUDA call failed; the CUDA error string is in gg_last_error() */
    GG_ERR_STATE = 5,         /* call not valid in the graph's current state */
    GG_ERR_TIMEOUT = 6,       /* reserved (no device-side waits) */
    GG_ERR_UNSUPPORTED = 7    /* combination not implemented */
} gg_status;

typedef enum {
    GG_APP_PAGERANK = 0,      /* Alg. 2: pull PageRank, FP32 ranks */
    GG_APP_SSSP = 1,          /* Sec. 4.1: single-source shortest paths, uint32 weights */
    GG_APP_BFS = 2,           /* unit-weight SSSP: levels */
    GG_APP_CC = 3,            /* Sec. 4.1 WCC: min-label propagation (symmetric graphs) */
    GG_APP_PPR = 4            /* beyond the paper: personalized PageRank from the source,
                                 rank_0 = e_s, rank' = (1-d) e_s + d * sum rank(v)/outdeg(v) */
} gg_app;

typedef enum {
    GG_POLICY_EXACT = 0,          /* accurate mode every iteration (the paper's baseline, Sec. 5) */
    GG_POLICY_NONE = 1,           /* SP: sparsify with sigma, never correct (Sec. 5.2) */
    GG_POLICY_STATIC_SWITCH = 2,  /* SMS: approximate for alpha iterations, one correction,
                                     then accurate to the end (Sec. 5.2) */
    GG_POLICY_ADAPTIVE = 3,       /* GG: a correction after every alpha approximate
                                     iterations (Sec. 3.4) */
    GG_POLICY_TRIGGERED = 4,      /* beyond the paper (which notes the correction points could
                                     vary, Sec. 3.4): a correction follows the approximate
                                     iteration whose change statistic is at most trigger_ratio
                                     times that of the first approximate iteration since the last
                                     correction, or the alpha-th one. Statistic: vertices changed
                                     (SSSP/BFS/CC, exact) or sum |old-new| (PageRank, the
                                     fixed-point sum of gg_iter_stats.sum_delta) */
    GG_POLICY_LEARNED = 5         /* beyond the paper: the GG schedule, but at a correction the
                                     scorer set by gg_set_scorer selects the vertices to correct
                                     (logit > select_logit): they gather over all in-edges and
                                     recompute their flags; every other vertex keeps its value and
                                     flags for that iteration. A selection holding more than
                                     fallback_frac of the arcs runs the full correction instead,
                                     and so does the correction after a learned one that changed
                                     no value (min applications: no vertex decreased; PageRank: no
                                     |old-new| above epsilon) */
} gg_policy;

typedef enum {
    GG_RESULT_VALUES = 0,     /* float[n] (PageRank) or uint32[n]: vertex values after the last run */
    GG_RESULT_MASK = 1,       /* uint32[ceil(m/32)]: edge flags, bit (k & 31) of word k/32 = CSC arc k */
    GG_RESULT_STATS = 2,      /* gg_stats */
    GG_RESULT_ITER_STATS = 3, /* gg_iter_stats[iterations] of the last run */
    GG_RESULT_CSC_PTR = 4,    /* int32[n+1]: in-edge row pointers */
    GG_RESULT_CSC_SRC = 5,    /* int32[m]: in-edge sources, each row ascending */
    GG_RESULT_CSC_W = 6,      /* uint32[m]: in-edge weights (graphs loaded with weights) */
    GG_RESULT_SPARSE_PTR = 7, /* int32[n+1]: row pointers of the packed active in-edges */
    GG_RESULT_SPARSE_SRC = 8, /* int32[nnz]: sources of the packed active in-edges */
    GG_RESULT_OUT_TO_IN = 9,  /* int32[m]: CSC position of every CSR arc */
    GG_RESULT_SCORES = 10     /* float[n]: logits of the last learned correction's scoring */
} gg_result_kind;

/* gg_load_csr gflags */
#define GG_DIRECTED 0u
#define GG_SYMMETRIC 1u       /* every arc u->v has a matching v->u; sampling keys on the
                                 unordered pair so both directions start with the same flag */
#define GG_DEVICE_PTRS 2u     /* rowptr / colidx / weights are device pointers */

/* gg_params.flags */
#define GG_STOP_QUIESCE 1u    /* PageRank: stop after an accurate iteration with no active vertex */
#define GG_EST_STRICT 2u      /* corrections also clear flags of arcs whose source is unreached */
#define GG_FORCE_PULL 4u      /* min applications: never use the push frontier */
#define GG_FORCE_PUSH 8u      /* min applications: always push from the frontier (no pull switch) */
#define GG_TIMING 16u         /* record per-kernel-class device time with CUDA events */
#define GG_INFL_SHARE 32u     /* PageRank corrections: influence = the arc's share of its row's total
                                 (order-free) instead of the running-prefix form of Alg. 2 */
#define GG_RENORM 64u         /* PageRank: approximate iterations divide a source's rank by its number
                                 of active out-arcs (no rank mass leaks through inactive arcs) */
#define GG_PULL_FILTER 128u   /* min applications: pull gathers read only the values of frontier sources
                                 (a bitmap of the frontier). Same results; off by default, since on
                                 GB300 the bitmap lookup per arc costs more than the reads it saves */

#define GG_INF 0xFFFFFFFFu
#define GG_ITER_PUSH 0x100u   /* gg_iter_stats.mode bit: iteration done by the push frontier */
#define GG_ITER_LEARNED 0x200u /* gg_iter_stats.mode bit: a correction of the selected vertices only */
#define GG_ITER_FILTER 0x400u /* gg_iter_stats.mode bit: a pull gather that read frontier sources only */

typedef struct {
    uint32_t alpha;       /* approximate window: approximate iterations between corrections (Sec. 3.4) */
    float theta;          /* influence threshold (Sec. 3.4, GG-EStatus) */
    uint32_t max_iters;   /* iteration cap T (PageRank runs exactly T unless GG_STOP_QUIESCE) */
    float damping;        /* PageRank d (Alg. 2 GG-Apply), e.g. 0.85 */
    float epsilon;        /* GG-VStatus threshold |old - new| > epsilon (PageRank) */
    int32_t source;       /* SSSP / BFS source vertex */
    uint64_t seed;        /* sampling seed (Sec. 3.4) */
    uint32_t flags;       /* GG_* flags above */
    float trigger_ratio;  /* GG_POLICY_TRIGGERED: fraction of the window's first change statistic
                             at or below which a correction follows; finite, >= 0 */
    float select_logit;   /* GG_POLICY_LEARNED: vertices whose logit exceeds this are corrected */
    float fallback_frac;  /* GG_POLICY_LEARNED: a selection with more in-edges than this x m runs
                             the full correction (1 = never; < 0 = always) */
    float select_cost;    /* GG_POLICY_LEARNED: a vertex with in-degree d is selected when its logit
                             exceeds fmaf(select_cost, L(d), select_logit), L(d) = bit length of d
                             (0 for d = 0): hub rows need stronger scores (0 = plain threshold) */
} gg_params;

typedef struct {
    uint32_t iterations;      /* iterations counted (no-op iterations skipped by R12 included) */
    uint32_t corrections;     /* correction iterations executed */
    uint32_t push_iterations; /* min applications: iterations done by the push frontier */
    uint32_t pull_iterations; /* iterations done by a pull gather (including corrections) */
    uint64_t arcs_processed;  /* sum over iterations of the iteration's edge-set size */
    uint64_t active_arcs;     /* arcs active at the end of the run */
    uint64_t changed_last;    /* vertices active after the last iteration */
    uint32_t device_error;    /* error flags of the device-side CSR validation (2: bad graph), else 0 */
    uint32_t kernels_load;    /* kernels this library launched during gg_load_csr */
    float ms_load;            /* device time of the last gg_load_csr (copy + validate + CSC build) */
    float ms_sample;          /* device time of the last sampling */
    float ms_run;             /* device time of the last gg_run (sampling included when it resampled) */
    float ms_gather;          /* GG_TIMING: total time of approximate / accurate pull gathers */
    float ms_correct;         /* GG_TIMING: total time of correction kernels */
    float ms_push;            /* GG_TIMING: total time of push-frontier kernels */
    uint32_t n_gather;        /* GG_TIMING: launches counted in ms_gather */
    uint32_t n_correct;       /* GG_TIMING: launches counted in ms_correct */
    uint32_t n_push;          /* GG_TIMING: launches counted in ms_push */
    uint32_t kernels_launched;/* kernels this library launched during the last gg_run */
    uint32_t learned_corrections; /* corrections of the selected vertices only (GG_POLICY_LEARNED) */
    uint64_t trace_rows;      /* rows written to the trace buffers since gg_set_trace */
} gg_stats;

typedef struct {
    uint32_t mode;            /* 0 approximate, 1 accurate, 2 correction, 3 skipped no-op;
                                 | GG_ITER_PUSH when the push frontier ran the iteration */
    uint32_t max_delta_bits;  /* max |old-new|: float bits (PageRank) or uint32 */
    uint64_t arcs;            /* size of the iteration's edge set */
    uint64_t changed;         /* vertices active after GG-VStatus */
    uint64_t sum_delta;       /* sum |old-new|: fixed point 2^-40 (PageRank) or exact integer
                                 over vertices that were reached before */
    uint64_t active_after;    /* active arcs after the iteration */
    uint64_t selected;        /* learned correction: vertices it corrected (else 0) */
} gg_iter_stats;

typedef struct gg_graph gg_graph;

/*
 * gg_load_csr - load a graph given by its out-edges (CSR) and build the
 * in-edge view the pull engine gathers over (Sec. 2.1 GAS gather over
 * incoming edges; Sec. 3.3 "one flag per edge", no new graph).
 *   g        out: new handle (set only on GG_OK)
 *   n, m     vertices and arcs; 1 <= n, 0 <= m < 2^31
 *   rowptr   int32[n+1], rowptr[0] = 0, non-decreasing, rowptr[n] = m
 *   colidx   int32[m], destinations in [0, n)
 *   weights  uint32[m] arc weights (needed by SSSP) or NULL
 *   gflags   GG_DIRECTED / GG_SYMMETRIC, | GG_DEVICE_PTRS for device inputs
 * The arrays are copied into library-owned device memory; the caller may
 * free them on return. The CSR is validated on the device; a bad graph
 * returns GG_ERR_BAD_GRAPH. In-edge rows list their sources in ascending
 * order (duplicates in CSR order); this order defines the running influence.
 */
gg_status gg_load_csr(gg_graph **g, int32_t n, int64_t m, const int32_t *rowptr,
                      const int32_t *colidx, const uint32_t *weights, uint32_t gflags);

/*
 * gg_sample_edges - set the initial edge flags by uniform sparsification
 * (Sec. 3.4, Fig. 1a): arc src->dst is active iff
 * SplitMix64(seed ^ (src<<32 | dst)) >> 32 < floor(sample_ratio * 2^32)
 * (the unordered pair on GG_SYMMETRIC graphs), and count the active in-edges.
 * The packed list of the active in-edges (GG_RESULT_SPARSE_*) is built when a
 * run's approximate gather or gg_result first needs it.
 *   sample_ratio  sigma in (0, 1]
 * Enqueued on the stream; returns before the work completes.
 */
gg_status gg_sample_edges(gg_graph *g, double sample_ratio, uint64_t seed);

/*
 * gg_run - one execution of a vertex program under a correction policy
 * (Sec. 3.3 modes, Sec. 3.4 adaptive correction, Sec. 5.2 SP / SMS).
 *   app           GG_APP_*; SSSP needs weights; CC expects a symmetric graph
 *   sample_ratio  sigma; the edges are (re)sampled with (sample_ratio,
 *                 p->seed) unless the current flags already are that
 *                 untouched sample. Ignored by GG_POLICY_EXACT.
 *   policy        GG_POLICY_*
 *   p             parameters (see gg_params); p->max_iters >= 1
 * PageRank runs p->max_iters iterations from rank 1/N. SSSP / BFS / CC run
 * until an accurate iteration changes nothing (or max_iters) and synchronise
 * the stream once per iteration to choose push or pull. Values stay on the
 * device until gg_result.
 */
gg_status gg_run(gg_graph *g, gg_app app, double sample_ratio, gg_policy policy,
                 const gg_params *p);

/*
 * gg_result - copy a result out (synchronises the stream).
 *   kind           GG_RESULT_*; sizes as listed in gg_result_kind
 *   dst            destination buffer (host, or device if dst_is_device)
 *   bytes          size of dst; must be at least the result's size
 * Returns GG_ERR_STATE if the result does not exist yet (e.g. VALUES before
 * any run, SPARSE_* before any sampling).
 */
gg_status gg_result(gg_graph *g, gg_result_kind kind, void *dst, size_t bytes,
                    int dst_is_device);

/* Size in bytes of a result (0 if it does not exist yet). Synchronises the
 * graph's stream. Returns GG_RESULT_SIZE_ERROR ((size_t)-1) if g is NULL or a
 * CUDA call failed; gg_last_error() then says which. */
#define GG_RESULT_SIZE_ERROR ((size_t)-1)
size_t gg_result_size(gg_graph *g, gg_result_kind kind);

/* gg_set_stream - enqueue all later work of g on this cudaStream_t (e.g.
 * torch.cuda.current_stream().cuda_stream). NULL = the legacy default stream. */
gg_status gg_set_stream(gg_graph *g, void *cuda_stream);

/* gg_free_graph - release every device buffer of g (NULL is a no-op). */
void gg_free_graph(gg_graph *g);

/* gg_last_error - message of the last failure on this thread. */
const char *gg_last_error(void);

/*
 * Learned correction (beyond the paper). The scorer is a per-vertex MLP
 * 8 -> 64 -> 64 -> 1 with ReLU after both hidden layers; its parameters are
 * GG_MLP_NPARAM floats, row-major: W1[64][8], b1[64], W2[64][64], b2[64],
 * w3[64], b3. Arithmetic: weights and each layer's inputs rounded to
 * bfloat16 (nearest even), products accumulated in FP32 on the tensor cores,
 * FP32 biases. Vertex features (FP32, in this order): sqrt(in-degree)/64,
 * sqrt(out-degree)/64, the change feature of the last three executed
 * iterations, newest first (PageRank: n |old - new|; SSSP / BFS / CC: 1 if the
 * value decreased, else 0; 0 before the run's start), the active fraction
 * of the in-edges (1 without in-edges), iteration / 64, application id.
 */
#define GG_MLP_NPARAM 4801

/* gg_set_scorer - copy host params[GG_MLP_NPARAM] into g for GG_POLICY_LEARNED. */
gg_status gg_set_scorer(gg_graph *g, const float *params);

/*
 * gg_set_trace - record training rows during later runs of g: at every full
 * correction, the features of all n vertices (device features[cap_rows][8])
 * before it and their labels (device labels[cap_rows], 0/1) after it: a
 * PageRank vertex is labelled 1 if |new - old| > label_tol * |new| (FP32), a
 * min-application vertex if its value decreased. Rows are appended (c*n + u)
 * across runs while cap_rows has room for all n; the count is
 * gg_stats.trace_rows. The buffers stay the caller's; features = NULL stops
 * recording.
 */
gg_status gg_set_trace(gg_graph *g, float *features, uint8_t *labels, uint64_t cap_rows, float label_tol);

/*
 * gg_mlp_score - logits of rows feature rows (device features[rows][8], 8-byte
 * aligned) into device logits[rows], with device params[GG_MLP_NPARAM].
 * Enqueued on stream (NULL = legacy default stream).
 */
gg_status gg_mlp_score(const float *features, uint64_t rows, const float *params, float *logits, void *stream);

/*
 * gg_mlp_train - `steps` steps of minibatch SGD on the mean logistic loss:
 * step s uses rows ((start + s*batch + j) mod rows) * stride mod rows,
 * j < batch (stride coprime to rows makes this a permutation). Forward in the
 * scorer's arithmetic; the backward contractions on the tensor cores
 * (bfloat16 operands, the FP32 gradients split into two bfloat16 parts, FP32
 * accumulation), one block per 128 rows of a step, the blocks' partial
 * gradients summed in block order (deterministic). Allocates its scratch
 * (about 19 KB per 128 rows of the batch) from the library's pool.
 *   features  device float[rows][8]; labels device uint8[rows] (0 / 1)
 *   rows      1 .. 2^32-1; stride < rows
 *   params    device float[GG_MLP_NPARAM], updated in place (FP32 masters)
 *   batch     1 .. 16384
 *   losses    device float[steps] (nullable): each step's mean loss
 *   grad_last device float[GG_MLP_NPARAM] (nullable): the last step's gradient
 */
gg_status gg_mlp_train(const float *features, const uint8_t *labels, uint64_t rows, float *params,
                       uint32_t batch, uint32_t steps, float lr, uint64_t stride, uint64_t start,
                       float *losses, float *grad_last, void *stream);

/*
 * Batched serving (beyond the paper): many BFS / SSSP / personalized-
 * PageRank queries over loaded graphs of uneven size in one persistent
 * launch, replayed as a captured CUDA graph. Queries on graphs with at least
 * big_arcs arcs are served by a whole thread-block cluster of `cluster`
 * CTAs (meeting at the cluster barrier between iterations), the others by
 * single CTAs; each team claims its next query (most estimated work first)
 * with one atomic, so no team waits on another. Vertices are binned by
 * degree: below warp_deg one thread handles a vertex, below cta_deg a warp,
 * else the whole CTA. BFS / SSSP run exactly to the fixed point (push
 * frontier); personalized PageRank runs `iters` pull iterations. The batch
 * reads the graphs' device arrays: the graphs must outlive it.
 */
typedef struct {
    int32_t graph;        /* index into the graphs given to gg_batch_create */
    int32_t app;          /* GG_APP_BFS, GG_APP_SSSP (weighted graph) or GG_APP_PPR */
    int32_t source;
    uint32_t iters;       /* GG_APP_PPR: iterations */
    float damping;        /* GG_APP_PPR: d in [0, 1] */
    int32_t warp_deg;     /* this query's degree bins (see gg_batch_config); 0, 0 = the batch's */
    int32_t cta_deg;
} gg_query;

typedef struct {
    int32_t cluster;      /* CTAs per cluster team: 1 (no cluster teams), 2, 4, 8 or 16 (16 is a
                             non-portable size: GG_ERR_CUDA where the device cannot place it) */
    int32_t warp_deg;     /* degree from which a warp handles a vertex (>= 1) */
    int32_t cta_deg;      /* degree from which the whole CTA does (>= warp_deg) */
    int32_t threads;      /* threads per CTA: 256, 512 or 1024 (0 = 256) */
    int64_t big_arcs;     /* graphs with at least this many arcs get cluster teams */
    int32_t small_first;  /* every small_first-th cluster serves the single-CTA queries first,
                             the rest start with the cluster-team queries (0: all start there) */
    int32_t order;        /* order in which teams claim queries: GG_ORDER_MOST_WORK (0, the largest
                             estimated work first: shortest makespan), GG_ORDER_LEAST_WORK (1, the
                             smallest first: lowest median latency), GG_ORDER_TRAVERSALS_FIRST (2,
                             BFS / SSSP before personalized PageRank, each largest first) */
} gg_batch_config;
#define GG_ORDER_MOST_WORK 0
#define GG_ORDER_LEAST_WORK 1
#define GG_ORDER_TRAVERSALS_FIRST 2

typedef struct {
    uint64_t latency_ns;  /* from the launch's start to the query's completion */
    uint64_t service_ns;  /* from the query's claim to its completion */
    uint64_t arcs;        /* arcs the query traversed (pushes, or iters x m pulls) */
    uint32_t iterations;
    uint32_t team;        /* CTAs that served it */
} gg_query_stats;

typedef struct gg_batch gg_batch;

/* Validate queries, lay out their state in one device arena, plan the teams. */
gg_status gg_batch_create(gg_graph *const *graphs, int32_t n_graphs, const gg_query *queries, int32_t n_queries,
                          const gg_batch_config *cfg, gg_batch **out);
/* Serve every query (one persistent launch; captured as a CUDA graph on the
 * first call, replayed afterwards); *ms = device time of the launch. */
gg_status gg_batch_run(gg_batch *b, float *ms);
/* Per-query latency, service time, arcs and iterations of the last run. */
gg_status gg_batch_query_stats(gg_batch *b, gg_query_stats *out, int32_t n);
/* Values of query q (uint32 distances / levels, or float ranks) into host dst. */
gg_status gg_batch_result(gg_batch *b, int32_t q, void *dst, size_t bytes);
void gg_batch_free(gg_batch *b);

/*
 * gg_sample_csc_noalloc - the sampling step of gg_sample_edges applied to a
 * caller-owned in-edge list, without allocating any device memory. The paper
 * has no counterpart: this entry point exists for callers that cannot
 * allocate device memory when they need the step: code that runs inside an
 * allocator's own callbacks, processes whose device memory budget is handed
 * out in full up front, or loops that must not call into the allocator.
 *   n, m       vertices and arcs, n >= 1, n + m <= GG_NOALLOC_MAX_ITEMS
 *   in_ptr     device int32[n+1], in_src device int32[m]: in-edge rows, each
 *              listing its sources (the order defines the packed order).
 *              in_ptr[0] must be 0, in_ptr[n] must be m and the row pointers
 *              must never decrease; the call checks this on the device and,
 *              if it fails, writes neither mask nor sp_ptr / sp_src and sets
 *              *sp_nnz = 0xFFFFFFFF
 *   sample_ratio, seed, symmetric: as in gg_sample_edges / GG_SYMMETRIC
 *   mask       device uint32[ceil(m/32)] out: flag bits of the m arcs (bits
 *              past m in the last word are left as they were)
 *   sp_ptr     device int32[n+1] out, sp_src device int32[m] out (the first
 *              *sp_nnz entries used), sp_nnz device uint32[1] out: the
 *              packed active in-edges
 *   stream     cudaStream_t to run on (NULL = legacy default stream)
 * Working memory is one fixed device array inside libgg.so (about 0.8 MB
 * per GPU that uses it, kept until the process exits). Every call on a
 * device shares it, so calls that overlap on the GPU race. The first call on
 * a device looks up the array's address (cudaGetSymbolAddress); under CUDA's
 * default lazy module loading that first call is also what loads the
 * library's module on the device and creates the array, so it does take
 * device memory once: callers with a fixed budget make it before they hand
 * the budget out, and before any stream capture. The cached address is not
 * refreshed after cudaDeviceReset. Sizes above the limit return
 * GG_ERR_INVALID_ARG. Returns after enqueueing the work.
 */
#define GG_NOALLOC_MAX_ITEMS (1u << 24)
gg_status gg_sample_csc_noalloc(int32_t n, int64_t m, const int32_t *in_ptr, const int32_t *in_src,
                                double sample_ratio, uint64_t seed, int symmetric, uint32_t *mask,
                                int32_t *sp_ptr, int32_t *sp_src, uint32_t *sp_nnz, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GG_H */

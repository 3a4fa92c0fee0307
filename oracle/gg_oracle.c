/*
 * gg_oracle.c - TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential-per-vertex CPU restatement of GraphGuess
 * (Ramezani, Kandemir, Sivasubramaniam, "GraphGuess: Approximate Graph
 * Processing System with Adaptive Correction", arXiv 2104.10039): exact and
 * approximate pull-based vertex-centric execution with correction steps.
 * Only the tests, the smoke check and the bench's CPU-baseline leg load this
 * file; the product path never does, and it shares no code, header, table or
 * helper with the CUDA library.
 *
 * Arithmetic: PageRank in FP64; SSSP / BFS / CC in exact integers
 * (uint32 values, 0xFFFFFFFF = unreached).
 *
 * Readings of the paper taken here:
 *  - Sec. 3.3: approximate mode gathers over active in-edges only, accurate
 *    mode over all in-edges; one flag per edge, no new graph.
 *  - Sec. 3.4: start from a sigma-fraction of active edges, run alpha
 *    approximate iterations, then one correction ("superstep") iteration in
 *    accurate mode that recomputes edge influence; afterwards exactly the
 *    edges with influence > theta are active. Repeated every alpha
 *    approximate iterations. Iteration i is a correction iff
 *    i mod (alpha+1) == alpha.
 *  - Sec. 3.4 sampling: independent Bernoulli(sigma) per arc decided by a
 *    stateless hash: h = SplitMix64 output for state (seed XOR key),
 *    key = src<<32 | dst (min<<32 | max on symmetric graphs), active iff
 *    (h >> 32) < floor(sigma * 2^32).
 *  - Alg. 2 GG-Gather: a separate accumulator starting at 0 (Alg. 1's
 *    new_property); in-edges visited in CSC order (source id ascending);
 *    influence = (acc_after - acc_before) / acc_after; v.degree = full
 *    out-degree.
 *  - Alg. 2 GG-Apply: rank = (1-d)/N + d * acc; initial rank 1/N; no
 *    dangling redistribution.
 *  - Alg. 2 GG-VStatus: vertex active iff |old - new| > epsilon (PageRank);
 *    iff its value decreased (min applications).
 *  - Alg. 2 GG-EStatus: edge active iff influence > theta.
 *  - Min applications (SSSP, BFS, CC) use the same running-accumulator form
 *    of influence on a min accumulator that starts "empty": the first
 *    finite candidate has influence 1, a later candidate that lowers the
 *    running minimum has (acc - cand) / acc, any other has 0. For CC the
 *    influence is binary (1 if it lowers the running label, else 0), as
 *    Sec. 5.2 states for WCC. The comparison with theta is done exactly in
 *    integers against theta rounded down to a multiple of 2^-32.
 *  - Arcs whose source is unreached (no candidate) keep their flag in a
 *    correction (the reset of Sec. 3.4 applies to evaluated arcs), unless
 *    ORC_EST_STRICT is set, which clears them too.
 *  - Synchronous (Jacobi) iterations: every gather reads the previous
 *    iteration's values.
 *  - SP (policy NONE) never corrects; SMS (STATIC_SWITCH) corrects once at
 *    iteration alpha and stays accurate afterwards (Sec. 5.2).
 *  - ORC_TRIGGERED (beyond the paper, which notes the correction points
 *    could vary, Sec. 3.4): a correction follows the approximate iteration
 *    whose change statistic (vertices that changed for the min
 *    applications, sum |old-new| for PageRank) is at most trigger_ratio times
 *    that of the window's first approximate iteration, or the alpha-th
 *    approximate iteration of the window.
 *  - ORC_LEARNED (beyond the paper; the scorer is this project's): the
 *    adaptive schedule, but at a correction a per-vertex MLP scores every
 *    vertex from 8 features and only the vertices scoring above
 *    select_logit are corrected (all in-edges gathered, influence and flags
 *    recomputed); the others keep their value and flags for that iteration.
 *    A selection holding more than fallback_frac of all arcs runs the full
 *    correction instead, and so does the correction after a learned one that
 *    changed no value. Scorer arithmetic: weights and every layer's inputs
 *    rounded to bfloat16 (nearest even), exact products summed (FP64 here,
 *    rounded to FP32 before the next rounding), FP32 biases, ReLU after the
 *    two hidden layers.
 *  - ORC_PPR (beyond the paper): personalized PageRank from `source`, the
 *    same gather with the restart mass on the source only: rank_0 = e_s,
 *    rank' = (1-d) e_s + d * sum over in-edges of rank(v) / outdeg(v).
 *  - Two PageRank variants beyond the paper (flags): ORC_INFL_SHARE takes
 *    an arc's influence as its share of the row's total (order-free) instead
 *    of the running-prefix form; ORC_RENORM divides a source's rank by its
 *    number of *active* out-arcs in approximate iterations, so no rank mass
 *    leaks through inactive arcs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_PAGERANK = 0, ORC_SSSP = 1, ORC_BFS = 2, ORC_CC = 3, ORC_PPR = 4 };
enum { ORC_EXACT = 0, ORC_NONE = 1, ORC_STATIC_SWITCH = 2, ORC_ADAPTIVE = 3, ORC_TRIGGERED = 4,
       ORC_LEARNED = 5 };
enum { ORC_MODE_APPROX = 0, ORC_MODE_ACCURATE = 1, ORC_MODE_CORRECTION = 2 };
#define ORC_STOP_QUIESCE 1u
#define ORC_EST_STRICT 2u
#define ORC_INFL_SHARE 32u
#define ORC_RENORM 64u
#define ORC_INF 0xFFFFFFFFu

typedef struct {
    int32_t app, policy;
    double sample_ratio;         /* sigma */
    uint64_t seed;
    uint32_t alpha;
    double theta;
    uint32_t max_iters;
    double damping;
    double epsilon;
    int32_t source;
    uint32_t flags;
    int32_t symmetric;
    int32_t nthreads;            /* <= 0: OpenMP default */
    const uint8_t *replay_masks; /* n_replay x m bytes in CSC order, or NULL */
    int32_t n_replay;
    double replay_tol;
    double trigger_ratio;        /* ORC_TRIGGERED: correct when the window's change falls to this fraction */
    const int8_t *replay_modes;  /* per iteration ORC_MODE_* to follow instead of the trigger, or NULL */
    const float *mlp;            /* ORC_LEARNED: scorer parameters, ORC_MLP_NPARAM floats */
    double select_logit;         /* ORC_LEARNED: vertices with a logit above this are corrected */
    double fallback_frac;        /* ORC_LEARNED: a selection with more arcs than this x m corrects fully */
    const uint8_t *replay_select;/* n_replay_select x n selections (0/1) to adopt, or NULL */
    int32_t n_replay_select;
    double replay_select_tol;    /* a differing selection must have |logit - select_logit| <= this */
    float *trace_x;              /* features (8 per row) at every full correction, rows c*n+u, or NULL */
    uint8_t *trace_y;            /* labels of those rows */
    int64_t trace_cap;           /* rows available in trace_x / trace_y */
    double label_tol;            /* PageRank label: |new-old| > label_tol * |new| */
    float select_cost;           /* ORC_LEARNED: the threshold of a vertex with in-degree d is
                                    fmaf(select_cost, L(d), select_logit) in float, L(d) = bit length of d */
} orc_params;

typedef struct {
    double *pr_values;           /* n, PageRank */
    uint32_t *int_values;        /* n, SSSP / BFS / CC */
    uint8_t *mask;               /* m, final flags in CSC order (nullable) */
    int64_t *iter_arcs;          /* max_iters: arcs in each iteration's edge set */
    int32_t *iter_mode;          /* max_iters: ORC_MODE_* (-1 = skipped) */
    int64_t *iter_changed;       /* max_iters: vertices active after VStatus */
    double *iter_sum_delta;      /* max_iters: sum |old-new| over vertices (nullable) */
    int64_t *iter_selected;      /* max_iters: vertices a learned correction corrected, else -1 (nullable) */
    double *logits;              /* n: logits of the last scored correction (nullable) */
    int32_t iterations;          /* iterations counted (skipped no-ops included) */
    int32_t corrections;
    int64_t replay_mismatch;
    double replay_max_margin;
    int64_t replay_violations;
    int64_t select_mismatch;     /* adopted selections that differ from the oracle's own */
    int64_t select_violations;   /* ... of which farther than replay_select_tol from the threshold */
    double select_max_margin;
    int64_t trace_rows;          /* rows written to the trace */
} orc_out;

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the output for a given
 * state: advance by the golden gamma, then the variant-13 finaliser. */
uint64_t orc_splitmix64(uint64_t state)
{
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Initial flag of arc src->dst (Sec. 3.4, uniform sparsification). */
int orc_arc_sampled(int32_t src, int32_t dst, int symmetric, double sigma, uint64_t seed)
{
    uint32_t a = (uint32_t)src, b = (uint32_t)dst;
    if (symmetric && a > b) { uint32_t t = a; a = b; b = t; }
    uint64_t key = ((uint64_t)a << 32) | (uint64_t)b;
    uint64_t h = orc_splitmix64(seed ^ key);
    uint64_t thr = (uint64_t)floor(sigma * 4294967296.0);
    return (h >> 32) < thr;
}

/* In-edge (CSC) view of a CSR graph: a stable counting sort of the arcs by
 * destination. CSR rows are visited in source order, so every in-row lists
 * its sources in ascending order, duplicates in CSR order. csr_pos[k] is
 * the CSR index of CSC arc k. */
int orc_csc_from_csr(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx,
                     const uint32_t *w, int32_t *in_ptr, int32_t *in_src, uint32_t *in_w,
                     int32_t *csr_pos)
{
    for (int32_t u = 0; u <= n; ++u) in_ptr[u] = 0;
    for (int64_t e = 0; e < m; ++e) {
        if (colidx[e] < 0 || colidx[e] >= n) return -1;
        in_ptr[colidx[e] + 1] += 1;
    }
    for (int32_t u = 0; u < n; ++u) in_ptr[u + 1] += in_ptr[u];
    int32_t *next = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!next) return -1;
    memcpy(next, in_ptr, (size_t)n * sizeof(int32_t));
    for (int32_t v = 0; v < n; ++v) {
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            int32_t u = colidx[e];
            int32_t k = next[u]++;
            in_src[k] = v;
            if (in_w) in_w[k] = w ? w[e] : 1u;
            if (csr_pos) csr_pos[k] = e;
        }
    }
    free(next);
    return 0;
}

/* Flags of all CSC arcs after sampling with ratio sigma. */
void orc_sample_mask(int32_t n, const int32_t *in_ptr, const int32_t *in_src, int symmetric,
                     double sigma, uint64_t seed, uint8_t *mask)
{
    for (int32_t u = 0; u < n; ++u)
        for (int32_t k = in_ptr[u]; k < in_ptr[u + 1]; ++k)
            mask[k] = (uint8_t)orc_arc_sampled(in_src[k], u, symmetric, sigma, seed);
}

/* Mode of iteration i under each policy (Sec. 3.4 and Sec. 5.2). */
int orc_iteration_mode(int policy, uint32_t alpha, uint32_t i)
{
    switch (policy) {
    case ORC_EXACT: return ORC_MODE_ACCURATE;
    case ORC_NONE: return ORC_MODE_APPROX;
    case ORC_STATIC_SWITCH:
        if (i < alpha) return ORC_MODE_APPROX;
        return i == alpha ? ORC_MODE_CORRECTION : ORC_MODE_ACCURATE;
    case ORC_ADAPTIVE:
    case ORC_LEARNED:
        return (i % (alpha + 1u)) == alpha ? ORC_MODE_CORRECTION : ORC_MODE_APPROX;
    default: return -1;
    }
}

/* First iteration index > i whose mode is a correction or accurate, or -1
 * when the policy never leaves approximate mode again. */
static int64_t next_accurate_iteration(int policy, uint32_t alpha, uint32_t i)
{
    if (policy == ORC_NONE) return -1;
    if (policy == ORC_STATIC_SWITCH) return i < alpha ? (int64_t)alpha : (int64_t)i + 1;
    if (policy == ORC_ADAPTIVE || policy == ORC_LEARNED) {
        uint64_t period = (uint64_t)alpha + 1u;
        return (int64_t)(((uint64_t)i / period) * period + alpha);
    }
    return (int64_t)i + 1;   /* EXACT, and TRIGGERED (a quiet window triggers at once) */
}

/* ------------------------------------------------------------ scorer ----
 * Parameters (FP32): W1[64][8], b1[64], W2[64][64], b2[64], w3[64], b3. */
#define ORC_MLP_IN 8
#define ORC_MLP_H 64
#define ORC_MLP_NPARAM (ORC_MLP_H * ORC_MLP_IN + ORC_MLP_H + ORC_MLP_H * ORC_MLP_H + ORC_MLP_H + ORC_MLP_H + 1)

/* bfloat16 value of x: round to nearest, ties to even, on the upper 16 bits. */
float orc_bf16(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    b += 0x7FFFu + ((b >> 16) & 1u);
    b &= 0xFFFF0000u;
    memcpy(&x, &b, 4);
    return x;
}

static double rnd(double v, int round) { return round ? (double)orc_bf16((float)v) : v; }

/* Logit of one row; h1 / h2 (64 each) receive the (rounded) hidden
 * activations and s1 / s2 their pre-activations when not NULL. */
static double mlp_row(const float *P, const float *x, int round, double *h1, double *h2, double *s1,
                      double *s2)
{
    const float *W1 = P, *b1 = P + 512, *W2 = P + 576, *b2 = P + 4672, *w3 = P + 4736;
    const float b3 = P[4800];
    double xb[ORC_MLP_IN], a1[ORC_MLP_H], a2[ORC_MLP_H];
    for (int f = 0; f < ORC_MLP_IN; ++f) xb[f] = rnd(x[f], round);
    for (int j = 0; j < ORC_MLP_H; ++j) {
        double acc = b1[j];
        for (int f = 0; f < ORC_MLP_IN; ++f) acc += rnd(W1[j * ORC_MLP_IN + f], round) * xb[f];
        if (s1) s1[j] = acc;
        a1[j] = acc > 0.0 ? rnd(round ? (double)(float)acc : acc, round) : 0.0;
        if (h1) h1[j] = a1[j];
    }
    for (int j = 0; j < ORC_MLP_H; ++j) {
        double acc = b2[j];
        for (int k = 0; k < ORC_MLP_H; ++k) acc += rnd(W2[j * ORC_MLP_H + k], round) * a1[k];
        if (s2) s2[j] = acc;
        a2[j] = acc > 0.0 ? rnd(round ? (double)(float)acc : acc, round) : 0.0;
        if (h2) h2[j] = a2[j];
    }
    double z = b3;
    for (int j = 0; j < ORC_MLP_H; ++j) z += rnd(w3[j], round) * a2[j];
    return z;
}

/* Logits of `rows` feature rows (8 floats each). */
void orc_mlp_forward(const float *P, const float *x, int64_t rows, int round, double *logits)
{
    for (int64_t r = 0; r < rows; ++r) logits[r] = mlp_row(P, x + r * ORC_MLP_IN, round, NULL, NULL, NULL, NULL);
}

/* Gradient of the mean logistic loss over the rows idx[0..b) (labels 0/1)
 * with respect to the parameters (same layout), the rounding treated as
 * the identity; returns the loss. */
double orc_mlp_grad(const float *P, const float *x, const uint8_t *y, const int64_t *idx, int64_t b, int round,
                    double *grad)
{
    const float *W2 = P + 576, *w3 = P + 4736;
    double *gW1 = grad, *gb1 = grad + 512, *gW2 = grad + 576, *gb2 = grad + 4672, *gw3 = grad + 4736;
    double h1[ORC_MLP_H], h2[ORC_MLP_H], s1[ORC_MLP_H], s2[ORC_MLP_H], d2[ORC_MLP_H];
    double loss = 0.0;
    for (int i = 0; i < ORC_MLP_NPARAM; ++i) grad[i] = 0.0;
    for (int64_t t = 0; t < b; ++t) {
        const float *xr = x + idx[t] * ORC_MLP_IN;
        const double lab = y[idx[t]] ? 1.0 : 0.0;
        const double z = mlp_row(P, xr, round, h1, h2, s1, s2);
        loss += (z > 0.0 ? z : 0.0) - z * lab + log1p(exp(-fabs(z)));
        const double dz = (1.0 / (1.0 + exp(-z)) - lab) / (double)b;
        grad[4800] += dz;
        for (int j = 0; j < ORC_MLP_H; ++j) {
            gw3[j] += dz * h2[j];
            d2[j] = s2[j] > 0.0 ? dz * rnd(w3[j], round) : 0.0;
            gb2[j] += d2[j];
            for (int k = 0; k < ORC_MLP_H; ++k) gW2[j * ORC_MLP_H + k] += d2[j] * h1[k];
        }
        for (int k = 0; k < ORC_MLP_H; ++k) {
            if (!(s1[k] > 0.0)) continue;
            double d1 = 0.0;
            for (int j = 0; j < ORC_MLP_H; ++j) d1 += rnd(W2[j * ORC_MLP_H + k], round) * d2[j];
            gb1[k] += d1;
            for (int f = 0; f < ORC_MLP_IN; ++f) gW1[k * ORC_MLP_IN + f] += d1 * rnd(xr[f], round);
        }
    }
    return loss / (double)(b > 0 ? b : 1);
}

/* The scorer's 8 features of vertex u before iteration i (FP32, each from
 * correctly rounded operations): sqrt(in-degree)/64, sqrt(out-degree)/64,
 * the change features of the last three executed iterations (newest first),
 * the active fraction of the in-edges (1 without in-edges), i/64, app id.
 * hist holds 3 rows of n; executed = iterations executed so far. */
static void vertex_features(int32_t u, int32_t n, uint32_t i, int app, const int32_t *in_ptr,
                            const int32_t *outdeg, const uint8_t *mask, const float *hist, uint32_t executed,
                            float *x)
{
    const int32_t indeg = in_ptr[u + 1] - in_ptr[u];
    int32_t act = 0;
    for (int32_t k = in_ptr[u]; k < in_ptr[u + 1]; ++k) act += mask[k] ? 1 : 0;
    x[0] = sqrtf((float)indeg) * 0.015625f;
    x[1] = sqrtf((float)outdeg[u]) * 0.015625f;
    for (uint32_t j = 1; j <= 3; ++j) x[1 + j] = hist[(size_t)((executed + 3u - j) % 3u) * (size_t)n + (size_t)u];
    x[5] = indeg > 0 ? (float)act / (float)indeg : 1.0f;
    x[6] = (float)i * 0.015625f;
    x[7] = (float)app;
}

/* Number of active out-arcs of every vertex under the flags `mask`. */
static void active_outdeg(int32_t n, const int32_t *in_ptr, const int32_t *in_src, const uint8_t *mask,
                          int32_t *act)
{
    for (int32_t v = 0; v < n; ++v) act[v] = 0;
    for (int32_t u = 0; u < n; ++u)
        for (int32_t k = in_ptr[u]; k < in_ptr[u + 1]; ++k)
            act[in_src[k]] += mask[k] ? 1 : 0;
}

/* Edge status for a min application (integers only).
 * returns 1 active, 0 inactive. */
static int min_app_estatus(int app, uint32_t acc, uint32_t cand, double theta)
{
    int improving = cand < acc;
    if (theta < 0.0) return 1;               /* influence >= 0 > theta */
    if (theta >= 1.0) return 0;              /* influence <= 1 <= theta */
    if (!improving) return 0;                /* influence 0 */
    if (acc == ORC_INF || app == ORC_CC) return 1;   /* influence 1 */
    uint64_t theta_fx = (uint64_t)floor(theta * 4294967296.0);
    uint64_t lhs = (uint64_t)(acc - cand) << 32;
    uint64_t rhs = theta_fx * (uint64_t)acc;
    return lhs > rhs;
}

/* Learned selection threshold of a vertex with in-degree d: select_logit
 * plus select_cost times the bit length of d, computed as one fused float
 * operation (the library computes it the same way). */
static double select_threshold(const orc_params *p, int64_t d)
{
    int bits = 0;
    while (d > 0) {
        bits += 1;
        d >>= 1;
    }
    return (double)fmaf(p->select_cost, (float)bits, (float)p->select_logit);
}

int orc_run(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx,
            const uint32_t *weights, const orc_params *p, orc_out *o)
{
    if (n <= 0 || m < 0 || !p || !o) return -1;
    if (p->app < ORC_PAGERANK || p->app > ORC_PPR) return -1;
    if (p->app != ORC_PAGERANK && p->app != ORC_CC && (p->source < 0 || p->source >= n)) return -1;
    if (!(p->sample_ratio > 0.0 && p->sample_ratio <= 1.0)) return -1;
    if (p->policy == ORC_LEARNED && !p->mlp) return -1;
#ifdef _OPENMP
    omp_set_num_threads(p->nthreads > 0 ? p->nthreads : omp_get_num_procs());
#endif
    int rc = -1;
    int32_t *in_ptr = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *in_src = (int32_t *)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    uint32_t *in_w = (uint32_t *)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
    uint8_t *mask = (uint8_t *)malloc((size_t)(m ? m : 1));
    uint8_t *new_mask = (uint8_t *)malloc((size_t)(m ? m : 1));
    double *infl = (double *)malloc((size_t)(m ? m : 1) * sizeof(double));
    int32_t *outdeg = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *act = NULL;
    float *hist = NULL;          /* change features of the last three executed iterations */
    uint8_t *sel = NULL;         /* vertices a learned correction corrects */
    double *logit = NULL;
    double *rank = NULL, *rank_next = NULL;
    uint32_t *val = NULL, *val_next = NULL;
    if (!in_ptr || !in_src || !in_w || !mask || !new_mask || !infl || !outdeg) goto done;
    if (orc_csc_from_csr(n, m, rowptr, colidx, weights, in_ptr, in_src, in_w, NULL) != 0) goto done;
    for (int32_t v = 0; v < n; ++v) outdeg[v] = rowptr[v + 1] - rowptr[v];
    orc_sample_mask(n, in_ptr, in_src, p->symmetric, p->sample_ratio, p->seed, mask);

    const int is_pr = p->app == ORC_PAGERANK || p->app == ORC_PPR;
    const int ppr = p->app == ORC_PPR;
    const int renorm = is_pr && (p->flags & ORC_RENORM);
    const int share = is_pr && (p->flags & ORC_INFL_SHARE);
    const int learned_policy = p->policy == ORC_LEARNED;
    if (learned_policy || p->trace_x) {
        hist = (float *)calloc((size_t)3 * (size_t)n, sizeof(float));
        sel = (uint8_t *)malloc((size_t)n);
        logit = (double *)malloc((size_t)n * sizeof(double));
        if (!hist || !sel || !logit) goto done;
    }
    if (renorm) {
        act = (int32_t *)malloc((size_t)n * sizeof(int32_t));
        if (!act) goto done;
        active_outdeg(n, in_ptr, in_src, mask, act);
    }
    if (is_pr) {
        rank = (double *)malloc((size_t)n * sizeof(double));
        rank_next = (double *)malloc((size_t)n * sizeof(double));
        if (!rank || !rank_next) goto done;
        for (int32_t u = 0; u < n; ++u) rank[u] = ppr ? (u == p->source ? 1.0 : 0.0) : 1.0 / (double)n;
    } else {
        val = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
        val_next = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
        if (!val || !val_next) goto done;
        for (int32_t u = 0; u < n; ++u) val[u] = (p->app == ORC_CC) ? (uint32_t)u : ORC_INF;
        if (p->app != ORC_CC) val[p->source] = 0;
    }

    o->iterations = 0;
    o->corrections = 0;
    o->replay_mismatch = 0;
    o->replay_max_margin = 0.0;
    o->replay_violations = 0;
    o->select_mismatch = 0;
    o->select_violations = 0;
    o->select_max_margin = 0.0;
    o->trace_rows = 0;
    uint32_t executed = 0;       /* iterations run (skipped no-ops excluded) */
    int force_full = 0;          /* the next correction is a full one */
    int32_t select_next = 0;
    const double d = p->damping;
    const double base = (1.0 - d) / (double)n;
    int32_t replay_next = 0;
    int trig_next = p->policy == ORC_TRIGGERED && p->alpha == 0;   /* correction comes next */
    uint32_t window = 0;
    double window_first = 0.0;

    for (uint32_t i = 0; i < p->max_iters; ++i) {
        int mode;
        if (p->replay_modes) mode = p->replay_modes[i];
        else if (p->policy == ORC_TRIGGERED) mode = trig_next ? ORC_MODE_CORRECTION : ORC_MODE_APPROX;
        else mode = orc_iteration_mode(p->policy, p->alpha, i);
        if (mode < 0 || mode > ORC_MODE_CORRECTION) goto done;
        double sum_delta = 0.0;
        const int accurate = mode != ORC_MODE_APPROX;
        const int correcting = mode == ORC_MODE_CORRECTION;
        int64_t arcs = 0, changed = 0;
        if (o->iter_selected) o->iter_selected[i] = -1;

        /* Learned correction: score every vertex, select, maybe fall back. */
        int learned = 0;
        if (correcting && learned_policy && !force_full) {
            int64_t nsel = 0, sel_arcs = 0;
#pragma omp parallel for schedule(dynamic, 1024)
            for (int32_t u = 0; u < n; ++u) {
                float x[ORC_MLP_IN];
                vertex_features(u, n, i, p->app, in_ptr, outdeg, mask, hist, executed, x);
                logit[u] = mlp_row(p->mlp, x, 1, NULL, NULL, NULL, NULL);
                sel[u] = logit[u] > select_threshold(p, in_ptr[u + 1] - in_ptr[u]);
            }
            if (o->logits) memcpy(o->logits, logit, (size_t)n * sizeof(double));
            if (p->replay_select && select_next < p->n_replay_select) {
                const uint8_t *given = p->replay_select + (size_t)select_next * (size_t)n;
                for (int32_t u = 0; u < n; ++u) {
                    if ((given[u] != 0) != (sel[u] != 0)) {
                        const double margin = fabs(logit[u] - select_threshold(p, in_ptr[u + 1] - in_ptr[u]));
                        o->select_mismatch += 1;
                        if (margin > o->select_max_margin) o->select_max_margin = margin;
                        if (!(margin <= p->replay_select_tol)) o->select_violations += 1;
                    }
                    sel[u] = given[u] ? 1 : 0;
                }
                select_next += 1;
            }
            for (int32_t u = 0; u < n; ++u) {
                nsel += sel[u];
                sel_arcs += sel[u] ? in_ptr[u + 1] - in_ptr[u] : 0;
            }
            learned = !((double)sel_arcs > p->fallback_frac * (double)m);
            if (learned && o->iter_selected) o->iter_selected[i] = nsel;
        }
        /* Trace: features before every full correction, labels after it. */
        const int tracing = correcting && !learned && p->trace_x && o->trace_rows + n <= p->trace_cap;
        if (tracing) {
#pragma omp parallel for schedule(static)
            for (int32_t u = 0; u < n; ++u)
                vertex_features(u, n, i, p->app, in_ptr, outdeg, mask, hist, executed,
                                p->trace_x + (size_t)(o->trace_rows + u) * ORC_MLP_IN);
        }
        float *hist_out = hist ? hist + (size_t)(executed % 3u) * (size_t)n : NULL;

        /* Gather (GG-Gather over in-edges, Alg. 1 / Alg. 2), Apply, VStatus */
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : arcs, changed, sum_delta)
        for (int32_t u = 0; u < n; ++u) {
            if (learned && !sel[u]) {   /* not selected: value and flags stay */
                if (is_pr) rank_next[u] = rank[u];
                else val_next[u] = val[u];
                for (int32_t k = in_ptr[u]; k < in_ptr[u + 1]; ++k) {
                    new_mask[k] = mask[k];
                    infl[k] = 1e300;
                }
                if (hist_out) hist_out[u] = 0.0f;
                continue;
            }
            if (is_pr) {
                double acc = 0.0;
                for (int32_t k = in_ptr[u]; k < in_ptr[u + 1]; ++k) {
                    if (!accurate && !mask[k]) continue;
                    int32_t v = in_src[k];
                    double before = acc;
                    const int32_t deg = (renorm && !accurate) ? act[v] : outdeg[v];
                    acc = rank[v] / (double)deg + acc;
                    arcs += 1;
                    if (correcting && !share) {
                        double f = acc != 0.0 ? (acc - before) / acc : 0.0;
                        infl[k] = f;
                        new_mask[k] = (uint8_t)(f > p->theta);
                    }
                }
                if (correcting && share) {   /* the arc's share of the row total */
                    for (int32_t k = in_ptr[u]; k < in_ptr[u + 1]; ++k) {
                        double c = rank[in_src[k]] / (double)outdeg[in_src[k]];
                        double f = acc != 0.0 ? c / acc : 0.0;
                        infl[k] = f;
                        new_mask[k] = (uint8_t)(f > p->theta);
                    }
                }
                double old = rank[u];
                double nw = (ppr ? (u == p->source ? 1.0 - d : 0.0) : base) + d * acc;
                rank_next[u] = nw;
                changed += fabs(old - nw) > p->epsilon;
                sum_delta += fabs(old - nw);
                if (hist_out) hist_out[u] = (float)((double)n * fabs(old - nw));
            } else {
                uint32_t acc = ORC_INF;
                for (int32_t k = in_ptr[u]; k < in_ptr[u + 1]; ++k) {
                    if (!accurate && !mask[k]) continue;
                    arcs += 1;
                    uint32_t vv = val[in_src[k]];
                    uint32_t cand;
                    if (p->app == ORC_CC) {
                        cand = vv;
                    } else {
                        uint64_t step = (p->app == ORC_BFS) ? 1u : in_w[k];
                        uint64_t c = (vv == ORC_INF) ? ORC_INF : (uint64_t)vv + step;
                        cand = c >= ORC_INF ? ORC_INF : (uint32_t)c;
                    }
                    if (cand == ORC_INF) {      /* no candidate: arc unevaluated */
                        if (correcting) {
                            new_mask[k] = (p->flags & ORC_EST_STRICT) ? 0 : mask[k];
                            infl[k] = -1.0;
                        }
                        continue;
                    }
                    if (correcting) {
                        new_mask[k] = (uint8_t)min_app_estatus(p->app, acc, cand, p->theta);
                        infl[k] = 0.0;
                    }
                    if (cand < acc) acc = cand;
                }
                uint32_t old = val[u];
                uint32_t nw = acc < old ? acc : old;
                val_next[u] = nw;
                changed += nw < old;
                if (hist_out) hist_out[u] = nw < old ? 1.0f : 0.0f;
            }
        }
        executed += 1;
        if (tracing) {
            for (int32_t u = 0; u < n; ++u) {
                const int y = is_pr ? fabs(rank_next[u] - rank[u]) > p->label_tol * fabs(rank_next[u])
                                    : val_next[u] < val[u];
                p->trace_y[o->trace_rows + u] = (uint8_t)y;
            }
            o->trace_rows += n;
        }
        if (!correcting) {
            /* nothing to do for the flags */
        } else if (p->replay_masks && replay_next < p->n_replay) {
            /* Mask replay: adopt the given post-correction flags after
             * checking each differing decision lies within tol of theta. */
            const uint8_t *given = p->replay_masks + (size_t)replay_next * (size_t)m;
            int64_t mism = 0, viol = 0;
            double maxmargin = o->replay_max_margin;
            for (int64_t k = 0; k < m; ++k) {
                if ((given[k] != 0) != (new_mask[k] != 0)) {
                    mism += 1;
                    double margin = is_pr ? fabs(infl[k] - p->theta) : INFINITY;
                    if (margin > maxmargin) maxmargin = margin;
                    if (!(margin <= p->replay_tol)) viol += 1;
                }
                mask[k] = given[k] ? 1 : 0;
            }
            o->replay_mismatch += mism;
            o->replay_violations += viol;
            o->replay_max_margin = maxmargin;
            replay_next += 1;
        } else {
            memcpy(mask, new_mask, (size_t)m);
        }
        if (correcting && renorm) active_outdeg(n, in_ptr, in_src, mask, act);
        if (is_pr) { double *t = rank; rank = rank_next; rank_next = t; }
        else { uint32_t *t = val; val = val_next; val_next = t; }

        if (o->iter_arcs) o->iter_arcs[i] = arcs;
        if (o->iter_mode) o->iter_mode[i] = mode;
        if (o->iter_changed) o->iter_changed[i] = changed;
        if (o->iter_sum_delta) o->iter_sum_delta[i] = sum_delta;
        o->iterations = (int32_t)i + 1;
        o->corrections += correcting;
        if (p->policy == ORC_TRIGGERED) {
            if (correcting) {
                window = 0;
                trig_next = p->alpha == 0;
            } else {
                const double metric = is_pr ? sum_delta : (double)changed;
                window += 1;
                if (window == 1) window_first = metric;
                trig_next = window >= p->alpha || metric <= p->trigger_ratio * window_first;
            }
        }

        if (correcting && learned_policy) force_full = learned && changed == 0;
        int stop_on_quiet = !is_pr || (p->flags & ORC_STOP_QUIESCE);
        if (stop_on_quiet && changed == 0 && !(accurate && learned)) {
            /* (a quiet learned correction only makes the next correction full) */
            if (accurate) break;                /* fixed point of the full graph */
            /* An approximate iteration that changed nothing leaves the state
             * as it was, so the approximate iterations until the next
             * accurate one are no-ops: skip them (they still count). */
            int64_t nxt = next_accurate_iteration(p->policy, p->alpha, i);
            if (nxt < 0) break;                 /* SP: nothing will change again */
            for (uint32_t j = i + 1; j < (uint32_t)nxt && j < p->max_iters; ++j) {
                if (o->iter_arcs) o->iter_arcs[j] = 0;
                if (o->iter_mode) o->iter_mode[j] = -1;
                if (o->iter_changed) o->iter_changed[j] = 0;
                if (o->iter_sum_delta) o->iter_sum_delta[j] = 0.0;
                o->iterations = (int32_t)j + 1;
            }
            if ((uint64_t)nxt >= p->max_iters) break;
            i = (uint32_t)nxt - 1;
        }
    }
    if (is_pr) { if (o->pr_values) memcpy(o->pr_values, rank, (size_t)n * sizeof(double)); }
    else if (o->int_values) memcpy(o->int_values, val, (size_t)n * sizeof(uint32_t));
    if (o->mask) memcpy(o->mask, mask, (size_t)m);
    rc = 0;
done:
    free(in_ptr); free(in_src); free(in_w); free(mask); free(new_mask); free(infl); free(outdeg); free(act);
    free(rank); free(rank_next); free(val); free(val_next); free(hist); free(sel); free(logit);
    return rc;
}

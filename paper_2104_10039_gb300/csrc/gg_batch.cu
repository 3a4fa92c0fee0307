// gg_batch.cu - batched serving (beyond the paper): many BFS / SSSP /
// personalized-PageRank queries over graphs of uneven size in one persistent
// launch.
//
// Teams. Queries on large graphs are served by a whole thread-block cluster
// (its CTAs split each iteration's work and meet at the hardware cluster
// barrier between iterations); the rest by single CTAs (__syncthreads). A
// team claims its next query with one atomic on a global counter (queries in
// the batch's order: by estimated work, descending or ascending, or BFS /
// SSSP before personalized PageRank), so no block ever waits for another
// team: the only waits are the cluster barriers inside a team, which every
// CTA of the cluster reaches the same number of times.
//
// Work inside a CTA is binned by degree: a vertex below warp_deg is handled
// by one thread, up to cta_deg by a warp (lanes over its arcs), above by the
// whole CTA (threads over its arcs, staged through shared memory). The bins
// are per query (the autotuner picks them per graph scale).
//
// BFS / SSSP push over a frontier (atomicMin relaxations, per-iteration
// stamps so a vertex enters the next frontier once); they run until the
// frontier is empty, which gives the unique shortest distances / levels.
// Personalized PageRank pulls over the in-edges for a fixed number of
// iterations: rank_0 = e_s, rank' = (1-d) e_s + d * sum rank(v) / outdeg(v),
// summed per row in a fixed order.
//
// Visibility: the team barrier orders each iteration's writes before the
// next iteration's reads (__syncthreads within a CTA; the cluster barrier
// has release / acquire semantics at cluster scope), so the rank arrays use
// plain, L1-cached loads; BFS / SSSP values, which other CTAs lower with
// atomics during an iteration, are read from L2.
#include <cooperative_groups.h>

#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "gg_graph.cuh"

namespace cg = cooperative_groups;

namespace gg {

namespace {

struct BatchGraph {
    int32_t n;
    int32_t m;
    const int32_t *out_ptr;
    const int32_t *out_dst;
    const uint32_t *out_w;
    const int32_t *in_ptr;
    const int32_t *in_src;
};

struct BatchQuery {
    int32_t graph;
    int32_t app;
    int32_t source;
    uint32_t iters;
    float damping;
    int32_t warp_deg;          // degree bins of this query
    int32_t cta_deg;
    uint32_t pad;
    unsigned long long off;    // first word of the query's state in the arena
};

struct QueryStatsDev {
    unsigned long long t_start, t_end, arcs;
    uint32_t iterations, team;
};

struct BatchArgs {
    const BatchGraph *graphs;
    const BatchQuery *queries;
    const int32_t *order_big;     // served by clusters, most work first
    int32_t n_big;
    const int32_t *order_small;   // served by single CTAs, most work first
    int32_t n_small;
    uint32_t *counters;           // [0] next big query, [1] next small query
    uint32_t *arena;
    QueryStatsDev *qs;
    unsigned long long *t0;
    int32_t warp_deg, cta_deg;
    int32_t cluster;
    int32_t small_first;          // every small_first-th cluster serves small queries first (0: none)
};

// BT = threads per CTA (256, 512 or 1024: an autotuned size); at most BT
// CTA-binned vertices are staged per pass.

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

struct CtaTeam {
    __device__ int rank() const { return 0; }
    __device__ int size() const { return 1; }
    __device__ void sync() const { __syncthreads(); }
};

struct ClusterTeam {
    cg::cluster_group cl;
    __device__ int rank() const { return (int)cl.block_rank(); }
    __device__ int size() const { return (int)cl.num_blocks(); }
    __device__ void sync() const { cl.sync(); }
};

template <int BT>
struct Shared {
    int32_t hub[BT];
    int32_t hub_n;
    int32_t claim;
    unsigned long long arcs;
    float red[BT / 32];
    float seg[BT];          // per warp: row parts of a chunk of light-row arcs
};

// Relax arc (v -> u) with candidate cand (BFS / SSSP push).
__device__ __forceinline__ void relax(uint32_t *val, uint32_t *stamp, uint32_t tag, int32_t *q_next,
                                      uint32_t *len_next, int32_t u, uint32_t cand)
{
    if (cand >= __ldcg(val + u)) return;
    const uint32_t old = atomicMin(val + u, cand);
    if (cand < old && atomicExch(stamp + u, tag) != tag) {
        const uint32_t pos = atomicAdd(len_next, 1u);
        q_next[pos] = u;
    }
}

__device__ __forceinline__ uint32_t cand_of(uint32_t vv, int app, const uint32_t *w, int32_t e)
{
    if (vv == kInf) return kInf;
    const unsigned long long c = (unsigned long long)vv + (app == GG_APP_BFS ? 1u : __ldg(w + e));
    return c >= kInf ? kInf : (uint32_t)c;
}

// ---------------------------------------------------------- BFS / SSSP --
template <int BT, class Team>
__device__ void serve_push(const BatchArgs &A, const BatchQuery &Q, const BatchGraph &G, const Team &team,
                           Shared<BT> &sh, QueryStatsDev *qs)
{
    const int32_t n = G.n;
    uint32_t *val = A.arena + Q.off;
    uint32_t *stamp = val + n;
    int32_t *qb[2] = {(int32_t *)(val + 2 * (size_t)n), (int32_t *)(val + 3 * (size_t)n)};
    uint32_t *L = val + 4 * (size_t)n;     // three rotating frontier lengths
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tr = team.rank(), ts = team.size();
    // init
    for (int32_t u = tr * BT + tid; u < n; u += ts * BT) {
        __stcg(val + u, u == Q.source ? 0u : kInf);
        __stcg(stamp + u, 0u);
    }
    if (tr == 0 && tid == 0) {
        __stcg((uint32_t *)qb[0], (uint32_t)Q.source);
        __stcg(L + 0, 1u);
        __stcg(L + 1, 0u);
        __stcg(L + 2, 0u);
    }
    if (tid == 0) sh.arcs = 0;
    team.sync();
    uint32_t it = 0;
    for (; it < (uint32_t)n + 1u; ++it) {
        const uint32_t len = __ldcg(L + it % 3);
        if (len == 0) break;
        const int32_t *q = qb[it & 1];
        int32_t *qn = qb[(it + 1) & 1];
        uint32_t *ln = L + (it + 1) % 3;
        if (tr == 0 && tid == 0) __stcg(L + (it + 2) % 3, 0u);
        const uint32_t tag = it + 1;
        const uint32_t lo = (uint32_t)(((unsigned long long)len * tr) / ts);
        const uint32_t hi = (uint32_t)(((unsigned long long)len * (tr + 1)) / ts);
        unsigned long long my_arcs = 0;
        for (uint32_t b0 = lo; b0 < hi; b0 += BT) {
            const uint32_t i = b0 + tid;
            int32_t v = -1, e0 = 0, deg = 0;
            if (i < hi) {
                v = __ldcg(q + i);
                e0 = __ldg(G.out_ptr + v);
                deg = __ldg(G.out_ptr + v + 1) - e0;
                my_arcs += (unsigned long long)deg;
            }
            if (tid == 0) sh.hub_n = 0;
            __syncthreads();
            // light vertices (degree below warp_deg) of this warp's 32 frontier
            // entries: the warp relaxes their out-arcs together, 32 at a time
            {
                const bool light = v >= 0 && deg < Q.warp_deg;
                const int32_t ld = light ? deg : 0;
                const uint32_t vv = light ? __ldcg(val + v) : kInf;
                int32_t incl = ld;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
                const int32_t excl = incl - ld;
                for (int32_t j0 = 0; j0 < tot; j0 += 32) {
                    const int32_t j = j0 + lane;
                    int r = 0;   // the entry whose out-arcs hold item j
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int c = r + step;
                        if (__shfl_sync(0xFFFFFFFFu, excl, c) <= j) r = c;
                    }
                    const int32_t re0 = __shfl_sync(0xFFFFFFFFu, e0, r);
                    const int32_t rex = __shfl_sync(0xFFFFFFFFu, excl, r);
                    const uint32_t rvv = __shfl_sync(0xFFFFFFFFu, vv, r);
                    if (j < tot) {
                        const int32_t e = re0 + (j - rex);
                        relax(val, stamp, tag, qn, ln, __ldg(G.out_dst + e), cand_of(rvv, Q.app, G.out_w, e));
                    }
                }
            }
            // warp bin
            unsigned mb = __ballot_sync(0xFFFFFFFFu, v >= 0 && deg >= Q.warp_deg && deg < Q.cta_deg);
            while (mb) {
                const int src = __ffs(mb) - 1;
                mb &= mb - 1;
                const int32_t wv = __shfl_sync(0xFFFFFFFFu, v, src);
                const int32_t we0 = __shfl_sync(0xFFFFFFFFu, e0, src);
                const int32_t wdeg = __shfl_sync(0xFFFFFFFFu, deg, src);
                const uint32_t vv = __ldcg(val + wv);
                for (int32_t k = lane; k < wdeg; k += 32) {
                    const int32_t e = we0 + k;
                    relax(val, stamp, tag, qn, ln, __ldg(G.out_dst + e), cand_of(vv, Q.app, G.out_w, e));
                }
            }
            // CTA bin
            if (v >= 0 && deg >= Q.cta_deg) sh.hub[atomicAdd(&sh.hub_n, 1)] = i;
            __syncthreads();
            for (int h = 0; h < sh.hub_n; ++h) {
                const int32_t hv = __ldcg(q + sh.hub[h]);
                const int32_t he0 = __ldg(G.out_ptr + hv);
                const int32_t hdeg = __ldg(G.out_ptr + hv + 1) - he0;
                const uint32_t vv = __ldcg(val + hv);
                for (int32_t k = tid; k < hdeg; k += BT) {
                    const int32_t e = he0 + k;
                    relax(val, stamp, tag, qn, ln, __ldg(G.out_dst + e), cand_of(vv, Q.app, G.out_w, e));
                }
            }
            __syncthreads();
        }
        (void)warp;
        if (my_arcs) atomicAdd(&sh.arcs, my_arcs);
        team.sync();
    }
    __syncthreads();
    if (tid == 0 && sh.arcs) atomicAdd(&qs->arcs, sh.arcs);
    if (tr == 0 && tid == 0) qs->iterations = it;
}

// ------------------------------------------------ personalized PageRank --
template <int BT, class Team>
__device__ void serve_ppr(const BatchArgs &A, const BatchQuery &Q, const BatchGraph &G, const Team &team,
                          Shared<BT> &sh, QueryStatsDev *qs)
{
    const int32_t n = G.n;
    float *rank[2] = {(float *)(A.arena + Q.off), (float *)(A.arena + Q.off + (size_t)n)};
    float *contrib[2] = {(float *)(A.arena + Q.off + 2 * (size_t)n), (float *)(A.arena + Q.off + 3 * (size_t)n)};
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tr = team.rank(), ts = team.size();
    const float d = Q.damping, restart = 1.0f - Q.damping;
    for (int32_t u = tr * BT + tid; u < n; u += ts * BT) {
        const int32_t od = __ldg(G.out_ptr + u + 1) - __ldg(G.out_ptr + u);
        const float r = u == Q.source ? 1.0f : 0.0f;
        rank[0][u] = r;
        contrib[0][u] = od > 0 ? __fdiv_rn(r, (float)od) : 0.0f;
    }
    team.sync();
    const int32_t lo = (int32_t)(((long long)n * tr) / ts), hi = (int32_t)(((long long)n * (tr + 1)) / ts);
    for (uint32_t it = 0; it < Q.iters; ++it) {
        const float *cc = contrib[it & 1];
        float *rn = rank[(it + 1) & 1];
        float *cn = contrib[(it + 1) & 1];
        auto apply = [&](int32_t u, float acc) {
            const float nw = __fmaf_rn(d, acc, u == Q.source ? restart : 0.0f);
            const int32_t od = __ldg(G.out_ptr + u + 1) - __ldg(G.out_ptr + u);
            rn[u] = nw;
            cn[u] = od > 0 ? __fdiv_rn(nw, (float)od) : 0.0f;
        };
        for (int32_t b0 = lo; b0 < hi; b0 += BT) {
            const int32_t u = b0 + tid;
            int32_t k0 = 0, deg = -1;
            if (u < hi) {
                k0 = __ldg(G.in_ptr + u);
                deg = __ldg(G.in_ptr + u + 1) - k0;
            }
            if (tid == 0) sh.hub_n = 0;
            __syncthreads();
            {
                // light rows (degree below warp_deg) of this warp's 32 rows: the
                // warp walks their arcs together, 32 at a time (consecutive source
                // reads), and a segmented scan in arc order sums each row's chunk
                // part, which the row's lane adds to its total
                const bool light = deg >= 0 && deg < Q.warp_deg;
                const int32_t ld = light ? deg : 0;
                int32_t incl = ld;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
                const int32_t excl = incl - ld;
                float acc = 0.0f;
                for (int32_t j0 = 0; j0 < tot; j0 += 32) {
                    const int32_t i = j0 + lane;
                    int r = 0;   // the lane whose row holds item i: last lane with excl <= i
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int c = r + step;
                        if (__shfl_sync(0xFFFFFFFFu, excl, c) <= i) r = c;
                    }
                    const int32_t rk0 = __shfl_sync(0xFFFFFFFFu, k0, r);
                    const int32_t rex = __shfl_sync(0xFFFFFFFFu, excl, r);
                    const bool valid = i < tot;
                    const int owner = valid ? r : 32 + lane;
                    float v = valid ? cc[__ldg(G.in_src + rk0 + (i - rex))] : 0.0f;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const float y = __shfl_up_sync(0xFFFFFFFFu, v, o);
                        const int yo = __shfl_up_sync(0xFFFFFFFFu, owner, o);
                        if (lane >= o && yo == owner) v = __fadd_rn(y, v);
                    }
                    const int next_owner = __shfl_down_sync(0xFFFFFFFFu, owner, 1);
                    sh.seg[warp * 32 + lane] = 0.0f;
                    __syncwarp();
                    if (valid && (lane == 31 || next_owner != owner)) sh.seg[warp * 32 + r] = v;
                    __syncwarp();
                    acc = __fadd_rn(acc, sh.seg[warp * 32 + lane]);
                    __syncwarp();
                }
                if (light) apply(u, acc);
            }
            unsigned mb = __ballot_sync(0xFFFFFFFFu, deg >= Q.warp_deg && deg < Q.cta_deg);
            while (mb) {
                const int src = __ffs(mb) - 1;
                mb &= mb - 1;
                const int32_t wu = __shfl_sync(0xFFFFFFFFu, u, src);
                const int32_t wk0 = __shfl_sync(0xFFFFFFFFu, k0, src);
                const int32_t wdeg = __shfl_sync(0xFFFFFFFFu, deg, src);
                float acc = 0.0f;
                for (int32_t k = lane; k < wdeg; k += 32) acc = __fadd_rn(acc, cc[__ldg(G.in_src + wk0 + k)]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, o));
                if (lane == src) apply(wu, acc);
            }
            if (deg >= Q.cta_deg) sh.hub[atomicAdd(&sh.hub_n, 1)] = u;
            __syncthreads();
            for (int h = 0; h < sh.hub_n; ++h) {
                const int32_t hu = sh.hub[h];
                const int32_t hk0 = __ldg(G.in_ptr + hu);
                const int32_t hdeg = __ldg(G.in_ptr + hu + 1) - hk0;
                float acc = 0.0f;
                for (int32_t k = tid; k < hdeg; k += BT) acc = __fadd_rn(acc, cc[__ldg(G.in_src + hk0 + k)]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, o));
                if (lane == 0) sh.red[warp] = acc;
                __syncthreads();
                if (tid == 0) {
                    float t = 0.0f;
                    for (int w = 0; w < BT / 32; ++w) t = __fadd_rn(t, sh.red[w]);
                    apply(hu, t);
                }
                __syncthreads();
            }
            __syncthreads();
        }
        team.sync();
    }
    if (tr == 0 && tid == 0) {
        qs->iterations = Q.iters;
        qs->arcs = (unsigned long long)Q.iters * (unsigned long long)G.m;
    }
}

template <int BT, class Team>
__device__ void serve(const BatchArgs &A, int32_t q, const Team &team, Shared<BT> &sh)
{
    const BatchQuery Q = A.queries[q];
    const BatchGraph G = A.graphs[Q.graph];
    QueryStatsDev *qs = A.qs + q;
    if (team.rank() == 0 && threadIdx.x == 0) {
        qs->t_start = globaltimer();
        qs->team = (uint32_t)team.size();
    }
    if (Q.app == GG_APP_PPR) serve_ppr<BT>(A, Q, G, team, sh, qs);
    else serve_push<BT>(A, Q, G, team, sh, qs);
    team.sync();
    if (team.rank() == 0 && threadIdx.x == 0) qs->t_end = globaltimer();
}

template <int BT>
__global__ void __launch_bounds__(BT) k_batch(BatchArgs A)
{
    __shared__ Shared<BT> sh;
    if (threadIdx.x == 0) atomicMin(A.t0, globaltimer());
    // Some clusters start with the small queries (so short queries do not
    // queue behind every large one), the others with the large ones; each
    // then serves the other kind until none is left.
    const int cid = (int)(blockIdx.x / (unsigned)(A.cluster > 1 ? A.cluster : 1));
    const bool small_first = A.cluster > 1 && A.small_first > 0 && cid % A.small_first == 0;
    for (int phase = 0; phase < 2; ++phase) {
        if ((phase == 0) != small_first) {
            if (A.cluster <= 1) continue;
            ClusterTeam team{cg::this_cluster()};
            for (;;) {
                if (team.rank() == 0 && threadIdx.x == 0) sh.claim = (int32_t)atomicAdd(&A.counters[0], 1u);
                team.sync();
                const int32_t idx = *team.cl.map_shared_rank(&sh.claim, 0);
                team.sync();
                if (idx >= A.n_big) break;
                serve<BT>(A, A.order_big[idx], team, sh);
            }
        } else {
            CtaTeam solo;
            for (;;) {
                if (threadIdx.x == 0) sh.claim = (int32_t)atomicAdd(&A.counters[1], 1u);
                __syncthreads();
                const int32_t idx = sh.claim;
                __syncthreads();
                if (idx >= A.n_small) break;
                serve<BT>(A, A.order_small[idx], solo, sh);
            }
        }
    }
}

}  // namespace

}  // namespace gg

// ------------------------------------------------------------------ host --
struct gg_batch {
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    gg_batch_config cfg{};
    int32_t n_queries = 0;
    std::vector<gg::BatchQuery> hq;
    std::vector<int32_t> hn;            // vertex count of each query's graph
    gg::DevBuf b_graphs, b_queries, b_order, b_counters, b_arena, b_qs;
    gg::BatchArgs args{};
    int grid = 0;
    int threads = 256;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
};

using namespace gg;

static const void *batch_kernel(int threads)
{
    switch (threads) {
    case 512: return (const void *)k_batch<512>;
    case 1024: return (const void *)k_batch<1024>;
    default: return (const void *)k_batch<256>;
    }
}

static cudaError_t launch_batch(gg_batch *b)
{
    cudaLaunchConfig_t lc{};
    lc.gridDim = dim3((unsigned)b->grid);
    lc.blockDim = dim3((unsigned)b->threads);
    lc.dynamicSmemBytes = 0;
    lc.stream = b->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)(b->cfg.cluster > 1 ? b->cfg.cluster : 1);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    void *args[] = {&b->args};
    return cudaLaunchKernelExC(&lc, batch_kernel(b->threads), args);
}

extern "C" {

gg_status gg_batch_create(gg_graph *const *graphs, int32_t n_graphs, const gg_query *queries, int32_t n_queries,
                          const gg_batch_config *cfg, gg_batch **out)
{
    if (!out) { set_error("gg_batch_create: out is NULL"); return GG_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!graphs || n_graphs < 1 || !queries || n_queries < 1 || !cfg) {
        set_error("gg_batch_create: empty or NULL graphs / queries / cfg");
        return GG_ERR_INVALID_ARG;
    }
    if (!(cfg->cluster == 1 || cfg->cluster == 2 || cfg->cluster == 4 || cfg->cluster == 8 || cfg->cluster == 16)) {
        set_error("gg_batch_create: cluster must be 1, 2, 4, 8 or 16");
        return GG_ERR_INVALID_ARG;
    }
    if (cfg->small_first < 0) { set_error("gg_batch_create: small_first must be >= 0"); return GG_ERR_INVALID_ARG; }
    if (cfg->order < GG_ORDER_MOST_WORK || cfg->order > GG_ORDER_TRAVERSALS_FIRST) {
        set_error("gg_batch_create: unknown order %d", (int)cfg->order);
        return GG_ERR_INVALID_ARG;
    }
    if (!(cfg->threads == 0 || cfg->threads == 256 || cfg->threads == 512 || cfg->threads == 1024)) {
        set_error("gg_batch_create: threads must be 0 (256), 256, 512 or 1024");
        return GG_ERR_INVALID_ARG;
    }
    if (cfg->warp_deg < 1 || cfg->cta_deg < cfg->warp_deg) {
        set_error("gg_batch_create: need 1 <= warp_deg <= cta_deg");
        return GG_ERR_INVALID_ARG;
    }
    for (int32_t i = 0; i < n_graphs; ++i)
        if (!graphs[i]) { set_error("gg_batch_create: graph %d is NULL", i); return GG_ERR_INVALID_ARG; }
    gg_batch *b = new (std::nothrow) gg_batch();
    if (!b) { set_error("gg_batch_create: host allocation failed"); return GG_ERR_OOM; }
    b->cfg = *cfg;
    b->threads = cfg->threads ? cfg->threads : 256;
    b->n_queries = n_queries;
    gg_status st = GG_OK;
    cudaError_t e;
    do {
        if ((e = cudaGetDevice(&b->device)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreate(&b->e0)) != cudaSuccess || (e = cudaEventCreate(&b->e1)) != cudaSuccess) {
            st = cuda_fail(e, "gg_batch_create (device setup)");
            break;
        }
        std::vector<BatchGraph> hg((size_t)n_graphs);
        for (int32_t i = 0; i < n_graphs; ++i) {
            gg_graph *g = graphs[i];
            if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) { st = cuda_fail(e, "graph stream"); break; }
            hg[i] = BatchGraph{g->n, (int32_t)g->m, g->out_ptr, g->out_dst, g->out_w, g->in_ptr, g->in_src};
        }
        if (st != GG_OK) break;
        b->hq.resize((size_t)n_queries);
        b->hn.resize((size_t)n_queries);
        std::vector<std::pair<double, int32_t>> big, small;
        unsigned long long words = 0;
        for (int32_t q = 0; q < n_queries; ++q) {
            const gg_query &Q = queries[q];
            if (Q.graph < 0 || Q.graph >= n_graphs) { set_error("query %d: graph %d out of range", q, Q.graph); st = GG_ERR_INVALID_ARG; break; }
            const gg_graph *g = graphs[Q.graph];
            if (!(Q.app == GG_APP_BFS || Q.app == GG_APP_SSSP || Q.app == GG_APP_PPR)) { set_error("query %d: app must be BFS, SSSP or PPR", q); st = GG_ERR_INVALID_ARG; break; }
            if (Q.source < 0 || Q.source >= g->n) { set_error("query %d: source %d outside [0, %d)", q, Q.source, g->n); st = GG_ERR_INVALID_ARG; break; }
            if (Q.app == GG_APP_SSSP && !g->has_w) { set_error("query %d: SSSP needs a weighted graph", q); st = GG_ERR_INVALID_ARG; break; }
            if (Q.app == GG_APP_PPR && !(Q.damping >= 0.0f && Q.damping <= 1.0f)) { set_error("query %d: damping must be in [0, 1]", q); st = GG_ERR_INVALID_ARG; break; }
            if ((Q.warp_deg != 0 || Q.cta_deg != 0) && !(Q.warp_deg >= 1 && Q.cta_deg >= Q.warp_deg)) {
                set_error("query %d: need 1 <= warp_deg <= cta_deg (or both 0)", q);
                st = GG_ERR_INVALID_ARG;
                break;
            }
            const int32_t wd = Q.warp_deg ? Q.warp_deg : cfg->warp_deg, cd = Q.warp_deg ? Q.cta_deg : cfg->cta_deg;
            BatchQuery bq{Q.graph, Q.app, Q.source, Q.iters, Q.damping, wd, cd, 0u, words};
            b->hq[q] = bq;
            b->hn[q] = g->n;
            words += 4ull * (unsigned long long)g->n + 8ull;
            words = (words + 31ull) & ~31ull;
            // estimated work: PPR iters * m; traversals ~ m (each arc relaxed about once);
            // the sort key gives the claim order (ascending key first)
            const double work = (Q.app == GG_APP_PPR ? (double)Q.iters : 1.0) * ((double)g->m + (double)g->n);
            double key = -work;
            if (cfg->order == GG_ORDER_LEAST_WORK) key = work;
            else if (cfg->order == GG_ORDER_TRAVERSALS_FIRST) key = (Q.app == GG_APP_PPR ? 1e300 : 0.0) - work;
            if (cfg->cluster > 1 && (int64_t)g->m >= cfg->big_arcs) big.push_back({key, q});
            else small.push_back({key, q});
        }
        if (st != GG_OK) break;
        std::stable_sort(big.begin(), big.end());
        std::stable_sort(small.begin(), small.end());
        std::vector<int32_t> order;
        for (auto &p : big) order.push_back(p.second);
        for (auto &p : small) order.push_back(p.second);
        if ((st = b->b_graphs.alloc(sizeof(BatchGraph) * hg.size())) != GG_OK ||
            (st = b->b_queries.alloc(sizeof(BatchQuery) * b->hq.size())) != GG_OK ||
            (st = b->b_order.alloc(sizeof(int32_t) * order.size())) != GG_OK ||
            (st = b->b_counters.alloc(16 + sizeof(unsigned long long))) != GG_OK ||
            (st = b->b_arena.alloc(4 * (size_t)words)) != GG_OK ||
            (st = b->b_qs.alloc(sizeof(QueryStatsDev) * (size_t)n_queries)) != GG_OK)
            break;
        if ((e = cudaMemcpy(b->b_graphs.p, hg.data(), sizeof(BatchGraph) * hg.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(b->b_queries.p, b->hq.data(), sizeof(BatchQuery) * b->hq.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(b->b_order.p, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
            st = cuda_fail(e, "gg_batch_create (upload)");
            break;
        }
        BatchArgs &A = b->args;
        A.graphs = (const BatchGraph *)b->b_graphs.p;
        A.queries = (const BatchQuery *)b->b_queries.p;
        A.order_big = b->b_order.i32();
        A.n_big = (int32_t)big.size();
        A.order_small = b->b_order.i32() + big.size();
        A.n_small = (int32_t)small.size();
        A.counters = b->b_counters.u32();
        A.t0 = (unsigned long long *)(b->b_counters.u32() + 4);
        A.arena = b->b_arena.u32();
        A.qs = (QueryStatsDev *)b->b_qs.p;
        A.warp_deg = cfg->warp_deg;
        A.cta_deg = cfg->cta_deg;
        A.cluster = cfg->cluster;
        A.small_first = cfg->small_first;
        // persistent grid: as many clusters (or CTAs) as fit at once
        const void *fn = batch_kernel(b->threads);
        if (cfg->cluster > 8 &&
            (e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess) {
            st = cuda_fail(e, "cluster size 16 (non-portable)");
            break;
        }
        cudaLaunchConfig_t lc{};
        lc.blockDim = dim3((unsigned)b->threads);
        lc.gridDim = dim3((unsigned)(b->num_sms * cfg->cluster));
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)cfg->cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        int clusters = 0;
        if ((e = cudaOccupancyMaxActiveClusters(&clusters, fn, &lc)) != cudaSuccess || clusters < 1) {
            if (e == cudaSuccess) e = cudaErrorInvalidConfiguration;
            st = cuda_fail(e, "cudaOccupancyMaxActiveClusters");
            break;
        }
        b->grid = clusters * cfg->cluster;
    } while (0);
    if (st != GG_OK) {
        gg_batch_free(b);
        return st;
    }
    *out = b;
    return GG_OK;
}

gg_status gg_batch_run(gg_batch *b, float *ms)
{
    if (!b) { set_error("gg_batch_run: batch is NULL"); return GG_ERR_INVALID_ARG; }
    if (!b->exec) {
        // one captured graph: reset the claim counters and the start time,
        // then the persistent launch
        GG_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemsetAsync(b->b_counters.p, 0, 16, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync((char *)b->b_counters.p + 16, 0xFF, 8, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->b_qs.p, 0, b->b_qs.bytes, b->stream);
        if (e == cudaSuccess) e = launch_batch(b);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e != cudaSuccess ? e : e2, "gg_batch_run (capture)");
        }
        b->graph = graph;
        GG_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
    GG_CUDA(cudaEventRecord(b->e0, b->stream));
    GG_CUDA(cudaGraphLaunch(b->exec, b->stream));
    GG_CUDA(cudaEventRecord(b->e1, b->stream));
    GG_CUDA(cudaStreamSynchronize(b->stream));
    if (ms) GG_CUDA(cudaEventElapsedTime(ms, b->e0, b->e1));
    return GG_OK;
}

gg_status gg_batch_query_stats(gg_batch *b, gg_query_stats *out, int32_t n)
{
    if (!b || !out || n < b->n_queries) { set_error("gg_batch_query_stats: bad arguments"); return GG_ERR_INVALID_ARG; }
    std::vector<QueryStatsDev> h((size_t)b->n_queries);
    unsigned long long t0 = 0;
    GG_CUDA(cudaStreamSynchronize(b->stream));
    GG_CUDA(cudaMemcpy(h.data(), b->b_qs.p, sizeof(QueryStatsDev) * h.size(), cudaMemcpyDeviceToHost));
    GG_CUDA(cudaMemcpy(&t0, b->args.t0, sizeof t0, cudaMemcpyDeviceToHost));
    for (int32_t q = 0; q < b->n_queries; ++q) {
        const QueryStatsDev &s = h[q];
        out[q].latency_ns = s.t_end >= t0 ? s.t_end - t0 : 0;
        out[q].service_ns = s.t_end >= s.t_start ? s.t_end - s.t_start : 0;
        out[q].arcs = s.arcs;
        out[q].iterations = s.iterations;
        out[q].team = s.team;
    }
    return GG_OK;
}

gg_status gg_batch_result(gg_batch *b, int32_t q, void *dst, size_t bytes)
{
    if (!b || !dst || q < 0 || q >= b->n_queries) { set_error("gg_batch_result: bad arguments"); return GG_ERR_INVALID_ARG; }
    const size_t n = (size_t)b->hn[q];
    if (bytes < 4 * n) { set_error("gg_batch_result: buffer of %zu bytes, result needs %zu", bytes, 4 * n); return GG_ERR_INVALID_ARG; }
    const BatchQuery &Q = b->hq[q];
    const uint32_t *src = b->b_arena.u32() + Q.off;
    if (Q.app == GG_APP_PPR) src += (Q.iters & 1u) ? n : 0;
    GG_CUDA(cudaStreamSynchronize(b->stream));
    GG_CUDA(cudaMemcpy(dst, src, 4 * n, cudaMemcpyDeviceToHost));
    return GG_OK;
}

void gg_batch_free(gg_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    b->b_graphs.release();
    b->b_queries.release();
    b->b_order.release();
    b->b_counters.release();
    b->b_arena.release();
    b->b_qs.release();
    if (b->stream) {
        cudaStreamSynchronize(b->stream);
        cudaStreamDestroy(b->stream);
    }
    delete b;
}

}  // extern "C"

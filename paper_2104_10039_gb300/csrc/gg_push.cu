// gg_push.cu - the push frontier of the min applications (SSSP, BFS, CC) and
// the small per-vertex kernels around the iterations (initial values, frontier
// degrees and value snapshots).
//
// Active vertices (Sec. 2.1): only vertices whose value changed in the last
// iteration can lower a neighbour, so an iteration may relax just their
// out-arcs (the active ones in approximate mode, Sec. 3.3) instead of
// pulling over every in-edge. Values pushed are the frontier's values at the
// end of the previous iteration (q_val), and targets are lowered in place with
// atomicMin, which gives exactly the synchronous pull result.
#include "gg_internal.cuh"

namespace gg {

__global__ void __launch_bounds__(kThreads) k_push(PushArgs a)
{
    __shared__ int slot;
    const uint32_t qn = *a.q_len;
    const uint32_t total = qn ? a.q_deg_ex[qn] : 0u;
    const uint32_t num_tiles = (total + kTile - 1) / kTile;
    const uint32_t lane = lane_id();
    const uint32_t lt = (1u << lane) - 1u;
    for (;;) {
        const int t = next_tile(a.sched, num_tiles, &slot);
        if (t < 0) break;
        const uint32_t g0 = (uint32_t)t * kTile;
#pragma unroll 1
        for (int r = 0; r < kIPT; ++r) {
            const uint32_t g = g0 + (uint32_t)r * kThreads + threadIdx.x;
            bool want = false;
            int32_t u = 0;
            if (g < total) {
                uint32_t lo = 0, hi = qn;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (a.q_deg_ex[mid] <= g) lo = mid;
                    else hi = mid;
                }
                const int32_t v = a.q[lo];
                const int32_t e = a.out_ptr[v] + (int32_t)(g - a.q_deg_ex[lo]);
                bool active = true;
                if (a.mask) {
                    const int32_t k = a.out_to_in[e];
                    active = (a.mask[k >> 5] >> (k & 31)) & 1u;
                }
                if (active) {
                    u = a.out_dst[e];
                    const uint32_t vv = a.q_val[lo];
                    uint32_t cand;
                    if (a.app == GG_APP_CC) {
                        cand = vv;
                    } else {
                        const uint32_t step = a.app == GG_APP_BFS ? 1u : a.out_w[e];
                        const unsigned long long c = (unsigned long long)vv + step;
                        cand = (vv == kInf || c >= kInf) ? kInf : (uint32_t)c;
                    }
                    if (cand != kInf && cand < a.val[u]) {
                        const uint32_t old = atomicMin(&a.val[u], cand);
                        if (cand < old) want = atomicExch(&a.stamp[u], a.stamp_tag) != a.stamp_tag;
                    }
                }
            }
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, want);
            if (b) {
                const int leader = __ffs(b) - 1;
                uint32_t base = 0;
                if ((int)lane == leader) base = atomicAdd(a.q_out_len, (uint32_t)__popc(b));
                base = __shfl_sync(0xFFFFFFFFu, base, leader);
                if (want) a.q_out[base + __popc(b & lt)] = u;
            }
        }
    }
    sched_leave(a.sched);
}

cudaError_t launch_push(const PushArgs &a, uint32_t max_arcs, int grid, cudaStream_t s)
{
    const uint32_t tiles = (max_arcs + kTile - 1) / kTile;
    int g = grid < (int)tiles ? grid : (int)tiles;
    if (g < 1) g = 1;
    k_push<<<g, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// Out-degrees of the frontier vertices (scanned afterwards into q_deg).
// Out-degree of every frontier vertex (the push scans them into arc offsets)
// and the frontier summary: its length, its out-arcs (sum is zeroed before the
// launch) and the packed list's arc count.
__global__ void k_qdeg(const int32_t *__restrict__ q, const uint32_t *__restrict__ q_len,
                       const int32_t *__restrict__ out_ptr, uint32_t *__restrict__ deg, FrontSum *sum,
                       const uint32_t *__restrict__ nnz)
{
    const uint32_t qn = *q_len;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sum->len = qn;
        sum->nnz = nnz ? *nnz : 0u;
    }
    unsigned long long arcs = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < qn; i += gridDim.x * blockDim.x) {
        const int32_t v = q[i];
        const uint32_t d = (uint32_t)(out_ptr[v + 1] - out_ptr[v]);
        deg[i] = d;
        arcs += d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) arcs += __shfl_xor_sync(0xFFFFFFFFu, arcs, o);
    if ((threadIdx.x & 31) == 0 && arcs) atomicAdd(&sum->arcs, arcs);
}

// Values of the frontier vertices at the end of a push iteration; with hist,
// also their change feature (1: the value decreased; the slot was zeroed).
__global__ void k_snapshot(const int32_t *__restrict__ q, const uint32_t *__restrict__ q_len,
                           const uint32_t *__restrict__ val, uint32_t *__restrict__ q_val, float *__restrict__ hist)
{
    const uint32_t qn = *q_len;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < qn; i += gridDim.x * blockDim.x) {
        const int32_t u = q[i];
        q_val[i] = val[u];
        if (hist) hist[u] = 1.0f;
    }
}

// GG-Apply's starting point for PageRank: rank 1/N, contribution rank/outdeg.
__global__ void k_init_pr(int32_t n, const int32_t *__restrict__ out_ptr, float *__restrict__ rank,
                          float *__restrict__ contrib)
{
    const float r0 = __fdiv_rn(1.0f, (float)n);
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int deg = out_ptr[u + 1] - out_ptr[u];
        rank[u] = r0;
        contrib[u] = deg > 0 ? __fdiv_rn(r0, (float)deg) : 0.0f;
    }
}

// Min applications: unreached everywhere but the source (SSSP, BFS), or own
// id (CC); the first frontier is the source, or every vertex.
__global__ void k_init_min(int32_t n, int app, int32_t source, uint32_t *__restrict__ val,
                           int32_t *__restrict__ q, uint32_t *__restrict__ q_val, uint32_t *__restrict__ q_len)
{
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        if (app == GG_APP_CC) {
            val[u] = (uint32_t)u;
            q[u] = u;
            q_val[u] = (uint32_t)u;
        } else {
            val[u] = u == source ? 0u : kInf;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (app == GG_APP_CC) {
            *q_len = (uint32_t)n;
        } else {
            q[0] = source;
            q_val[0] = 0u;
            *q_len = 1u;
        }
    }
}

__global__ void k_iter_header(IterStatsDev *s, uint32_t mode, const uint32_t *arcs_dev, unsigned long long arcs,
                              unsigned long long selected)
{
    s->mode = mode;
    s->arcs = arcs_dev ? (unsigned long long)*arcs_dev : arcs;
    s->selected = selected;
}

// After a learned correction: the frontier of the next push iteration also
// takes the vertices that changed in the iteration before it (the rows the
// correction left alone did not gather them), unless already in it.
__global__ void k_append_frontier(const int32_t *__restrict__ q_src, uint32_t len, const float *__restrict__ hist_now,
                                  const uint32_t *__restrict__ val, int32_t *__restrict__ q_dst,
                                  uint32_t *__restrict__ q_dst_val, uint32_t *__restrict__ q_dst_len)
{
    const uint32_t lane = lane_id();
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t i0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; i0 < len; i0 += gridDim.x * blockDim.x) {
        const uint32_t i = i0 + lane;
        int32_t u = 0;
        bool want = false;
        if (i < len) {
            u = q_src[i];
            want = hist_now[u] == 0.0f;
        }
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, want);
        if (b) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(q_dst_len, (uint32_t)__popc(b));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (want) {
                q_dst[base + __popc(b & lt)] = u;
                q_dst_val[base + __popc(b & lt)] = val[u];
            }
        }
    }
}

cudaError_t launch_append_frontier(const int32_t *q_src, uint32_t len, const float *hist_now, const uint32_t *val,
                                   int32_t *q_dst, uint32_t *q_dst_val, uint32_t *q_dst_len, int num_sms,
                                   cudaStream_t s)
{
    if (len == 0) return cudaSuccess;
    int blocks = (int)((len + 255) / 256);
    if (blocks > num_sms * 8) blocks = num_sms * 8;
    k_append_frontier<<<blocks, 256, 0, s>>>(q_src, len, hist_now, val, q_dst, q_dst_val, q_dst_len);
    return cudaGetLastError();
}

__global__ void k_iter_changed(IterStatsDev *s, const uint32_t *q_len) { s->changed = *q_len; }

cudaError_t launch_qdeg(const int32_t *q, const uint32_t *q_len, const int32_t *out_ptr, uint32_t *deg,
                        FrontSum *sum, const uint32_t *nnz, uint32_t max_n, int num_sms, cudaStream_t s)
{
    int blocks = (int)((max_n + 255) / 256);
    if (blocks > num_sms * 8) blocks = num_sms * 8;
    if (blocks < 1) blocks = 1;
    k_qdeg<<<blocks, 256, 0, s>>>(q, q_len, out_ptr, deg, sum, nnz);
    return cudaGetLastError();
}

cudaError_t launch_snapshot(const int32_t *q, const uint32_t *q_len, const uint32_t *val, uint32_t *q_val,
                            float *hist, uint32_t max_n, int num_sms, cudaStream_t s)
{
    int blocks = (int)((max_n + 255) / 256);
    if (blocks > num_sms * 8) blocks = num_sms * 8;
    if (blocks < 1) blocks = 1;
    k_snapshot<<<blocks, 256, 0, s>>>(q, q_len, val, q_val, hist);
    return cudaGetLastError();
}

cudaError_t launch_init_pr(int32_t n, const int32_t *out_ptr, float *rank, float *contrib, int num_sms,
                           cudaStream_t s)
{
    k_init_pr<<<num_sms * 8, 256, 0, s>>>(n, out_ptr, rank, contrib);
    return cudaGetLastError();
}

cudaError_t launch_init_min(int32_t n, int app, int32_t source, uint32_t *val, int32_t *q, uint32_t *q_val,
                            uint32_t *q_len, int num_sms, cudaStream_t s)
{
    k_init_min<<<num_sms * 8, 256, 0, s>>>(n, app, source, val, q, q_val, q_len);
    return cudaGetLastError();
}

cudaError_t launch_iter_header(IterStatsDev *st, uint32_t mode, const uint32_t *arcs_dev,
                               unsigned long long arcs, cudaStream_t s, unsigned long long selected)
{
    k_iter_header<<<1, 1, 0, s>>>(st, mode, arcs_dev, arcs, selected);
    return cudaGetLastError();
}

cudaError_t launch_iter_changed(IterStatsDev *st, const uint32_t *q_len, cudaStream_t s)
{
    k_iter_changed<<<1, 1, 0, s>>>(st, q_len);
    return cudaGetLastError();
}

__global__ void k_active_outdeg(const int32_t *__restrict__ sp_src, const uint32_t *__restrict__ sp_nnz,
                                const int32_t *__restrict__ hub_ids, int32_t *__restrict__ act)
{
    const uint32_t nnz = *sp_nnz;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x) {
        const int32_t v = sp_src[k];   // hub-coded
        atomicAdd(&act[v < 0 ? hub_ids[-v - 1] : v], 1);
    }
}

cudaError_t launch_active_outdeg(const int32_t *sp_src, const uint32_t *sp_nnz, uint32_t max_arcs, int32_t n,
                                 const int32_t *hub_ids, int32_t *act, int num_sms, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(act, 0, sizeof(int32_t) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    int blocks = (int)((max_arcs + 255) / 256);
    if (blocks > num_sms * 8) blocks = num_sms * 8;
    if (blocks < 1) blocks = 1;
    k_active_outdeg<<<blocks, 256, 0, s>>>(sp_src, sp_nnz, hub_ids, act);
    return cudaGetLastError();
}

// contrib = rank / degree, the degree being deg[u] (active out-arcs) or, when
// deg is null, the full out-degree from out_ptr.
__global__ void k_contrib(int32_t n, const float *__restrict__ rank, const int32_t *__restrict__ deg,
                          const int32_t *__restrict__ out_ptr, float *__restrict__ contrib)
{
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int d = deg ? deg[u] : out_ptr[u + 1] - out_ptr[u];
        contrib[u] = d > 0 ? __fdiv_rn(rank[u], (float)d) : 0.0f;
    }
}

cudaError_t launch_contrib(int32_t n, const float *rank, const int32_t *deg, const int32_t *out_ptr,
                           float *contrib, int num_sms, cudaStream_t s)
{
    k_contrib<<<num_sms * 8, 256, 0, s>>>(n, rank, deg, out_ptr, contrib);
    return cudaGetLastError();
}

}  // namespace gg

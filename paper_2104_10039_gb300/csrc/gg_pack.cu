// gg_pack.cu - the packed active in-edges (the list approximate gathers
// stream, Sec. 3.4: the graph keeps every edge, flagged active or not) from
// the flag bitmap of the full in-edge list, after every sampling pass and
// every correction.
//
// Tiles of 256 consecutive arcs (the pull path's tiles):
//   k_pack_counts  active arcs per tile (popcount of its 8 flag words); a
//                  correction's flag pass writes these itself
//   (scan)         tile offsets in the packed list
//   k_pack_arcs    one warp per tile: each active arc's source (hub-coded for
//                  PageRank, as its gathers read them) and weight to tile
//                  offset + its rank among the tile's active arcs,
//                  sources read with 16-byte loads, staged in shared memory
//                  and stored by consecutive lanes
//   k_pack_ptr     one thread per vertex: its packed row start = the offset
//                  of the tile holding its first arc + the active arcs of
//                  that tile before it
// The packed order is the list order, so the result is the same whatever
// the tiling. The last two steps wait until an approximate gather or a
// result needs the list (ensure_packed): a min application that only pushes
// before its next correction, or a run that ends on a correction, never
// builds it; PageRank builds it without weights.
//
// The active-arc count (scan total) is always set at once: the push/pull
// switch and the iteration statistics need it.
#include "gg_graph.cuh"

namespace gg {

namespace {

constexpr int kPT = 256;   // arcs per tile

// Flag bits of arcs [32w, 32w + 32) that lie before arc m.
__device__ __forceinline__ uint32_t word_in_list(uint32_t word, long long w, long long m)
{
    const long long lo = 32 * w;
    if (lo + 32 <= m) return word;
    if (lo >= m) return 0u;
    return word & ((1u << (uint32_t)(m - lo)) - 1u);
}

__global__ void k_pack_counts(const uint32_t *__restrict__ mask, long long m, uint32_t *__restrict__ cnt)
{
    const long long nt = (m + kPT - 1) / kPT;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += (long long)gridDim.x * blockDim.x) {
        uint32_t c = 0;
        const long long nw = (m + 31) / 32;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const long long w = 8 * t + i;
            if (w < nw) c += (uint32_t)__popc(word_in_list(mask[w], w, m));
        }
        cnt[t] = c;
    }
}

template <bool WEIGHTED>
__global__ void __launch_bounds__(256) k_pack_arcs(const uint32_t *__restrict__ mask, long long m,
                                                   const uint32_t *__restrict__ off, const int32_t *__restrict__ src,
                                                   const uint32_t *__restrict__ w, int32_t *__restrict__ sp_src,
                                                   uint32_t *__restrict__ sp_w)
{
    // each warp stages its tile's active arcs in order, then stores them with
    // consecutive lanes on consecutive positions
    __shared__ int32_t s_src[8 * kPT];
    __shared__ uint32_t s_w[WEIGHTED ? 8 * kPT : 1];
    const uint32_t lane = threadIdx.x & 31u;
    int32_t *st = s_src + (threadIdx.x >> 5) * kPT;
    uint32_t *sw = s_w + (WEIGHTED ? (threadIdx.x >> 5) * kPT : 0);
    const long long nt = (m + kPT - 1) / kPT;
    const long long nw = (m + 31) / 32;
    const long long W = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nt; t += W) {
        const long long a0 = t * kPT;
        const bool full = a0 + kPT <= m;
        // the tile's flag words (lanes 0..7 load one each, then broadcast)
        uint32_t mw = 0;
        if (lane < 8 && 8 * t + lane < nw) mw = word_in_list(mask[8 * t + lane], 8 * t + lane, m);
        const uint32_t base = off[t];
        uint32_t before = 0;   // active arcs of the tile before this half
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t wi = 4u * (uint32_t)h + (lane >> 3), sh = 4u * (lane & 7u);
            const uint32_t word = __shfl_sync(0xFFFFFFFFu, mw, (int)wi);
            const uint32_t f = (word >> sh) & 0xFu;
            uint32_t rank = before + (uint32_t)__popc(word & ((1u << sh) - 1u));
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t wk = __shfl_sync(0xFFFFFFFFu, mw, 4 * h + k);
                if ((uint32_t)k < (lane >> 3)) rank += (uint32_t)__popc(wk);
            }
            if (f) {
                const long long q0 = a0 + 128 * h + 4 * (long long)lane;
                int32_t s4[4];
                uint32_t w4[4] = {0u, 0u, 0u, 0u};
                if (full) {
                    const int4 x = __ldg(reinterpret_cast<const int4 *>(src + q0));
                    s4[0] = x.x; s4[1] = x.y; s4[2] = x.z; s4[3] = x.w;
                    if (WEIGHTED) {
                        const uint4 y = __ldg(reinterpret_cast<const uint4 *>(w + q0));
                        w4[0] = y.x; w4[1] = y.y; w4[2] = y.z; w4[3] = y.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        s4[j] = ((f >> j) & 1u) ? src[q0 + j] : 0;   // flagged arcs lie before m
                        if (WEIGHTED) w4[j] = ((f >> j) & 1u) ? w[q0 + j] : 0u;
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if ((f >> j) & 1u) {
                        st[rank] = s4[j];
                        if (WEIGHTED) sw[rank] = w4[j];
                        ++rank;
                    }
                }
            }
            uint32_t hw = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) hw += (uint32_t)__popc(__shfl_sync(0xFFFFFFFFu, mw, 4 * h + k));
            before += hw;
        }
        __syncwarp();
        for (uint32_t k = lane; k < before; k += 32u) {
            sp_src[base + k] = st[k];
            if (WEIGHTED) sp_w[base + k] = sw[k];
        }
        __syncwarp();
    }
}

__global__ void k_pack_ptr(const int32_t *__restrict__ in_ptr, int32_t n, const uint32_t *__restrict__ mask,
                           long long m, const uint32_t *__restrict__ off, int32_t *__restrict__ sp_ptr)
{
    const long long nt = (m + kPT - 1) / kPT;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += (long long)gridDim.x * blockDim.x) {
        const long long p = in_ptr[v];
        const long long t = p / kPT;
        uint32_t r = 0;
        if (t < nt) {
            const long long wp = p >> 5;
            for (long long wd = 8 * t; wd < wp; ++wd) r += (uint32_t)__popc(mask[wd]);   // words wholly before p (< m)
            if ((p & 31) != 0) r += (uint32_t)__popc(mask[wp] & ((1u << (uint32_t)(p & 31)) - 1u));
        }
        sp_ptr[v] = (int32_t)(off[t < nt ? t : nt] + r);
    }
}

// The arc count of a deferred pack (the scan's total) and the correction's
// active_after statistic.
__global__ void k_pack_total(const uint32_t *__restrict__ off, long long nt, uint32_t *__restrict__ sp_nnz,
                             IterStatsDev *stats)
{
    const uint32_t q = off[nt];
    *sp_nnz = q;
    if (stats) stats->active_after = q;
}

// The packed arcs and row pointers from the scanned tile counts.
gg_status pack_lists(gg_graph *g, bool weighted, bool hubs)
{
    const int32_t *src = hubs ? g->in_src_h : g->in_src;
    cudaStream_t s = g->stream;
    const long long m = g->m;
    const long long nt = (m + kPT - 1) / kPT;
    long long ab = (nt * 32 + 255) / 256;
    if (ab > (long long)g->num_sms * 8) ab = (long long)g->num_sms * 8;
    if (ab < 1) ab = 1;
    if (nt > 0) {
        if (weighted) {
            k_pack_arcs<true><<<(unsigned)ab, 256, 0, s>>>(g->mask, m, g->tile_off, src, g->in_w, g->sp_src,
                                                           g->sp_w);
        } else {
            k_pack_arcs<false><<<(unsigned)ab, 256, 0, s>>>(g->mask, m, g->tile_off, src, nullptr, g->sp_src,
                                                            nullptr);
        }
        GG_CUDA(cudaGetLastError());
        g->launches += 1;
    }
    long long vb = ((long long)g->n + 1 + 255) / 256;
    if (vb > (long long)g->num_sms * 8) vb = (long long)g->num_sms * 8;
    k_pack_ptr<<<(unsigned)vb, 256, 0, s>>>(g->in_ptr, g->n, g->mask, m, g->tile_off, g->sp_ptr);
    GG_CUDA(cudaGetLastError());
    g->launches += 1;
    g->sp_stale = false;
    g->sp_has_w = weighted;
    g->sp_hubs = hubs;
    g->plan[1].valid = false;
    return GG_OK;
}

}  // namespace

gg_status pack_active(gg_graph *g, IterStatsDev *stats, bool have_counts)
{
    cudaStream_t s = g->stream;
    const long long m = g->m;
    const long long nt = (m + kPT - 1) / kPT;
    int grid = (int)((nt + 255) / 256);
    if (grid > g->num_sms * 8) grid = g->num_sms * 8;
    if (grid < 1) grid = 1;
    if (!have_counts) {
        k_pack_counts<<<grid, 256, 0, s>>>(g->mask, m, g->tile_cnt);
        GG_CUDA(cudaGetLastError());
        g->launches += 1;
    }
    GG_CUDA(launch_scan_u32(g->tile_cnt, g->tile_off, (size_t)nt, g->scan_tmp, s));
    k_pack_total<<<1, 1, 0, s>>>(g->tile_off, nt, g->sp_nnz, stats);
    GG_CUDA(cudaGetLastError());
    g->launches += nt > 0 ? 4 : 2;   // scan: three launches over a non-empty list, one otherwise
    g->sp_stale = true;
    g->plan[1].valid = false;
    return GG_OK;
}

// tile_off holds the scan of the current flags' tile counts: pack_active
// runs after every change of the flags, and nothing else writes it.
gg_status ensure_packed(gg_graph *g, bool weighted, PackCoding coding)
{
    weighted = weighted && g->has_w;
    const bool hubs = coding == PACK_ANY ? (g->sp_stale ? false : g->sp_hubs) : coding == PACK_HUBS;
    if (!g->sp_stale && (g->sp_has_w || !weighted) && g->sp_hubs == hubs) return GG_OK;
    return pack_lists(g, weighted, hubs);
}

}  // namespace gg

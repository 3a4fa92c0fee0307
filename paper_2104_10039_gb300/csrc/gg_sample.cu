// gg_sample.cu - sparsification of the full in-edge list (Sec. 3.4): every
// arc's initial flag from the hash of its endpoints, and the per-tile counts
// the pack of the active in-edges starts from.
//
// The hash needs both endpoints, so the list keeps each arc's row (in_dst)
// next to its source: the sampler is then one coalesced pass over two arrays
// with a ballot per 32 flags, and no merge path. The counts walk the
// merge-path tiles of the list once, reading only flag words and row ends.
#include "gg_hash.cuh"
#include "gg_internal.cuh"

namespace gg {

namespace {

constexpr int kSampleBatch = 8;   // flag words whose arcs are loaded at once

// One warp per chunk of 32 flag words (1 024 arcs): lane l takes arc 32 j + l
// of word j; the ballot of word j lands in lane j, which stores it.
__global__ void __launch_bounds__(256) k_sample(const int32_t *__restrict__ in_src,
                                                const int32_t *__restrict__ in_dst, long long m, int symmetric,
                                                unsigned long long seed, unsigned long long thr,
                                                uint32_t *__restrict__ mask)
{
    const uint32_t lane = lane_id();
    const long long words = (m + 31) >> 5;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c * 32 < words; c += warps) {
        uint32_t mine = 0;
#pragma unroll 1
        for (int b = 0; b < 32; b += kSampleBatch) {
            int32_t sv[kSampleBatch], dv[kSampleBatch];
#pragma unroll
            for (int j = 0; j < kSampleBatch; ++j) {
                const long long k = ((c * 32 + b + j) << 5) + lane;
                sv[j] = k < m ? __ldcs(in_src + k) : 0;
                dv[j] = k < m ? __ldcs(in_dst + k) : 0;
            }
#pragma unroll
            for (int j = 0; j < kSampleBatch; ++j) {
                const long long k = ((c * 32 + b + j) << 5) + lane;
                const uint32_t fl = k < m ? sampled_flag(sv[j], dv[j], symmetric, seed, thr) : 0u;
                const uint32_t word = __ballot_sync(0xFFFFFFFFu, fl != 0u);
                if ((int)lane == b + j) mine = word;
            }
        }
        const long long w = c * 32 + lane;
        if (w < words) mask[w] = mine;
    }
}

__device__ __forceinline__ uint32_t warp_incl_add(uint32_t v)
{
    const uint32_t lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= (uint32_t)o) v += y;
    }
    return v;
}

// One warp per tile t (items [t kWT, (t+1) kWT) of the merged sequence of
// arcs and row ends): the tile's arcs [a0, a1) span at most kWT / 32 + 1 flag
// words, one per lane; a warp scan of their popcounts gives the active arcs
// before any position. tile_cnt[t] = active arcs of the tile; for every row u
// ending in the tile, sp_ptr[u + 1] = active arcs in [a0, row_ptr[u + 1]).
__global__ void __launch_bounds__(256) k_tile_counts(const int32_t *__restrict__ tile_info, uint32_t num_tiles,
                                                     long long total_items, const int32_t *__restrict__ row_ptr,
                                                     const uint32_t *__restrict__ mask,
                                                     uint32_t *__restrict__ tile_cnt, int32_t *__restrict__ sp_ptr)
{
    const uint32_t lane = lane_id();
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < num_tiles; t += warps) {
        const int32_t r0 = tile_info[t] & 0x7FFFFFFF, r1 = tile_info[t + 1] & 0x7FFFFFFF;
        const long long d1 = (t + 1) * kWT < total_items ? (t + 1) * kWT : total_items;
        const int32_t a0 = (int32_t)(t * kWT - r0), a1 = (int32_t)(d1 - r1);
        const int32_t wb = a0 >> 5;
        const int nw = a1 > a0 ? ((a1 - 1) >> 5) - wb + 1 : 0;
        uint32_t rw = 0;
        if ((int)lane < nw) {
            const int32_t w0 = (wb + (int32_t)lane) * 32;
            const int32_t lo = a0 > w0 ? a0 : w0, hi = a1 < w0 + 32 ? a1 : w0 + 32;
            const uint32_t range = hi - lo == 32 ? 0xFFFFFFFFu : ((1u << (hi - lo)) - 1u) << (lo & 31);
            rw = mask[wb + (int32_t)lane] & range;
        }
        const uint32_t c = __popc(rw);
        const uint32_t incl = warp_incl_add(c);
        const uint32_t excl = incl - c;
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        if (lane == 0) tile_cnt[t] = total;
        for (int32_t base = r0; base < r1; base += 32) {
            const int32_t u = base + (int32_t)lane;
            const bool valid = u < r1;
            const int32_t e = valid ? row_ptr[u + 1] : a0;
            const int j = (e >> 5) - wb;   // 0 <= j <= nw
            const int js = j < 31 ? j : 31;
            const uint32_t ex_j = __shfl_sync(0xFFFFFFFFu, excl, js);
            const uint32_t rw_j = __shfl_sync(0xFFFFFFFFu, rw, js);
            const uint32_t before = j < nw ? ex_j + __popc(rw_j & ((1u << (e & 31)) - 1u)) : total;
            if (valid) sp_ptr[u + 1] = (int32_t)before;
        }
    }
}

}  // namespace

cudaError_t launch_sample(const int32_t *in_src, const int32_t *in_dst, long long m, int symmetric,
                          unsigned long long seed, unsigned long long thr, uint32_t *mask, int num_sms,
                          cudaStream_t s)
{
    const long long chunks = (m + 1023) / 1024;
    long long blocks = (chunks + 7) / 8;
    if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
    if (blocks < 1) return cudaSuccess;
    k_sample<<<(unsigned)blocks, 256, 0, s>>>(in_src, in_dst, m, symmetric, seed, thr, mask);
    return cudaGetLastError();
}

cudaError_t launch_tile_counts(const int32_t *tile_info, uint32_t num_tiles, long long total_items,
                               const int32_t *row_ptr, const uint32_t *mask, uint32_t *tile_cnt, int32_t *sp_ptr,
                               int num_sms, cudaStream_t s)
{
    long long blocks = ((long long)num_tiles * 32 + 255) / 256;
    if (blocks > (long long)num_sms * 16) blocks = (long long)num_sms * 16;
    if (blocks < 1) return cudaSuccess;
    k_tile_counts<<<(unsigned)blocks, 256, 0, s>>>(tile_info, num_tiles, total_items, row_ptr, mask, tile_cnt,
                                                   sp_ptr);
    return cudaGetLastError();
}

}  // namespace gg

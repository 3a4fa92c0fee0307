// gg_sample.cu - sparsification of the full in-edge list (Sec. 3.4): every
// arc's initial flag from the hash of its endpoints (the pack, gg_pack.cu,
// then builds the packed active in-edges from the flags).
//
// The hash needs both endpoints. An arc's source is in in_src; its row (the
// destination) comes from the full list's pull plan: the rank of the row
// holding the tile's first arc, plus the row starts in the tile up to the
// arc, indexes the vertices of the non-empty rows. So the sampler streams
// 4 bytes per arc (plus one row-start bit), with a ballot per 32 flags.
#include "gg_hash.cuh"
#include "gg_internal.cuh"

namespace gg {

namespace {

constexpr int kSampleBatch = 8;   // flag words whose arcs are loaded at once

// One warp per chunk of 32 flag words (1 024 arcs, four 256-arc plan tiles):
// lane l takes arc 32 j + l of word j; the ballot of word j lands in lane j,
// which stores it. The row of arc k in tile t at position q is
// nzv[trow[t] + (row starts at positions 1..q of the tile)].
__global__ void __launch_bounds__(256) k_sample(const int32_t *__restrict__ in_src, const uint32_t *__restrict__ hb,
                                                const int32_t *__restrict__ trow, const int32_t *__restrict__ nzv,
                                                long long m, int symmetric, unsigned long long seed,
                                                unsigned long long thr, uint32_t *__restrict__ mask)
{
    const uint32_t lane = lane_id();
    const long long words = (m + 31) >> 5;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const uint32_t upto = (2u << lane) - 1u;   // bits 0..lane (lane 31: all)
    for (long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c * 32 < words; c += warps) {
        uint32_t mine = 0;
        int32_t base = 0;    // rank of the row holding the current tile's first arc, minus its bit 0
        uint32_t run = 0;    // row starts in the tile's earlier words
#pragma unroll 1
        for (int b = 0; b < 32; b += kSampleBatch) {
            int32_t sv[kSampleBatch], dv[kSampleBatch];
#pragma unroll
            for (int j = 0; j < kSampleBatch; ++j) {
                const long long w = c * 32 + b + j;
                const long long k = (w << 5) + lane;
                const uint32_t h = w < words ? __ldg(hb + w) : 0u;
                if ((w & 7) == 0) {
                    base = w < words ? __ldg(trow + (w >> 3)) - (int32_t)(h & 1u) : 0;
                    run = 0;
                }
                sv[j] = k < m ? __ldcs(in_src + k) : 0;
                dv[j] = k < m ? __ldg(nzv + base + (int32_t)(run + (uint32_t)__popc(h & upto))) : 0;
                run += (uint32_t)__popc(h);
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

}  // namespace

cudaError_t launch_sample(const int32_t *in_src, const uint32_t *hb, const int32_t *trow, const int32_t *nzv,
                          long long m, int symmetric, unsigned long long seed, unsigned long long thr, uint32_t *mask,
                          int num_sms, cudaStream_t s)
{
    const long long chunks = (m + 1023) / 1024;
    long long blocks = (chunks + 7) / 8;
    if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
    if (blocks < 1) return cudaSuccess;
    k_sample<<<(unsigned)blocks, 256, 0, s>>>(in_src, hb, trow, nzv, m, symmetric, seed, thr, mask);
    return cudaGetLastError();
}

}  // namespace gg

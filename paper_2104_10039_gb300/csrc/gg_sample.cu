// gg_sample.cu - sparsification of the full in-edge list (Sec. 3.4): every
// arc's initial flag from the hash of its endpoints (the pack, gg_pack.cu,
// then builds the packed active in-edges from the flags).
//
// The hash needs both endpoints, so the list keeps each arc's row (in_dst)
// next to its source: the sampler is then one coalesced pass over two arrays
// with a ballot per 32 flags, and no merge path.
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

}  // namespace gg

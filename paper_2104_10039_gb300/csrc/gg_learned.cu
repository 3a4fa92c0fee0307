// gg_learned.cu - the learned correction's list plumbing (beyond the paper):
// the vertices the scorer selected are corrected over all their in-edges
// while every other vertex keeps its value and flags for that iteration.
//
// The selected rows' in-edges are copied into a sub-list (sources, weights,
// old flags, and each arc's position in the full in-edge list) that the
// ordinary correction kernels walk with a row -> vertex map; the sub-list's
// new flags are then written back to the full bitmap.
#include "gg_internal.cuh"

namespace gg {

namespace {

// rows[p] / sub_ptr[p] for the p-th selected vertex (p = sel_pos[u]);
// counts = {selected vertices, their in-edges}.
__global__ void k_sel_compact(int32_t n, const uint32_t *__restrict__ sel_flag, const uint32_t *__restrict__ sel_pos,
                              const uint32_t *__restrict__ sel_off, int32_t *__restrict__ rows,
                              int32_t *__restrict__ sub_ptr, uint32_t *__restrict__ counts)
{
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        if (sel_flag[u]) {
            const uint32_t p = sel_pos[u];
            rows[p] = u;
            sub_ptr[p] = (int32_t)sel_off[u];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t nsel = sel_pos[n], total = sel_off[n];
        sub_ptr[nsel] = (int32_t)total;
        counts[0] = nsel;
        counts[1] = total;
    }
}

// Last row r in [lo, hi] with sub_ptr[r] <= j (the row holding sub-list arc j).
__device__ __forceinline__ int32_t row_of(const int32_t *__restrict__ sub_ptr, int32_t lo, int32_t hi, uint32_t j)
{
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if ((uint32_t)sub_ptr[mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

constexpr int kChunk = 2048;   // sub-list arcs per block of k_sub_copy (8 per thread)

__global__ void __launch_bounds__(256) k_sub_copy(const int32_t *__restrict__ sub_ptr, int32_t nsel, uint32_t total,
                                                  const int32_t *__restrict__ rows, const int32_t *__restrict__ in_ptr,
                                                  const int32_t *__restrict__ in_src, const uint32_t *__restrict__ in_w,
                                                  const uint32_t *__restrict__ mask, int32_t *__restrict__ sub_src,
                                                  uint32_t *__restrict__ sub_w, int32_t *__restrict__ sub_pos,
                                                  uint32_t *__restrict__ sub_mask)
{
    __shared__ int32_t bounds[2];
    const uint32_t j0 = blockIdx.x * (uint32_t)kChunk;
    if (threadIdx.x == 0) {
        const uint32_t jl = j0 + kChunk - 1 < total ? j0 + kChunk - 1 : total - 1;
        bounds[0] = row_of(sub_ptr, 0, nsel - 1, j0);
        bounds[1] = row_of(sub_ptr, bounds[0], nsel - 1, jl);
    }
    __syncthreads();
    const int32_t lo = bounds[0], hi = bounds[1];
#pragma unroll 1
    for (int i = 0; i < kChunk / 256; ++i) {
        const uint32_t j = j0 + (uint32_t)(i * 256) + threadIdx.x;
        uint32_t flag = 0;
        if (j < total) {
            const int32_t r = row_of(sub_ptr, lo, hi, j);
            const int32_t k = in_ptr[rows[r]] + (int32_t)(j - (uint32_t)sub_ptr[r]);
            sub_src[j] = in_src[k];
            if (in_w) sub_w[j] = in_w[k];
            sub_pos[j] = k;
            flag = (mask[k >> 5] >> (k & 31)) & 1u;
        }
        const uint32_t word = __ballot_sync(0xFFFFFFFFu, flag);
        if ((threadIdx.x & 31) == 0 && j < total) sub_mask[j >> 5] = word;
    }
}

__global__ void k_keep_values(int32_t n, const float *__restrict__ rank_cur, float *__restrict__ rank_next,
                              const float *__restrict__ contrib_cur, float *__restrict__ contrib_next,
                              const uint32_t *__restrict__ val_cur, uint32_t *__restrict__ val_next,
                              float *__restrict__ hist)
{
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        if (rank_cur) {
            rank_next[u] = rank_cur[u];
            contrib_next[u] = contrib_cur[u];
        } else {
            val_next[u] = val_cur[u];
        }
        if (hist) hist[u] = 0.0f;
    }
}

// Flags of the sub-list back into the full bitmap. A warp takes 32
// consecutive sub-list arcs; their full-list positions increase, so the lanes
// that hit one bitmap word are consecutive and a segmented OR gathers the
// word's bits at its first lane, which writes it: a plain store when the
// warp owns all 32 bits, else an AND/OR pair limited to its bits.
__global__ void k_scatter_flags(const int32_t *__restrict__ sub_pos, const uint32_t *__restrict__ sub_mask,
                                uint32_t total, uint32_t *__restrict__ mask)
{
    const uint32_t lane = lane_id();
    const uint32_t nw = (total + 31) / 32;
    for (uint32_t wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wi < nw; wi += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t j = wi * 32 + lane;
        const bool live = j < total;
        const int32_t k = live ? sub_pos[j] : -1;
        const uint32_t word = live ? (uint32_t)k >> 5 : 0xFFFFFFFFu;
        const uint32_t bit = live ? 1u << (k & 31) : 0u;
        uint32_t set = ((sub_mask[wi] >> lane) & 1u) && live ? bit : 0u;
        uint32_t rng = bit;
        const uint32_t grp = __match_any_sync(0xFFFFFFFFu, word);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t s2 = __shfl_down_sync(0xFFFFFFFFu, set, o);
            const uint32_t r2 = __shfl_down_sync(0xFFFFFFFFu, rng, o);
            if (lane + o < 32 && ((grp >> (lane + o)) & 1u)) {
                set |= s2;
                rng |= r2;
            }
        }
        const bool first = live && (__ffs(grp) - 1) == (int)lane;
        if (first) {
            if (rng == 0xFFFFFFFFu) {
                mask[word] = set;
            } else {
                atomicAnd(&mask[word], ~rng);
                atomicOr(&mask[word], set);
            }
        }
    }
}

}  // namespace

cudaError_t launch_sel_compact(int32_t n, const uint32_t *sel_flag, const uint32_t *sel_pos, const uint32_t *sel_off,
                               int32_t *rows, int32_t *sub_ptr, uint32_t *counts, int num_sms, cudaStream_t s)
{
    k_sel_compact<<<num_sms * 8, 256, 0, s>>>(n, sel_flag, sel_pos, sel_off, rows, sub_ptr, counts);
    return cudaGetLastError();
}

cudaError_t launch_sub_copy(const int32_t *sub_ptr, int32_t nsel, uint32_t total, const int32_t *rows,
                            const int32_t *in_ptr, const int32_t *in_src, const uint32_t *in_w, const uint32_t *mask,
                            int32_t *sub_src, uint32_t *sub_w, int32_t *sub_pos, uint32_t *sub_mask, cudaStream_t s)
{
    if (total == 0 || nsel <= 0) return cudaSuccess;
    const uint32_t blocks = (total + kChunk - 1) / kChunk;
    k_sub_copy<<<blocks, 256, 0, s>>>(sub_ptr, nsel, total, rows, in_ptr, in_src, in_w, mask, sub_src, sub_w, sub_pos,
                                      sub_mask);
    return cudaGetLastError();
}

cudaError_t launch_keep_values(int32_t n, const float *rank_cur, float *rank_next, const float *contrib_cur,
                               float *contrib_next, const uint32_t *val_cur, uint32_t *val_next, float *hist,
                               int num_sms, cudaStream_t s)
{
    k_keep_values<<<num_sms * 8, 256, 0, s>>>(n, rank_cur, rank_next, contrib_cur, contrib_next, val_cur, val_next,
                                              hist);
    return cudaGetLastError();
}

cudaError_t launch_scatter_flags(const int32_t *sub_pos, const uint32_t *sub_mask, uint32_t total, uint32_t *mask,
                                 int num_sms, cudaStream_t s)
{
    if (total == 0) return cudaSuccess;
    long long warps = ((long long)total + 31) / 32;
    long long blocks = (warps + 7) / 8;
    if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
    k_scatter_flags<<<(unsigned)blocks, 256, 0, s>>>(sub_pos, sub_mask, total, mask);
    return cudaGetLastError();
}

}  // namespace gg

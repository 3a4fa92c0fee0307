// gg_noalloc.cu - gg_sample_csc_noalloc: edge sampling of a caller-owned
// in-edge list that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need this
// step: code running inside an allocator's own callbacks, a process whose
// device memory budget is fixed up front and already handed out, or a loop
// that must not call into the allocator. They pass their own inputs and outputs; the working memory this
// step needs (the tile partition, the per-tile active counts and their scan)
// lives in one fixed file-scope device array below, sized for
// n + m <= GG_NOALLOC_MAX_ITEMS. Every GPU that loads the library holds that
// array until the process exits, and every call on a device shares it, so
// calls that overlap on the GPU race; the array keeps the last call's
// contents and every call rewrites what it reads.
#include <atomic>
#include <cmath>

#include "gg_tile.cuh"

namespace gg {

constexpr uint32_t kNoallocMaxItems = GG_NOALLOC_MAX_ITEMS;
constexpr uint32_t kNoallocTiles = kNoallocMaxItems / kWT + 2;
constexpr uint32_t kNoallocPartials = kNoallocTiles / 4096 + 4;
// words: tile_info | tile_cnt | tile_off | scan partials | scalars
constexpr size_t kNoallocWords = 3 * ((size_t)kNoallocTiles + 2) + kNoallocPartials + 8;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoallocWords];

// Device address of the scratch array on the current device. Host code may
// not use the symbol itself as an address; the address is looked up once per
// device and cached (several host threads may race to fill an entry: they
// store the same address). The cache is not refreshed after cudaDeviceReset.
static uint32_t *noalloc_scratch(gg_status *st)
{
    static std::atomic<uint32_t *> ptrs[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { *st = cuda_fail(e, "cudaGetDevice"); return nullptr; }
    if (dev < 0 || dev >= 64) { set_error("gg_sample_csc_noalloc: device %d not supported", dev); *st = GG_ERR_UNSUPPORTED; return nullptr; }
    uint32_t *p = ptrs[dev].load(std::memory_order_acquire);
    if (!p) {
        void *a = nullptr;
        e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
        if (e != cudaSuccess) { *st = cuda_fail(e, "cudaGetSymbolAddress"); return nullptr; }
        p = (uint32_t *)a;
        ptrs[dev].store(p, std::memory_order_release);
    }
    *st = GG_OK;
    return p;
}

// scal[0] = m, scal[2] = 0 (the row-pointer check below sets it).
__global__ void k_na_set(uint32_t *scal, uint32_t m)
{
    scal[0] = m;
    scal[2] = 0u;
}

// The in-edge row pointers must start at 0, end at m and never decrease;
// otherwise the partition and the tile kernels would index outside the
// caller's arrays. A failed check sets scal[2]: the tile kernels then do
// nothing and *sp_nnz is set to 0xFFFFFFFF.
__global__ void k_na_check(const int32_t *__restrict__ in_ptr, int32_t n, uint32_t m, uint32_t *scal)
{
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        bad |= in_ptr[i] > in_ptr[i + 1];
    if (blockIdx.x == 0 && threadIdx.x == 0) bad |= in_ptr[0] != 0 || (uint32_t)in_ptr[n] != m;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(scal + 2, 1u);
}

struct NaSmem {
    int32_t rowend[kWT + 1];
    int32_t src[kPadded];
    uint32_t bits[kWT / 32 + 2];
};

// Merge-path coordinates of this lane inside tile t (rows r0.., arcs a0..).
__device__ __forceinline__ void na_lane_start(const NaSmem &s, int tile_items, int nrows, int narcs, int a0,
                                              int *lx, int *ly, int *cnt)
{
    const int lane = (int)lane_id();
    const int ld = lane * kIPT < tile_items ? lane * kIPT : tile_items;
    int c = tile_items - ld;
    *cnt = c < kIPT ? c : kIPT;
    int lo = ld - narcs > 0 ? ld - narcs : 0;
    int hi = ld < nrows ? ld : nrows;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s.rowend[mid] - a0 <= ld - mid - 1) lo = mid + 1;
        else hi = mid;
    }
    *lx = lo;
    *ly = ld - lo;
}

// Pass 1: sampled flags (Sec. 3.4) into the caller's bitmap, active count per tile.
__global__ void __launch_bounds__(kThreads)
k_na_flags(const int32_t *__restrict__ in_ptr, const int32_t *__restrict__ in_src, int32_t n,
           const uint32_t *__restrict__ scal, const int32_t *__restrict__ tile_info, int symmetric,
           unsigned long long seed, unsigned long long thr, uint32_t *__restrict__ mask,
           uint32_t *__restrict__ tile_cnt)
{
    __shared__ NaSmem smem[kWarps];
    NaSmem &s = smem[threadIdx.x >> 5];
    const uint32_t lane = lane_id();
    const long long total = (long long)n + scal[0];
    const int num_tiles = scal[2] ? 0 : (int)scal[1];   // rejected row pointers: no work
    const int W = (int)((gridDim.x * kThreads) >> 5);
    for (int t = (int)((blockIdx.x * kThreads + threadIdx.x) >> 5); t < num_tiles; t += W) {
        const int32_t r0 = tile_info[t] & 0x7FFFFFFF, r1 = tile_info[t + 1] & 0x7FFFFFFF;
        const long long d0 = (long long)t * kWT, d1 = d0 + kWT < total ? d0 + kWT : total;
        const int32_t a0 = (int32_t)(d0 - r0), a1 = (int32_t)(d1 - r1);
        const int nrows = r1 - r0, narcs = a1 - a0, w0 = a0 >> 5;
        const int nwords = narcs > 0 ? ((a1 - 1) >> 5) - w0 + 1 : 0;
        for (int i = (int)lane; i < nrows; i += 32) s.rowend[i] = in_ptr[r0 + i + 1];
        if (lane == 0) s.rowend[nrows] = 0x7FFFFFFF;
        for (int k = (int)lane; k < narcs; k += 32) s.src[pad(k)] = in_src[a0 + k];
        for (int i = (int)lane; i < nwords; i += 32) s.bits[i] = 0u;
        __syncwarp();
        int lx, ly, cnt;
        na_lane_start(s, (int)(d1 - d0), nrows, narcs, a0, &lx, &ly, &cnt);
        uint32_t active = 0;
        for (int i = 0, x = lx, y = ly; i < cnt; ++i) {
            if (y < s.rowend[x] - a0) {
                if (sampled_flag(s.src[pad(y)], r0 + x, symmetric, seed, thr)) {
                    const int k = a0 + y;
                    atomicOr(&s.bits[(k >> 5) - w0], 1u << (k & 31));
                    ++active;
                }
                ++y;
            } else {
                ++x;
            }
        }
        const uint32_t incl = warp_incl_sum_u32(active);
        if (lane == 31) tile_cnt[t] = incl;
        __syncwarp();
        for (int i = (int)lane; i < nwords; i += 32) {
            const int w = w0 + i;
            const int lo = a0 > w * 32 ? a0 : w * 32;
            const int hi = a1 < w * 32 + 32 ? a1 : w * 32 + 32;
            if (hi - lo == 32) {
                mask[w] = s.bits[i];
            } else {
                const uint32_t range = ((1u << (hi - lo)) - 1u) << (lo & 31);
                atomicAnd(&mask[w], ~range);
                atomicOr(&mask[w], s.bits[i]);
            }
        }
        __syncwarp();
    }
}

// Pass 2: pack the flagged arcs at their tile's offset, row pointers of the
// packed list.
__global__ void __launch_bounds__(kThreads)
k_na_pack(const int32_t *__restrict__ in_ptr, const int32_t *__restrict__ in_src, int32_t n,
          const uint32_t *__restrict__ scal, const int32_t *__restrict__ tile_info,
          const uint32_t *__restrict__ mask, const uint32_t *__restrict__ tile_off,
          int32_t *__restrict__ sp_ptr, int32_t *__restrict__ sp_src, uint32_t *__restrict__ sp_nnz)
{
    __shared__ NaSmem smem[kWarps];
    NaSmem &s = smem[threadIdx.x >> 5];
    const uint32_t lane = lane_id();
    const long long total = (long long)n + scal[0];
    const int num_tiles = scal[2] ? 0 : (int)scal[1];   // rejected row pointers: no work
    const int W = (int)((gridDim.x * kThreads) >> 5);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (scal[2]) {
            *sp_nnz = 0xFFFFFFFFu;
        } else {
            sp_ptr[0] = 0;
            *sp_nnz = tile_off[num_tiles];
        }
    }
    for (int t = (int)((blockIdx.x * kThreads + threadIdx.x) >> 5); t < num_tiles; t += W) {
        const int32_t r0 = tile_info[t] & 0x7FFFFFFF, r1 = tile_info[t + 1] & 0x7FFFFFFF;
        const long long d0 = (long long)t * kWT, d1 = d0 + kWT < total ? d0 + kWT : total;
        const int32_t a0 = (int32_t)(d0 - r0), a1 = (int32_t)(d1 - r1);
        const int nrows = r1 - r0, narcs = a1 - a0;
        for (int i = (int)lane; i < nrows; i += 32) s.rowend[i] = in_ptr[r0 + i + 1];
        if (lane == 0) s.rowend[nrows] = 0x7FFFFFFF;
        __syncwarp();
        int lx, ly, cnt;
        na_lane_start(s, (int)(d1 - d0), nrows, narcs, a0, &lx, &ly, &cnt);
        uint32_t active = 0;
        for (int i = 0, x = lx, y = ly; i < cnt; ++i) {
            if (y < s.rowend[x] - a0) {
                const int k = a0 + y;
                active += (mask[k >> 5] >> (k & 31)) & 1u;
                ++y;
            } else {
                ++x;
            }
        }
        const uint32_t incl = warp_incl_sum_u32(active);
        uint32_t off = tile_off[t] + incl - active;
        for (int i = 0, x = lx, y = ly; i < cnt; ++i) {
            if (y < s.rowend[x] - a0) {
                const int k = a0 + y;
                if ((mask[k >> 5] >> (k & 31)) & 1u) sp_src[off++] = in_src[k];
                ++y;
            } else {
                sp_ptr[r0 + x + 1] = (int32_t)off;
                ++x;
            }
        }
        __syncwarp();
    }
}

}  // namespace gg

using namespace gg;

extern "C" gg_status gg_sample_csc_noalloc(int32_t n, int64_t m, const int32_t *in_ptr, const int32_t *in_src,
                                           double sample_ratio, uint64_t seed, int symmetric, uint32_t *mask,
                                           int32_t *sp_ptr, int32_t *sp_src, uint32_t *sp_nnz, void *stream)
{
    if (n < 1 || m < 0) {
        set_error("gg_sample_csc_noalloc: need n >= 1 and m >= 0");
        return GG_ERR_INVALID_ARG;
    }
    if ((uint64_t)n + (uint64_t)m > kNoallocMaxItems) {
        set_error("gg_sample_csc_noalloc: n + m = %lld exceeds the fixed scratch limit %u "
                  "(GG_NOALLOC_MAX_ITEMS); use gg_sample_edges", (long long)n + (long long)m, kNoallocMaxItems);
        return GG_ERR_INVALID_ARG;
    }
    if (!in_ptr || !sp_ptr || !sp_nnz || (m > 0 && (!in_src || !mask || !sp_src))) {
        set_error("gg_sample_csc_noalloc: NULL array");
        return GG_ERR_INVALID_ARG;
    }
    if (!(sample_ratio > 0.0 && sample_ratio <= 1.0)) {
        set_error("gg_sample_csc_noalloc: sample_ratio must be in (0, 1], got %g", sample_ratio);
        return GG_ERR_INVALID_ARG;
    }
    gg_status st;
    uint32_t *scratch = noalloc_scratch(&st);
    if (!scratch) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *tile_info = (int32_t *)scratch;
    uint32_t *tile_cnt = scratch + (kNoallocTiles + 2);
    uint32_t *tile_off = scratch + 2 * ((size_t)kNoallocTiles + 2);
    uint32_t *partials = scratch + 3 * ((size_t)kNoallocTiles + 2);
    uint32_t *scal = partials + kNoallocPartials;   // [0] arcs, [1] tiles, [2] row pointers rejected
    const uint32_t nt = (uint32_t)(((uint64_t)n + (uint64_t)m + kWT - 1) / kWT);
    const unsigned long long thr = (unsigned long long)std::floor(sample_ratio * 4294967296.0);
    int dev = 0, sms = 0;
    GG_CUDA(cudaGetDevice(&dev));
    GG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int grid = (int)((nt + kWarps - 1) / kWarps);
    if (grid > sms * 4) grid = sms * 4;
    if (grid < 1) grid = 1;
    k_na_set<<<1, 1, 0, s>>>(scal, (uint32_t)m);
    GG_CUDA(cudaGetLastError());
    int cgrid = (int)(((long long)n + 255) / 256);
    if (cgrid > sms * 4) cgrid = sms * 4;
    k_na_check<<<cgrid, 256, 0, s>>>(in_ptr, n, (uint32_t)m, scal);
    GG_CUDA(cudaGetLastError());
    GG_CUDA(launch_partition(in_ptr, n, scal, nt, tile_info, scal + 1, s));
    k_na_flags<<<grid, kThreads, 0, s>>>(in_ptr, in_src, n, scal, tile_info, symmetric ? 1 : 0, seed, thr,
                                         mask, tile_cnt);
    GG_CUDA(cudaGetLastError());
    GG_CUDA(launch_scan_u32(tile_cnt, tile_off, nt, partials, s));
    k_na_pack<<<grid, kThreads, 0, s>>>(in_ptr, in_src, n, scal, tile_info, mask, tile_off, sp_ptr, sp_src,
                                        sp_nnz);
    GG_CUDA(cudaGetLastError());
    return GG_OK;
}

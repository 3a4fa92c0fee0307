// gg_build.cu - graph loading on the device: CSR validation, in-edge (CSC)
// construction by a stable LSD radix sort of the arcs by destination, the
// merge-path partition of a list into tiles, and a device-wide exclusive scan.
//
// Ordering contract (the in-edge order defines the running edge influence of
// Alg. 2): CSR arcs are taken in CSR order, which lists sources in ascending
// order; a stable sort by destination therefore leaves every in-row sorted by
// source, duplicates in CSR order.
#include <vector>

#include "gg_graph.cuh"

namespace gg {

// ------------------------------------------------------------- partition ----
// tile_info[t] = rows whose end item precedes diagonal t*kWT of the merged
// (row ends, arcs) sequence (Merrill-Garland merge-path search), with bit 31
// set when the row open at that diagonal already has arcs in earlier tiles.
__global__ void k_partition(const int32_t *__restrict__ row_ptr, int32_t n,
                            const uint32_t *__restrict__ list_nnz, uint32_t max_tiles,
                            int32_t *__restrict__ tile_info, uint32_t *__restrict__ num_tiles)
{
    const uint32_t nnz = *list_nnz;
    const long long total = (long long)n + nnz;
    const uint32_t nt = (uint32_t)((total + kWT - 1) / kWT);
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) *num_tiles = nt;
    if (t > nt || t > max_tiles) return;
    long long d = (long long)t * kWT;
    if (d > total) d = total;
    long long lo = d - (long long)nnz > 0 ? d - (long long)nnz : 0;
    long long hi = d < n ? d : n;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if ((long long)row_ptr[mid + 1] <= d - mid - 1) lo = mid + 1;
        else hi = mid;
    }
    const int32_t r = (int32_t)lo;
    const long long arcs_before = d - lo;
    const bool open = t < nt && r < n && arcs_before > row_ptr[r];
    tile_info[t] = (int32_t)((uint32_t)r | (open ? 0x80000000u : 0u));
}

cudaError_t launch_partition(const int32_t *row_ptr, int32_t n, const uint32_t *list_nnz,
                             uint32_t max_tiles, int32_t *tile_info, uint32_t *num_tiles,
                             cudaStream_t s)
{
    const uint32_t threads = 256;
    const uint32_t blocks = (max_tiles + 1 + threads - 1) / threads;
    k_partition<<<blocks, threads, 0, s>>>(row_ptr, n, list_nnz, max_tiles, tile_info, num_tiles);
    return cudaGetLastError();
}


// ------------------------------------------------------------------ scan ----
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t *s_warp, uint32_t *total)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t w = lane < (uint32_t)nw ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= (uint32_t)o) wi += y;
        }
        if (lane < (uint32_t)nw) s_warp[lane] = wi - w;
        if (lane == (uint32_t)nw - 1) s_warp[32] = wi;
    }
    __syncthreads();
    const uint32_t r = s_warp[warp] + x - v;
    if (total) *total = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const uint32_t *__restrict__ in, size_t n, uint32_t *__restrict__ partial)
{
    __shared__ uint32_t s_warp[33];
    const size_t base = (size_t)blockIdx.x * kScanTile;
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const size_t k = base + threadIdx.x + (size_t)i * kScanThreads;
        if (k < n) sum += in[k];
    }
    uint32_t tot;
    block_excl_scan_u32(sum, s_warp, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Single block: exclusive scan of the tile sums in place; total at [nb].
__global__ void k_scan_partials(uint32_t *partial, uint32_t nb, uint32_t *out, size_t n)
{
    __shared__ uint32_t s_warp[33];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nb; base += blockDim.x) {
        const uint32_t k = base + threadIdx.x;
        const uint32_t v = k < nb ? partial[k] : 0u;
        uint32_t tot;
        const uint32_t ex = block_excl_scan_u32(v, s_warp, &tot);
        if (k < nb) partial[k] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        partial[nb] = carry;
        if (out) out[n] = carry;
    }
}

__global__ void k_scan_down(const uint32_t *in, uint32_t *out, size_t n, const uint32_t *__restrict__ partial)
{
    __shared__ uint32_t s_data[kScanTile];
    __shared__ uint32_t s_warp[33];
    const size_t base = (size_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int j = threadIdx.x + i * kScanThreads;
        s_data[j] = base + j < n ? in[base + j] : 0u;
    }
    __syncthreads();
    uint32_t local[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        local[i] = s_data[threadIdx.x * kScanItems + i];
        sum += local[i];
    }
    uint32_t run = partial[blockIdx.x] + block_excl_scan_u32(sum, s_warp, nullptr);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        s_data[threadIdx.x * kScanItems + i] = run;
        run += local[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int j = threadIdx.x + i * kScanThreads;
        if (base + j < n) out[base + j] = s_data[j];
    }
}

size_t scan_tmp_words(size_t n) { return (n + kScanTile - 1) / kScanTile + 2; }

// out[0..n) = exclusive prefix of in[0..n); out[n] = total (out needs n+1
// words). in and out may alias.
cudaError_t launch_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *tmp, cudaStream_t s)
{
    const uint32_t nb = (uint32_t)((n + kScanTile - 1) / kScanTile);
    if (nb > 0) k_scan_reduce<<<nb, kScanThreads, 0, s>>>(in, n, tmp);
    k_scan_partials<<<1, 1024, 0, s>>>(tmp, nb, out, n);
    if (nb > 0) k_scan_down<<<nb, kScanThreads, 0, s>>>(in, out, n, tmp);
    return cudaGetLastError();
}

// ------------------------------------------------------------ validation ----
// colidx (library-owned, 16-byte aligned) is read with 16-byte loads, four in
// flight per thread.
__global__ void k_validate(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
                           int32_t n, long long m, uint32_t *err)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    for (long long i = tid; i <= n; i += stride) {
        const int32_t r = rowptr[i];
        bad |= (i == 0 && r != 0) || (i == n && (long long)r != m) || r < 0 || (long long)r > m;
        if (i < n && rowptr[i + 1] < r) bad = true;
    }
    auto out = [n](int32_t c) { return c < 0 || c >= n; };
    constexpr int U = 4;
    const long long m4 = m >> 2;
    const int4 *c4 = reinterpret_cast<const int4 *>(colidx);
    for (long long q0 = tid; q0 < m4; q0 += U * stride) {
        int4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long q = q0 + u * stride;
            v[u] = q < m4 ? __ldcs(c4 + q) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) bad |= out(v[u].x) || out(v[u].y) || out(v[u].z) || out(v[u].w);
    }
    for (long long i = 4 * m4 + tid; i < m; i += stride) bad |= out(colidx[i]);
    if (bad) atomicOr(err, DEVERR_BAD_GRAPH);
}

// Source vertex of every CSR arc. A warp takes 32 consecutive rows; when
// their arcs are few (the usual case) the warp walks those arcs with
// coalesced stores and finds each arc's row by a binary search over the 32
// row starts held in its lanes; a warp whose rows hold many arcs walks them
// row by row.
__global__ void k_expand_src(const int32_t *__restrict__ rowptr, int32_t n, int32_t *__restrict__ src_of)
{
    constexpr int32_t kShort = 2048;
    const int lane = threadIdx.x & 31;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long v0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; v0 < n; v0 += warps * 32) {
        const long long v = v0 + lane;
        const int32_t b = rowptr[v < n ? v : n];   // rows past n start at m
        const int32_t start = __shfl_sync(0xFFFFFFFFu, b, 0);
        const int32_t end = __shfl_sync(0xFFFFFFFFu, lane == 0 ? rowptr[v0 + 32 < n ? v0 + 32 : n] : 0, 0);
        if (end - start <= kShort) {
            for (int32_t base = start; base < end; base += 32) {
                const int32_t k = base + lane;
                int lo = 0;   // the last lane whose row starts at or before k
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int32_t bb = __shfl_sync(0xFFFFFFFFu, b, lo + step);
                    if (bb <= k) lo += step;
                }
                if (k < end) src_of[k] = (int32_t)(v0 + lo);
            }
        } else {
            for (int l = 0; l < 32; ++l) {
                const int32_t rb = __shfl_sync(0xFFFFFFFFu, b, l);
                const int32_t re = l < 31 ? __shfl_sync(0xFFFFFFFFu, b, l + 1) : end;
                for (int32_t k = rb + lane; k < re; k += 32) src_of[k] = (int32_t)(v0 + l);
            }
        }
    }
}

// ------------------------------------------------------------ radix sort ----
// Stable LSD radix sort of the CSR arcs by destination, 8 bits per pass. The
// arcs' payload travels with them: the CSR position e (for the CSR -> CSC
// map), the source and the weight; the first pass reads them from the CSR
// (e = position), the last pass writes the in-edge arrays themselves and the
// hub-coded copy of the sources.
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kRadixThreads * kRadixItems;
constexpr int kRadixWarps = kRadixThreads / 32;

struct RadixIO {
    const uint32_t *keys_in;
    uint32_t *keys_out;
    const uint32_t *e_in;   // nullptr: the input position (first pass)
    uint32_t *e_out;
    const int32_t *src_in;
    int32_t *src_out;
    int32_t *src_h_out;     // last pass: sources with hubs coded -(slot + 1)
    const int32_t *hub_slot;
    const uint32_t *w_in;   // nullptr: no weights
    uint32_t *w_out;
};

__global__ void k_radix_upsweep(const uint32_t *__restrict__ keys, long long m, int shift,
                                uint32_t num_tiles, uint32_t *__restrict__ counts)
{
    __shared__ uint32_t hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRadixTile;
#pragma unroll
    for (int i = 0; i < kRadixItems; ++i) {
        const long long k = base + threadIdx.x + (long long)i * kRadixThreads;
        if (k < m) atomicAdd(&hist[(keys[k] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * num_tiles + blockIdx.x] = hist[threadIdx.x];
}

// Stable scatter of one 8-bit digit. Warp w ranks positions
// [w*512, w*512+512) of the tile in rounds of 32, so the order of equal
// digits inside the tile is (warp, round, lane) = input order. The keys go
// through shared memory in tile order first, which fixes every item's global
// position; each payload array then follows through the same staging buffer.
__global__ void __launch_bounds__(kRadixThreads, 3)
k_radix_downsweep(RadixIO io, long long m, int shift, uint32_t num_tiles, const uint32_t *__restrict__ offsets)
{
    __shared__ uint32_t s_stage[kRadixTile];
    __shared__ uint32_t s_gpos[kRadixTile];
    __shared__ uint32_t s_whist[kRadixWarps][256];
    __shared__ uint32_t s_tile_excl[256];
    __shared__ uint32_t s_glob[256];
    __shared__ uint32_t s_warp[33];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long base = (long long)blockIdx.x * kRadixTile;
    const int count = (int)((m - base) < kRadixTile ? (m - base) : kRadixTile);
    for (int i = tid; i < kRadixWarps * 256; i += kRadixThreads) (&s_whist[0][0])[i] = 0;
    __syncthreads();

    uint32_t key[kRadixItems], lp[kRadixItems];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const int p = warp * (kRadixItems * 32) + r * 32 + lane;
        key[r] = p < count ? io.keys_in[base + p] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const int p = warp * (kRadixItems * 32) + r * 32 + lane;
        const bool valid = p < count;
        const uint32_t digit = valid ? ((key[r] >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, digit);
        uint32_t before = 0;
        if (valid) before = s_whist[warp][digit];
        __syncwarp();
        if (valid && (peers & lt) == 0) s_whist[warp][digit] = before + __popc(peers);
        __syncwarp();
        lp[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    {
        const int d = tid;   // 256 threads = 256 digits
        uint32_t run = 0;
        for (int w = 0; w < kRadixWarps; ++w) {
            const uint32_t c = s_whist[w][d];
            s_whist[w][d] = run;
            run += c;
        }
        s_glob[d] = offsets[(size_t)d * num_tiles + blockIdx.x];
        s_tile_excl[d] = block_excl_scan_u32(run, s_warp, nullptr);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const int p = warp * (kRadixItems * 32) + r * 32 + lane;
        if (p < count) {
            const uint32_t digit = (key[r] >> shift) & 255u;
            lp[r] += s_tile_excl[digit] + s_whist[warp][digit];
            s_stage[lp[r]] = key[r];
        }
    }
    __syncthreads();
    for (int i = tid; i < count; i += kRadixThreads) {
        const uint32_t k = s_stage[i];
        const uint32_t digit = (k >> shift) & 255u;
        const uint32_t g = s_glob[digit] + (uint32_t)i - s_tile_excl[digit];
        io.keys_out[g] = k;
        s_gpos[i] = g;
    }
    // one payload array: loaded in the keys' order, staged, stored in place
    auto move = [&](auto load, auto store) {
        uint32_t v[kRadixItems];
#pragma unroll
        for (int r = 0; r < kRadixItems; ++r) {
            const int p = warp * (kRadixItems * 32) + r * 32 + lane;
            v[r] = p < count ? load(base + p) : 0u;
        }
        __syncthreads();   // the previous array's stores have read s_stage
#pragma unroll
        for (int r = 0; r < kRadixItems; ++r) {
            const int p = warp * (kRadixItems * 32) + r * 32 + lane;
            if (p < count) s_stage[lp[r]] = v[r];
        }
        __syncthreads();
        for (int i = tid; i < count; i += kRadixThreads) store(s_gpos[i], s_stage[i]);
    };
    move([&](long long q) { return io.e_in ? __ldcs(io.e_in + q) : (uint32_t)q; },
         [&](uint32_t g, uint32_t x) { io.e_out[g] = x; });
    move([&](long long q) { return (uint32_t)__ldcs(io.src_in + q); },
         [&](uint32_t g, uint32_t x) {
             io.src_out[g] = (int32_t)x;
             if (io.src_h_out) {
                 const int32_t slot = __ldg(io.hub_slot + x);
                 io.src_h_out[g] = slot >= 0 ? -(slot + 1) : (int32_t)x;
             }
         });
    if (io.w_in)
        move([&](long long q) { return __ldcs(io.w_in + q); }, [&](uint32_t g, uint32_t x) { io.w_out[g] = x; });
}

// in_ptr from destination-sorted keys: every boundary writes the row starts
// of the rows it opens (empty rows included).
// Four keys per thread (one 16-byte load; keys are library-owned and 16-byte
// aligned).
__global__ void k_csc_rowptr(const uint32_t *__restrict__ keys, long long m, int32_t n, int32_t *__restrict__ in_ptr)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long q_end = (m + 3) >> 2;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < q_end; q += stride) {
        const long long k0 = 4 * q;
        uint32_t c[4];
        if (k0 + 4 <= m) {
            const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(keys) + q);
            c[0] = v.x, c[1] = v.y, c[2] = v.z, c[3] = v.w;
        } else {
            for (int i = 0; i < 4; ++i) c[i] = k0 + i < m ? keys[k0 + i] : 0u;
        }
        int32_t prev = k0 == 0 ? -1 : (int32_t)keys[k0 - 1];
        for (int i = 0; i < 4 && k0 + i < m; ++i) {
            const int32_t u = (int32_t)c[i];
            for (int32_t v = prev + 1; v <= u; ++v) in_ptr[v] = (int32_t)(k0 + i);
            if (k0 + i == m - 1)
                for (int32_t v = u + 1; v <= n; ++v) in_ptr[v] = (int32_t)m;
            prev = u;
        }
    }
}

// CSR -> CSC map: out_to_in[e] = k for the sorted position k of CSR arc e. The
// stores are random, so they are made in windows of e small enough to stay in
// L2 until every word of a sector is written; each launch reads the sorted
// positions once.
constexpr long long kMapWindow = 16ll << 20;   // 64 MB of out_to_in per launch

__global__ void k_out_to_in(const uint32_t *__restrict__ e_sorted, long long m, long long lo, long long hi,
                            int32_t *__restrict__ out_to_in)
{
    constexpr int U = 4;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; k0 < m; k0 += U * stride) {
        uint32_t e[U];
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const long long k = k0 + i * stride;
            e[i] = k < m ? __ldcs(e_sorted + k) : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const long long k = k0 + i * stride;
            if (k < m && (long long)e[i] >= lo && (long long)e[i] < hi) out_to_in[e[i]] = (int32_t)k;
        }
    }
}

// -------------------------------------------------------------- host side ----
gg_status build_csc(gg_graph *g)
{
    cudaStream_t s = g->stream;
    const long long m = g->m;
    const int32_t n = g->n;
    const int grid = g->num_sms * 8;
    if (m == 0) {
        GG_CUDA(cudaMemsetAsync(g->in_ptr, 0, sizeof(int32_t) * ((size_t)n + 1), s));
        return GG_OK;
    }
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < (int64_t)n) ++bits;
    const int passes = (bits + 7) / 8;
    const uint32_t num_tiles = (uint32_t)((m + kRadixTile - 1) / kRadixTile);
    const size_t ncounts = (size_t)256 * num_tiles;

    // working arrays: keys, sources and weights alternate between a
    // temporary and the final in-edge array (the last pass lands in the
    // final one); the CSR positions alternate between two temporaries
    DevBuf tmp;
    const size_t words = 5 * (size_t)m + ncounts + 1 + scan_tmp_words(ncounts) + (size_t)m;
    gg_status st = tmp.alloc(words * sizeof(uint32_t), s);
    if (st != GG_OK) return st;
    uint32_t *t_keys = tmp.u32(), *t_src = t_keys + m, *t_w = t_src + m;
    uint32_t *t_e[2] = {t_w + m, t_w + 2 * m};
    uint32_t *counts = t_w + 3 * m;
    uint32_t *scan_tmp = counts + ncounts + 1;
    int32_t *src_of = (int32_t *)(scan_tmp + scan_tmp_words(ncounts));

    k_expand_src<<<grid, 256, 0, s>>>(g->out_ptr, n, src_of);
    RadixIO io{};
    io.keys_in = (const uint32_t *)g->out_dst;
    io.e_in = nullptr;
    io.src_in = src_of;
    io.w_in = g->out_w;
    io.hub_slot = g->hub_slot;
    for (int p = 0; p < passes; ++p) {
        const bool to_final = ((passes - 1 - p) & 1) == 0;
        const bool last = p == passes - 1;
        io.keys_out = to_final ? (uint32_t *)g->in_dst : t_keys;
        io.e_out = t_e[p & 1];
        io.src_out = to_final ? g->in_src : (int32_t *)t_src;
        io.src_h_out = last ? g->in_src_h : nullptr;
        io.w_out = g->out_w ? (to_final ? g->in_w : t_w) : nullptr;
        k_radix_upsweep<<<num_tiles, kRadixThreads, 0, s>>>(io.keys_in, m, 8 * p, num_tiles, counts);
        GG_CUDA(launch_scan_u32(counts, counts, ncounts, scan_tmp, s));
        k_radix_downsweep<<<num_tiles, kRadixThreads, 0, s>>>(io, m, 8 * p, num_tiles, counts);
        io.keys_in = io.keys_out;
        io.e_in = io.e_out;
        io.src_in = io.src_out;
        io.w_in = io.w_out;
    }
    k_csc_rowptr<<<grid, 256, 0, s>>>((const uint32_t *)g->in_dst, m, n, g->in_ptr);
    for (long long lo = 0; lo < m; lo += kMapWindow)
        k_out_to_in<<<grid, 256, 0, s>>>(io.e_in, m, lo, lo + kMapWindow, g->out_to_in);
    g->load_launches += 2 + 5 * passes + (uint32_t)((m + kMapWindow - 1) / kMapWindow);
    GG_CUDA(cudaGetLastError());
    // the temporaries are released only after the queued work has used them
    GG_CUDA(cudaStreamSynchronize(s));
    return GG_OK;
}

// ------------------------------------------------------------ hub cache ----
// The sources read most often by pull gathers are the vertices with the most
// out-arcs. They get slots (build_hubs), and the last pass of the in-edge sort
// codes their in-arcs as -(slot + 1) in in_src_h, so the slots are chosen
// before the sort.
constexpr uint32_t kDegBins = 65536;

// Out-degree histogram (degrees clamped to kDegBins - 1); the many small
// degrees are counted in shared memory first, so their global counters see
// one atomic per block.
constexpr int kDegLow = 4096;

__global__ void k_deg_hist(const int32_t *__restrict__ out_ptr, int32_t n, uint32_t *__restrict__ hist)
{
    __shared__ uint32_t low[kDegLow];
    for (int i = threadIdx.x; i < kDegLow; i += blockDim.x) low[i] = 0u;
    __syncthreads();
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int32_t d = out_ptr[v + 1] - out_ptr[v];
        if (d < kDegLow) atomicAdd(&low[d], 1u);
        else atomicAdd(&hist[d < (int32_t)kDegBins - 1 ? d : (int32_t)kDegBins - 1], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kDegLow; i += blockDim.x)
        if (low[i]) atomicAdd(&hist[i], low[i]);
}

// Tier of each vertex: 1 (out-degree >= thr1), 2 (thr2 <= out-degree < thr1)
// or none.
__global__ void k_hub_flag(const int32_t *__restrict__ out_ptr, int32_t n, int32_t thr1, int32_t thr2,
                           uint32_t *__restrict__ flag1, uint32_t *__restrict__ flag2)
{
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int32_t d = out_ptr[v + 1] - out_ptr[v];
        flag1[v] = d >= thr1 ? 1u : 0u;
        flag2[v] = (d >= thr2 && d < thr1) ? 1u : 0u;
    }
}

// Slots: tier 1 in vertex order, then tier 2 in vertex order.
__global__ void k_hub_fill(int32_t n, const uint32_t *__restrict__ flag1, const uint32_t *__restrict__ pos1,
                           const uint32_t *__restrict__ flag2, const uint32_t *__restrict__ pos2, uint32_t n1,
                           int32_t *__restrict__ hub_slot, int32_t *__restrict__ hub_ids)
{
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int32_t slot = -1;
        if (flag1[v]) slot = (int32_t)pos1[v];
        else if (flag2[v]) slot = (int32_t)(n1 + pos2[v]);
        hub_slot[v] = slot;
        if (slot >= 0) hub_ids[slot] = v;
    }
}

// The hubs: with out-degree >= T1 (the smallest threshold, at least 2, that
// admits no more than kHubs vertices) the first tier; with T2 <= out-degree
// < T1 (T2 the same for kHubCodes) the second.
gg_status build_hubs(gg_graph *g)
{
    cudaStream_t s = g->stream;
    const int32_t n = g->n;
    const int grid = g->num_sms * 8;
    DevBuf tmp;
    gg_status st = tmp.alloc(4 * ((size_t)kDegBins + 4 * ((size_t)n + 1)), s);
    if (st != GG_OK) return st;
    uint32_t *hist = tmp.u32(), *flag1 = hist + kDegBins, *pos1 = flag1 + n + 1, *flag2 = pos1 + n + 1,
             *pos2 = flag2 + n + 1;
    GG_CUDA(cudaMemsetAsync(hist, 0, 4 * (size_t)kDegBins, s));
    k_deg_hist<<<grid, 256, 0, s>>>(g->out_ptr, n, hist);
    std::vector<uint32_t> h(kDegBins);
    GG_CUDA(cudaMemcpyAsync(h.data(), hist, 4 * (size_t)kDegBins, cudaMemcpyDeviceToHost, s));
    GG_CUDA(cudaStreamSynchronize(s));
    uint64_t above = 0, n1 = 0;
    int32_t thr1 = 0x7FFFFFFF, thr2 = 0x7FFFFFFF;   // no hub
    bool tier1 = true;
    for (int32_t d = (int32_t)kDegBins - 1; d >= 2; --d) {
        if (tier1 && above + h[d] > (uint64_t)kHubs) tier1 = false;
        if (above + h[d] > (uint64_t)kHubCodes) break;
        above += h[d];
        thr2 = d;
        if (tier1) { thr1 = d; n1 = above; }
    }
    k_hub_flag<<<grid, 256, 0, s>>>(g->out_ptr, n, thr1, thr2, flag1, flag2);
    GG_CUDA(launch_scan_u32(flag1, pos1, (size_t)n, g->scan_tmp, s));
    GG_CUDA(launch_scan_u32(flag2, pos2, (size_t)n, g->scan_tmp, s));
    k_hub_fill<<<grid, 256, 0, s>>>(n, flag1, pos1, flag2, pos2, (uint32_t)n1, g->hub_slot, g->hub_ids);
    g->n_hubs = (int32_t)above;
    g->load_launches += 10;
    GG_CUDA(cudaGetLastError());
    GG_CUDA(cudaStreamSynchronize(s));
    return GG_OK;
}

__global__ void k_decode_src(const int32_t *__restrict__ coded, const uint32_t *__restrict__ count,
                             const int32_t *__restrict__ hub_ids, int32_t *__restrict__ out)
{
    const uint32_t c = *count;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < c; k += gridDim.x * blockDim.x) {
        const int32_t v = coded[k];
        out[k] = v < 0 ? hub_ids[-v - 1] : v;
    }
}

cudaError_t launch_decode_src(const int32_t *coded, const uint32_t *count, uint32_t max_count, const int32_t *hub_ids,
                              int32_t *out, int num_sms, cudaStream_t s)
{
    long long blocks = ((long long)max_count + 255) / 256;
    if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
    if (blocks < 1) blocks = 1;
    k_decode_src<<<(unsigned)blocks, 256, 0, s>>>(coded, count, hub_ids, out);
    return cudaGetLastError();
}

gg_status validate_csr(gg_graph *g)
{
    cudaStream_t s = g->stream;
    GG_CUDA(cudaMemsetAsync(g->dev_err, 0, sizeof(uint32_t), s));
    k_validate<<<g->num_sms * 8, 256, 0, s>>>(g->out_ptr, g->out_dst, g->n, g->m, g->dev_err);
    g->load_launches += 1;
    GG_CUDA(cudaGetLastError());
    uint32_t err = 0;
    GG_CUDA(cudaMemcpyAsync(&err, g->dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GG_CUDA(cudaStreamSynchronize(s));
    if (err & DEVERR_BAD_GRAPH) {
        set_error("gg_load_csr: invalid CSR (rowptr not monotone / not 0..m, or colidx outside [0,n))");
        return GG_ERR_BAD_GRAPH;
    }
    return GG_OK;
}

}  // namespace gg

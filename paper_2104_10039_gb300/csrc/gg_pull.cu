// gg_pull.cu - the pull iterations of every application: approximate and
// accurate gathers (Alg. 1 / Alg. 2: GG-Gather over a row's flagged in-edges,
// GG-Apply, GG-VStatus) and corrections (influence, GG-EStatus) over a
// precomputed plan of the list they walk.
//
// A gather reads one 4-byte value per arc at a random address, and on this
// GPU those reads are bounded by how many scattered L1 misses each SM keeps
// in flight (the L1 capacity left beside shared memory), not by DRAM. These
// kernels therefore keep the arc work free of shared memory: every lane holds
// its arcs' values in registers, row boundaries come from a bit per arc
// computed once per list, and the vertex work (apply, change statistics,
// frontier) is a separate coalesced pass.
//
//   k_pull_arcs  warp tiles of kPT = 256 consecutive arcs; lane L takes arcs
//                4L..4L+3 and 128+4L..128+4L+3 (two 16-byte source loads, and
//                weights for SSSP), fetches their values, and a segmented
//                fold over the tile (lane-local, then a warp scan) gives every
//                row's total: a sum of contributions for PageRank, a minimum of
//                candidates for SSSP / BFS / CC. A row whose first arc lies in
//                the tile writes its total (or, if it continues past the tile,
//                the part in the tile) to acc[v]; the part of the tile before
//                its first row start goes to lead[tile]. PageRank's sources
//                are hub-coded: a hub's contribution comes from the dense copy
//                k_hub_values writes before the launch. With a frontier
//                bitmap (k_front_bits, GG_PULL_FILTER) the min applications
//                read only the frontier sources' values.
//   k_long_rows  one block per long row: its total and, for a correction,
//                every tile's carry (the row's value before the tile).
//   k_carries    a correction's carries of the tiles inside shorter rows.
//   k_prc_flags, k_minc_flags
//                a correction's second pass (lane L: arcs 8L..8L+7): every
//                arc's influence from the running value of its row before and
//                after it (the values kept by the first pass, the carry of a
//                continued row from acc and the leads), one flag bit per arc,
//                and each tile's count of active arcs for the pack.
//   k_pr_apply, k_min_apply
//                one thread per four consecutive vertices: the row's total (acc[v] folded with the
//                later tiles' leading parts of a row continued across tile
//                ends, in tile order; the identity for a row with no arcs in
//                the list), then GG-Apply and GG-VStatus (PageRank: rank',
//                contrib', change statistics; SSSP / BFS / CC: the minimum with
//                the old value, the changed vertices appended to the frontier).
//
// The sums use a fixed grouping (lane-local prefix, warp scan, tile order),
// so PageRank results are deterministic (the minimum is exact anyway).
//
// The plan of a list (built by build_pull_plan whenever the list changes):
//   hb[w]     bit j: arc 32w + j is the first arc of a row
//   trow[t]   rank among non-empty rows of the row holding arc 256t
//   nzv[k]    vertex of the k-th non-empty row
//   topen[t]  the row holding arc 256t: vertex, tile of its first arc, long flag
//   lrows     the long rows (more than kLongTiles tiles past their first one)
//   nzb, nzc  non-empty-row bitmap and counts (to rank the rows)
#include "gg_graph.cuh"

namespace gg {

namespace {

constexpr int kPT = 256;          // arcs per pull tile
constexpr int kPullThreads = 256;
constexpr int32_t kNoArc = (int32_t)0x80000000;   // a lane's position past the list's end
// A row whose arcs reach more than kLongTiles tiles past the tile of its
// first arc is "long": one block completes its sum and its tiles' carries
// (k_long_rows); shorter rows fold at most kLongTiles leading parts inline.
constexpr int kLongTiles = 8;

// ------------------------------------------------------------------ plan ----
__global__ void k_plan_nz(const int32_t *__restrict__ ptr, int32_t n, uint32_t *__restrict__ nzb,
                          uint32_t *__restrict__ nzcnt)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); v0 < n; v0 += stride) {
        const long long v = v0 + (threadIdx.x & 31u);
        const bool ne = v < n && ptr[v + 1] > ptr[v];
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, ne);
        if ((threadIdx.x & 31u) == 0) {
            nzb[v0 >> 5] = b;
            nzcnt[v0 >> 5] = (uint32_t)__popc(b);
        }
    }
}

__global__ void k_plan_heads(const int32_t *__restrict__ ptr, int32_t n, const uint32_t *__restrict__ nzb,
                             const uint32_t *__restrict__ nzc, uint32_t *__restrict__ hb,
                             int32_t *__restrict__ trow, int32_t *__restrict__ nzv, int2 *__restrict__ topen,
                             int32_t *__restrict__ lrows, uint32_t *__restrict__ nlong)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t s = ptr[v], e = ptr[v + 1];
        if (e <= s) continue;
        const uint32_t w = (uint32_t)(v >> 5), bit = (uint32_t)(v & 31);
        const int32_t k = (int32_t)(nzc[w] + (uint32_t)__popc(nzb[w] & ((1u << bit) - 1u)));
        atomicOr(hb + (s >> 5), 1u << (s & 31));
        nzv[k] = (int32_t)v;
        const int32_t t0 = s / kPT, t1 = (e - 1) / kPT;
        const bool is_long = t1 - t0 > kLongTiles;
        if (is_long) lrows[atomicAdd(nlong, 1u)] = (int32_t)v;
        for (long long t = ((long long)s + kPT - 1) / kPT; t * kPT < e; ++t) {
            trow[t] = k;
            topen[t] = make_int2((int32_t)v, t0 | (is_long ? (int32_t)0x80000000 : 0));
        }
    }
}

}  // namespace

namespace {

__device__ __forceinline__ uint32_t pick4(const uint4 &w, uint32_t i)
{
    return i == 0 ? w.x : (i == 1 ? w.y : (i == 2 ? w.z : w.w));
}

// Row-start bits of word i of a tile holding `rel` valid arcs: positions at
// or past `rel` count as row starts (each a one-arc segment that is skipped),
// so the last real row ends at the last valid arc.
__device__ __forceinline__ uint32_t tail_bits(uint32_t word, int i, uint32_t rel)
{
    const uint32_t lo = 32u * (uint32_t)i;
    if (rel <= lo) return 0xFFFFFFFFu;
    if (rel >= lo + 32u) return word;
    return word | ~((1u << (rel - lo)) - 1u);
}

// What a pull gather folds per application: PageRank sums contributions
// (FP32, identity 0); SSSP / BFS / CC take the minimum of candidates (exact,
// identity INF): SSSP value + weight and BFS value + 1, saturating at INF (a
// candidate that would reach INF is no candidate), CC the label itself.
template <int APP>
struct PullOp {
    using T = uint32_t;
    static __device__ __forceinline__ T id() { return kInf; }
    static __device__ __forceinline__ T op(T x, T y) { return x < y ? x : y; }
    static __device__ __forceinline__ T cand(const PullArgs &a, int32_t src, uint32_t w)
    {
        const uint32_t u = __ldg(a.val_cur + src);
        if (APP == GG_APP_CC) return u;
        const unsigned long long c = (unsigned long long)u + (APP == GG_APP_BFS ? 1u : w);
        return (u == kInf || c >= kInf) ? kInf : (uint32_t)c;
    }
};
template <>
struct PullOp<GG_APP_PAGERANK> {
    using T = float;
    static __device__ __forceinline__ T id() { return 0.0f; }
    static __device__ __forceinline__ T op(T x, T y) { return x + y; }
    static __device__ __forceinline__ T cand(const PullArgs &a, int32_t src, uint32_t)
    {
        // one load: a hub's contribution from the dense hub copy, any other from the vector
        return __ldg(src < 0 ? reinterpret_cast<const float *>(a.hubv) + (-src - 1) : a.contrib + src);
    }
};

// ---------------------------------------------------------------- gather ----
// PF: the next tile's sources (and weights) are loaded while this tile's
// values are in flight (full tiles only). a.vals != nullptr (a correction's
// first pass): every arc's value is also stored, in list order.
template <int APP, int MINB, bool PF, bool FILT = false>
__global__ void __launch_bounds__(kPullThreads, MINB) k_pull_arcs(PullArgs a)
{
    using Op = PullOp<APP>;
    using T = typename Op::T;
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    constexpr bool kW = APP == GG_APP_SSSP;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nnz = *a.nnz;
    const long long nt = ((long long)nnz + kPT - 1) / kPT;
    const long long W = (long long)gridDim.x * (kPullThreads / 32);
    const bool has_w = kW && a.w != nullptr;
    int32_t pf[8];
    uint32_t pw[kW ? 8 : 1];
    bool have_pf = false;
    for (long long t = (long long)blockIdx.x * (kPullThreads / 32) + (threadIdx.x >> 5); t < nt; t += W) {
        const long long a0 = t * kPT;
        const uint32_t rel = nnz - (uint32_t)a0 < (uint32_t)kPT ? nnz - (uint32_t)a0 : (uint32_t)kPT;
        // ---- sources (16-byte loads), weights, and the arcs' values ----------
        int32_t s[8];
        uint32_t w[kW ? 8 : 1];
        if (PF && have_pf) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                s[i] = pf[i];
                if constexpr (kW) w[i] = pw[i];
            }
        } else if (rel == (uint32_t)kPT) {
            const int4 x = __ldg(reinterpret_cast<const int4 *>(a.src + a0) + lane);
            const int4 y = __ldg(reinterpret_cast<const int4 *>(a.src + a0 + 128) + lane);
            s[0] = x.x; s[1] = x.y; s[2] = x.z; s[3] = x.w;
            s[4] = y.x; s[5] = y.y; s[6] = y.z; s[7] = y.w;
            if constexpr (kW) {
                if (has_w) {
                    const uint4 p = __ldg(reinterpret_cast<const uint4 *>(a.w + a0) + lane);
                    const uint4 q = __ldg(reinterpret_cast<const uint4 *>(a.w + a0 + 128) + lane);
                    w[0] = p.x; w[1] = p.y; w[2] = p.z; w[3] = p.w;
                    w[4] = q.x; w[5] = q.y; w[6] = q.z; w[7] = q.w;
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) w[i] = 1u;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t q = 4u * lane + (uint32_t)j;
                s[j] = q < rel ? a.src[a0 + q] : kNoArc;
                s[4 + j] = q + 128u < rel ? a.src[a0 + 128 + q] : kNoArc;
                if constexpr (kW) {
                    w[j] = (has_w && q < rel) ? a.w[a0 + q] : 1u;
                    w[4 + j] = (has_w && q + 128u < rel) ? a.w[a0 + 128 + q] : 1u;
                }
            }
        }
        T v[8];
        if constexpr (FILT) {
            // only a frontier source can lower a row: every other source's
            // value was taken in when it last changed
            uint32_t fw[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                fw[i] = s[i] != kNoArc ? (__ldg(a.front + (s[i] >> 5)) >> (s[i] & 31)) & 1u : 0u;
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = fw[i] ? Op::cand(a, s[i], kW ? w[kW ? i : 0] : 1u) : Op::id();
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = s[i] != kNoArc ? Op::cand(a, s[i], kW ? w[kW ? i : 0] : 1u) : Op::id();
        }
        if (a.vals) {
            uint32_t *vb = reinterpret_cast<uint32_t *>(a.vals);
            uint32_t b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if constexpr (APP == GG_APP_PAGERANK) b[i] = __float_as_uint(v[i]);
                else b[i] = v[i];
            }
            if (rel == (uint32_t)kPT) {
                reinterpret_cast<uint4 *>(vb + a0)[lane] = make_uint4(b[0], b[1], b[2], b[3]);
                reinterpret_cast<uint4 *>(vb + a0 + 128)[lane] = make_uint4(b[4], b[5], b[6], b[7]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t q = 4u * lane + (uint32_t)j;
                    if (q < rel) vb[a0 + q] = b[j];
                    if (q + 128u < rel) vb[a0 + 128 + q] = b[4 + j];
                }
            }
        }
        if (PF) {
            const long long tn = t + W;
            have_pf = tn < nt && (tn + 1) * kPT <= (long long)nnz;
            if (have_pf) {
                const int4 x = __ldg(reinterpret_cast<const int4 *>(a.src + tn * kPT) + lane);
                const int4 y = __ldg(reinterpret_cast<const int4 *>(a.src + tn * kPT + 128) + lane);
                pf[0] = x.x; pf[1] = x.y; pf[2] = x.z; pf[3] = x.w;
                pf[4] = y.x; pf[5] = y.y; pf[6] = y.z; pf[7] = y.w;
                if constexpr (kW) {
                    if (has_w) {
                        const uint4 p = __ldg(reinterpret_cast<const uint4 *>(a.w + tn * kPT) + lane);
                        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(a.w + tn * kPT + 128) + lane);
                        pw[0] = p.x; pw[1] = p.y; pw[2] = p.z; pw[3] = p.w;
                        pw[4] = q.x; pw[5] = q.y; pw[6] = q.z; pw[7] = q.w;
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i) pw[i] = 1u;
                    }
                }
            }
        }
        // ---- row starts of the tile ------------------------------------------
        uint4 h0 = __ldg(reinterpret_cast<const uint4 *>(a.hb + t * 8));
        uint4 h1 = __ldg(reinterpret_cast<const uint4 *>(a.hb + t * 8 + 4));
        const uint32_t next_head = a0 + kPT >= (long long)nnz ? 1u : (__ldg(a.hb + (t + 1) * 8) & 1u);
        if (rel < (uint32_t)kPT) {
            h0.x = tail_bits(h0.x, 0, rel); h0.y = tail_bits(h0.y, 1, rel);
            h0.z = tail_bits(h0.z, 2, rel); h0.w = tail_bits(h0.w, 3, rel);
            h1.x = tail_bits(h1.x, 4, rel); h1.y = tail_bits(h1.y, 5, rel);
            h1.z = tail_bits(h1.z, 6, rel); h1.w = tail_bits(h1.w, 7, rel);
        }
        // first row start in the tile (kPT: none)
        uint32_t fh = kPT;
        {
            const uint32_t wv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
#pragma unroll
            for (int i = 7; i >= 0; --i)
                if (wv[i]) fh = 32u * (uint32_t)i + (uint32_t)(__ffs(wv[i]) - 1);
        }
        const int32_t tr = __ldg(a.trow + t);
        const uint32_t h0bit = h0.x & 1u;
        T carry = Op::id();      // running value of the segment open at the end of the previous half
        uint32_t before = 0;     // row starts in earlier halves
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint4 hw = h ? h1 : h0;
            const uint32_t wi = lane >> 3, sh = 4u * (lane & 7u);
            const uint32_t word = pick4(hw, wi);
            const uint32_t f = (word >> sh) & 0xFu;     // bit j: arc j of this lane starts a row
            uint32_t cnt = before + (uint32_t)__popc(word & ((1u << sh) - 1u));
            cnt += wi > 0 ? (uint32_t)__popc(hw.x) : 0u;
            cnt += wi > 1 ? (uint32_t)__popc(hw.y) : 0u;
            cnt += wi > 2 ? (uint32_t)__popc(hw.z) : 0u;
            // does a row start right after this lane's last arc?
            uint32_t nxt = __shfl_down_sync(FULL, f, 1) & 1u;
            if (lane == 31) nxt = h == 0 ? (h1.x & 1u) : next_head;
            // lane-local running values, restarting at row starts
            const T v0 = v[4 * h], v1 = v[4 * h + 1], v2 = v[4 * h + 2], v3 = v[4 * h + 3];
            const T r0 = v0;
            const T r1 = (f & 2u) ? v1 : Op::op(r0, v1);
            const T r2 = (f & 4u) ? v2 : Op::op(r1, v2);
            const T r3 = (f & 8u) ? v3 : Op::op(r2, v3);
            // warp segmented inclusive scan of the lanes' open tails
            const uint32_t heads = __ballot_sync(FULL, f != 0u);
            const uint32_t le = heads & (FULL >> (31u - lane));
            const int start = le ? 31 - __clz(le) : -1;   // lane where the segment open at this lane's end starts
            T x = r3;
            if (lane == 0 && f == 0u) x = Op::op(carry, r3);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const T y = __shfl_up_sync(FULL, x, o);
                if ((int)lane >= o && (int)lane - o >= start) x = Op::op(y, x);
            }
            T E = __shfl_up_sync(FULL, x, 1);
            if (lane == 0) E = carry;
            const uint32_t fj = f ? (uint32_t)(__ffs(f) - 1) : 4u;   // first row start in the lane
            T run[4];
            run[0] = fj > 0 ? Op::op(E, r0) : r0;
            run[1] = fj > 1 ? Op::op(E, r1) : r1;
            run[2] = fj > 2 ? Op::op(E, r2) : r2;
            run[3] = fj > 3 ? Op::op(E, r3) : r3;
            // segment ends: a row starts at the next arc, or the tile ends
            const uint32_t ends = (f >> 1) | (nxt << 3) | ((h == 1 && lane == 31) ? 8u : 0u);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t q = 128u * (uint32_t)h + 4u * lane + (uint32_t)j;
                if (((ends >> j) & 1u) && q < rel) {
                    T *lead = reinterpret_cast<T *>(a.lead);
                    T *acc = reinterpret_cast<T *>(a.acc);
                    if (q < fh) {
                        lead[t] = run[j];    // the row continued from an earlier tile
                    } else {
                        const uint32_t c = cnt + (uint32_t)__popc(f & ((2u << j) - 1u)) - h0bit;
                        acc[__ldg(a.nzv + tr + (int32_t)c)] = run[j];
                    }
                }
            }
            before += (uint32_t)(__popc(hw.x) + __popc(hw.y) + __popc(hw.z) + __popc(hw.w));
            carry = __shfl_sync(FULL, x, 31);
        }
    }
}

}  // namespace

namespace {

// ------------------------------------------------------------- long rows ----
// One block per long row (its arcs reach more than kLongTiles tiles past the
// tile of its first arc): the leading parts of its later tiles folded in tile
// order onto its first part, 256 at a time (a block scan with a fixed
// grouping). With a.carry, every such tile's carry (the row's value before
// the tile) is stored for the correction's flag pass; acc[v] ends as the
// row's total. Runs after k_pull_arcs, before the flag pass and the apply.
template <int APP>
__global__ void __launch_bounds__(kPullThreads) k_long_rows(PullArgs a)
{
    using Op = PullOp<APP>;
    using T = typename Op::T;
    __shared__ T s_w[kPullThreads / 32];
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    T *acc = reinterpret_cast<T *>(a.acc);
    const T *lead = reinterpret_cast<const T *>(a.lead);
    T *carry = reinterpret_cast<T *>(a.carry);
    const uint32_t nl = *a.nlong;
    for (uint32_t r = blockIdx.x; r < nl; r += gridDim.x) {
        const int32_t v = a.lrows[r];
        const int32_t t0 = __ldg(a.row_ptr + v) / kPT, t1 = (__ldg(a.row_ptr + v + 1) - 1) / kPT;
        T run = acc[v];
        for (int32_t base = t0 + 1; base <= t1; base += kPullThreads) {
            const int32_t u = base + (int32_t)threadIdx.x;
            T x = u <= t1 ? lead[u] : Op::id();
            // inclusive warp scan, then the warps' totals in order
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if ((int)lane >= o) x = Op::op(y, x);
            }
            if (lane == 31) s_w[wid] = x;
            __syncthreads();
            T before_warp = Op::id(), chunk = Op::id();
#pragma unroll
            for (int i = 0; i < kPullThreads / 32; ++i) {
                if (i < (int)wid) before_warp = Op::op(before_warp, s_w[i]);
                chunk = Op::op(chunk, s_w[i]);
            }
            const T excl_lane = __shfl_up_sync(0xFFFFFFFFu, x, 1);
            const T excl = lane ? Op::op(before_warp, excl_lane) : before_warp;
            if (carry && u <= t1) carry[u] = Op::op(run, excl);
            run = Op::op(run, chunk);
            __syncthreads();
        }
        if (threadIdx.x == 0) acc[v] = run;
        __syncthreads();
    }
}

// Carry of every tile that starts inside a short row (a correction's flag
// pass reads it): the row's first part and the leading parts of the tiles in
// between, in tile order. One thread per tile; long rows' carries come from
// k_long_rows.
template <int APP>
__global__ void __launch_bounds__(kPullThreads) k_carries(PullArgs a)
{
    using Op = PullOp<APP>;
    using T = typename Op::T;
    const T *acc = reinterpret_cast<const T *>(a.acc);
    const T *lead = reinterpret_cast<const T *>(a.lead);
    T *carry = reinterpret_cast<T *>(a.carry);
    const uint32_t nnz = *a.nnz;
    const long long nt = ((long long)nnz + kPT - 1) / kPT;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
        const int2 op = __ldg(a.topen + t);
        if (op.y < 0 || op.y >= t) continue;   // long row, or the tile starts with a row
        T c = acc[op.x];
        for (long long u = (long long)op.y + 1; u < t; ++u) c = Op::op(c, lead[u]);
        carry[t] = c;
    }
}

// ------------------------------------------------------ correction flags ----
// Second pass of a PageRank correction (Sec. 3.4, Alg. 2 GG-Gather influence
// and GG-EStatus) over the full in-edge list, after k_pull_arcs stored every
// arc's contribution: the running sum of its row before and after each arc,
// influence (after - before) / after > theta tested as
// (after - before) > theta * after, one flag bit per arc. The row continued
// from earlier tiles starts from its carry (k_carries / k_long_rows): its
// part in the tile of its first arc plus the leading parts of the tiles in
// between, in tile order. Lane L takes the tile's arcs 8L .. 8L + 7 (two
// 16-byte loads of the kept values, one byte of a flag word), so a single
// segmented warp scan covers the tile.
__global__ void __launch_bounds__(kPullThreads, 4) k_prc_flags(PullArgs a)
{
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nnz = *a.nnz;
    const long long nt = ((long long)nnz + kPT - 1) / kPT;
    const long long mask_words = ((long long)nnz + 31) / 32;
    const long long W = (long long)gridDim.x * (kPullThreads / 32);
    const uint32_t sh = 8u * (lane & 3u);                // this lane's byte in its flag word
    uint4 pf0 = make_uint4(0u, 0u, 0u, 0u), pf1 = pf0;   // the next full tile's values, loaded ahead
    bool have_pf = false;
    for (long long t = (long long)blockIdx.x * (kPullThreads / 32) + (threadIdx.x >> 5); t < nt; t += W) {
        const long long a0 = t * kPT;
        const uint32_t rel = nnz - (uint32_t)a0 < (uint32_t)kPT ? nnz - (uint32_t)a0 : (uint32_t)kPT;
        // lane L: arcs 8L .. 8L + 7 of the tile
        float v[8];
        if (rel == (uint32_t)kPT) {
            uint4 x = pf0, y = pf1;
            if (!have_pf) {
                x = reinterpret_cast<const uint4 *>(a.vals + a0 + 8 * lane)[0];
                y = reinterpret_cast<const uint4 *>(a.vals + a0 + 8 * lane)[1];
            }
            v[0] = __uint_as_float(x.x); v[1] = __uint_as_float(x.y); v[2] = __uint_as_float(x.z);
            v[3] = __uint_as_float(x.w); v[4] = __uint_as_float(y.x); v[5] = __uint_as_float(y.y);
            v[6] = __uint_as_float(y.z); v[7] = __uint_as_float(y.w);
            const long long tn = t + W;
            have_pf = tn < nt && (tn + 1) * kPT <= (long long)nnz;
            if (have_pf) {
                pf0 = reinterpret_cast<const uint4 *>(a.vals + tn * kPT + 8 * lane)[0];
                pf1 = reinterpret_cast<const uint4 *>(a.vals + tn * kPT + 8 * lane)[1];
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t q = 8u * lane + (uint32_t)j;
                v[j] = q < rel ? a.vals[a0 + q] : 0.0f;
            }
        }
        uint32_t hw = __ldg(a.hb + t * 8 + (lane >> 2));
        if (rel < (uint32_t)kPT) hw = tail_bits(hw, (int)(lane >> 2), rel);
        const uint32_t f = (hw >> sh) & 0xFFu;   // bit j: arc j of this lane starts a row
        // carry of the row open at the tile start (k_carries, k_long_rows)
        float carry = 0.0f;
        if (lane == 0 && !(hw & 1u)) carry = a.carry[t];
        // the lane's tail: its arcs from its last row start (or all of them)
        float r = v[0];
#pragma unroll
        for (int j = 1; j < 8; ++j) r = ((f >> j) & 1u) ? v[j] : r + v[j];
        // warp segmented inclusive scan of the tails
        const uint32_t heads = __ballot_sync(FULL, f != 0u);
        const uint32_t le = heads & (FULL >> (31u - lane));
        const int start = le ? 31 - __clz(le) : -1;   // lane where the segment open at this lane's end starts
        float x = r;
        if (lane == 0 && f == 0u) x = carry + r;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(FULL, x, o);
            if ((int)lane >= o && (int)lane - o >= start) x = y + x;
        }
        float run = __shfl_up_sync(FULL, x, 1);
        if (lane == 0) run = carry;
        // running sums before / after each arc, in arc order from the
        // segment's value at the lane start
        uint32_t byte = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t q = 8u * lane + (uint32_t)j;
            const float before = ((f >> j) & 1u) ? 0.0f : run;
            const float after = __fadd_rn(before, v[j]);
            run = after;
            const bool fl = after != 0.0f ? __fsub_rn(after, before) > __fmul_rn(a.theta, after) : 0.0f > a.theta;
            if (fl && q < rel) byte |= 1u << j;
        }
        uint32_t word = byte << sh;
        word |= __shfl_xor_sync(FULL, word, 1);
        word |= __shfl_xor_sync(FULL, word, 2);
        const long long wi = t * 8 + (lane >> 2);
        if ((lane & 3u) == 0 && wi < mask_words) a.mask[wi] = word;
        const uint32_t tile_active = __reduce_add_sync(FULL, (uint32_t)__popc(byte));
        if (lane == 0 && a.tcnt) a.tcnt[t] = tile_active;
    }
}

// Second pass of a correction of SSSP / BFS / CC (Sec. 3.4; influence on a
// min accumulator as the reading of Alg. 2 for these applications): the
// running minimum of its row before each arc (INF before the first), the
// candidate's influence, one flag bit per arc. An arc without a candidate
// (source unreached) keeps its flag (cleared under GG_EST_STRICT); theta < 0
// sets every other flag, theta >= 1 clears it; otherwise the flag is set when
// the candidate lowers the running minimum by more than theta of it
// ((before - cand) 2^32 > theta_fx before, exact), or is the row's first
// candidate (or, for CC, lowers it at all).
template <int APP>
__global__ void __launch_bounds__(kPullThreads, 4) k_minc_flags(PullArgs a)
{
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nnz = *a.nnz;
    const long long nt = ((long long)nnz + kPT - 1) / kPT;
    const long long mask_words = ((long long)nnz + 31) / 32;
    const long long W = (long long)gridDim.x * (kPullThreads / 32);
    const uint32_t *cv = reinterpret_cast<const uint32_t *>(a.vals);
    const uint32_t sh = 8u * (lane & 3u);                // this lane's byte in its flag word
    uint4 pf0 = make_uint4(0u, 0u, 0u, 0u), pf1 = pf0;   // the next full tile's candidates, loaded ahead
    bool have_pf = false;
    for (long long t = (long long)blockIdx.x * (kPullThreads / 32) + (threadIdx.x >> 5); t < nt; t += W) {
        const long long a0 = t * kPT;
        const uint32_t rel = nnz - (uint32_t)a0 < (uint32_t)kPT ? nnz - (uint32_t)a0 : (uint32_t)kPT;
        // lane L: arcs 8L .. 8L + 7 of the tile
        uint32_t v[8];
        if (rel == (uint32_t)kPT) {
            uint4 x = pf0, y = pf1;
            if (!have_pf) {
                x = reinterpret_cast<const uint4 *>(cv + a0 + 8 * lane)[0];
                y = reinterpret_cast<const uint4 *>(cv + a0 + 8 * lane)[1];
            }
            v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
            v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
            const long long tn = t + W;
            have_pf = tn < nt && (tn + 1) * kPT <= (long long)nnz;
            if (have_pf) {
                pf0 = reinterpret_cast<const uint4 *>(cv + tn * kPT + 8 * lane)[0];
                pf1 = reinterpret_cast<const uint4 *>(cv + tn * kPT + 8 * lane)[1];
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t q = 8u * lane + (uint32_t)j;
                v[j] = q < rel ? cv[a0 + q] : kInf;
            }
        }
        const long long wi = t * 8 + (lane >> 2);
        uint32_t hw = __ldg(a.hb + t * 8 + (lane >> 2));
        if (rel < (uint32_t)kPT) hw = tail_bits(hw, (int)(lane >> 2), rel);
        const uint32_t f = (hw >> sh) & 0xFFu;   // bit j: arc j of this lane starts a row
        const uint32_t old = ((wi < mask_words) ? a.mask[wi] : 0u) >> sh;   // this lane's flags, before
        // running minimum of the row open at the tile start (k_carries, k_long_rows)
        uint32_t carry = kInf;
        if (lane == 0 && !(hw & 1u)) carry = reinterpret_cast<const uint32_t *>(a.carry)[t];
        uint32_t r = v[0];
#pragma unroll
        for (int j = 1; j < 8; ++j) r = ((f >> j) & 1u) ? v[j] : min(r, v[j]);
        const uint32_t heads = __ballot_sync(FULL, f != 0u);
        const uint32_t le = heads & (FULL >> (31u - lane));
        const int start = le ? 31 - __clz(le) : -1;
        uint32_t x = r;
        if (lane == 0 && f == 0u) x = min(carry, r);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if ((int)lane >= o && (int)lane - o >= start) x = min(y, x);
        }
        uint32_t run = __shfl_up_sync(FULL, x, 1);
        if (lane == 0) run = carry;
        uint32_t byte = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t q = 8u * lane + (uint32_t)j;
            const uint32_t before = ((f >> j) & 1u) ? kInf : run;
            const uint32_t c = v[j];
            run = min(before, c);
            uint32_t fl = 0;
            if (c == kInf) {
                fl = a.est_strict ? 0u : (old >> j) & 1u;
            } else if (a.theta_case == 1) {
                fl = 1u;
            } else if (a.theta_case == 2) {
                fl = 0u;
            } else if (c < before) {
                if (before == kInf || APP == GG_APP_CC) fl = 1u;
                else fl = ((unsigned long long)(before - c) << 32) > a.theta_fx * (unsigned long long)before ? 1u : 0u;
            }
            if (fl && q < rel) byte |= 1u << j;
        }
        uint32_t word = byte << sh;
        word |= __shfl_xor_sync(FULL, word, 1);
        word |= __shfl_xor_sync(FULL, word, 2);
        if ((lane & 3u) == 0 && wi < mask_words) a.mask[wi] = word;
        const uint32_t tile_active = __reduce_add_sync(FULL, (uint32_t)__popc(byte));
        if (lane == 0 && a.tcnt) a.tcnt[t] = tile_active;
    }
}

// ----------------------------------------------------------------- apply ----
// Loads of the four consecutive vertices v0 .. v0 + 3 (16-byte loads when
// all four exist): row pointers (5), row sums, old values, degrees.
struct Quad {
    int32_t rp[5];
    uint32_t acc[4], old[4];
    int32_t deg[4];
};

template <bool PR>
__device__ __forceinline__ void load_quad(const PullArgs &a, long long v0, Quad &q)
{
    const uint32_t *accu = reinterpret_cast<const uint32_t *>(a.acc);
    const uint32_t *oldu = PR ? reinterpret_cast<const uint32_t *>(a.rank_cur) : a.val_cur;
    if (v0 + 4 <= a.n) {
        const int4 r = __ldg(reinterpret_cast<const int4 *>(a.row_ptr + v0));
        q.rp[0] = r.x; q.rp[1] = r.y; q.rp[2] = r.z; q.rp[3] = r.w;
        q.rp[4] = __ldg(a.row_ptr + v0 + 4);
        const uint4 c = *reinterpret_cast<const uint4 *>(accu + v0);
        q.acc[0] = c.x; q.acc[1] = c.y; q.acc[2] = c.z; q.acc[3] = c.w;
        const uint4 o = *reinterpret_cast<const uint4 *>(oldu + v0);
        q.old[0] = o.x; q.old[1] = o.y; q.old[2] = o.z; q.old[3] = o.w;
        if (PR) {
            if (a.deg_apply) {
                const int4 d = *reinterpret_cast<const int4 *>(a.deg_apply + v0);
                q.deg[0] = d.x; q.deg[1] = d.y; q.deg[2] = d.z; q.deg[3] = d.w;
            } else {
                const int4 p = __ldg(reinterpret_cast<const int4 *>(a.out_ptr + v0));
                const int32_t pn = __ldg(a.out_ptr + v0 + 4);
                q.deg[0] = p.y - p.x; q.deg[1] = p.z - p.y; q.deg[2] = p.w - p.z; q.deg[3] = pn - p.w;
            }
        }
    } else {
        // the last, partial group: rows past n read as empty (row_ptr[n])
#pragma unroll
        for (int i = 0; i < 5; ++i) q.rp[i] = __ldg(a.row_ptr + (v0 + i < a.n ? v0 + i : (long long)a.n));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const long long v = v0 + i;
            const bool live = v < a.n;
            q.acc[i] = live ? accu[v] : 0u;
            q.old[i] = live ? oldu[v] : 0u;
            q.deg[i] = 0;
            if (PR && live) q.deg[i] = a.deg_apply ? a.deg_apply[v] : __ldg(a.out_ptr + v + 1) - __ldg(a.out_ptr + v);
        }
    }
}

// GG-Apply + GG-VStatus (Alg. 2) for PageRank, four consecutive vertices per
// thread and step. A row's sum is acc[v] (written by the tile holding its
// first arc), plus, for a row continued across at most kLongTiles tile ends,
// the leading parts of the later tiles it covers, in tile order (a long row's
// acc[v] is complete already); a row with no arcs in the list sums to 0.
__global__ void __launch_bounds__(kPullThreads) k_pr_apply(PullArgs a)
{
    unsigned long long changed = 0, sum = 0;
    uint32_t mx = 0;
    const long long S = (long long)gridDim.x * blockDim.x;
    const long long ng = ((long long)a.n + 3) / 4;
    for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < ng; gi += S) {
        const long long v0 = 4 * gi;
        Quad q;
        load_quad<true>(a, v0, q);
        float nw[4], cb[4], hv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float acc = 0.0f;
            if (q.rp[i + 1] > q.rp[i]) {
                acc = __uint_as_float(q.acc[i]);
                const int32_t t0 = q.rp[i] / kPT, t1 = (q.rp[i + 1] - 1) / kPT;
                if (t1 - t0 <= kLongTiles)
                    for (int32_t u = t0 + 1; u <= t1; ++u) acc += a.lead[u];
            }
            nw[i] = __fmaf_rn(a.damping, acc, a.base);
            const float delta = fabsf(__fsub_rn(nw[i], __uint_as_float(q.old[i])));
            cb[i] = q.deg[i] > 0 ? __fdiv_rn(nw[i], (float)q.deg[i]) : 0.0f;
            hv[i] = __fmul_rn(a.n_f, delta);
            if (v0 + i < a.n) {
                changed += delta > a.epsilon ? 1ull : 0ull;
                sum += __float2ull_rz(delta * 1099511627776.0f);   // fixed point 2^-40
                const uint32_t db = __float_as_uint(delta);
                mx = db > mx ? db : mx;
            }
        }
        if (v0 + 4 <= a.n) {
            *reinterpret_cast<float4 *>(a.rank_next + v0) = make_float4(nw[0], nw[1], nw[2], nw[3]);
            *reinterpret_cast<float4 *>(a.contrib_next + v0) = make_float4(cb[0], cb[1], cb[2], cb[3]);
            if (a.hist_out) *reinterpret_cast<float4 *>(a.hist_out + v0) = make_float4(hv[0], hv[1], hv[2], hv[3]);
        } else {
            for (int i = 0; i < 4 && v0 + i < a.n; ++i) {
                a.rank_next[v0 + i] = nw[i];
                a.contrib_next[v0 + i] = cb[i];
                if (a.hist_out) a.hist_out[v0 + i] = hv[i];
            }
        }
    }
    if (!a.stats) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        changed += __shfl_xor_sync(0xFFFFFFFFu, changed, o);
        sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
        const uint32_t om = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
        mx = om > mx ? om : mx;
    }
    if ((threadIdx.x & 31u) == 0 && (changed | sum | mx)) {
        atomicAdd(&a.stats->changed, changed);
        atomicAdd(&a.stats->sum_delta, sum);
        atomicMax(&a.stats->max_delta_bits, mx);
    }
}

// GG-Apply + GG-VStatus for SSSP / BFS / CC, four consecutive vertices per
// thread and step: new = min(old, the row's minimum candidate); a vertex
// whose value decreased joins the next frontier (vertex, new value); each
// block reserves its entries with one atomic per step (many vertices change
// in the first iterations).
template <int APP>
__global__ void __launch_bounds__(kPullThreads) k_min_apply(PullArgs a)
{
    const uint32_t *lead = reinterpret_cast<const uint32_t *>(a.lead);
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    __shared__ uint32_t s_cnt[kPullThreads / 32];
    __shared__ uint32_t s_base;
    unsigned long long changed = 0, sum = 0;
    uint32_t mx = 0;
    const long long S = (long long)gridDim.x * blockDim.x;
    const long long ng = ((long long)a.n + 3) / 4;
    const long long nround = (ng + S - 1) / S * S;   // whole blocks stay in the loop (block-wide reservation)
    for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < nround; gi += S) {
        const long long v0 = 4 * gi;
        Quad q;
        uint32_t nw[4];
        uint32_t chm = 0;
        if (gi < ng) {
            load_quad<false>(a, v0, q);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t m = kInf;
                if (q.rp[i + 1] > q.rp[i]) {
                    m = q.acc[i];
                    const int32_t t0 = q.rp[i] / kPT, t1 = (q.rp[i + 1] - 1) / kPT;
                    if (t1 - t0 <= kLongTiles)
                        for (int32_t u = t0 + 1; u <= t1; ++u) m = min(m, lead[u]);
                }
                nw[i] = min(q.old[i], m);
                if (v0 + i < a.n && nw[i] < q.old[i]) {
                    chm |= 1u << i;
                    changed += 1;
                    if (q.old[i] != kInf) {
                        sum += q.old[i] - nw[i];
                        mx = (q.old[i] - nw[i]) > mx ? (q.old[i] - nw[i]) : mx;
                    }
                }
            }
            if (v0 + 4 <= a.n) {
                *reinterpret_cast<uint4 *>(a.val_next + v0) = make_uint4(nw[0], nw[1], nw[2], nw[3]);
                if (a.hist_out)
                    *reinterpret_cast<float4 *>(a.hist_out + v0) =
                        make_float4(chm & 1u ? 1.0f : 0.0f, chm & 2u ? 1.0f : 0.0f, chm & 4u ? 1.0f : 0.0f,
                                    chm & 8u ? 1.0f : 0.0f);
            } else {
                for (int i = 0; i < 4 && v0 + i < a.n; ++i) {
                    a.val_next[v0 + i] = nw[i];
                    if (a.hist_out) a.hist_out[v0 + i] = (chm >> i) & 1u ? 1.0f : 0.0f;
                }
            }
        }
        // frontier: the block's changed vertices at one offset
        if (a.q_out) {
            const uint32_t c = (uint32_t)__popc(chm);
            uint32_t incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if ((int)lane >= o) incl += y;
            }
            if (lane == 31) s_cnt[wid] = incl;
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t tot = 0;
#pragma unroll
                for (int i = 0; i < kPullThreads / 32; ++i) {
                    const uint32_t x = s_cnt[i];
                    s_cnt[i] = tot;
                    tot += x;
                }
                s_base = tot ? atomicAdd(a.q_out_len, tot) : 0u;
            }
            __syncthreads();
            uint32_t pos = s_base + s_cnt[wid] + incl - c;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if ((chm >> i) & 1u) {
                    a.q_out[pos] = (int32_t)(v0 + i);
                    a.q_out_val[pos] = nw[i];
                    ++pos;
                }
            }
            __syncthreads();
        }
    }
    if (!a.stats) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        changed += __shfl_xor_sync(0xFFFFFFFFu, changed, o);
        sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
        const uint32_t om = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
        mx = om > mx ? om : mx;
    }
    if (lane == 0 && (changed | sum | mx)) {
        atomicAdd(&a.stats->changed, changed);
        atomicAdd(&a.stats->sum_delta, sum);
        atomicMax(&a.stats->max_delta_bits, mx);
    }
}

// The contribution of every hub slot, which the PageRank pull gathers read in
// place of the hubs' scattered contributions.
__global__ void k_hub_values(PullArgs a)
{
    const uint32_t *v = reinterpret_cast<const uint32_t *>(a.contrib);
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < a.n_hubs; j += gridDim.x * blockDim.x)
        a.hubv[j] = v[a.hub_ids[j]];
}

// bit v of bits: vertex v is in the frontier queue (bits cleared beforehand)
__global__ void k_front_bits(const int32_t *__restrict__ q, const uint32_t *__restrict__ q_len,
                             uint32_t *__restrict__ bits, int32_t n)
{
    const uint32_t len = *q_len;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
        const int32_t v = q[i];
        if (v >= 0 && v < n) atomicOr(bits + (v >> 5), 1u << (v & 31));
    }
}

}  // namespace

namespace {

template <int APP>
void launch_arcs(const PullArgs &a, uint32_t max_tiles, int num_sms, cudaStream_t s)
{
    constexpr int arc_blocks_per_sm = 4;
    long long blocks = ((long long)max_tiles + kPullThreads / 32 - 1) / (kPullThreads / 32);
    if (blocks > (long long)num_sms * arc_blocks_per_sm) blocks = (long long)num_sms * arc_blocks_per_sm;
    if (blocks < 1) blocks = 1;
    if constexpr (APP != GG_APP_PAGERANK) {
        if (a.front) {
            k_pull_arcs<APP, arc_blocks_per_sm, true, true><<<(unsigned)blocks, kPullThreads, 0, s>>>(a);
            return;
        }
    }
    k_pull_arcs<APP, arc_blocks_per_sm, true><<<(unsigned)blocks, kPullThreads, 0, s>>>(a);
}

template <int APP>
void launch_flags(const PullArgs &a, uint32_t max_tiles, int num_sms, cudaStream_t s)
{
    long long blocks = ((long long)max_tiles + kPullThreads / 32 - 1) / (kPullThreads / 32);
    if (blocks > (long long)num_sms * 4) blocks = (long long)num_sms * 4;
    if (blocks < 1) blocks = 1;
    if constexpr (APP == GG_APP_PAGERANK) k_prc_flags<<<(unsigned)blocks, kPullThreads, 0, s>>>(a);
    else k_minc_flags<APP><<<(unsigned)blocks, kPullThreads, 0, s>>>(a);
}

template <int APP>
void launch_apply(const PullArgs &a, int num_sms, cudaStream_t s)
{
    // persistent: the blocks one wave holds (PageRank's apply 4 blocks of 256
    // per SM, the min apply 8), four vertices per thread and step
    const int per_sm = APP == GG_APP_PAGERANK ? 4 : 8;
    long long ab = ((long long)a.n / 4 + kPullThreads) / kPullThreads;
    if (ab > (long long)num_sms * per_sm) ab = (long long)num_sms * per_sm;
    if (ab < 1) ab = 1;
    if constexpr (APP == GG_APP_PAGERANK) k_pr_apply<<<(unsigned)ab, kPullThreads, 0, s>>>(a);
    else k_min_apply<APP><<<(unsigned)ab, kPullThreads, 0, s>>>(a);
}

template <int APP>
cudaError_t pull_iteration(PullArgs a, bool correct, uint32_t max_tiles, int num_sms, cudaStream_t s)
{
    if (APP == GG_APP_PAGERANK && a.n_hubs > 0)
        k_hub_values<<<(unsigned)((a.n_hubs + kPullThreads - 1) / kPullThreads), kPullThreads, 0, s>>>(a);
    launch_arcs<APP>(a, max_tiles, num_sms, s);
    if (!correct) a.carry = nullptr;
    k_long_rows<APP><<<(unsigned)(num_sms * 4), kPullThreads, 0, s>>>(a);
    if (correct) {
        long long cb = ((long long)max_tiles + kPullThreads - 1) / kPullThreads;
        if (cb > (long long)num_sms * 8) cb = (long long)num_sms * 8;
        if (cb < 1) cb = 1;
        k_carries<APP><<<(unsigned)cb, kPullThreads, 0, s>>>(a);
        launch_flags<APP>(a, max_tiles, num_sms, s);
    }
    launch_apply<APP>(a, num_sms, s);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_front_bits(const int32_t *q, const uint32_t *q_len, uint32_t *bits, int32_t n, int num_sms,
                              cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bits, 0, 4 * (((size_t)n + 31) / 32), s);
    if (e != cudaSuccess) return e;
    k_front_bits<<<(unsigned)(num_sms * 8), 256, 0, s>>>(q, q_len, bits, n);
    return cudaGetLastError();
}

cudaError_t launch_pull(int app, const PullArgs &a, bool correct, uint32_t max_tiles, int num_sms, cudaStream_t s)
{
    switch (app) {
    case GG_APP_PAGERANK: return pull_iteration<GG_APP_PAGERANK>(a, correct, max_tiles, num_sms, s);
    case GG_APP_SSSP: return pull_iteration<GG_APP_SSSP>(a, correct, max_tiles, num_sms, s);
    case GG_APP_BFS: return pull_iteration<GG_APP_BFS>(a, correct, max_tiles, num_sms, s);
    case GG_APP_CC: return pull_iteration<GG_APP_CC>(a, correct, max_tiles, num_sms, s);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------- plan (host) ----
gg_status ensure_pull(gg_graph *g)
{
    if (g->pull_ready) return GG_OK;
    const size_t tiles = ((size_t)g->m + kPT - 1) / kPT + 1;
    const size_t nzw = ((size_t)g->n + 31) / 32 + 1;
    // per plan: hb (8 words per tile + 8), topen (2 words per tile + 2), trow (tiles + 1), lrows, nlong,
    // nzb, nzc, nzcnt, nzv (n + 4)
    const size_t nlr = tiles / kLongTiles + 2;
    const size_t words = 8 * tiles + 8 + 2 * (tiles + 1) + (tiles + 1) + nlr + 4 + 3 * nzw + ((size_t)g->n + 4) + 8;
    for (int i = 0; i < 2; ++i) {
        PullPlan &p = g->plan[i];
        gg_status st = p.buf.alloc(4 * words, g->stream);
        if (st != GG_OK) return st;
        uint32_t *w = p.buf.u32();
        p.hb = w; w += 8 * tiles + 8;
        p.topen = (int2 *)w; w += 2 * (tiles + 1);
        p.trow = (int32_t *)w; w += tiles + 1;
        p.lrows = (int32_t *)w; w += nlr;
        p.nlong = w; w += 4;
        p.nzb = w; w += nzw;
        p.nzc = w; w += nzw;
        p.nzcnt = w; w += nzw;
        p.nzv = (int32_t *)w;
        p.hb_words = 8 * tiles + 8;
        p.tiles = tiles;
        p.nzw = nzw;
        p.valid = false;
    }
    const size_t fwords = ((size_t)g->n + 31) / 32 + 4;
    gg_status st = g->b_pull.alloc(4 * ((size_t)g->n + 2 * tiles + 16 + fwords + kHubCodes), g->stream);
    if (st != GG_OK) return st;
    g->pull_acc = g->b_pull.f32();
    g->pull_lead = g->pull_acc + g->n + 4;
    g->pull_carry = g->pull_lead + tiles + 4;
    g->pull_front = reinterpret_cast<uint32_t *>(g->pull_carry + tiles + 4);
    g->pull_hubv = g->pull_front + fwords;
    g->pull_ready = true;
    return GG_OK;
}

// Plan of the full in-edge list (which 0) or of the packed active list (1).
gg_status build_pull_plan(gg_graph *g, int which)
{
    PullPlan &p = g->plan[which];
    const int32_t *ptr = which ? g->sp_ptr : g->in_ptr;
    cudaStream_t s = g->stream;
    GG_CUDA(cudaMemsetAsync(p.hb, 0, 4 * p.hb_words, s));
    GG_CUDA(cudaMemsetAsync(p.nlong, 0, 4, s));
    int grid = (int)(((size_t)g->n + 255) / 256);
    if (grid > g->num_sms * 8) grid = g->num_sms * 8;
    if (grid < 1) grid = 1;
    k_plan_nz<<<grid, 256, 0, s>>>(ptr, g->n, p.nzb, p.nzcnt);
    GG_CUDA(cudaGetLastError());
    // exclusive scan of the words' counts (it also writes the total at
    // nzc[words], inside the array: nzw = words + 1)
    const size_t words = ((size_t)g->n + 31) / 32;
    GG_CUDA(launch_scan_u32(p.nzcnt, p.nzc, words, g->scan_tmp, s));
    k_plan_heads<<<grid, 256, 0, s>>>(ptr, g->n, p.nzb, p.nzc, p.hb, p.trow, p.nzv, p.topen, p.lrows, p.nlong);
    GG_CUDA(cudaGetLastError());
    g->launches += 8;
    p.valid = true;
    return GG_OK;
}

}  // namespace gg

// gg_tile.cuh - the merge-path tile engine behind the pull gather (approximate
// and accurate iterations), the correction iteration and the edge sampler.
//
// A list (CSC rows: row_ptr + per-arc source/weight) is viewed as the merged
// sequence "arcs of row 0, end of row 0, arcs of row 1, end of row 1, ...".
// Tile t owns kTile consecutive items of that sequence; its first row and
// arc come from a precomputed partition (tile_row). Within a tile:
//   load    row ends into shared memory; arcs' values gathered into shared
//           memory with coalesced loads of the arc arrays and random loads of
//           the source values (the GG-Gather reads of Alg. 1 / Alg. 2);
//   pass 1  each thread folds its kIPT items into (has_row_end, partial);
//           a block segmented scan gives every thread the running value of
//           the row open at its start;
//   carry   a row that began in earlier tiles takes the sum of those tiles'
//           published partials, added in tile order (deterministic);
//   pass 2  walk again with the carry: per arc, influence and new flag
//           (correction, Alg. 2 GG-Gather + GG-EStatus) or sampled flag
//           (Sec. 3.4); per row end, GG-Apply + GG-VStatus;
//   pass 3  (correction, sampling) stream-compact the active arcs into the
//           packed active-CSC through a decoupled look-back over tile counts.
#pragma once

#include "gg_internal.cuh"

namespace gg {

// ------------------------------------------------------------- value ops ----
template <int APP>
struct Acc {  // min applications: uint32, min, identity = unreached
    using T = uint32_t;
    __device__ static __forceinline__ T id() { return kInf; }
    __device__ static __forceinline__ T op(T a, T b) { return a < b ? a : b; }
    __device__ static __forceinline__ uint32_t bits(T v) { return v; }
    __device__ static __forceinline__ T from_bits(uint32_t b) { return b; }
};
template <>
struct Acc<GG_APP_PAGERANK> {  // PageRank: FP32 sum
    using T = float;
    __device__ static __forceinline__ T id() { return 0.0f; }
    __device__ static __forceinline__ T op(T a, T b) { return __fadd_rn(a, b); }
    __device__ static __forceinline__ uint32_t bits(T v) { return __float_as_uint(v); }
    __device__ static __forceinline__ T from_bits(uint32_t b) { return __uint_as_float(b); }
};

// SplitMix64 output for one state (Steele, Lea, Flood 2014): advance by the
// golden gamma, then the variant-13 finaliser.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long state)
{
    unsigned long long z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Initial flag of arc src -> dst under ratio threshold thr = floor(sigma*2^32).
__device__ __forceinline__ uint32_t sampled_flag(int32_t src, int32_t dst, int symmetric,
                                                 unsigned long long seed, unsigned long long thr)
{
    uint32_t a = (uint32_t)src, b = (uint32_t)dst;
    if (symmetric && a > b) { uint32_t t = a; a = b; b = t; }
    unsigned long long key = ((unsigned long long)a << 32) | b;
    return (splitmix64(seed ^ key) >> 32) < thr ? 1u : 0u;
}

// ------------------------------------------------------------ warp scans ----
template <int APP>
__device__ __forceinline__ void warp_seg_scan_incl(typename Acc<APP>::T &v, uint32_t &f)
{
    const uint32_t lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        typename Acc<APP>::T ov = __shfl_up_sync(0xFFFFFFFFu, v, o);
        uint32_t of = __shfl_up_sync(0xFFFFFFFFu, f, o);
        if (lane >= (uint32_t)o) {
            if (!f) v = Acc<APP>::op(ov, v);
            f |= of;
        }
    }
}

__device__ __forceinline__ uint32_t warp_incl_sum_u32(uint32_t v)
{
    const uint32_t lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t ov = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= (uint32_t)o) v += ov;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Exclusive prefix (over earlier tiles) of the published per-tile counts:
// decoupled look-back with a warp; integer sums, so the grouping does not
// matter. Call with the whole warp; the result is valid in every lane.
__device__ __forceinline__ uint32_t lookback_count(unsigned long long *st, int t, uint32_t epoch,
                                                   uint32_t *err)
{
    const uint32_t lane = lane_id();
    uint32_t excl = 0;
    for (int base = t - 1; base >= 0; base -= 32) {
        int j = base - (int)lane;
        uint32_t flag = 0, val = 0;
        bool valid = j >= 0;
        if (valid) {
            unsigned long long w = wait_status(&st[j], epoch, err, pack_status(epoch, 1u, 0u));
            flag = status_flag(w);
            val = status_value(w);
        }
        unsigned ball = __ballot_sync(0xFFFFFFFFu, valid && flag);
        if (ball) {
            int stop = __ffs(ball) - 1;
            excl += warp_sum_u32((int)lane <= stop ? val : 0u);
            break;
        }
        excl += warp_sum_u32(valid ? val : 0u);
    }
    return excl;
}

// Carry of the row open at the start of tile t: the partials published by
// the tiles from the one where that row began (the nearest earlier tile with
// a row end) up to t-1, combined in tile order. Whole warp; valid in lane 0.
template <int APP>
__device__ __forceinline__ typename Acc<APP>::T lookback_carry(unsigned long long *st, int t,
                                                               uint32_t epoch, uint32_t *err)
{
    using T = typename Acc<APP>::T;
    const uint32_t lane = lane_id();
    int jstar = 0;
    const unsigned long long fallback = pack_status(epoch, 1u, Acc<APP>::bits(Acc<APP>::id()));
    for (int base = t - 1; base >= 0; base -= 32) {
        int j = base - (int)lane;
        uint32_t f = 0;
        if (j >= 0) f = status_flag(wait_status(&st[j], epoch, err, fallback));
        unsigned ball = __ballot_sync(0xFFFFFFFFu, f != 0u);
        if (ball) {
            jstar = base - (__ffs(ball) - 1);
            break;
        }
    }
    T acc = Acc<APP>::id();
    for (int s0 = jstar; s0 < t; s0 += 32) {
        int j = s0 + (int)lane;
        T v = Acc<APP>::id();
        if (j < t) {
            unsigned long long w = ld_acquire_u64(&st[j]);
            if (status_epoch(w) == epoch) v = Acc<APP>::from_bits(status_value(w));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            T ov = __shfl_down_sync(0xFFFFFFFFu, v, o);
            v = Acc<APP>::op(v, ov);
        }
        acc = Acc<APP>::op(acc, __shfl_sync(0xFFFFFFFFu, v, 0));
    }
    return acc;
}

// ----------------------------------------------------------- tile kernel ----
template <int APP, int KIND>
struct TileSmem {
    using T = typename Acc<APP>::T;
    int32_t rowend[kTile + 1];
    T val[kTile];
    int32_t src[(KIND == K_GATHER) ? 1 : kTile];
    uint32_t w[(KIND == K_GATHER) ? 1 : kTile];
    uint8_t flag[(KIND == K_GATHER) ? 1 : kTile];
    uint32_t oldw[(KIND == K_CORRECT && APP != GG_APP_PAGERANK) ? (kTile / 32 + 2) : 1];
    T warp_v[kWarps];
    uint32_t warp_f[kWarps];
    uint32_t warp_c[kWarps];
    T carry;
    uint32_t tile_excl;
    int32_t r0, r1, a0, a1, row_start;
    int slot;
};

template <int APP, int KIND>
__global__ void __launch_bounds__(kThreads)
k_tile(TileArgs a)
{
    using T = typename Acc<APP>::T;
    using A = Acc<APP>;
    constexpr bool kCarry = KIND != K_SAMPLE;
    constexpr bool kCompact = KIND != K_GATHER;
    constexpr bool kMin = APP != GG_APP_PAGERANK;
    constexpr bool kWeighted = APP == GG_APP_SSSP;
    __shared__ TileSmem<APP, KIND> sm;

    const int tid = threadIdx.x;
    const uint32_t lane = lane_id();
    const int warp = tid >> 5;
    const uint32_t nnz = *a.list_nnz;
    const uint32_t num_tiles = *a.num_tiles;
    const long long total = (long long)a.n + nnz;
    const bool has_w = (a.arc_w != nullptr);

    unsigned long long my_changed = 0, my_sum = 0;
    uint32_t my_max = 0;

    for (;;) {
        const int t = next_tile(a.sched, num_tiles, &sm.slot);
        if (t < 0) break;
        const long long d0 = (long long)t * kTile;
        const long long d1 = d0 + kTile < total ? d0 + kTile : total;
        if (tid == 0) {
            int32_t r0 = a.tile_row[t], r1 = a.tile_row[t + 1];
            sm.r0 = r0;
            sm.r1 = r1;
            sm.a0 = (int32_t)(d0 - r0);
            sm.a1 = (int32_t)(d1 - r1);
            sm.row_start = a.row_ptr[r0 < a.n ? r0 : a.n];
        }
        __syncthreads();
        const int32_t r0 = sm.r0, r1 = sm.r1, a0 = sm.a0, a1 = sm.a1;
        const int nrows = r1 - r0;     // row ends inside the tile
        const int narcs = a1 - a0;     // arcs inside the tile

        // ---- load: row ends and arc values ---------------------------------
        for (int i = tid; i < nrows; i += kThreads) sm.rowend[i] = a.row_ptr[r0 + i + 1];
        if (tid == 0) sm.rowend[nrows] = 0x7FFFFFFF;   // row r1 stays open past the tile
        if (KIND == K_CORRECT && kMin) {
            if (narcs > 0) {
                const int w0 = a0 >> 5, w1 = (a1 - 1) >> 5;
                for (int w = w0 + tid; w <= w1; w += kThreads) sm.oldw[w - w0] = a.mask[w];
            }
        }
        {
            int32_t s[kIPT];
#pragma unroll
            for (int i = 0; i < kIPT; ++i) {
                const int k = tid + i * kThreads;
                s[i] = k < narcs ? __ldg(a.arc_src + a0 + k) : 0;
            }
            uint32_t wv[kIPT];
#pragma unroll
            for (int i = 0; i < kIPT; ++i) {
                const int k = tid + i * kThreads;
                wv[i] = (has_w && (kWeighted || KIND == K_SAMPLE) && k < narcs) ? __ldg(a.arc_w + a0 + k) : 1u;
            }
#pragma unroll
            for (int i = 0; i < kIPT; ++i) {
                const int k = tid + i * kThreads;
                if (k < narcs) {
                    if (KIND != K_GATHER) {
                        sm.src[k] = s[i];
                        sm.w[k] = wv[i];
                    }
                    if (KIND != K_SAMPLE) {
                        if constexpr (APP == GG_APP_PAGERANK) {
                            sm.val[k] = __ldg(a.contrib_cur + s[i]);
                        } else {
                            const uint32_t vv = __ldg(a.val_cur + s[i]);
                            uint32_t cand;
                            if constexpr (APP == GG_APP_CC) {
                                cand = vv;
                            } else {
                                const uint32_t step = (APP == GG_APP_BFS) ? 1u : wv[i];
                                const unsigned long long c = (unsigned long long)vv + step;
                                cand = (vv == kInf || c >= kInf) ? kInf : (uint32_t)c;
                            }
                            sm.val[k] = cand;
                        }
                    }
                }
            }
        }
        __syncthreads();

        // ---- per-thread merge-path coordinates inside the tile -------------
        const int tile_items = (int)(d1 - d0);
        const int ld = tid * kIPT < tile_items ? tid * kIPT : tile_items;
        int cnt = tile_items - ld;
        cnt = cnt < kIPT ? cnt : kIPT;
        int lx, ly;
        {
            int lo = ld - narcs > 0 ? ld - narcs : 0;
            int hi = ld < nrows ? ld : nrows;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (sm.rowend[mid] - a0 <= ld - mid - 1) lo = mid + 1;
                else hi = mid;
            }
            lx = lo;
            ly = ld - lo;
        }

        // ---- pass 1 + block segmented scan + carry ---------------------------
        T carry_in = A::id();
        if constexpr (kCarry) {
            T v = A::id();
            uint32_t f = 0;
            {
                int x = lx, y = ly;
                for (int i = 0; i < cnt; ++i) {
                    if (y < sm.rowend[x] - a0) { v = A::op(v, sm.val[y]); ++y; }
                    else { f = 1; v = A::id(); ++x; }
                }
            }
            warp_seg_scan_incl<APP>(v, f);
            T lane_ev = __shfl_up_sync(0xFFFFFFFFu, v, 1);
            uint32_t lane_ef = __shfl_up_sync(0xFFFFFFFFu, f, 1);
            if (lane == 0) { lane_ev = A::id(); lane_ef = 0; }
            if (lane == 31) { sm.warp_v[warp] = v; sm.warp_f[warp] = f; }
            __syncthreads();
            if (warp == 0) {
                T wv = lane < kWarps ? sm.warp_v[lane] : A::id();
                uint32_t wf = lane < kWarps ? sm.warp_f[lane] : 0u;
                warp_seg_scan_incl<APP>(wv, wf);
                T ev = __shfl_up_sync(0xFFFFFFFFu, wv, 1);
                uint32_t ef = __shfl_up_sync(0xFFFFFFFFu, wf, 1);
                if (lane == 0) { ev = A::id(); ef = 0; }
                // publish the tile's own partial (the open row's part in this tile)
                T tv = __shfl_sync(0xFFFFFFFFu, wv, kWarps - 1);
                uint32_t tf = __shfl_sync(0xFFFFFFFFu, wf, kWarps - 1);
                if (lane == 0) st_release_u64(&a.st_carry[t], pack_status(a.epoch, tf, A::bits(tv)));
                if (lane < kWarps) { sm.warp_v[lane] = ev; sm.warp_f[lane] = ef; }
                // the carry of the row open at the tile start
                T c = A::id();
                if (a0 > sm.row_start) c = lookback_carry<APP>(a.st_carry, t, a.epoch, a.err);
                if (lane == 0) sm.carry = c;
            }
            __syncthreads();
            // exclusive prefix of this thread = warp prefix (+) lane prefix, behind the carry
            T ex_v = sm.warp_v[warp];
            uint32_t ex_f = sm.warp_f[warp];
            if (lane_ef) ex_v = lane_ev; else ex_v = A::op(ex_v, lane_ev);
            ex_f |= lane_ef;
            carry_in = ex_f ? ex_v : A::op(sm.carry, ex_v);
        }

        // ---- pass 2: influence / flags per arc, apply per row end ----------
        uint32_t my_active = 0;
        int32_t q_u[kMin ? kIPT : 1];
        uint32_t q_v[kMin ? kIPT : 1];
        int q_n = 0;
        {
            T acc = carry_in;
            int x = lx, y = ly;
            for (int i = 0; i < cnt; ++i) {
                if (y < sm.rowend[x] - a0) {
                    if constexpr (KIND == K_SAMPLE) {
                        const uint32_t fl = sampled_flag(sm.src[y], r0 + x, a.symmetric, a.seed, a.thr);
                        sm.flag[y] = (uint8_t)fl;
                        my_active += fl;
                    } else {
                        const T v = sm.val[y];
                        if constexpr (KIND == K_CORRECT) {
                            uint32_t fl;
                            if constexpr (APP == GG_APP_PAGERANK) {
                                // GG-Gather's returned influence (Alg. 2): (new - old) / new
                                const float after = __fadd_rn(acc, v);
                                const float infl = after != 0.0f ? __fdiv_rn(__fsub_rn(after, acc), after) : 0.0f;
                                fl = infl > a.theta ? 1u : 0u;
                            } else {
                                if (v == kInf) {   // no candidate: the arc keeps its flag
                                    const int k = a0 + y;
                                    fl = a.est_strict ? 0u : (sm.oldw[(k >> 5) - (a0 >> 5)] >> (k & 31)) & 1u;
                                } else if (a.theta_case == 1) {
                                    fl = 1u;
                                } else if (a.theta_case == 2) {
                                    fl = 0u;
                                } else if (v < acc) {
                                    if (acc == kInf || APP == GG_APP_CC) fl = 1u;
                                    else fl = ((unsigned long long)(acc - v) << 32) > a.theta_fx * (unsigned long long)acc ? 1u : 0u;
                                } else {
                                    fl = 0u;
                                }
                            }
                            sm.flag[y] = (uint8_t)fl;
                            my_active += fl;
                        }
                        acc = A::op(acc, v);
                    }
                    ++y;
                } else {
                    if constexpr (KIND != K_SAMPLE) {
                        const int32_t u = r0 + x;
                        if constexpr (APP == GG_APP_PAGERANK) {
                            // GG-Apply + GG-VStatus (Alg. 2)
                            const float nw = __fmaf_rn(a.damping, acc, a.base);
                            const float old = a.rank_cur[u];
                            const float delta = fabsf(__fsub_rn(nw, old));
                            const int deg = a.out_ptr[u + 1] - a.out_ptr[u];
                            a.rank_next[u] = nw;
                            a.contrib_next[u] = deg > 0 ? __fdiv_rn(nw, (float)deg) : 0.0f;
                            my_changed += delta > a.epsilon ? 1ull : 0ull;
                            my_sum += __float2ull_rz(delta * 1099511627776.0f);
                            const uint32_t db = __float_as_uint(delta);
                            my_max = db > my_max ? db : my_max;
                        } else {
                            const uint32_t old = a.val_cur[u];
                            const uint32_t nw = acc < old ? acc : old;
                            a.val_next[u] = nw;
                            if (nw < old) {
                                my_changed += 1;
                                if (old != kInf) {
                                    my_sum += old - nw;
                                    my_max = (old - nw) > my_max ? (old - nw) : my_max;
                                }
                                q_u[q_n] = u;
                                q_v[q_n] = nw;
                                ++q_n;
                            }
                        }
                    }
                    acc = A::id();
                    ++x;
                }
            }
        }

        // ---- frontier output (min applications) ----------------------------
        if constexpr (kMin && KIND != K_SAMPLE) {
            if (a.q_out) {
                const uint32_t incl = warp_incl_sum_u32((uint32_t)q_n);
                const uint32_t wtot = __shfl_sync(0xFFFFFFFFu, incl, 31);
                uint32_t base = 0;
                if (lane == 31 && wtot) base = atomicAdd(a.q_out_len, wtot);
                base = __shfl_sync(0xFFFFFFFFu, base, 31);
                const uint32_t pos = base + incl - (uint32_t)q_n;
                for (int i = 0; i < q_n; ++i) {
                    a.q_out[pos + i] = q_u[i];
                    a.q_out_val[pos + i] = q_v[i];
                }
            }
        }

        // ---- pass 3: flags to the bitmap, compaction of active arcs --------
        if constexpr (kCompact) {
            const uint32_t incl = warp_incl_sum_u32(my_active);
            if (lane == 31) sm.warp_c[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                uint32_t wc = lane < kWarps ? sm.warp_c[lane] : 0u;
                const uint32_t wincl = warp_incl_sum_u32(wc);
                const uint32_t tile_total = __shfl_sync(0xFFFFFFFFu, wincl, kWarps - 1);
                if (lane < kWarps) sm.warp_c[lane] = wincl - wc;
                if (lane == 0) {
                    st_release_u64(&a.st_count[t], pack_status(a.epoch, t == 0 ? 1u : 0u, tile_total));
                }
                uint32_t excl = 0;
                if (t > 0) excl = lookback_count(a.st_count, t, a.epoch, a.err);
                if (lane == 0) {
                    if (t > 0) st_release_u64(&a.st_count[t], pack_status(a.epoch, 1u, excl + tile_total));
                    sm.tile_excl = excl;
                    if (t == (int)num_tiles - 1) {
                        *a.sp_nnz = excl + tile_total;
                        if (a.stats) a.stats->active_after = excl + tile_total;
                    }
                    if (t == 0) a.sp_ptr[0] = 0;
                }
            }
            __syncthreads();
            uint32_t off = sm.tile_excl + sm.warp_c[warp] + incl - my_active;
            {
                int x = lx, y = ly;
                for (int i = 0; i < cnt; ++i) {
                    if (y < sm.rowend[x] - a0) {
                        if (sm.flag[y]) {
                            a.sp_src[off] = sm.src[y];
                            if (a.sp_w && has_w) a.sp_w[off] = sm.w[y];
                            ++off;
                        }
                        ++y;
                    } else {
                        a.sp_ptr[r0 + x + 1] = (int32_t)off;
                        ++x;
                    }
                }
            }
            if (narcs > 0) {
                const int w0 = a0 >> 5, w1 = (a1 - 1) >> 5;
                for (int w = w0 + tid; w <= w1; w += kThreads) {
                    const int lo = a0 > w * 32 ? a0 : w * 32;
                    const int hi = a1 < w * 32 + 32 ? a1 : w * 32 + 32;
                    uint32_t bits = 0;
                    for (int k = lo; k < hi; ++k) bits |= (uint32_t)sm.flag[k - a0] << (k & 31);
                    if (hi - lo == 32) {
                        a.mask[w] = bits;
                    } else {
                        const uint32_t range = ((1u << (hi - lo)) - 1u) << (lo & 31);
                        atomicAnd(&a.mask[w], ~range);
                        atomicOr(&a.mask[w], bits);
                    }
                }
            }
        }
    }

    // ---- statistics of this launch -----------------------------------------
    if constexpr (KIND != K_SAMPLE) {
        if (a.stats) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                my_changed += __shfl_xor_sync(0xFFFFFFFFu, my_changed, o);
                my_sum += __shfl_xor_sync(0xFFFFFFFFu, my_sum, o);
                const uint32_t om = __shfl_xor_sync(0xFFFFFFFFu, my_max, o);
                my_max = om > my_max ? om : my_max;
            }
            if (lane == 0 && (my_changed | my_sum | my_max)) {
                atomicAdd(&a.stats->changed, my_changed);
                atomicAdd(&a.stats->sum_delta, my_sum);
                atomicMax(&a.stats->max_delta_bits, my_max);
            }
        }
    }
    sched_leave(a.sched);
}

}  // namespace gg

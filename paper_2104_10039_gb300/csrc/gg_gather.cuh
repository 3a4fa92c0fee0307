// gg_gather.cuh - the arc-parallel tile kernels: the pull gather of
// approximate and accurate iterations (Alg. 1 / Alg. 2: GG-Gather over a row's
// flagged in-edges, GG-Apply, GG-VStatus) and the first launch of a correction
// iteration (the gather over all in-edges that stashes, for every arc, the
// running value before it: the "old" value of Alg. 2's influence).
//
// A warp tile covers kWT consecutive items of the merged sequence of arcs and
// row ends (the merge-path partition of the tile engine, with the same
// per-tile partials, so k_fixup completes the rows that began in an earlier
// tile and k_correct2 finds the carry of a continued row). Inside the tile
// the work is arc-parallel rather than item by item:
//   * sources are loaded coalesced (prefetched one tile ahead) and every
//     arc's value is fetched with one random load (or from the block's hub
//     cache) and staged in shared memory in arc order;
//   * every row ending in the tile marks its tile-local end position in a
//     257-bit "segment head" bitmap (a row's arcs are the positions from the
//     previous row's end up to its own end);
//   * lane L takes arcs 8L .. 8L+7 and folds them with a running sum (or
//     min) that restarts at every head; a warp segmented scan carries the
//     segment open at each lane's start;
//   * gather: the running value at the last arc of every segment replaces
//     that arc's staged value, so the row ending at position e reads its
//     total at e - 1, and the rows are applied one per lane, in row order;
//   * stash: the running value before every arc is staged next to its value
//     and both are stored with coalesced 8-byte stores.
#pragma once

#include "gg_tile.cuh"

namespace gg {

template <int APP, int KIND>
struct ArcSmem {
    static constexpr bool kApply = KIND == K_GATHER;
    int32_t end[kWT];                // tile-local arc position where each row of the tile ends
    uint32_t val[kPadded];           // arc values in arc order; gather: segment totals at segment ends
    uint32_t vtx[kApply ? kWT : 1];  // rows' current value; min applications: then the frontier values
    int32_t aux[kApply ? kWT : 1];   // PageRank: rows' out-degree; min applications: frontier vertices
    uint32_t bef[KIND == K_STASH ? kPadded : 1];   // stash: running value before each arc
    uint32_t head[kWT / 32 + 2];     // bit p: a row ends at arc position p (p = 0 .. kWT)
};

template <int APP, int KIND>
__global__ void __launch_bounds__(kThreads, 4)
k_arcs(TileArgs a)
{
    static_assert(KIND == K_GATHER || KIND == K_STASH, "gather or stash");
    using T = typename Acc<APP>::T;
    using A = Acc<APP>;
    constexpr bool kMin = APP != GG_APP_PAGERANK;
    constexpr bool kWeighted = APP == GG_APP_SSSP;
    constexpr bool kApply = KIND == K_GATHER;
    __shared__ ArcSmem<APP, KIND> smem[kWarps];
    ArcSmem<APP, KIND> &s = smem[threadIdx.x >> 5];
    // hub cache: the values of the most-read sources, one copy per block
    __shared__ uint32_t s_hub[kHubs];
    const int nh = a.n_hubs < kHubs ? a.n_hubs : kHubs;   // slots past these are read from global memory
    {
        for (int j = (int)threadIdx.x; j < nh; j += kThreads) {
            const int32_t v = a.hub_ids[j];
            if constexpr (APP == GG_APP_PAGERANK) s_hub[j] = __float_as_uint(__ldg(a.contrib_cur + v));
            else s_hub[j] = __ldg(a.val_cur + v);
        }
        __syncthreads();
    }

    const uint32_t lane = lane_id();
    const int gw = (int)((blockIdx.x * kThreads + threadIdx.x) >> 5);
    const int W = (int)((gridDim.x * kThreads) >> 5);
    const uint32_t nnz = *a.list_nnz;
    const int num_tiles = (int)*a.num_tiles;
    const long long total = (long long)a.n + nnz;
    const bool load_w = kWeighted && a.arc_w != nullptr;
    ApplyStats st;

    // ---- software pipeline: headers two tiles ahead, sources one ahead ------
    uint32_t hdr_cur = 0, hdr_nxt = 0;
    if (lane < 2 && gw < num_tiles) hdr_cur = (uint32_t)a.tile_info[gw + (int)lane];
    if (lane < 2 && gw + W < num_tiles) hdr_nxt = (uint32_t)a.tile_info[gw + W + (int)lane];
    int32_t src_cur[kIPT];
    uint32_t w_cur[kWeighted ? kIPT : 1];
    auto load_arcs = [&](int tt, uint32_t hdr, int32_t *srcv, uint32_t *wv) {
        const uint32_t h0 = __shfl_sync(0xFFFFFFFFu, hdr, 0), h1 = __shfl_sync(0xFFFFFFFFu, hdr, 1);
        const long long e0 = (long long)tt * kWT;
        const long long e1 = e0 + kWT < total ? e0 + kWT : total;
        const int32_t b0 = (int32_t)(e0 - (int32_t)(h0 & 0x7FFFFFFFu));
        const int32_t b1 = (int32_t)(e1 - (int32_t)(h1 & 0x7FFFFFFFu));
        const bool live = tt < num_tiles;
#pragma unroll
        for (int i = 0; i < kIPT; ++i) {
            const int k = (int)lane + 32 * i;
            const bool ok = live && k < b1 - b0;
            srcv[i] = ok ? __ldg(a.arc_src + b0 + k) : 0;
            if constexpr (kWeighted) wv[i] = (ok && load_w) ? __ldg(a.arc_w + b0 + k) : 1u;
        }
    };
    load_arcs(gw, hdr_cur, src_cur, w_cur);

    for (int t = gw; t < num_tiles; t += W) {
        const uint32_t i0 = __shfl_sync(0xFFFFFFFFu, hdr_cur, 0);
        const uint32_t i1 = __shfl_sync(0xFFFFFFFFu, hdr_cur, 1);
        const int32_t r0 = (int32_t)(i0 & 0x7FFFFFFFu), r1 = (int32_t)(i1 & 0x7FFFFFFFu);
        const bool need_carry = (i0 >> 31) != 0u;   // row r0 began in an earlier tile
        const long long d0 = (long long)t * kWT;
        const long long d1 = d0 + kWT < total ? d0 + kWT : total;
        const int32_t a0 = (int32_t)(d0 - r0), a1 = (int32_t)(d1 - r1);
        const int nrows = r1 - r0, narcs = a1 - a0;

        // ---- issue this tile's value reads (GG-Gather) -----------------------
        uint32_t gv[kIPT];
#pragma unroll
        for (int i = 0; i < kIPT; ++i) {
            const int k = (int)lane + 32 * i;
            const int32_t sv = src_cur[i];   // a hub is coded -(slot + 1)
            const int32_t hs = -sv - 1;
            const int32_t u = (sv < 0 && hs >= nh) ? __ldg(a.hub_ids + hs) : sv;
            if constexpr (APP == GG_APP_PAGERANK)
                gv[i] = k < narcs ? (u < 0 ? s_hub[hs] : __float_as_uint(__ldg(a.contrib_cur + u))) : 0u;
            else
                gv[i] = k < narcs ? (u < 0 ? s_hub[hs] : __ldg(a.val_cur + u)) : kInf;
        }
        if (lane < kWT / 32 + 2) s.head[lane] = 0u;
        __syncwarp();
        // ---- rows ending in the tile: end positions, heads (vertex data) ------
        for (int rb = 0; rb < nrows; rb += 32) {
            const int x = rb + (int)lane;
            int32_t e = 0;
            if (x < nrows) {
                e = a.row_ptr[r0 + x + 1] - a0;   // 0 <= e <= narcs
                s.end[x] = e;
                if constexpr (kApply) {
                    const int32_t v = a.row_vtx ? a.row_vtx[r0 + x] : r0 + x;
                    if constexpr (APP == GG_APP_PAGERANK) {
                        s.vtx[x] = __float_as_uint(a.rank_cur[v]);
                        s.aux[x] = a.deg_apply ? a.deg_apply[v] : a.out_ptr[v + 1] - a.out_ptr[v];
                    } else {
                        s.vtx[x] = a.val_cur[v];
                    }
                }
            }
            // head bits: the batch's ends do not decrease with x, so its words
            // run from the first lane's end to the last valid lane's; each word
            // is the OR over the lanes (no shared-memory atomics)
            const int last = nrows - 1 - rb < 31 ? nrows - 1 - rb : 31;
            const int wl = __shfl_sync(0xFFFFFFFFu, e, 0) >> 5, wh = __shfl_sync(0xFFFFFFFFu, e, last) >> 5;
            for (int w = wl; w <= wh; ++w) {
                const uint32_t word = __reduce_or_sync(0xFFFFFFFFu, (x < nrows && (e >> 5) == w) ? 1u << (e & 31) : 0u);
                if (lane == 0) s.head[w] |= word;
            }
        }
        // ---- prefetch: next tile's sources, header two tiles ahead ----------
        int32_t src_nxt[kIPT];
        uint32_t w_nxt[kWeighted ? kIPT : 1];
        load_arcs(t + W, hdr_nxt, src_nxt, w_nxt);
        uint32_t hdr_far = 0;
        if (lane < 2 && t + 2 * W < num_tiles) hdr_far = (uint32_t)a.tile_info[t + 2 * W + (int)lane];

        // ---- stage values (candidates for the min applications) in arc order --
#pragma unroll
        for (int i = 0; i < kIPT; ++i) {
            const int k = (int)lane + 32 * i;
            if (k < narcs) {
                uint32_t v = gv[i];
                if constexpr (kMin && APP != GG_APP_CC) {
                    const uint32_t step = (APP == GG_APP_BFS) ? 1u : w_cur[kWeighted ? i : 0];
                    const unsigned long long c = (unsigned long long)v + step;
                    v = (v == kInf || c >= kInf) ? kInf : (uint32_t)c;
                }
                s.val[pad(k)] = v;
            }
        }
        __syncwarp();

        // ---- lane L: arcs 8L .. 8L+7, running value restarting at each head ---
        const int p0 = (int)lane * kIPT;
        // heads at positions p0 .. p0 + 8 (bit j: a row ends at p0 + j)
        const uint32_t hw = (uint32_t)(((unsigned long long)s.head[(lane >> 2) + 1] << 32 | s.head[lane >> 2]) >>
                                       (8u * (lane & 3u))) & 0x1FFu;
        T run[kIPT];
        T r = A::id();
#pragma unroll
        for (int j = 0; j < kIPT; ++j) {
            const T v = p0 + j < narcs ? A::from_bits(s.val[pad(p0 + j)]) : A::id();
            r = ((hw >> j) & 1u) ? v : A::op(r, v);
            run[j] = r;
        }
        // the segment open at this lane's start, carried from the lanes before
        // (lane 0: the row open at the tile start begins from the identity; its
        // earlier part comes from the partials of the tiles before)
        T ex_v;
        {
            T v = r;
            uint32_t f = (hw & 0xFFu) != 0u;
            warp_seg_scan_incl<APP>(v, f);
            ex_v = __shfl_up_sync(0xFFFFFFFFu, v, 1);
            if (lane == 0) ex_v = A::id();
        }
        const uint32_t first = (hw & 0xFFu) ? (uint32_t)(__ffs(hw & 0xFFu) - 1) : 8u;   // first head in the lane
        if constexpr (KIND == K_GATHER) {
            // segment totals at segment ends (a head follows) and at the last arc
#pragma unroll
            for (int j = 0; j < kIPT; ++j) {
                const int p = p0 + j;
                if (p < narcs && (((hw >> (j + 1)) & 1u) || p == narcs - 1)) {
                    const T v = (uint32_t)j < first ? A::op(ex_v, run[j]) : run[j];
                    s.val[pad(p)] = A::bits(v);
                }
            }
        } else {
            // the running value before every arc
#pragma unroll
            for (int j = 0; j < kIPT; ++j) {
                const int p = p0 + j;
                if (p < narcs) {
                    T b = A::id();
                    if (!((hw >> j) & 1u)) {
                        if (j == 0) b = ex_v;
                        else b = (uint32_t)(j - 1) < first ? A::op(ex_v, run[j - 1]) : run[j - 1];
                    }
                    s.bef[pad(p)] = A::bits(b);
                }
            }
        }
        __syncwarp();
        // ---- tile partials (k_fixup, k_correct2): (has a row end, part after
        // the last end) and the part before the first end -----------------------
        if (lane == 0) {
            // running value at position p (its segment up to and including p)
            auto upto = [&](int p) -> T {
                if constexpr (KIND == K_GATHER) return A::from_bits(s.val[pad(p)]);
                else return A::op(A::from_bits(s.bef[pad(p)]), A::from_bits(s.val[pad(p)]));
            };
            T tail = A::id();
            if (narcs > 0 && !((s.head[narcs >> 5] >> (narcs & 31)) & 1u)) tail = upto(narcs - 1);
            T head_t = tail;
            if (nrows > 0) {
                const int e0 = s.end[0];
                head_t = e0 > 0 ? upto(e0 - 1) : A::id();
            }
            a.part[t] = make_uint2(nrows > 0 ? 1u : 0u, A::bits(tail));
            a.part_head[t] = A::bits(head_t);
        }

        if constexpr (KIND == K_STASH) {
#pragma unroll
            for (int i = 0; i < kIPT; ++i) {
                const int k = (int)lane + 32 * i;
                if (k < narcs) __stcs(a.stash + a0 + k, make_uint2(s.bef[pad(k)], s.val[pad(k)]));
            }
        } else {
            // ---- apply every row ending in the tile (GG-Apply, GG-VStatus) ---
            // min applications: the changed vertices are collected in shared
            // memory (entry q of the tile overwrites aux / vtx slot q <= its
            // row, read before) and appended to the frontier once per tile
            uint32_t q_n = 0;
            for (int rb = 0; rb < nrows; rb += 32) {
                const int x = rb + (int)lane;
                bool ch = false;
                int32_t u = 0;
                uint32_t nw = 0;
                if (x < nrows && !(x == 0 && need_carry)) {   // row r0 continued: k_fixup
                    const int32_t e = s.end[x];
                    const int32_t eb = x > 0 ? s.end[x - 1] : 0;
                    const T acc = e > eb ? A::from_bits(s.val[pad(e - 1)]) : A::id();
                    u = a.row_vtx ? a.row_vtx[r0 + x] : r0 + x;
                    if constexpr (APP == GG_APP_PAGERANK) {
                        apply_pr(a, u, acc, __uint_as_float(s.vtx[x]), s.aux[x], st);
                    } else {
                        nw = apply_min(a, u, acc, s.vtx[x], st, &ch);
                    }
                }
                if constexpr (kMin) {
                    const unsigned b = __ballot_sync(0xFFFFFFFFu, ch);
                    if (ch) {
                        const uint32_t q = q_n + __popc(b & ((1u << lane) - 1u));
                        s.aux[q] = u;
                        s.vtx[q] = nw;
                    }
                    q_n += __popc(b);
                }
            }
            if constexpr (kMin) {
                if (a.q_out && q_n) {
                    __syncwarp();
                    uint32_t base = 0;
                    if (lane == 0) base = atomicAdd(a.q_out_len, q_n);
                    base = __shfl_sync(0xFFFFFFFFu, base, 0);
                    for (uint32_t i = lane; i < q_n; i += 32) {
                        a.q_out[base + i] = s.aux[i];
                        a.q_out_val[base + i] = s.vtx[i];
                    }
                }
            }
        }
        __syncwarp();

        // ---- rotate the pipeline --------------------------------------------
        hdr_cur = hdr_nxt;
        hdr_nxt = hdr_far;
#pragma unroll
        for (int i = 0; i < kIPT; ++i) {
            src_cur[i] = src_nxt[i];
            if constexpr (kWeighted) w_cur[i] = w_nxt[i];
        }
    }
    if constexpr (kApply) flush_stats(a, st);
}

}  // namespace gg

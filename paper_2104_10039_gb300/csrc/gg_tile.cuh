// gg_tile.cuh - the merge-path tile engine: shared pieces of the tile
// kernels (value ops, warp scans, partial carries, the row apply), the
// second launches of a correction iteration (k_correct2, k_share) and the
// completion of rows split across tiles (k_fixup).
//
// A list (CSC rows: row_ptr + per-arc source/weight) is viewed as the merged
// sequence "arcs of row 0, end of row 0, arcs of row 1, end of row 1, ...".
// Warp tile t owns kWT consecutive items of that sequence; its first row (and
// whether that row began in an earlier tile) comes from a precomputed
// partition. Every warp works on its own tiles (t = warp, warp + W, ...) with
// no barrier and no wait on another warp, and loads the next tile's header
// and arc data while it works on the current one. Each tile publishes two
// partials: whether it holds a row end with the part of the row open at its
// end, and the part before its first row end.
// A row that began in an earlier tile needs those tiles' partials. The gather
// (k_arcs<., K_GATHER>, gg_gather.cuh) leaves that row to k_fixup. The
// correction, whose per-arc influence needs the running value before each arc
// (Alg. 2, GG-Gather's return), runs in two launches: k_arcs<., K_STASH>
// gathers the values, publishes the partials and stashes, for every arc in
// arc order, its value and the running value before it; k_correct2 then
// reads those pairs back with coalesced loads and takes its carry from the
// finished partials. The share influence, which needs whole rows first, runs
// k_share over the stashed values instead.
#pragma once

#include "gg_hash.cuh"
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

// Shared-memory slot of tile-local item k: one padding word per 8 items, so
// lanes reading their own 8 consecutive items hit distinct banks.
__device__ __forceinline__ int pad(int k) { return k + (k >> 3); }
constexpr int kPadded = kWT + kWT / 8 + 1;

// ------------------------------------------------------------ warp scans ----
template <int APP>
__device__ __forceinline__ void warp_seg_scan_incl(typename Acc<APP>::T &v, uint32_t &f)
{
    const uint32_t lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const typename Acc<APP>::T ov = __shfl_up_sync(0xFFFFFFFFu, v, o);
        const uint32_t of = __shfl_up_sync(0xFFFFFFFFu, f, o);
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
        const uint32_t ov = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= (uint32_t)o) v += ov;
    }
    return v;
}

// Carry of the row open at the start of tile t, from the finished partials of
// earlier tiles: the part after the last row end of the nearest tile with a
// row end, then every later tile whole, in tile order. Whole warp; valid in
// all lanes. `prev` is part[t-1], already loaded.
template <int APP>
__device__ __forceinline__ typename Acc<APP>::T carry_from_parts(const uint2 *part, int t, uint2 prev)
{
    using T = typename Acc<APP>::T;
    if (prev.x) return Acc<APP>::from_bits(prev.y);
    const uint32_t lane = lane_id();
    int jstar = 0;
    for (int base = t - 2; base >= 0; base -= 32) {
        const int j = base - (int)lane;
        const uint32_t f = j >= 0 ? part[j].x : 0u;
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, f != 0u);
        if (ball) {
            jstar = base - (__ffs(ball) - 1);
            break;
        }
    }
    T acc = Acc<APP>::id();
    for (int s0 = jstar; s0 < t; s0 += 32) {
        const int j = s0 + (int)lane;
        T v = j < t ? Acc<APP>::from_bits(part[j].y) : Acc<APP>::id();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = __shfl_down_sync(0xFFFFFFFFu, v, o);
            v = Acc<APP>::op(v, ov);
        }
        acc = Acc<APP>::op(acc, __shfl_sync(0xFFFFFFFFu, v, 0));
    }
    return acc;
}

// Later part of the row open at the end of tile t: the whole tiles after t
// without a row end, then the part before the first row end of the next tile
// that has one (from the finished partials, in tile order). Whole warp.
template <int APP>
__device__ __forceinline__ typename Acc<APP>::T lookahead_parts(const uint2 *part, const uint32_t *part_head,
                                                                int t, int num_tiles)
{
    using T = typename Acc<APP>::T;
    const uint32_t lane = lane_id();
    T acc = Acc<APP>::id();
    for (int s0 = t + 1; s0 < num_tiles; s0 += 32) {
        const int j = s0 + (int)lane;
        const uint32_t f = j < num_tiles ? part[j].x : 1u;
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, f != 0u);
        const int stop = ball ? __ffs(ball) - 1 : 32;
        T v = Acc<APP>::id();
        if ((int)lane < stop) v = Acc<APP>::from_bits(part[j].y);
        else if ((int)lane == stop && j < num_tiles) v = Acc<APP>::from_bits(part_head[j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = __shfl_down_sync(0xFFFFFFFFu, v, o);
            v = Acc<APP>::op(v, ov);
        }
        acc = Acc<APP>::op(acc, __shfl_sync(0xFFFFFFFFu, v, 0));
        if (ball) break;
    }
    return acc;
}

// ------------------------------------------------------------- row apply ----
// GG-Apply + GG-VStatus of Alg. 2 for PageRank; min for the min applications
// (a vertex is active when its value decreased). Shared by the gather, k_fixup,
// k_correct2 and k_share.
struct ApplyStats {
    unsigned long long changed = 0, sum = 0;
    uint32_t max = 0;
};

__device__ __forceinline__ void apply_pr(const TileArgs &a, int32_t u, float acc, float old, int deg,
                                         ApplyStats &st)
{
    const float nw = __fmaf_rn(a.damping, acc, a.base);
    const float delta = fabsf(__fsub_rn(nw, old));
    a.rank_next[u] = nw;
    a.contrib_next[u] = deg > 0 ? __fdiv_rn(nw, (float)deg) : 0.0f;
    if (a.hist_out) a.hist_out[u] = __fmul_rn(a.n_f, delta);
    st.changed += delta > a.epsilon ? 1ull : 0ull;
    st.sum += __float2ull_rz(delta * 1099511627776.0f);   // fixed point 2^-40
    const uint32_t db = __float_as_uint(delta);
    st.max = db > st.max ? db : st.max;
}

// Returns the new value; *changed tells whether it decreased.
__device__ __forceinline__ uint32_t apply_min(const TileArgs &a, int32_t u, uint32_t acc, uint32_t old,
                                              ApplyStats &st, bool *changed)
{
    const uint32_t nw = acc < old ? acc : old;
    a.val_next[u] = nw;
    *changed = nw < old;
    if (a.hist_out) a.hist_out[u] = nw < old ? 1.0f : 0.0f;
    if (nw < old) {
        st.changed += 1;
        if (old != kInf) {
            st.sum += old - nw;
            st.max = (old - nw) > st.max ? (old - nw) : st.max;
        }
    }
    return nw;
}

// Warp-aggregated append of this lane's (vertex, value) pairs to the frontier.
__device__ __forceinline__ void frontier_append(const TileArgs &a, const int32_t *qu, const uint32_t *qv, int qn)
{
    const uint32_t lane = lane_id();
    const uint32_t incl = warp_incl_sum_u32((uint32_t)qn);
    const uint32_t wtot = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (wtot == 0) return;
    uint32_t base = 0;
    if (lane == 31) base = atomicAdd(a.q_out_len, wtot);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    const uint32_t pos = base + incl - (uint32_t)qn;
    for (int i = 0; i < qn; ++i) {
        a.q_out[pos + i] = qu[i];
        a.q_out_val[pos + i] = qv[i];
    }
}

__device__ __forceinline__ void flush_stats(const TileArgs &a, ApplyStats st)
{
    if (!a.stats) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        st.changed += __shfl_xor_sync(0xFFFFFFFFu, st.changed, o);
        st.sum += __shfl_xor_sync(0xFFFFFFFFu, st.sum, o);
        const uint32_t om = __shfl_xor_sync(0xFFFFFFFFu, st.max, o);
        st.max = om > st.max ? om : st.max;
    }
    if (lane_id() == 0 && (st.changed | st.sum | st.max)) {
        atomicAdd(&a.stats->changed, st.changed);
        atomicAdd(&a.stats->sum_delta, st.sum);
        atomicMax(&a.stats->max_delta_bits, st.max);
    }
}

// ------------------------------------------------- share-influence pass ----
// The correction's second launch when a PageRank arc's influence is its share
// of the row total (GG_INFL_SHARE): the stashing gather has left every arc's
// value in the stash and the tile partials, so this pass walks the tile's
// merged items again (merge path: each lane takes kIPT consecutive items), adds
// up rows with a warp segmented scan, finds the total of every row in the tile
// (the row still open at the tile end adds the later tiles' partials), tests
// each arc's share against theta (GG-EStatus), applies the rows ending in the
// tile (GG-Apply, GG-VStatus) and writes the new flags (the pack recounts
// them).
struct ShareSmem {
    int32_t rowend[kWT + 1];
    uint32_t val[kPadded];      // arc values
    uint32_t vtx[kWT];          // rows' current rank
    int32_t deg[kWT];           // rows' out-degree
    uint32_t bits[kWT / 32 + 2];
    float rowtot[kWT + 1];      // row totals
};

template <int APP>
__global__ void __launch_bounds__(kThreads, 4)
k_share(TileArgs a)
{
    static_assert(APP == GG_APP_PAGERANK, "the share influence is PageRank's");
    using T = float;
    using A = Acc<GG_APP_PAGERANK>;
    __shared__ ShareSmem smem[kWarps];
    ShareSmem &s = smem[threadIdx.x >> 5];

    const uint32_t lane = lane_id();
    const int gw = (int)((blockIdx.x * kThreads + threadIdx.x) >> 5);
    const int W = (int)((gridDim.x * kThreads) >> 5);
    const uint32_t nnz = *a.list_nnz;
    const int num_tiles = (int)*a.num_tiles;
    const long long total = (long long)a.n + nnz;
    ApplyStats st;

    // ---- software pipeline: headers two tiles ahead, values one ahead -------
    uint32_t hdr_cur = 0, hdr_nxt = 0;
    if (lane < 2 && gw < num_tiles) hdr_cur = (uint32_t)a.tile_info[gw + (int)lane];
    if (lane < 2 && gw + W < num_tiles) hdr_nxt = (uint32_t)a.tile_info[gw + W + (int)lane];
    uint32_t v_cur[kIPT];
    auto load_vals = [&](int tt, uint32_t hdr, uint32_t *vv) {
        const uint32_t h0 = __shfl_sync(0xFFFFFFFFu, hdr, 0), h1 = __shfl_sync(0xFFFFFFFFu, hdr, 1);
        const long long e0 = (long long)tt * kWT;
        const long long e1 = e0 + kWT < total ? e0 + kWT : total;
        const int32_t b0 = (int32_t)(e0 - (int32_t)(h0 & 0x7FFFFFFFu));
        const int32_t b1 = (int32_t)(e1 - (int32_t)(h1 & 0x7FFFFFFFu));
        const bool live = tt < num_tiles;
#pragma unroll
        for (int i = 0; i < kIPT; ++i) {
            const int k = (int)lane + 32 * i;
            vv[i] = (live && k < b1 - b0) ? __ldcs(&a.stash[b0 + k].y) : 0u;
        }
    };
    load_vals(gw, hdr_cur, v_cur);

    for (int t = gw; t < num_tiles; t += W) {
        const uint32_t i0 = __shfl_sync(0xFFFFFFFFu, hdr_cur, 0);
        const uint32_t i1 = __shfl_sync(0xFFFFFFFFu, hdr_cur, 1);
        const int32_t r0 = (int32_t)(i0 & 0x7FFFFFFFu), r1 = (int32_t)(i1 & 0x7FFFFFFFu);
        const bool need_carry = (i0 >> 31) != 0u;
        const long long d0 = (long long)t * kWT;
        const long long d1 = d0 + kWT < total ? d0 + kWT : total;
        const int32_t a0 = (int32_t)(d0 - r0), a1 = (int32_t)(d1 - r1);
        const int nrows = r1 - r0, narcs = a1 - a0;
        const int w0 = a0 >> 5;
        const int nwords = narcs > 0 ? ((a1 - 1) >> 5) - w0 + 1 : 0;

        uint2 prev_part = make_uint2(1u, A::bits(A::id()));
        if (need_carry && lane == 0) prev_part = a.part[t - 1];
        for (int i = (int)lane; i < nrows; i += 32) {
            s.rowend[i] = a.row_ptr[r0 + i + 1];
            const int32_t v = a.row_vtx ? a.row_vtx[r0 + i] : r0 + i;
            s.vtx[i] = __float_as_uint(a.rank_cur[v]);
            s.deg[i] = a.deg_apply ? a.deg_apply[v] : a.out_ptr[v + 1] - a.out_ptr[v];
        }
        if (lane == 0) s.rowend[nrows] = 0x7FFFFFFF;   // row r1 stays open past the tile
        for (int i = (int)lane; i < nwords; i += 32) s.bits[i] = 0u;
        // ---- prefetch: next tile's values, header two tiles ahead ----------
        uint32_t v_nxt[kIPT];
        load_vals(t + W, hdr_nxt, v_nxt);
        uint32_t hdr_far = 0;
        if (lane < 2 && t + 2 * W < num_tiles) hdr_far = (uint32_t)a.tile_info[t + 2 * W + (int)lane];
#pragma unroll
        for (int i = 0; i < kIPT; ++i) {
            const int k = (int)lane + 32 * i;
            if (k < narcs) s.val[pad(k)] = v_cur[i];
        }
        __syncwarp();

        // ---- this lane's items into registers (merge-path search) ----------
        const int tile_items = (int)(d1 - d0);
        const int ld = (int)lane * kIPT < tile_items ? (int)lane * kIPT : tile_items;
        int cnt = tile_items - ld;
        cnt = cnt < kIPT ? cnt : kIPT;
        int lx, ly;
        {
            int lo = ld - narcs > 0 ? ld - narcs : 0;
            int hi = ld < nrows ? ld : nrows;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s.rowend[mid] - a0 <= ld - mid - 1) lo = mid + 1;
                else hi = mid;
            }
            lx = lo;
            ly = ld - lo;
        }
        uint32_t item_v[kIPT];
        uint32_t arcmask = 0;   // bit i: item i is an arc (else a row end)
        {
            int x = lx, y = ly;
#pragma unroll
            for (int i = 0; i < kIPT; ++i) {
                item_v[i] = 0;
                if (i < cnt) {
                    if (y < s.rowend[x] - a0) {
                        item_v[i] = s.val[pad(y)];
                        arcmask |= 1u << i;
                        ++y;
                    } else {
                        ++x;
                    }
                }
            }
        }
        const uint32_t endmask = ((1u << cnt) - 1u) & ~arcmask;

        // ---- fold + warp segmented scan; carry of the continued row ---------
        T carry_in;
        {
            T v = A::id();
            uint32_t f = 0;
#pragma unroll
            for (int i = 0; i < kIPT; ++i) {
                if ((arcmask >> i) & 1u) {
                    v = A::op(v, A::from_bits(item_v[i]));
                } else if ((endmask >> i) & 1u) {
                    f = 1u;
                    v = A::id();
                }
            }
            warp_seg_scan_incl<GG_APP_PAGERANK>(v, f);
            T ex_v = __shfl_up_sync(0xFFFFFFFFu, v, 1);
            uint32_t ex_f = __shfl_up_sync(0xFFFFFFFFu, f, 1);
            if (lane == 0) {
                ex_v = A::id();
                ex_f = 0u;
            }
            T c = A::id();
            if (need_carry) {
                prev_part.x = __shfl_sync(0xFFFFFFFFu, prev_part.x, 0);
                prev_part.y = __shfl_sync(0xFFFFFFFFu, prev_part.y, 0);
                c = carry_from_parts<GG_APP_PAGERANK>(a.part, t, prev_part);
            }
            carry_in = ex_f ? ex_v : A::op(c, ex_v);
        }

        // ---- row totals and the apply of every row ending in the tile --------
        T end_run;
        {
            T acc = carry_in;
            int x = lx;
#pragma unroll
            for (int i = 0; i < kIPT; ++i) {
                if ((arcmask >> i) & 1u) {
                    acc = A::op(acc, A::from_bits(item_v[i]));
                } else if ((endmask >> i) & 1u) {
                    s.rowtot[x] = acc;
                    const int32_t u = a.row_vtx ? a.row_vtx[r0 + x] : r0 + x;
                    apply_pr(a, u, acc, __uint_as_float(s.vtx[x]), s.deg[x], st);
                    acc = A::id();
                    ++x;
                }
            }
            end_run = acc;
        }
        // the row still open at the tile end: the later tiles' parts
        {
            const int last = (tile_items - 1) / kIPT;
            const float tail_run = __shfl_sync(0xFFFFFFFFu, end_run, last);
            const float later = lookahead_parts<GG_APP_PAGERANK>(a.part, a.part_head, t, num_tiles);
            if (lane == 0) s.rowtot[nrows] = __fadd_rn(tail_run, later);
        }
        __syncwarp();
        // ---- flags: share c / total > theta, tested as c > theta * total -----
        uint32_t my_flags = 0;
        {
            int x = lx;
#pragma unroll
            for (int i = 0; i < kIPT; ++i) {
                if ((arcmask >> i) & 1u) {
                    const float tot = s.rowtot[x];
                    const bool hit = tot != 0.0f ? __uint_as_float(item_v[i]) > __fmul_rn(a.theta, tot)
                                                 : 0.0f > a.theta;
                    my_flags |= (hit ? 1u : 0u) << i;
                } else if ((endmask >> i) & 1u) {
                    ++x;
                }
            }
        }

        // ---- new flags into the bitmap ----------------------------------------
        {
            // this lane's arcs are the consecutive list positions a0+ly ..,
            // so its flags form one run of at most kIPT bits: at most two
            // shared-memory ORs per lane
            uint32_t run = 0;
            int na = 0;
#pragma unroll
            for (int i = 0; i < kIPT; ++i) {
                if ((arcmask >> i) & 1u) {
                    if ((my_flags >> i) & 1u) run |= 1u << na;
                    ++na;
                }
            }
            if (run) {
                const int k0 = a0 + ly;
                const int sh = k0 & 31, wi = (k0 >> 5) - w0;
                atomicOr(&s.bits[wi], run << sh);
                if (sh + na > 32) atomicOr(&s.bits[wi + 1], run >> (32 - sh));
            }
        }
        __syncwarp();
        for (int i = (int)lane; i < nwords; i += 32) {
            const int w = w0 + i;
            const int lo = a0 > w * 32 ? a0 : w * 32;
            const int hi = a1 < w * 32 + 32 ? a1 : w * 32 + 32;
            const uint32_t bits = s.bits[i];
            if (hi - lo == 32) {
                a.mask[w] = bits;
            } else {
                const uint32_t range = ((1u << (hi - lo)) - 1u) << (lo & 31);
                atomicAnd(&a.mask[w], ~range);
                atomicOr(&a.mask[w], bits);
            }
        }
        __syncwarp();

        // ---- rotate the pipeline --------------------------------------------
        hdr_cur = hdr_nxt;
        hdr_nxt = hdr_far;
#pragma unroll
        for (int i = 0; i < kIPT; ++i) v_cur[i] = v_nxt[i];
    }
    flush_stats(a, st);
}

// ----------------------------------------------------------------- fixup ----
// Rows of a gather that began in an earlier tile and end in tile t: their
// value is the partials of the tiles from the one where the row began up to
// t-1, then tile t's part before its first row end, added in tile order.
// One thread per tile (warp-uniform loop); runs after k_arcs<., K_GATHER>.
template <int APP>
__global__ void __launch_bounds__(kThreads)
k_fixup(TileArgs a)
{
    using T = typename Acc<APP>::T;
    using A = Acc<APP>;
    constexpr bool kMin = APP != GG_APP_PAGERANK;
    const long long num_tiles = (long long)*a.num_tiles;
    const uint32_t lane = lane_id();
    ApplyStats st;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long wb = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); wb < num_tiles; wb += stride) {
        const long long t = wb + lane;
        int32_t qu[1];
        uint32_t qv[1];
        int qn = 0;
        if (t < num_tiles) {
            const uint32_t info = (uint32_t)a.tile_info[t];
            const uint2 me = a.part[t];
            if ((info >> 31) && me.x) {
                // row r began after the end of row r - 1, the item at merged
                // index row_ptr[r] + r - 1: its tile j is the nearest earlier
                // tile with a row end, and the tiles between hold only row r
                const int32_t r = (int32_t)(info & 0x7FFFFFFFu);
                const long long j = r > 0 ? ((long long)a.row_ptr[r] + r - 1) / kWT : 0;
                T acc = A::from_bits(a.part[j].y);
                for (long long k = j + 1; k < t; ++k) acc = A::op(acc, A::from_bits(a.part[k].y));
                acc = A::op(acc, A::from_bits(a.part_head[t]));
                const int32_t u = a.row_vtx ? a.row_vtx[r] : r;
                if constexpr (APP == GG_APP_PAGERANK) {
                    apply_pr(a, u, acc, a.rank_cur[u],
                             a.deg_apply ? a.deg_apply[u] : a.out_ptr[u + 1] - a.out_ptr[u], st);
                } else {
                    bool ch;
                    const uint32_t nw = apply_min(a, u, acc, a.val_cur[u], st, &ch);
                    if (ch) {
                        qu[0] = u;
                        qv[0] = nw;
                        qn = 1;
                    }
                }
            }
        }
        if constexpr (kMin) {
            if (a.q_out) frontier_append(a, qu, qv, qn);
        }
    }
    flush_stats(a, st);
}


// ------------------------------------------------------ correction, pass 2 --
// The correction's second launch when the influence is the running-prefix
// form: k_arcs<., K_STASH> left, for every arc, the running value before it
// within its tile and its value, so no merge path or scan is needed here. Per
// warp tile: the carry of the row continued from earlier tiles (the finished
// partials), each arc's influence test (Alg. 2 GG-EStatus) from (carry +) its
// running values, the new flag words, every row ending in the tile applied
// (GG-Apply, GG-VStatus); the pack recounts the flags. The stash pairs, the
// ends of the tile's first 32 rows and the old flag words are loaded one tile
// ahead; the pairs are also staged in shared memory, where a row finds its
// total (the pair at its last arc); the first 32 rows' vertex data are
// requested before the flag work.
template <int APP>
__global__ void __launch_bounds__(kThreads, 4)
k_correct2(TileArgs a)
{
    using T = typename Acc<APP>::T;
    using A = Acc<APP>;
    constexpr bool kMin = APP != GG_APP_PAGERANK;
    constexpr int kW = kWT / 32 + 2;
    __shared__ uint32_t s_bits[kWarps][kW];
    __shared__ uint32_t s_old[kWarps][kMin ? kW : 1];
    __shared__ uint2 s_pair[kWarps][kWT];
    const int wi = (int)(threadIdx.x >> 5);
    uint32_t *bits = s_bits[wi], *oldw = s_old[wi];
    uint2 *pair = s_pair[wi];
    const uint32_t lane = lane_id();
    const int gw = (int)((blockIdx.x * kThreads + threadIdx.x) >> 5);
    const int W = (int)((gridDim.x * kThreads) >> 5);
    const uint32_t nnz = *a.list_nnz;
    const int num_tiles = (int)*a.num_tiles;
    const long long total = (long long)a.n + nnz;
    ApplyStats st;
    // software pipeline: headers two tiles ahead; the stash pairs, the ends of
    // the first 32 rows and (min applications) the old flag words one ahead
    auto load_tile = [&](int tt, uint32_t hdr, uint2 *pv, int32_t &re, uint32_t &ow) {
        const uint32_t h0 = __shfl_sync(0xFFFFFFFFu, hdr, 0), h1 = __shfl_sync(0xFFFFFFFFu, hdr, 1);
        const int32_t q0 = (int32_t)(h0 & 0x7FFFFFFFu), q1 = (int32_t)(h1 & 0x7FFFFFFFu);
        const long long e0 = (long long)tt * kWT;
        const long long e1 = e0 + kWT < total ? e0 + kWT : total;
        const int32_t b0 = (int32_t)(e0 - q0);
        const int32_t b1 = (int32_t)(e1 - q1);
        const bool live = tt < num_tiles;
#pragma unroll
        for (int j = 0; j < kIPT; ++j) {
            const int k = (int)lane + 32 * j;
            pv[j] = (live && k < b1 - b0) ? __ldcs(a.stash + b0 + k) : make_uint2(0u, 0u);
        }
        re = (live && (int)lane < q1 - q0) ? a.row_ptr[q0 + (int)lane + 1] : 0;
        if constexpr (kMin) {
            const int nw = (live && b1 > b0) ? ((b1 - 1) >> 5) - (b0 >> 5) + 1 : 0;
            ow = (int)lane < nw ? a.mask[(b0 >> 5) + (int)lane] : 0u;
        }
    };
    uint32_t hdr_cur = 0, hdr_nxt = 0;
    if (lane < 2 && gw < num_tiles) hdr_cur = (uint32_t)a.tile_info[gw + (int)lane];
    if (lane < 2 && gw + W < num_tiles) hdr_nxt = (uint32_t)a.tile_info[gw + W + (int)lane];
    uint2 pv_cur[kIPT];
    int32_t re_cur = 0;
    uint32_t ow_cur = 0;
    load_tile(gw, hdr_cur, pv_cur, re_cur, ow_cur);
    for (int t = gw; t < num_tiles; t += W) {
        const uint32_t i0 = __shfl_sync(0xFFFFFFFFu, hdr_cur, 0), i1 = __shfl_sync(0xFFFFFFFFu, hdr_cur, 1);
        const int32_t r0 = (int32_t)(i0 & 0x7FFFFFFFu), r1 = (int32_t)(i1 & 0x7FFFFFFFu);
        const bool need_carry = (i0 >> 31) != 0u;
        const long long d0 = (long long)t * kWT;
        const long long d1 = d0 + kWT < total ? d0 + kWT : total;
        const int32_t a0 = (int32_t)(d0 - r0), a1 = (int32_t)(d1 - r1);
        const int nrows = r1 - r0, narcs = a1 - a0;
        const int w0 = a0 >> 5;
        const int nwords = narcs > 0 ? ((a1 - 1) >> 5) - w0 + 1 : 0;
        // vertex data of the tile's first 32 rows, requested before the flag work
        int32_t u_first = 0;
        uint32_t old_first = 0;
        int32_t deg_first = 0;
        if ((int)lane < nrows) {
            u_first = a.row_vtx ? a.row_vtx[r0 + (int)lane] : r0 + (int)lane;
            if constexpr (APP == GG_APP_PAGERANK) {
                old_first = __float_as_uint(a.rank_cur[u_first]);
                deg_first = a.deg_apply ? a.deg_apply[u_first] : a.out_ptr[u_first + 1] - a.out_ptr[u_first];
            } else {
                old_first = a.val_cur[u_first];
            }
        }
        // the row continued from earlier tiles: its carry and its arcs here
        T c = A::id();
        int32_t first_end = a0;
        if (need_carry) {
            uint2 prev = make_uint2(0u, 0u);
            if (lane == 0) prev = a.part[t - 1];
            prev.x = __shfl_sync(0xFFFFFFFFu, prev.x, 0);
            prev.y = __shfl_sync(0xFFFFFFFFu, prev.y, 0);
            c = carry_from_parts<APP>(a.part, t, prev);
            // row r0's end, or past the tile when the tile holds no row end
            const int32_t e = __shfl_sync(0xFFFFFFFFu, re_cur, 0);
            first_end = (nrows > 0 && e < a1) ? e : a1;
        }
        if ((int)lane < nwords) {   // nwords <= kWT / 32 + 1
            bits[lane] = 0u;
            if constexpr (kMin) oldw[lane] = ow_cur;
        }
        uint2 pv_nxt[kIPT];
        int32_t re_nxt;
        uint32_t ow_nxt = 0;
        load_tile(t + W, hdr_nxt, pv_nxt, re_nxt, ow_nxt);
        uint32_t hdr_far = 0;
        if (lane < 2 && t + 2 * W < num_tiles) hdr_far = (uint32_t)a.tile_info[t + 2 * W + (int)lane];
        __syncwarp();
        // ---- flags: arcs a0 + lane + 32 j (coalesced), one ballot per 32 ----
        uint32_t active = 0;
#pragma unroll
        for (int j = 0; j < kIPT; ++j) {
            const int k = (int)lane + 32 * j;
            const int32_t p = a0 + k;
            uint32_t fl = 0;
            if (k < narcs) {
                const uint2 sv = pv_cur[j];
                pair[k] = sv;
                T before = A::from_bits(sv.x);
                const T v = A::from_bits(sv.y);
                if (p < first_end) before = A::op(c, before);
                if constexpr (APP == GG_APP_PAGERANK) {
                    // Alg. 2: influence (new - old) / new > theta, as (new - old) > theta * new
                    const float after = __fadd_rn(before, v);
                    fl = (after != 0.0f ? __fsub_rn(after, before) > __fmul_rn(a.theta, after) : 0.0f > a.theta)
                             ? 1u : 0u;
                } else {
                    if (v == kInf) {   // no candidate: the arc keeps its flag
                        fl = a.est_strict ? 0u : (oldw[(p >> 5) - w0] >> (p & 31)) & 1u;
                    } else if (a.theta_case == 1) {
                        fl = 1u;
                    } else if (a.theta_case == 2) {
                        fl = 0u;
                    } else if (v < before) {
                        if (before == kInf || APP == GG_APP_CC) fl = 1u;
                        else fl = ((unsigned long long)(before - v) << 32) > a.theta_fx * (unsigned long long)before
                                      ? 1u : 0u;
                    }
                }
            }
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, fl != 0u);
            active += __popc(b);
            if (lane == 0 && b) {
                const int q = a0 + 32 * j;   // position of lane 0's arc
                const int sh = q & 31, wq = (q >> 5) - w0;
                bits[wq] |= b << sh;
                if (sh) bits[wq + 1] |= b >> (32 - sh);
            }
        }
        __syncwarp();
        __syncwarp();
        // ---- rows ending in this tile: apply ---------------------------------
        int32_t prev_e = a0;   // where the batch's first row starts (row r0: the tile start)
        for (int rb = 0; rb < nrows; rb += 32) {
            const int ri = rb + (int)lane;
            int32_t e = 0;
            if (ri < nrows) e = rb == 0 ? re_cur : a.row_ptr[r0 + ri + 1];   // the row's arcs end before e
            int32_t start = __shfl_up_sync(0xFFFFFFFFu, e, 1);
            if (lane == 0) start = prev_e;
            prev_e = __shfl_sync(0xFFFFFFFFu, e, 31);
            int32_t qu[1];
            uint32_t qv[1];
            int qn = 0;
            if (ri < nrows) {
                const int32_t r = r0 + ri;
                // the row's total: the running value after its last arc when
                // that arc lies in this tile (plus the carry for the continued
                // row), else the carry (continued row ending at the tile start)
                // or nothing (a row without arcs)
                const bool continued = ri == 0 && need_carry;
                T tot = continued ? c : A::id();
                if (e > start) {
                    const uint2 sv = pair[e - 1 - a0];
                    tot = A::op(A::from_bits(sv.x), A::from_bits(sv.y));
                    if (continued) tot = A::op(c, tot);
                }
                int32_t u = u_first;
                uint32_t old = old_first;
                int32_t deg = deg_first;
                if (rb > 0) {
                    u = a.row_vtx ? a.row_vtx[r] : r;
                    if constexpr (APP == GG_APP_PAGERANK) {
                        old = __float_as_uint(a.rank_cur[u]);
                        deg = a.deg_apply ? a.deg_apply[u] : a.out_ptr[u + 1] - a.out_ptr[u];
                    } else {
                        old = a.val_cur[u];
                    }
                }
                if constexpr (APP == GG_APP_PAGERANK) {
                    apply_pr(a, u, tot, __uint_as_float(old), deg, st);
                } else {
                    bool ch;
                    const uint32_t nw = apply_min(a, u, tot, old, st, &ch);
                    if (ch) {
                        qu[0] = u;
                        qv[0] = nw;
                        qn = 1;
                    }
                }
            }
            if constexpr (kMin) {
                if (a.q_out) frontier_append(a, qu, qv, qn);
            }
        }
        // ---- flag words: plain stores where the tile owns the word ----------
        for (int i = (int)lane; i < nwords; i += 32) {
            const int w = w0 + i;
            const int lo = a0 > w * 32 ? a0 : w * 32;
            const int hi = a1 < w * 32 + 32 ? a1 : w * 32 + 32;
            if (hi - lo == 32) {
                a.mask[w] = bits[i];
            } else {
                const uint32_t range = ((1u << (hi - lo)) - 1u) << (lo & 31);
                atomicAnd(&a.mask[w], ~range);
                atomicOr(&a.mask[w], bits[i]);
            }
        }
        __syncwarp();
        hdr_cur = hdr_nxt;
        hdr_nxt = hdr_far;
        re_cur = re_nxt;
        ow_cur = ow_nxt;
#pragma unroll
        for (int j = 0; j < kIPT; ++j) pv_cur[j] = pv_nxt[j];
    }
    flush_stats(a, st);
}

}  // namespace gg

// gg_internal.cuh - shared definitions of the libgg CUDA sources (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "gg.h"

namespace gg {

// ---------------------------------------------------------------- tiling ----
// Every gather-type kernel walks a merged list of row ends and arcs
// ("merge path", Merrill & Garland 2016) cut into warp tiles of kWT items
// (kIPT per lane), so a tile costs the same whatever the degree skew.
constexpr int kThreads = 256;
constexpr int kIPT = 8;
constexpr int kWT = 32 * kIPT;
constexpr int kTile = kThreads * kIPT;   // push-frontier tiles (block-wide)
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kInf = 0xFFFFFFFFu;
// Hub coding: the (at most) kHubCodes sources with the most out-arcs are
// coded -(slot + 1) in in_src_h, slots in two tiers (the kHubs with the most
// out-arcs first). The PageRank pull gathers read a hub's contribution from
// a dense per-launch copy (64 KB, L1-resident); the merge-path kernels keep
// the first kHubs slots in each block's shared memory. The pull gathers of
// SSSP / BFS / CC read plain ids: with the hub copy they ran slower.
constexpr int kHubs = 3072;   // 12 KB: 4 blocks of the merge-path gather still fit an SM
constexpr int kHubCodes = 16384;

// Device error flags (the graph's error word; k_validate sets them).
enum DevErr : uint32_t {
    DEVERR_BAD_GRAPH = 2u,
};

// Per-launch dynamic tile scheduler. Tiles are handed out in increasing order
// by an atomic counter; the last block to leave resets both counters for the
// next launch.
struct TileSched {
    uint32_t next_tile;
    uint32_t done_blocks;
};

// Per-iteration statistics as the kernels accumulate them (same layout as
// gg_iter_stats).
struct IterStatsDev {
    uint32_t mode;
    uint32_t max_delta_bits;
    unsigned long long arcs;
    unsigned long long changed;
    unsigned long long sum_delta;
    unsigned long long active_after;
    unsigned long long selected;
};
static_assert(sizeof(IterStatsDev) == sizeof(gg_iter_stats), "stats layout");

// Arguments of the tile kernels (one struct for every kind; unused fields are
// ignored by a given instantiation).
struct TileArgs {
    // the list being walked: CSC rows (full, or packed active in-edges)
    const int32_t *row_ptr;     // n+1
    const int32_t *arc_src;     // list arcs: source vertex
    const uint32_t *arc_w;      // list arcs: weight (SSSP) or nullptr
    int32_t n;
    const uint32_t *list_nnz;   // device scalar: arcs in the list
    const int32_t *tile_info;   // per tile: rows before it | (row open at its start began earlier) << 31
    const uint32_t *num_tiles;  // device scalar
    // vertex state
    const float *contrib_cur;
    const float *rank_cur;
    float *rank_next;
    float *contrib_next;
    const int32_t *out_ptr;     // CSR row pointers (full out-degree)
    const uint32_t *val_cur;
    uint32_t *val_next;
    float base;                 // (1-d)/N
    float damping;
    float epsilon;
    const int32_t *deg_apply;   // degrees for the next contributions (renormalised), or nullptr = out-degree
    int infl_share;             // PageRank corrections: influence = share of the row total
    // flags (correction)
    uint32_t *mask;             // CSC-order bitmap
    float theta;
    unsigned long long theta_fx;
    int theta_case;             // 0 compare, 1 theta < 0, 2 theta >= 1
    int est_strict;
    // per-tile partials of a gather for k_fixup: (has row end, part after the
    // last end) and the part before the first end
    uint2 *part;
    uint32_t *part_head;
    // correction: per arc in list order, written by k_arcs<., K_STASH>: the row's running
    // value before the arc within its tile (rows continued from an earlier
    // tile start from the identity there) and the arc's value (candidate)
    uint2 *stash;
    // set by the host, not read by the current kernels
    unsigned long long *st_carry;
    uint32_t epoch;
    uint32_t *err;
    // statistics and frontier output
    IterStatsDev *stats;
    int32_t *q_out;
    uint32_t *q_out_val;
    uint32_t *q_out_len;
    // learned correction: the vertex of every list row (nullptr: row = vertex),
    // and the change feature of every applied vertex (nullptr: not kept)
    const int32_t *row_vtx;
    float *hist_out;
    float n_f;                  // vertex count (PageRank change feature = n |old - new|)
    // hub cache: vertex of every slot, and the number of slots in use
    const int32_t *hub_ids;
    int32_t n_hubs;
};

// K_GATHER: approximate / accurate pull iteration (k_arcs<., K_GATHER>).
// K_CORRECT: a correction iteration as the launchers take it, run as
// k_arcs<., K_STASH> then k_correct2 (or k_share for the share influence).
enum TileKind { K_GATHER = 0, K_CORRECT = 1, K_STASH = 2 };

// The PageRank pull path (gg_pull.cu): a list (sources as vertex ids), its
// plan, and the vertex state of one iteration.
struct PullArgs {
    const int32_t *src;         // list arcs: source vertex (PageRank: hubs coded -(slot + 1))
    const int32_t *row_ptr;     // list row pointers (n + 1)
    const uint32_t *nnz;        // device scalar: arcs in the list
    const uint32_t *hb;         // plan: row-start bit per arc
    const int32_t *trow;        // plan: per tile, non-empty-row rank of the row holding its first arc
    const int32_t *nzv;         // plan: vertex of each non-empty row
    const int2 *topen;          // plan: per tile, the row open at its start: vertex, its first tile | long << 31
    const int32_t *lrows;       // plan: the long rows (vertices)
    const uint32_t *nlong;      // plan: device scalar, number of long rows
    float *carry;               // correction: per tile inside a long row, the row's value before the tile
    uint32_t *tcnt;             // correction: per tile, its arcs flagged active (for the pack)
    const float *contrib;       // gathered vector (rank / degree of the previous iteration)
    float *acc;                 // per vertex: its row's sum over the tile holding the row's first arc
    float *lead;                // per tile: the part before its first row start
    float *vals;                // correction: every arc's value (contribution / candidate), in list order
    uint32_t *mask;             // correction: the flag bitmap of the list (old flags in, new flags out)
    float theta;                // PageRank correction threshold
    int theta_case;             // SSSP / BFS / CC correction: 0 compare, 1 theta < 0, 2 theta >= 1
    unsigned long long theta_fx;   // ... floor(theta 2^32)
    int est_strict;             // ... arcs without a candidate lose their flag
    const uint32_t *w;          // SSSP: list arcs' weights, or nullptr (weight 1)
    const uint32_t *front;      // SSSP / BFS / CC gathers: bitmap of the frontier (bit v: v changed in the
                                // previous iteration); only its vertices' arcs are read. nullptr: every arc
    const int32_t *hub_ids;     // PageRank: vertex of each hub slot (sources coded -(slot + 1) in src)
    int32_t n_hubs;
    uint32_t *hubv;             // ... the contribution of each hub slot (k_hub_values, per launch)
    const uint32_t *val_cur;    // SSSP / BFS / CC values
    uint32_t *val_next;
    int32_t *q_out;             // SSSP / BFS / CC: next frontier (vertex, value), length
    uint32_t *q_out_val;
    uint32_t *q_out_len;
    int32_t n;
    const float *rank_cur;
    float *rank_next;
    float *contrib_next;
    const int32_t *out_ptr;     // CSR row pointers (full out-degree)
    const int32_t *deg_apply;   // degrees for the next contributions (renormalised), or nullptr
    float base;                 // (1-d)/N
    float damping;
    float epsilon;
    float n_f;
    float *hist_out;            // change feature of every vertex (learned policy / traces), or nullptr
    IterStatsDev *stats;
};

// Inputs of the learned correction's vertex features.
struct FeatArgs {
    int32_t n;
    const int32_t *in_ptr;
    const int32_t *out_ptr;
    const int32_t *sp_ptr;      // packed active in-edges (current flags)
    const float *hist1;         // change features of the last three executed iterations, newest first
    const float *hist2;
    const float *hist3;
    float iter_f;               // iteration / 64
    float app_f;                // application id
};

struct PushArgs {
    const int32_t *q;           // frontier vertices
    const uint32_t *q_val;      // their values at the end of the previous iteration
    const uint32_t *q_len;      // device scalar
    const uint32_t *q_deg_ex;   // exclusive prefix of their out-degrees (q_len + 1)
    const int32_t *out_ptr;
    const int32_t *out_dst;
    const uint32_t *out_w;
    const int32_t *out_to_in;
    const uint32_t *mask;       // nullptr: accurate mode (every arc)
    uint32_t *val;              // relaxed in place (atomicMin)
    uint32_t *stamp;
    uint32_t stamp_tag;
    int32_t *q_out;
    uint32_t *q_out_len;
    TileSched *sched;
    uint32_t *err;
    int app;
};

// ------------------------------------------------------- device helpers ----
#ifdef __CUDACC__
// Fetch the next tile of a launch (block-uniform); returns -1 when exhausted.
__device__ __forceinline__ int next_tile(TileSched *s, uint32_t num_tiles, int *s_slot)
{
    __syncthreads();
    if (threadIdx.x == 0) *s_slot = (int)atomicAdd(&s->next_tile, 1u);
    __syncthreads();
    int t = *s_slot;
    return (uint32_t)t < num_tiles ? t : -1;
}

// Called by every block once it has left its tile loop.
__device__ __forceinline__ void sched_leave(TileSched *s)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        uint32_t done = atomicAdd(&s->done_blocks, 1u);
        if (done == gridDim.x - 1) {
            s->next_tile = 0;
            s->done_blocks = 0;
            __threadfence();
        }
    }
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
#endif

// ------------------------------------------------------------ host side ----
void set_error(const char *fmt, ...);
gg_status cuda_fail(cudaError_t e, const char *what);

#define GG_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Launchers (each defined in its own translation unit).
struct Graph;
cudaError_t launch_partition(const int32_t *row_ptr, int32_t n, const uint32_t *list_nnz,
                             uint32_t max_tiles, int32_t *tile_info, uint32_t *num_tiles,
                             cudaStream_t s);
// Tile kernels run a persistent grid: min(max_tiles, resident warps).
cudaError_t launch_tile_pr(int kind, const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s);
cudaError_t launch_tile_min(int app, int kind, const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s);
// Sampling (Sec. 3.4): the flag of every arc of the full in-edge list from
// the hash of its endpoints (in_dst: each arc's row).
cudaError_t launch_sample(const int32_t *in_src, const int32_t *in_dst, long long m, int symmetric,
                          unsigned long long seed, unsigned long long thr, uint32_t *mask, int num_sms,
                          cudaStream_t s);
// Rows a gather left open at tile starts (one launch after every gather).
cudaError_t launch_fixup(int app, const TileArgs &a, int max_tiles, int num_sms, cudaStream_t s);
cudaError_t launch_push(const PushArgs &a, uint32_t max_arcs, int grid, cudaStream_t s);
cudaError_t launch_scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *tmp, cudaStream_t s);
size_t scan_tmp_words(size_t n);
// What the host reads about a frontier after an iteration, in one copy: the
// out-arcs of its vertices, its length, and the packed list's arc count.
struct FrontSum {
    unsigned long long arcs;
    uint32_t len;
    uint32_t nnz;
};
cudaError_t launch_qdeg(const int32_t *q, const uint32_t *q_len, const int32_t *out_ptr, uint32_t *deg,
                        FrontSum *sum, const uint32_t *nnz, uint32_t max_n, int num_sms, cudaStream_t s);
cudaError_t launch_snapshot(const int32_t *q, const uint32_t *q_len, const uint32_t *val, uint32_t *q_val,
                            float *hist, uint32_t max_n, int num_sms, cudaStream_t s);
cudaError_t launch_init_pr(int32_t n, const int32_t *out_ptr, float *rank, float *contrib, int num_sms,
                           cudaStream_t s);
cudaError_t launch_init_min(int32_t n, int app, int32_t source, uint32_t *val, int32_t *q, uint32_t *q_val,
                            uint32_t *q_len, int num_sms, cudaStream_t s);
cudaError_t launch_iter_header(IterStatsDev *st, uint32_t mode, const uint32_t *arcs_dev,
                               unsigned long long arcs, cudaStream_t s, unsigned long long selected = 0);
cudaError_t launch_append_frontier(const int32_t *q_src, uint32_t len, const float *hist_now, const uint32_t *val,
                                   int32_t *q_dst, uint32_t *q_dst_val, uint32_t *q_dst_len, int num_sms,
                                   cudaStream_t s);
cudaError_t launch_iter_changed(IterStatsDev *st, const uint32_t *q_len, cudaStream_t s);
// Active out-degree of every vertex from the packed active in-edges.
cudaError_t launch_active_outdeg(const int32_t *sp_src, const uint32_t *sp_nnz, uint32_t max_arcs, int32_t n,
                                 const int32_t *hub_ids, int32_t *act, int num_sms, cudaStream_t s);
// Source ids of a hub-coded list back to vertex ids (count read on the device).
cudaError_t launch_decode_src(const int32_t *coded, const uint32_t *count, uint32_t max_count, const int32_t *hub_ids,
                              int32_t *out, int num_sms, cudaStream_t s);
// Pull iteration of an application (gg_pull.cu): arcs, then apply; with
// `correct`, arcs (values kept), influence and flags, then apply.
cudaError_t launch_front_bits(const int32_t *q, const uint32_t *q_len, uint32_t *bits, int32_t n, int num_sms,
                              cudaStream_t s);
cudaError_t launch_pull(int app, const PullArgs &a, bool correct, uint32_t max_tiles, int num_sms, cudaStream_t s);
// contrib[u] = rank[u] / deg[u], or / the full out-degree when deg is null (0 when the degree is 0).
cudaError_t launch_contrib(int32_t n, const float *rank, const int32_t *deg, const int32_t *out_ptr,
                           float *contrib, int num_sms, cudaStream_t s);

// Scorer (gg_mlp.cu).
cudaError_t launch_mlp_score(const float *x, long long rows, const float *P, float *logits, int num_sms,
                             cudaStream_t s);
cudaError_t launch_mlp_select(const FeatArgs &fa, const float *P, float tau, float cost, uint32_t *sel_flag,
                              uint32_t *sel_deg, float *logits, int num_sms, cudaStream_t s);
cudaError_t launch_trace_features(const FeatArgs &fa, float *out, int num_sms, cudaStream_t s);
cudaError_t launch_trace_labels(int32_t n, const float *rc, const float *rn, const uint32_t *vc, const uint32_t *vn,
                                float tol, uint8_t *y, int num_sms, cudaStream_t s);
cudaError_t launch_mlp_train(const float *x, const uint8_t *y, unsigned long long rows, float *params, int B,
                             int steps, float lr, unsigned long long stride, unsigned long long start, float *losses,
                             float *grad_last, float *scratch, cudaStream_t s);
size_t mlp_train_scratch(int B);
// Learned correction plumbing (gg_learned.cu).
cudaError_t launch_sel_compact(int32_t n, const uint32_t *sel_flag, const uint32_t *sel_pos, const uint32_t *sel_off,
                               int32_t *rows, int32_t *sub_ptr, uint32_t *counts, int num_sms, cudaStream_t s);
cudaError_t launch_sub_copy(const int32_t *sub_ptr, int32_t nsel, uint32_t total, const int32_t *rows,
                            const int32_t *in_ptr, const int32_t *in_src, const uint32_t *in_w, const uint32_t *mask,
                            int32_t *sub_src, uint32_t *sub_w, int32_t *sub_pos, uint32_t *sub_mask, cudaStream_t s);
cudaError_t launch_keep_values(int32_t n, const float *rank_cur, float *rank_next, const float *contrib_cur,
                               float *contrib_next, const uint32_t *val_cur, uint32_t *val_next, float *hist,
                               int num_sms, cudaStream_t s);
cudaError_t launch_scatter_flags(const int32_t *sub_pos, const uint32_t *sub_mask, uint32_t total, uint32_t *mask,
                                 int num_sms, cudaStream_t s);

}  // namespace gg

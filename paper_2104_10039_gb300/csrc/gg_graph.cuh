// gg_graph.cuh - host-side state of a loaded graph (not part of the ABI).
#pragma once

#include <vector>

#include "gg_internal.cuh"

namespace gg {

// The library's stream-ordered memory pool on the current device: freed
// blocks stay in the pool (release threshold = unlimited), so loading graph
// after graph reuses memory instead of calling the driver each time.
cudaMemPool_t device_pool();

// Owning device buffer, allocated from device_pool() in stream order.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release()
    {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        bytes = 0;
    }
    gg_status alloc(size_t b, cudaStream_t stream = nullptr)
    {
        release();
        if (b == 0) b = 16;
        s = stream;
        cudaMemPool_t pool = device_pool();
        cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, b, pool, s) : cudaErrorMemoryAllocation;
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            set_error("device allocation of %zu bytes failed: %s", b, cudaGetErrorString(e));
            return GG_ERR_OOM;
        }
        bytes = b;
        return GG_OK;
    }
    uint32_t *u32() const { return (uint32_t *)p; }
    int32_t *i32() const { return (int32_t *)p; }
    float *f32() const { return (float *)p; }
};

// Plan of one list for the PageRank pull path (gg_pull.cu): row-start bits,
// per-tile row ranks, the vertex of every non-empty row, and the non-empty-row
// bitmap and counts that rank them.
struct PullPlan {
    DevBuf buf;
    uint32_t *hb = nullptr;
    int32_t *trow = nullptr, *nzv = nullptr, *lrows = nullptr;
    int2 *topen = nullptr;
    uint32_t *nlong = nullptr;
    uint32_t *nzb = nullptr, *nzc = nullptr, *nzcnt = nullptr;
    size_t hb_words = 0, tiles = 0, nzw = 0;
    bool valid = false;
};

struct TimedLaunch {
    int cls;               // 0 gather, 1 correct, 2 push
    cudaEvent_t start, stop;
};

}  // namespace gg

struct gg_graph {
    int32_t n = 0;
    int64_t m = 0;
    bool symmetric = false;
    bool has_w = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;

    // CSR (out-arcs)
    gg::DevBuf b_out_ptr, b_out_dst, b_out_w;
    int32_t *out_ptr = nullptr, *out_dst = nullptr;
    uint32_t *out_w = nullptr;
    // CSC (in-arcs; in_dst = each arc's row, for the sampling hash), CSR ->
    // CSC positions
    gg::DevBuf b_in_ptr, b_in_src, b_in_dst, b_in_w, b_out_to_in;
    int32_t *in_ptr = nullptr, *in_src = nullptr, *in_dst = nullptr, *out_to_in = nullptr;
    // hub cache: in-arc sources with hubs coded -(slot + 1), each hub's slot
    // (-1 otherwise) and each slot's vertex
    gg::DevBuf b_hub;
    int32_t *in_src_h = nullptr, *hub_slot = nullptr, *hub_ids = nullptr;
    int32_t n_hubs = 0;
    uint32_t *in_w = nullptr;
    // partition of the full CSC (merge-path kernels)
    gg::DevBuf b_full_tile_info, b_scalars;
    int32_t *full_tile_info = nullptr;
    uint32_t *full_num_tiles = nullptr, *sp_num_tiles = nullptr, *full_nnz = nullptr, *sp_nnz = nullptr;
    uint32_t *dev_err = nullptr, *q_len = nullptr;  // q_len[2]
    uint32_t max_tiles = 0;     // upper bound on tiles of any list
    uint32_t full_tiles = 0;    // tiles of the full in-edge list
    // active arcs per tile of a correction / sampling pass and their scan;
    // gather partials; the correction's value stash
    gg::DevBuf b_tile_cnt, b_part, b_stash, b_act;
    int32_t *act_outdeg = nullptr;   // active out-degrees (GG_RENORM)
    uint2 *stash = nullptr;
    uint2 *part = nullptr;
    uint32_t *part_head = nullptr;
    uint32_t *tile_cnt = nullptr, *tile_off = nullptr;
    // flags and packed active in-edges
    gg::DevBuf b_mask, b_sp_ptr, b_sp_src, b_sp_w;
    uint32_t *mask = nullptr;
    size_t mask_words = 0;
    int32_t *sp_ptr = nullptr, *sp_src = nullptr;
    uint32_t *sp_w = nullptr;
    bool sampled = false;        // sp_* / mask hold a sample
    bool sample_clean = false;   // ... and no correction has changed it since
    double sample_ratio = 0.0;
    uint64_t sample_seed = 0;
    uint32_t sp_nnz_host = 0;
    // frontier summary on the device and its host copy
    gg::FrontSum *front_dev = nullptr;
    gg::FrontSum front_host{};
    // vertex values (double-buffered)
    gg::DevBuf b_vals;
    float *rank[2] = {nullptr, nullptr}, *contrib[2] = {nullptr, nullptr};
    uint32_t *val[2] = {nullptr, nullptr};
    int cur = 0;
    int last_app = -1;
    // frontier
    gg::DevBuf b_front;
    int32_t *q[2] = {nullptr, nullptr};
    uint32_t *q_val[2] = {nullptr, nullptr};
    uint32_t *q_deg = nullptr;
    uint32_t *stamp = nullptr;
    uint32_t stamp_tag = 0;
    // push-frontier tile scheduler; per-tile status words (unused)
    gg::DevBuf b_sched, b_status;
    gg::TileSched *sched = nullptr;
    unsigned long long *st_carry = nullptr;
    uint32_t epoch = 0;
    gg::DevBuf b_scan_tmp;
    uint32_t *scan_tmp = nullptr;
    // statistics
    gg::DevBuf b_iter;
    gg::IterStatsDev *iter_stats = nullptr;
    uint32_t iter_cap = 0;
    uint32_t iterations = 0;
    gg_stats stats{};
    cudaEvent_t ev_run0 = nullptr, ev_run1 = nullptr, ev_s0 = nullptr, ev_s1 = nullptr;
    bool run_timed = false, sample_timed = false;
    std::vector<gg::TimedLaunch> timed;
    size_t timed_used = 0;
    uint32_t launches = 0;
    uint32_t load_launches = 0;
    // learned correction: scorer, change features of the last three executed
    // iterations, selection and the selected rows' sub-list
    gg::DevBuf b_mlp, b_hist, b_sel, b_sub, b_sub_tiles;
    float *mlp = nullptr;
    bool has_scorer = false;
    float *hist = nullptr;           // 3 x n
    bool keep_hist = false;          // this run keeps change features
    uint32_t executed = 0;           // iterations executed in this run
    bool force_full = false;         // the next correction is a full one
    uint32_t *sel_flag = nullptr, *sel_pos = nullptr, *sel_off = nullptr, *sel_counts = nullptr;
    int32_t *sel_rows = nullptr, *sub_ptr = nullptr;
    float *logits = nullptr;
    bool logits_valid = false;
    int32_t *sub_src = nullptr, *sub_pos = nullptr;
    uint32_t *sub_w = nullptr, *sub_mask = nullptr;
    int32_t *sub_tile_info = nullptr;
    uint32_t *sub_num_tiles = nullptr;
    // PageRank pull path: plans of the full (0) and packed (1) lists, row sums
    // and tile leading parts; whether sp_src holds vertex ids (not hub-coded)
    gg::PullPlan plan[2];
    gg::DevBuf b_pull;
    float *pull_acc = nullptr, *pull_lead = nullptr, *pull_carry = nullptr;
    uint32_t *pull_front = nullptr;   // frontier bitmap of a filtered pull (n bits)
    uint32_t *pull_hubv = nullptr;    // hub slots' values for the pull gathers (kHubCodes)
    bool pull_ready = false;
    bool sp_stale = false;     // the mask's tile counts are scanned, the packed list not yet built
    bool sp_has_w = false;     // the packed list carries the weights
    bool sp_hubs = false;      // ... and hub-coded sources
    // training trace (caller-owned device buffers)
    float *trace_x = nullptr;
    uint8_t *trace_y = nullptr;
    uint64_t trace_cap = 0, trace_rows = 0;
    float label_tol = 0.0f;
};

namespace gg {
gg_status build_csc(gg_graph *g);
gg_status build_hubs(gg_graph *g);
gg_status validate_csr(gg_graph *g);
gg_status sample_edges(gg_graph *g, double ratio, uint64_t seed);
// Packed active in-edges from the flag bitmap (gg_pack.cu); have_counts: the
// per-tile active counts are in tile_cnt already (a correction's flag pass).
// After the flags changed: counts the active arcs of the bitmap per 256-arc
// tile (unless the correction's flag pass did: have_counts) and scans them;
// the packed list's arc count (and stats->active_after) are then set. The
// list itself is built by ensure_packed.
gg_status pack_active(gg_graph *g, IterStatsDev *stats, bool have_counts);
// Source coding of the packed list: vertex ids, hubs coded -(slot + 1) (the
// PageRank pull gathers), or whichever it has.
enum PackCoding { PACK_PLAIN = 0, PACK_HUBS = 1, PACK_ANY = 2 };
// Builds the packed list of the current flags if it is not built yet, lacks
// the weights a caller needs (weighted) or has another source coding.
gg_status ensure_packed(gg_graph *g, bool weighted, PackCoding coding);
gg_status run(gg_graph *g, gg_app app, double ratio, gg_policy policy, const gg_params *p);
uint32_t next_epoch(gg_graph *g);
gg_status ensure_pull(gg_graph *g);
gg_status build_pull_plan(gg_graph *g, int which);
}  // namespace gg

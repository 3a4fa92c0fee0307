// gg_api.cu - the C ABI (gg.h) and the host schedule of GraphGuess runs:
// sampling (Sec. 3.4), the approximate / accurate / correction iteration
// sequence of each policy (Sec. 3.4, Sec. 5.2), and the push/pull choice of
// the min applications.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "gg_graph.cuh"

namespace gg {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

gg_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
    return GG_ERR_CUDA;
}

cudaMemPool_t device_pool()
{
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = pool;
    }
    return pools[dev];
}

// A frontier whose out-arcs number less than the list's arcs / this factor is
// pushed instead of pulled (push pays atomics and a flag lookup per arc).
constexpr uint64_t kPushFactor = 4;

enum { MODE_APPROX = 0, MODE_ACCURATE = 1, MODE_CORRECTION = 2, MODE_SKIPPED = 3 };

// Mode of iteration i (Sec. 3.4: alpha approximate iterations, then a
// correction; Sec. 5.2: SP never corrects, SMS corrects once then stays
// accurate; the exact baseline is accurate throughout).
static int policy_mode(gg_policy p, uint32_t alpha, uint32_t i)
{
    switch (p) {
    case GG_POLICY_EXACT: return MODE_ACCURATE;
    case GG_POLICY_NONE: return MODE_APPROX;
    case GG_POLICY_STATIC_SWITCH:
        return i < alpha ? MODE_APPROX : (i == alpha ? MODE_CORRECTION : MODE_ACCURATE);
    case GG_POLICY_ADAPTIVE:
    case GG_POLICY_LEARNED: return (i % (alpha + 1u)) == alpha ? MODE_CORRECTION : MODE_APPROX;
    default: break;
    }
    return MODE_ACCURATE;
}

// First accurate or correction iteration after approximate iteration i, or
// -1 if the policy stays approximate for good.
static int64_t next_accurate(gg_policy p, uint32_t alpha, uint32_t i)
{
    if (p == GG_POLICY_NONE) return -1;
    if (p == GG_POLICY_STATIC_SWITCH) return i < alpha ? (int64_t)alpha : (int64_t)i + 1;
    if (p == GG_POLICY_ADAPTIVE || p == GG_POLICY_LEARNED) {
        const uint64_t period = (uint64_t)alpha + 1u;
        return (int64_t)(((uint64_t)i / period) * period + alpha);
    }
    return (int64_t)i + 1;
}

// GG_POLICY_TRIGGERED: a window starts at the run's start and after every
// correction; a correction follows the approximate iteration whose change
// statistic is at most ratio x that of the window's first approximate
// iteration, or the alpha-th approximate iteration of the window.
struct Trigger {
    bool on = false;
    uint32_t alpha = 0;
    double ratio = 0.0;
    bool correct_next = false;
    uint32_t window = 0;
    double first = 0.0;

    Trigger(gg_policy p, const gg_params *prm)
    {
        on = p == GG_POLICY_TRIGGERED;
        alpha = prm->alpha;
        ratio = (double)prm->trigger_ratio;
        correct_next = on && alpha == 0;
    }
    int mode(gg_policy p, uint32_t i) const
    {
        if (!on) return policy_mode(p, alpha, i);
        return correct_next ? MODE_CORRECTION : MODE_APPROX;
    }
    // The mode iteration i+1 gets if iteration i (of mode `cur`) does not
    // trigger a correction by its statistic.
    int next_unless_triggered(gg_policy p, uint32_t i, int cur) const
    {
        if (!on) return policy_mode(p, alpha, i + 1);
        if (cur == MODE_CORRECTION) return alpha == 0 ? MODE_CORRECTION : MODE_APPROX;
        return window + 1 >= alpha ? MODE_CORRECTION : MODE_APPROX;
    }
    void after(bool correcting, double metric)
    {
        if (!on) return;
        if (correcting) {
            window = 0;
            correct_next = alpha == 0;
            return;
        }
        window += 1;
        if (window == 1) first = metric;
        correct_next = window >= alpha || metric <= ratio * first;
    }
};

uint32_t next_epoch(gg_graph *g)
{
    if (g->epoch >= (1u << 30)) {
        cudaMemsetAsync(g->st_carry, 0, sizeof(unsigned long long) * (g->max_tiles + 2), g->stream);
        g->epoch = 0;
    }
    return ++g->epoch;
}

static void timed_begin(gg_graph *g, bool on, int cls, size_t *slot)
{
    *slot = (size_t)-1;
    if (!on) return;
    if (g->timed_used == g->timed.size()) {
        TimedLaunch t{};
        t.cls = cls;
        if (cudaEventCreate(&t.start) != cudaSuccess || cudaEventCreate(&t.stop) != cudaSuccess) return;
        g->timed.push_back(t);
    }
    TimedLaunch &t = g->timed[g->timed_used];
    t.cls = cls;
    cudaEventRecord(t.start, g->stream);
    *slot = g->timed_used++;
}

static void timed_end(gg_graph *g, size_t slot)
{
    if (slot != (size_t)-1) cudaEventRecord(g->timed[slot].stop, g->stream);
}

static void fill_list(const gg_graph *g, bool sparse, TileArgs &a)
{
    a.n = g->n;
    a.out_ptr = g->out_ptr;
    if (sparse) {
        a.row_ptr = g->sp_ptr;
        a.arc_src = g->sp_src;
        a.arc_w = g->has_w ? g->sp_w : nullptr;
        a.list_nnz = g->sp_nnz;
        a.tile_info = nullptr;   // the pull path walks the packed list through its plan
        a.num_tiles = nullptr;
    } else {
        a.row_ptr = g->in_ptr;
        a.arc_src = g->in_src_h;
        a.arc_w = g->has_w ? g->in_w : nullptr;
        a.list_nnz = g->full_nnz;
        a.tile_info = g->full_tile_info;
        a.num_tiles = g->full_num_tiles;
    }
    a.st_carry = g->st_carry;
    a.err = g->dev_err;
    a.hub_ids = g->hub_ids;
    a.n_hubs = g->n_hubs;
    a.part = g->part;
    a.part_head = g->part_head;
    a.stash = g->stash;
}

gg_status sample_edges(gg_graph *g, double ratio, uint64_t seed)
{
    if (!(ratio > 0.0 && ratio <= 1.0)) {
        set_error("sample_ratio must be in (0, 1], got %g", ratio);
        return GG_ERR_INVALID_ARG;
    }
    GG_CUDA(cudaEventRecord(g->ev_s0, g->stream));
    // the hash keys on vertex ids (in_src, not the hub-coded copy)
    GG_CUDA(launch_sample(g->in_src, g->in_dst, g->m, g->symmetric ? 1 : 0, seed,
                          (unsigned long long)std::floor(ratio * 4294967296.0), g->mask, g->num_sms, g->stream));
    g->launches += 1;
    gg_status st = pack_active(g, nullptr, false);
    if (st != GG_OK) return st;
    GG_CUDA(cudaEventRecord(g->ev_s1, g->stream));
    g->sample_timed = true;
    g->sampled = true;
    g->sample_clean = true;
    g->sample_ratio = ratio;
    g->sample_seed = seed;
    return GG_OK;
}

static gg_status ensure_iter_cap(gg_graph *g, uint32_t iters)
{
    if (g->iter_cap < iters) {
        gg_status st = g->b_iter.alloc(sizeof(IterStatsDev) * iters);
        if (st != GG_OK) return st;
        g->iter_stats = (IterStatsDev *)g->b_iter.p;
        g->iter_cap = iters;
    }
    GG_CUDA(cudaMemsetAsync(g->iter_stats, 0, sizeof(IterStatsDev) * iters, g->stream));
    return GG_OK;
}

// Active out-degrees of the current flags (GG_RENORM).
static gg_status refresh_active_outdeg(gg_graph *g)
{
    gg_status st = ensure_packed(g, false, PACK_HUBS);   // PageRank's coding
    if (st != GG_OK) return st;
    GG_CUDA(launch_active_outdeg(g->sp_src, g->sp_nnz, (uint32_t)g->m, g->n, g->hub_ids, g->act_outdeg, g->num_sms,
                                 g->stream));
    g->launches += 2;
    return GG_OK;
}

#define GG_ALLOC_BUF(buf, bytes)                                  \
    do {                                                          \
        const gg_status s_ = (buf).alloc((bytes), g->stream);     \
        if (s_ != GG_OK) return s_;                               \
    } while (0)

// Stride between the per-vertex arrays carved from one buffer: n rounded up
// to a multiple of 4, so each array starts on a 16-byte boundary (the apply
// passes use 16-byte loads and stores).
static size_t vstride(const gg_graph *g) { return ((size_t)g->n + 3) & ~(size_t)3; }

// ---------------------------------------------- learned correction, traces --
static gg_status ensure_hist(gg_graph *g)
{
    if (!g->hist) {
        GG_ALLOC_BUF(g->b_hist, 4 * 3 * vstride(g));
        g->hist = g->b_hist.f32();
    }
    GG_CUDA(cudaMemsetAsync(g->hist, 0, 4 * 3 * vstride(g), g->stream));
    return GG_OK;
}

static gg_status ensure_learned(gg_graph *g)
{
    if (g->sel_flag) return GG_OK;
    const size_t n = (size_t)g->n, m = (size_t)g->m;
    GG_ALLOC_BUF(g->b_sel, 4 * (6 * n + 8));
    GG_ALLOC_BUF(g->b_sub, 4 * (3 * m + m / 32 + 4));
    GG_ALLOC_BUF(g->b_sub_tiles, 4 * ((size_t)g->max_tiles + 4));
    uint32_t *s = g->b_sel.u32();
    g->sel_flag = s;
    g->sel_pos = s + n;               // n + 1
    g->sel_off = s + 2 * n + 1;       // n + 1
    g->sel_rows = (int32_t *)(s + 3 * n + 2);
    g->sub_ptr = (int32_t *)(s + 4 * n + 2);   // n + 1
    g->logits = (float *)(s + 5 * n + 3);
    g->sel_counts = s + 6 * n + 4;    // 2
    uint32_t *b = g->b_sub.u32();
    g->sub_src = (int32_t *)b;
    g->sub_w = b + m;
    g->sub_pos = (int32_t *)(b + 2 * m);
    g->sub_mask = b + 3 * m;
    g->sub_tile_info = g->b_sub_tiles.i32();
    g->sub_num_tiles = g->b_sub_tiles.u32() + g->max_tiles + 2;
    return GG_OK;
}

// Change-feature slot of the iteration about to execute (or nullptr).
static float *hist_slot(gg_graph *g)
{
    return g->keep_hist ? g->hist + (size_t)(g->executed % 3u) * vstride(g) : nullptr;
}

static FeatArgs feat_args(gg_graph *g, gg_app app, uint32_t i)
{
    FeatArgs fa{};
    fa.n = g->n;
    fa.in_ptr = g->in_ptr;
    fa.out_ptr = g->out_ptr;
    fa.sp_ptr = g->sp_ptr;
    const uint32_t e = g->executed;
    fa.hist1 = g->hist + (size_t)((e + 2u) % 3u) * vstride(g);
    fa.hist2 = g->hist + (size_t)((e + 1u) % 3u) * vstride(g);
    fa.hist3 = g->hist + (size_t)(e % 3u) * vstride(g);
    fa.iter_f = (float)i * 0.015625f;
    fa.app_f = (float)app;
    return fa;
}

// Trace rows of a full correction: features now (before it runs).
static gg_status trace_features(gg_graph *g, gg_app app, uint32_t i, bool *tracing)
{
    *tracing = g->trace_x && g->trace_rows + (uint64_t)g->n <= g->trace_cap;
    if (!*tracing) return GG_OK;
    // the active in-degree feature (coded as the application's gathers read it)
    gg_status st = ensure_packed(g, false, app == GG_APP_PAGERANK ? PACK_HUBS : PACK_PLAIN);
    if (st != GG_OK) return st;
    GG_CUDA(launch_trace_features(feat_args(g, app, i), g->trace_x + g->trace_rows * 8, g->num_sms, g->stream));
    g->launches += 1;
    return GG_OK;
}

// ... and labels once the correction has produced the next values.
static gg_status trace_labels(gg_graph *g, bool pr)
{
    const int c = g->cur, nx = g->cur ^ 1;
    GG_CUDA(launch_trace_labels(g->n, pr ? g->rank[c] : nullptr, pr ? g->rank[nx] : nullptr, pr ? nullptr : g->val[c],
                                pr ? nullptr : g->val[nx], g->label_tol, g->trace_y + g->trace_rows, g->num_sms,
                                g->stream));
    g->launches += 1;
    g->trace_rows += (uint64_t)g->n;
    return GG_OK;
}

// Learned correction, selection: score every vertex, compact the selected
// rows and their in-edge offsets; *learned = the selection is small enough
// (else the full correction runs).
static gg_status learned_select(gg_graph *g, gg_app app, const gg_params *p, uint32_t i, bool *learned,
                                uint32_t *nsel, uint32_t *total)
{
    *learned = false;
    // the active in-degree feature (coded as the application's gathers read it)
    gg_status st = ensure_packed(g, false, app == GG_APP_PAGERANK ? PACK_HUBS : PACK_PLAIN);
    if (st != GG_OK) return st;
    GG_CUDA(launch_mlp_select(feat_args(g, app, i), g->mlp, p->select_logit, p->select_cost, g->sel_flag,
                              g->sel_off, g->logits, g->num_sms, g->stream));
    GG_CUDA(launch_scan_u32(g->sel_flag, g->sel_pos, (size_t)g->n, g->scan_tmp, g->stream));
    GG_CUDA(launch_scan_u32(g->sel_off, g->sel_off, (size_t)g->n, g->scan_tmp, g->stream));
    GG_CUDA(launch_sel_compact(g->n, g->sel_flag, g->sel_pos, g->sel_off, g->sel_rows, g->sub_ptr, g->sel_counts,
                               g->num_sms, g->stream));
    g->launches += 8;
    g->logits_valid = true;
    uint32_t counts[2] = {0, 0};
    GG_CUDA(cudaMemcpyAsync(counts, g->sel_counts, sizeof counts, cudaMemcpyDeviceToHost, g->stream));
    GG_CUDA(cudaStreamSynchronize(g->stream));
    *nsel = counts[0];
    *total = counts[1];
    *learned = !((double)counts[1] > (double)p->fallback_frac * (double)g->m);
    return GG_OK;
}

// Learned correction, the corrected rows: every vertex keeps its value, then
// the correction kernels walk the selected rows' sub-list and overwrite
// theirs; the new flags go back to the full bitmap, whose tile counts are
// recounted for the pack. `a` carries the application's fields.
static gg_status learned_correct(gg_graph *g, gg_app app, TileArgs a, uint32_t nsel, uint32_t total)
{
    const bool pr = app == GG_APP_PAGERANK;
    const bool weighted = app == GG_APP_SSSP && g->has_w;
    GG_CUDA(launch_sub_copy(g->sub_ptr, (int32_t)nsel, total, g->sel_rows, g->in_ptr, g->in_src_h,
                            weighted ? g->in_w : nullptr, g->mask, g->sub_src, g->sub_w, g->sub_pos, g->sub_mask,
                            g->stream));
    const uint32_t sub_tiles = (uint32_t)(((uint64_t)nsel + total + kWT - 1) / kWT) + 1;
    GG_CUDA(launch_partition(g->sub_ptr, (int32_t)nsel, g->sel_counts + 1, sub_tiles, g->sub_tile_info,
                             g->sub_num_tiles, g->stream));
    float *hs = hist_slot(g);
    const int c = g->cur, nx = g->cur ^ 1;
    GG_CUDA(launch_keep_values(g->n, pr ? g->rank[c] : nullptr, pr ? g->rank[nx] : nullptr,
                               pr ? g->contrib[c] : nullptr, pr ? g->contrib[nx] : nullptr,
                               pr ? nullptr : g->val[c], pr ? nullptr : g->val[nx], hs, g->num_sms, g->stream));
    a.row_ptr = g->sub_ptr;
    a.arc_src = g->sub_src;
    a.arc_w = weighted ? g->sub_w : nullptr;
    a.n = (int32_t)nsel;
    a.list_nnz = g->sel_counts + 1;
    a.tile_info = g->sub_tile_info;
    a.num_tiles = g->sub_num_tiles;
    a.row_vtx = g->sel_rows;
    a.mask = g->sub_mask;
    a.hist_out = hs;
    a.epoch = next_epoch(g);
    if (nsel > 0) {
        if (pr) GG_CUDA(launch_tile_pr(K_CORRECT, a, (int)sub_tiles, g->num_sms, g->stream));
        else GG_CUDA(launch_tile_min((int)app, K_CORRECT, a, (int)sub_tiles, g->num_sms, g->stream));
    }
    GG_CUDA(launch_scatter_flags(g->sub_pos, g->sub_mask, total, g->mask, g->num_sms, g->stream));
    g->launches += 7;
    g->stats.learned_corrections += 1;
    return GG_OK;
}

// Kernels one pull iteration launches: the hubs' values (when the graph has
// hubs), the arcs, the long rows, (a correction's carries and flags,) the
// apply.
static int pull_launches(const gg_graph *g, bool correct, bool pr)
{
    return (correct ? 5 : 3) + (pr && g->n_hubs > 0 ? 1 : 0);
}

// Arguments of the pull path over the full in-edge list (which 0) or the
// packed active list (1), from the iteration's tile arguments; builds the
// list's plan if it is not current (and, on the graph's first pull, the
// plans' and row sums' buffers).
static gg_status pull_args(gg_graph *g, int which, bool pagerank, const TileArgs &a, PullArgs *pa)
{
    gg_status st = ensure_pull(g);   // plans and row-sum buffers (first pull on this graph)
    if (st != GG_OK) return st;
    if (!g->plan[which].valid) {
        st = build_pull_plan(g, which);
        if (st != GG_OK) return st;
    }
    const PullPlan &pl = g->plan[which];
    // PageRank reads hub-coded sources (the packed list was built to match)
    pa->src = which ? g->sp_src : (pagerank ? g->in_src_h : g->in_src);
    pa->hub_ids = g->hub_ids;
    pa->n_hubs = pagerank ? g->n_hubs : 0;
    pa->hubv = g->pull_hubv;
    pa->row_ptr = which ? g->sp_ptr : g->in_ptr;
    pa->nnz = which ? g->sp_nnz : g->full_nnz;
    pa->hb = pl.hb;
    pa->trow = pl.trow;
    pa->nzv = pl.nzv;
    pa->topen = pl.topen;
    pa->lrows = pl.lrows;
    pa->nlong = pl.nlong;
    pa->carry = g->pull_carry;
    pa->contrib = a.contrib_cur;
    pa->acc = g->pull_acc;
    pa->lead = g->pull_lead;
    pa->n = g->n;
    pa->rank_cur = a.rank_cur;
    pa->rank_next = a.rank_next;
    pa->contrib_next = a.contrib_next;
    pa->out_ptr = g->out_ptr;
    pa->deg_apply = a.deg_apply;
    pa->base = a.base;
    pa->damping = a.damping;
    pa->epsilon = a.epsilon;
    pa->n_f = a.n_f;
    pa->hist_out = a.hist_out;
    pa->stats = a.stats;
    pa->val_cur = a.val_cur;
    pa->val_next = a.val_next;
    pa->q_out = a.q_out;
    pa->q_out_val = a.q_out_val;
    pa->q_out_len = a.q_out_len;
    return GG_OK;
}

static gg_status run_pagerank(gg_graph *g, gg_policy policy, const gg_params *p)
{
    const bool timing = (p->flags & GG_TIMING) != 0;
    const bool renorm = (p->flags & GG_RENORM) != 0 && policy != GG_POLICY_EXACT;
    const bool learned_policy = policy == GG_POLICY_LEARNED;
    Trigger trig(policy, p);
    g->cur = 0;
    GG_CUDA(launch_init_pr(g->n, g->out_ptr, g->rank[0], g->contrib[0], g->num_sms, g->stream));
    g->launches += 1;
    if (renorm) {
        gg_status st = refresh_active_outdeg(g);
        if (st != GG_OK) return st;
        if (trig.mode(policy, 0) == MODE_APPROX) {
            GG_CUDA(launch_contrib(g->n, g->rank[0], g->act_outdeg, nullptr, g->contrib[0], g->num_sms,
                                   g->stream));
            g->launches += 1;
        }
    }
    const float base = (1.0f - p->damping) / (float)g->n;
    for (uint32_t i = 0; i < p->max_iters; ++i) {
        const int mode = trig.mode(policy, i);
        const int next = i + 1 < p->max_iters ? trig.next_unless_triggered(policy, i, mode) : MODE_ACCURATE;
        const int kind = mode == MODE_CORRECTION ? K_CORRECT : K_GATHER;
        TileArgs a{};
        a.infl_share = (p->flags & GG_INFL_SHARE) ? 1 : 0;
        // the next iteration gathers active arcs only: renormalised contributions
        a.deg_apply = (renorm && next == MODE_APPROX && kind != K_CORRECT) ? g->act_outdeg : nullptr;
        if (mode == MODE_APPROX) {
            gg_status st = ensure_packed(g, false, PACK_HUBS);
            if (st != GG_OK) return st;
        }
        fill_list(g, mode == MODE_APPROX, a);
        a.contrib_cur = g->contrib[g->cur];
        a.rank_cur = g->rank[g->cur];
        a.rank_next = g->rank[g->cur ^ 1];
        a.contrib_next = g->contrib[g->cur ^ 1];
        a.base = base;
        a.damping = p->damping;
        a.epsilon = p->epsilon;
        a.epoch = next_epoch(g);
        a.stats = g->iter_stats + i;
        a.hist_out = hist_slot(g);
        a.n_f = (float)g->n;
        if (kind == K_CORRECT) {
            a.mask = g->mask;
            a.theta = p->theta;
        }
        bool learned = false;
        bool counted = false;   // the correction's flag pass counted each tile's active arcs
        uint32_t nsel = 0, sel_arcs = 0;
        if (kind == K_CORRECT && learned_policy && !g->force_full) {
            gg_status st = learned_select(g, GG_APP_PAGERANK, p, i, &learned, &nsel, &sel_arcs);
            if (st != GG_OK) return st;
        }
        size_t slot;
        if (learned) {
            GG_CUDA(launch_iter_header(a.stats, (uint32_t)mode | GG_ITER_LEARNED, nullptr, sel_arcs, g->stream, nsel));
            timed_begin(g, timing, 1, &slot);
            gg_status st = learned_correct(g, GG_APP_PAGERANK, a, nsel, sel_arcs);
            if (st != GG_OK) return st;
            timed_end(g, slot);
            g->launches += 1;
        } else {
            bool tracing = false;
            if (kind == K_CORRECT) {
                gg_status st = trace_features(g, GG_APP_PAGERANK, i, &tracing);
                if (st != GG_OK) return st;
            }
            GG_CUDA(launch_iter_header(a.stats, (uint32_t)mode, a.list_nnz, 0, g->stream));
            if (kind == K_GATHER || !a.infl_share) {
                // pull path: gathers over either list, corrections over the full one
                const int which = mode == MODE_APPROX ? 1 : 0;
                PullArgs pa{};
                gg_status st = pull_args(g, which, true, a, &pa);
                if (st != GG_OK) return st;
                timed_begin(g, timing, kind == K_CORRECT ? 1 : 0, &slot);
                if (kind == K_GATHER) {
                    GG_CUDA(launch_pull(GG_APP_PAGERANK, pa, false, (uint32_t)g->plan[which].tiles, g->num_sms,
                                        g->stream));
                    g->launches += pull_launches(g, false, true);
                } else {
                    pa.vals = reinterpret_cast<float *>(g->stash);
                    pa.mask = g->mask;
                    pa.tcnt = g->tile_cnt;
                    pa.theta = p->theta;
                    GG_CUDA(launch_pull(GG_APP_PAGERANK, pa, true, (uint32_t)g->plan[which].tiles, g->num_sms,
                                        g->stream));
                    g->launches += pull_launches(g, true, true);
                    counted = true;
                }
                timed_end(g, slot);
            } else {
                // share influence: the merge-path correction (stash + share pass)
                timed_begin(g, timing, 1, &slot);
                GG_CUDA(launch_tile_pr(kind, a, (int)g->max_tiles, g->num_sms, g->stream));
                timed_end(g, slot);
                g->launches += 2;
            }
            if (tracing) {
                gg_status st = trace_labels(g, true);
                if (st != GG_OK) return st;
            }
        }
        if (kind == K_CORRECT) {
            // the packed list itself is built when an approximate gather needs it
            gg_status st = pack_active(g, a.stats, counted);
            if (st != GG_OK) return st;
            g->sample_clean = false;
            g->stats.corrections += 1;
            if (renorm) {
                st = refresh_active_outdeg(g);
                if (st != GG_OK) return st;
                if (next == MODE_APPROX) {
                    GG_CUDA(launch_contrib(g->n, g->rank[g->cur ^ 1], g->act_outdeg, nullptr,
                                           g->contrib[g->cur ^ 1], g->num_sms, g->stream));
                    g->launches += 1;
                }
            }
            if (learned_policy) {
                // a learned correction that changed no value makes the next one full
                unsigned long long changed = 0;
                if (learned) {
                    GG_CUDA(cudaMemcpyAsync(&changed, &g->iter_stats[i].changed, sizeof changed,
                                            cudaMemcpyDeviceToHost, g->stream));
                    GG_CUDA(cudaStreamSynchronize(g->stream));
                }
                g->force_full = learned && changed == 0;
            }
        }
        g->stats.pull_iterations += 1;
        g->cur ^= 1;
        g->iterations = i + 1;
        g->executed += 1;
        if (trig.on) {
            double metric = 0.0;
            if (mode == MODE_APPROX) {
                unsigned long long sd = 0;
                GG_CUDA(cudaMemcpyAsync(&sd, &g->iter_stats[i].sum_delta, sizeof sd, cudaMemcpyDeviceToHost,
                                        g->stream));
                GG_CUDA(cudaStreamSynchronize(g->stream));
                metric = (double)sd;
            }
            trig.after(mode == MODE_CORRECTION, metric);
            if (renorm && next == MODE_APPROX && trig.correct_next && i + 1 < p->max_iters) {
                // contributions were divided by active out-degrees for an
                // approximate iteration; the correction needs full degrees
                GG_CUDA(launch_contrib(g->n, g->rank[g->cur], nullptr, g->out_ptr, g->contrib[g->cur],
                                       g->num_sms, g->stream));
                g->launches += 1;
            }
        }
        if ((p->flags & GG_STOP_QUIESCE) && mode != MODE_APPROX && !learned) {
            unsigned long long changed = 0;
            GG_CUDA(cudaMemcpyAsync(&changed, &g->iter_stats[i].changed, sizeof changed, cudaMemcpyDeviceToHost,
                                    g->stream));
            GG_CUDA(cudaStreamSynchronize(g->stream));
            if (changed == 0) break;
        }
    }
    return GG_OK;
}

// The frontier q[qc] after an iteration, in one device-to-host read: its
// length, the out-arcs of its vertices (each vertex's out-degree stays in
// q_deg for the scan a push needs) and the packed list's arc count.
static gg_status frontier_summary(gg_graph *g, int qc, uint32_t *qlen, uint64_t *arcs)
{
    GG_CUDA(cudaMemsetAsync(g->front_dev, 0, sizeof(FrontSum), g->stream));
    GG_CUDA(launch_qdeg(g->q[qc], &g->q_len[qc], g->out_ptr, g->q_deg, g->front_dev, g->sp_nnz, (uint32_t)g->n,
                        g->num_sms, g->stream));
    GG_CUDA(cudaMemcpyAsync(&g->front_host, g->front_dev, sizeof(FrontSum), cudaMemcpyDeviceToHost, g->stream));
    GG_CUDA(cudaStreamSynchronize(g->stream));
    g->launches += 1;
    *qlen = g->front_host.len;
    *arcs = g->front_host.arcs;
    g->sp_nnz_host = g->front_host.nnz;
    return GG_OK;
}

static gg_status run_min(gg_graph *g, gg_app app, gg_policy policy, const gg_params *p)
{
    const bool timing = (p->flags & GG_TIMING) != 0;
    const bool learned_policy = policy == GG_POLICY_LEARNED;
    g->cur = 0;
    int qc = 0;
    GG_CUDA(launch_init_min(g->n, (int)app, p->source, g->val[0], g->q[0], g->q_val[0], &g->q_len[0], g->num_sms,
                            g->stream));
    g->launches += 1;
    uint32_t qlen = 0;
    uint64_t front_arcs = 0;
    gg_status st = frontier_summary(g, qc, &qlen, &front_arcs);
    if (st != GG_OK) return st;
    int theta_case = 0;
    unsigned long long theta_fx = 0;
    const double th = (double)p->theta;
    if (th < 0.0) theta_case = 1;
    else if (th >= 1.0) theta_case = 2;
    else theta_fx = (unsigned long long)std::floor(th * 4294967296.0);

    Trigger trig(policy, p);
    for (uint32_t i = 0; i < p->max_iters; ++i) {
        const int mode = trig.mode(policy, i);
        const int nq = qc ^ 1;
        GG_CUDA(cudaMemsetAsync(&g->q_len[nq], 0, sizeof(uint32_t), g->stream));
        const uint64_t list_nnz = mode == MODE_APPROX ? g->sp_nnz_host : (uint64_t)g->m;
        bool push = mode != MODE_CORRECTION && !(p->flags & GG_FORCE_PULL) &&
                    ((p->flags & GG_FORCE_PUSH) || front_arcs * kPushFactor < list_nnz);
        IterStatsDev *sti = g->iter_stats + i;
        float *hs = hist_slot(g);
        bool learned = false;
        if (push) {
            GG_CUDA(launch_iter_header(sti, (uint32_t)mode | GG_ITER_PUSH, nullptr, list_nnz, g->stream));
            g->launches += 1;
            if (++g->stamp_tag == 0) {
                GG_CUDA(cudaMemsetAsync(g->stamp, 0, sizeof(uint32_t) * g->n, g->stream));
                g->stamp_tag = 1;
            }
            if (hs) GG_CUDA(cudaMemsetAsync(hs, 0, sizeof(float) * g->n, g->stream));
            // arc offsets of the frontier vertices (their degrees are in q_deg)
            GG_CUDA(launch_scan_u32(g->q_deg, g->q_deg, qlen, g->scan_tmp, g->stream));
            g->launches += 3;
            PushArgs pa{};
            pa.q = g->q[qc];
            pa.q_val = g->q_val[qc];
            pa.q_len = &g->q_len[qc];
            pa.q_deg_ex = g->q_deg;
            pa.out_ptr = g->out_ptr;
            pa.out_dst = g->out_dst;
            pa.out_w = g->out_w;
            pa.out_to_in = g->out_to_in;
            pa.mask = mode == MODE_APPROX ? g->mask : nullptr;
            pa.val = g->val[g->cur];
            pa.stamp = g->stamp;
            pa.stamp_tag = g->stamp_tag;
            pa.q_out = g->q[nq];
            pa.q_out_len = &g->q_len[nq];
            pa.sched = g->sched;
            pa.err = g->dev_err;
            pa.app = (int)app;
            size_t slot;
            timed_begin(g, timing, 2, &slot);
            GG_CUDA(launch_push(pa, (uint32_t)front_arcs, g->num_sms * 8, g->stream));
            timed_end(g, slot);
            GG_CUDA(launch_snapshot(g->q[nq], &g->q_len[nq], g->val[g->cur], g->q_val[nq], hs, (uint32_t)g->n,
                                    g->num_sms, g->stream));
            GG_CUDA(launch_iter_changed(sti, &g->q_len[nq], g->stream));
            g->launches += 3;
            g->stats.push_iterations += 1;
        } else {
            const int kind = mode == MODE_CORRECTION ? K_CORRECT : K_GATHER;
            TileArgs a{};
            if (mode == MODE_APPROX) {
                st = ensure_packed(g, app == GG_APP_SSSP && g->has_w, PACK_PLAIN);
                if (st != GG_OK) return st;
            }
            fill_list(g, mode == MODE_APPROX, a);
            a.val_cur = g->val[g->cur];
            a.val_next = g->val[g->cur ^ 1];
            a.epoch = next_epoch(g);
            a.stats = sti;
            a.q_out = g->q[nq];
            a.q_out_val = g->q_val[nq];
            a.q_out_len = &g->q_len[nq];
            a.hist_out = hs;
            if (app != GG_APP_SSSP) a.arc_w = nullptr;
            if (kind == K_CORRECT) {
                a.mask = g->mask;
                a.theta_case = theta_case;
                a.theta_fx = theta_fx;
                a.est_strict = (p->flags & GG_EST_STRICT) ? 1 : 0;
            }
            uint32_t nsel = 0, sel_arcs = 0;
            if (kind == K_CORRECT && learned_policy && !g->force_full) {
                st = learned_select(g, app, p, i, &learned, &nsel, &sel_arcs);
                if (st != GG_OK) return st;
            }
            size_t slot;
            if (learned) {
                GG_CUDA(launch_iter_header(sti, (uint32_t)mode | GG_ITER_LEARNED, nullptr, sel_arcs, g->stream,
                                           nsel));
                timed_begin(g, timing, 1, &slot);
                st = learned_correct(g, app, a, nsel, sel_arcs);
                if (st != GG_OK) return st;
                timed_end(g, slot);
                g->launches += 1;
            } else {
                bool tracing = false;
                if (kind == K_CORRECT) {
                    st = trace_features(g, app, i, &tracing);
                    if (st != GG_OK) return st;
                }
                // GG_PULL_FILTER: a gather skips the arcs of sources outside the
                // frontier, whose values were taken in when they last changed (as
                // a push does)
                const bool filter = kind == K_GATHER && (p->flags & GG_PULL_FILTER) != 0;
                GG_CUDA(launch_iter_header(sti, (uint32_t)mode | (filter ? GG_ITER_FILTER : 0u), nullptr, list_nnz,
                                           g->stream));
                const int which = mode == MODE_APPROX ? 1 : 0;
                PullArgs pa{};
                st = pull_args(g, which, false, a, &pa);
                if (st != GG_OK) return st;
                pa.w = (app == GG_APP_SSSP && g->has_w) ? (which ? g->sp_w : g->in_w) : nullptr;
                timed_begin(g, timing, kind == K_CORRECT ? 1 : 0, &slot);
                if (filter) {
                    GG_CUDA(launch_front_bits(g->q[qc], &g->q_len[qc], g->pull_front, g->n, g->num_sms, g->stream));
                    g->launches += 1;
                    pa.front = g->pull_front;
                }
                if (kind == K_CORRECT) {
                    pa.vals = reinterpret_cast<float *>(g->stash);
                    pa.mask = g->mask;
                    pa.tcnt = g->tile_cnt;
                    pa.theta_case = theta_case;
                    pa.theta_fx = theta_fx;
                    pa.est_strict = (p->flags & GG_EST_STRICT) ? 1 : 0;
                }
                GG_CUDA(launch_pull((int)app, pa, kind == K_CORRECT, (uint32_t)g->plan[which].tiles, g->num_sms,
                                    g->stream));
                timed_end(g, slot);
                g->launches += pull_launches(g, kind == K_CORRECT, false);
                if (tracing) {
                    st = trace_labels(g, false);
                    if (st != GG_OK) return st;
                }
            }
            if (kind == K_CORRECT) {
                // the packed list itself is built when an approximate pull needs it
                st = pack_active(g, sti, !learned);
                if (st != GG_OK) return st;
                g->sample_clean = false;
                g->stats.corrections += 1;
            }
            g->cur ^= 1;
            g->stats.pull_iterations += 1;
        }
        const uint32_t prev_qlen = qlen;
        const int prev_qc = qc;
        qc = nq;
        st = frontier_summary(g, qc, &qlen, &front_arcs);
        if (st != GG_OK) return st;
        g->iterations = i + 1;
        g->executed += 1;
        trig.after(mode == MODE_CORRECTION, (double)qlen);
        if (learned_policy && mode == MODE_CORRECTION) g->force_full = learned && qlen == 0;
        if (learned && prev_qlen > 0) {
            // the rows left alone did not gather the previous iteration's
            // changes: the next frontier takes those vertices too
            GG_CUDA(launch_append_frontier(g->q[prev_qc], prev_qlen, hs, g->val[g->cur], g->q[qc], g->q_val[qc],
                                           &g->q_len[qc], g->num_sms, g->stream));
            g->launches += 1;
            st = frontier_summary(g, qc, &qlen, &front_arcs);
            if (st != GG_OK) return st;
        }
        if (qlen == 0 && !learned) {
            // Quiet iteration: an accurate one means a fixed point of the full
            // graph; an approximate one makes every approximate iteration up to
            // the next accurate one a no-op (skipped, still counted).
            if (mode != MODE_APPROX) break;
            const int64_t nxt = next_accurate(policy, p->alpha, i);
            if (nxt < 0) break;
            for (uint32_t j = i + 1; j < (uint32_t)nxt && j < p->max_iters; ++j) {
                GG_CUDA(launch_iter_header(g->iter_stats + j, MODE_SKIPPED, nullptr, 0, g->stream));
                g->launches += 1;
                g->iterations = j + 1;
            }
            if ((uint64_t)nxt >= p->max_iters) break;
            i = (uint32_t)nxt - 1;
            front_arcs = 0;
            continue;
        }
    }
    return GG_OK;
}

gg_status run(gg_graph *g, gg_app app, double ratio, gg_policy policy, const gg_params *p)
{
    if (!p) { set_error("gg_run: params is NULL"); return GG_ERR_INVALID_ARG; }
    if ((int)app < GG_APP_PAGERANK || (int)app > GG_APP_CC) { set_error("gg_run: unknown app %d", (int)app); return GG_ERR_INVALID_ARG; }
    if ((int)policy < GG_POLICY_EXACT || (int)policy > GG_POLICY_LEARNED) { set_error("gg_run: unknown policy %d", (int)policy); return GG_ERR_INVALID_ARG; }
    if (policy == GG_POLICY_LEARNED) {
        if (!g->has_scorer) { set_error("gg_run: GG_POLICY_LEARNED needs a scorer (gg_set_scorer)"); return GG_ERR_STATE; }
        if (p->fallback_frac != p->fallback_frac || p->select_logit != p->select_logit ||
            p->select_cost != p->select_cost) {
            set_error("gg_run: select_logit / fallback_frac / select_cost is NaN");
            return GG_ERR_INVALID_ARG;
        }
    }
    if (policy == GG_POLICY_TRIGGERED && !(p->trigger_ratio >= 0.0f && p->trigger_ratio <= 3.0e38f)) {
        set_error("gg_run: trigger_ratio must be finite and >= 0");
        return GG_ERR_INVALID_ARG;
    }
    if (p->max_iters < 1) { set_error("gg_run: max_iters must be >= 1"); return GG_ERR_INVALID_ARG; }
    if (app == GG_APP_SSSP && !g->has_w) { set_error("gg_run: SSSP needs arc weights"); return GG_ERR_INVALID_ARG; }
    if ((app == GG_APP_SSSP || app == GG_APP_BFS) && (p->source < 0 || p->source >= g->n)) {
        set_error("gg_run: source %d outside [0, %d)", p->source, g->n);
        return GG_ERR_INVALID_ARG;
    }
    if (app == GG_APP_PAGERANK && !(p->damping >= 0.0f && p->damping <= 1.0f)) {
        set_error("gg_run: damping must be in [0, 1]");
        return GG_ERR_INVALID_ARG;
    }
    if (policy != GG_POLICY_EXACT && !(ratio > 0.0 && ratio <= 1.0)) {
        set_error("gg_run: sample_ratio must be in (0, 1], got %g", ratio);
        return GG_ERR_INVALID_ARG;
    }
    if (p->alpha == 0xFFFFFFFFu) { set_error("gg_run: alpha too large"); return GG_ERR_INVALID_ARG; }
    gg_status st = ensure_iter_cap(g, p->max_iters);
    if (st != GG_OK) return st;
    {
        const float ms_load = g->stats.ms_load;
        const uint32_t kl = g->stats.kernels_load;
        g->stats = gg_stats{};
        g->stats.ms_load = ms_load;
        g->stats.kernels_load = kl;
    }
    g->timed_used = 0;
    g->launches = 0;
    g->iterations = 0;
    g->last_app = -1;
    g->executed = 0;
    g->force_full = false;
    g->keep_hist = policy == GG_POLICY_LEARNED || g->trace_x != nullptr;
    if (g->keep_hist) {
        st = ensure_hist(g);
        if (st != GG_OK) return st;
    }
    if (policy == GG_POLICY_LEARNED) {
        st = ensure_learned(g);
        if (st != GG_OK) return st;
    }
    GG_CUDA(cudaMemsetAsync(g->dev_err, 0, sizeof(uint32_t), g->stream));
    GG_CUDA(cudaEventRecord(g->ev_run0, g->stream));
    if (policy != GG_POLICY_EXACT &&
        !(g->sampled && g->sample_clean && g->sample_ratio == ratio && g->sample_seed == p->seed)) {
        st = sample_edges(g, ratio, p->seed);
        if (st != GG_OK) return st;
    }
    st = app == GG_APP_PAGERANK ? run_pagerank(g, policy, p) : run_min(g, app, policy, p);
    GG_CUDA(cudaEventRecord(g->ev_run1, g->stream));
    g->run_timed = true;
    if (st != GG_OK) return st;
    g->last_app = (int)app;
    g->stats.iterations = g->iterations;
    g->stats.kernels_launched = g->launches;
    return GG_OK;
}

}  // namespace gg

using namespace gg;

static gg_status alloc_graph(gg_graph *g)
{
    const size_t n = (size_t)g->n, m = (size_t)g->m;
    gg_status st;
#define GG_ALLOC(buf, bytes)                    \
    do {                                        \
        if ((st = (buf).alloc(bytes)) != GG_OK) \
            return st;                          \
    } while (0)
    GG_ALLOC(g->b_out_ptr, 4 * (n + 1));
    GG_ALLOC(g->b_out_dst, 4 * m);
    GG_ALLOC(g->b_in_ptr, 4 * (n + 1));
    GG_ALLOC(g->b_in_src, 4 * m);
    GG_ALLOC(g->b_in_dst, 4 * m);
    GG_ALLOC(g->b_hub, 4 * (m + n + (size_t)kHubCodes + 4));
    GG_ALLOC(g->b_out_to_in, 4 * m);
    GG_ALLOC(g->b_sp_ptr, 4 * (n + 1));
    GG_ALLOC(g->b_sp_src, 4 * m);
    if (g->has_w) {
        GG_ALLOC(g->b_out_w, 4 * m);
        GG_ALLOC(g->b_in_w, 4 * m);
        GG_ALLOC(g->b_sp_w, 4 * m);
    }
    g->full_tiles = (uint32_t)(((uint64_t)n + m + kWT - 1) / kWT);
    g->max_tiles = g->full_tiles + 1;
    GG_ALLOC(g->b_full_tile_info, 4 * ((size_t)g->max_tiles + 2));
    GG_ALLOC(g->b_tile_cnt, 4 * (2 * (size_t)g->max_tiles + 4));
    GG_ALLOC(g->b_act, 4 * n);
    GG_ALLOC(g->b_part, 12 * ((size_t)g->max_tiles + 2));
    GG_ALLOC(g->b_stash, 8 * m);
    GG_ALLOC(g->b_scalars, 4 * 16);
    g->mask_words = (m + 31) / 32;
    GG_ALLOC(g->b_mask, 4 * (g->mask_words + 1));
    const size_t nv = (n + 3) & ~(size_t)3;   // 16-byte aligned per-vertex arrays
    GG_ALLOC(g->b_vals, 4 * 4 * nv);
    GG_ALLOC(g->b_front, 4 * (6 * n + 2));
    GG_ALLOC(g->b_sched, sizeof(TileSched) * 2);
    GG_ALLOC(g->b_status, sizeof(unsigned long long) * ((size_t)g->max_tiles + 2));
    GG_ALLOC(g->b_scan_tmp, 4 * scan_tmp_words((n + 1 > (size_t)g->max_tiles + 1 ? n + 1 : (size_t)g->max_tiles + 1)));
#undef GG_ALLOC
    g->out_ptr = g->b_out_ptr.i32();
    g->out_dst = g->b_out_dst.i32();
    g->out_w = g->has_w ? g->b_out_w.u32() : nullptr;
    g->in_ptr = g->b_in_ptr.i32();
    g->in_src = g->b_in_src.i32();
    g->in_dst = g->b_in_dst.i32();
    g->in_src_h = g->b_hub.i32();
    g->hub_slot = g->in_src_h + m;
    g->hub_ids = g->hub_slot + n;
    g->in_w = g->has_w ? g->b_in_w.u32() : nullptr;
    g->out_to_in = g->b_out_to_in.i32();
    g->sp_ptr = g->b_sp_ptr.i32();
    g->sp_src = g->b_sp_src.i32();
    g->sp_w = g->has_w ? g->b_sp_w.u32() : nullptr;
    g->full_tile_info = g->b_full_tile_info.i32();
    g->tile_cnt = g->b_tile_cnt.u32();
    g->tile_off = g->tile_cnt + g->max_tiles + 2;
    g->act_outdeg = g->b_act.i32();
    g->part = (uint2 *)g->b_part.p;
    g->part_head = (uint32_t *)(g->part + g->max_tiles + 2);
    g->stash = (uint2 *)g->b_stash.p;
    uint32_t *sc = g->b_scalars.u32();
    g->full_num_tiles = sc + 0;
    g->sp_num_tiles = sc + 1;
    g->full_nnz = sc + 2;
    g->sp_nnz = sc + 3;
    g->dev_err = sc + 4;
    g->q_len = sc + 6;  // two entries
    g->front_dev = reinterpret_cast<FrontSum *>(sc + 8);
    g->mask = g->b_mask.u32();
    float *v = g->b_vals.f32();
    g->rank[0] = v;
    g->rank[1] = v + nv;
    g->contrib[0] = v + 2 * nv;
    g->contrib[1] = v + 3 * nv;
    g->val[0] = (uint32_t *)g->rank[0];
    g->val[1] = (uint32_t *)g->rank[1];
    uint32_t *f = g->b_front.u32();
    g->q[0] = (int32_t *)f;
    g->q[1] = (int32_t *)(f + n);
    g->q_val[0] = f + 2 * n;
    g->q_val[1] = f + 3 * n;
    g->stamp = f + 4 * n;
    g->q_deg = f + 5 * n;
    g->sched = (TileSched *)g->b_sched.p;
    g->st_carry = (unsigned long long *)g->b_status.p;
    g->scan_tmp = g->b_scan_tmp.u32();
    return GG_OK;
}

extern "C" {

gg_status gg_load_csr(gg_graph **out, int32_t n, int64_t m, const int32_t *rowptr, const int32_t *colidx,
                      const uint32_t *weights, uint32_t gflags)
{
    if (!out) { set_error("gg_load_csr: out is NULL"); return GG_ERR_INVALID_ARG; }
    *out = nullptr;
    if (n < 1) { set_error("gg_load_csr: n must be >= 1, got %d", n); return GG_ERR_INVALID_ARG; }
    if (m < 0 || m >= ((int64_t)1 << 31) - 1) { set_error("gg_load_csr: m must be in [0, 2^31-1), got %lld", (long long)m); return GG_ERR_INVALID_ARG; }
    if (!rowptr || (m > 0 && !colidx)) { set_error("gg_load_csr: rowptr/colidx is NULL"); return GG_ERR_INVALID_ARG; }
    if (gflags & ~(GG_SYMMETRIC | GG_DEVICE_PTRS)) { set_error("gg_load_csr: unknown flags 0x%x", gflags); return GG_ERR_INVALID_ARG; }
    gg_graph *g = new (std::nothrow) gg_graph();
    if (!g) { set_error("gg_load_csr: host allocation failed"); return GG_ERR_OOM; }
    g->n = n;
    g->m = m;
    g->symmetric = (gflags & GG_SYMMETRIC) != 0;
    g->has_w = weights != nullptr;
    gg_status st = GG_OK;
    cudaError_t e;
    do {
        if ((e = cudaGetDevice(&g->device)) != cudaSuccess) { st = cuda_fail(e, "cudaGetDevice"); break; }
        if ((e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device)) != cudaSuccess) {
            st = cuda_fail(e, "cudaDeviceGetAttribute");
            break;
        }
        if ((e = cudaEventCreate(&g->ev_run0)) != cudaSuccess || (e = cudaEventCreate(&g->ev_run1)) != cudaSuccess ||
            (e = cudaEventCreate(&g->ev_s0)) != cudaSuccess || (e = cudaEventCreate(&g->ev_s1)) != cudaSuccess) {
            st = cuda_fail(e, "cudaEventCreate");
            break;
        }
        if ((st = alloc_graph(g)) != GG_OK) break;
        cudaEvent_t l0, l1;
        cudaEventCreate(&l0);
        cudaEventCreate(&l1);
        cudaEventRecord(l0, g->stream);
        const cudaMemcpyKind kind = (gflags & GG_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if ((e = cudaMemcpyAsync(g->out_ptr, rowptr, 4 * ((size_t)n + 1), kind, g->stream)) != cudaSuccess ||
            (m > 0 && (e = cudaMemcpyAsync(g->out_dst, colidx, 4 * (size_t)m, kind, g->stream)) != cudaSuccess) ||
            (g->has_w && m > 0 && (e = cudaMemcpyAsync(g->out_w, weights, 4 * (size_t)m, kind, g->stream)) != cudaSuccess)) {
            st = cuda_fail(e, "cudaMemcpyAsync (graph upload)");
            cudaEventDestroy(l0);
            cudaEventDestroy(l1);
            break;
        }
        uint32_t mm = (uint32_t)m;
        if ((st = validate_csr(g)) != GG_OK || (st = build_hubs(g)) != GG_OK || (st = build_csc(g)) != GG_OK) {
            cudaEventDestroy(l0);
            cudaEventDestroy(l1);
            break;
        }
        if ((e = cudaMemcpyAsync(g->full_nnz, &mm, 4, cudaMemcpyHostToDevice, g->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(g->b_sched.p, 0, g->b_sched.bytes, g->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(g->b_status.p, 0, g->b_status.bytes, g->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(g->stamp, 0, 4 * (size_t)n, g->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(g->mask, 0, 4 * (g->mask_words + 1), g->stream)) != cudaSuccess) {
            st = cuda_fail(e, "cudaMemsetAsync (graph state)");
            cudaEventDestroy(l0);
            cudaEventDestroy(l1);
            break;
        }
        if ((e = launch_partition(g->in_ptr, n, g->full_nnz, g->max_tiles, g->full_tile_info, g->full_num_tiles,
                                  g->stream)) != cudaSuccess) {
            st = cuda_fail(e, "partition");
            cudaEventDestroy(l0);
            cudaEventDestroy(l1);
            break;
        }
        cudaEventRecord(l1, g->stream);
        if ((e = cudaStreamSynchronize(g->stream)) != cudaSuccess) {
            st = cuda_fail(e, "cudaStreamSynchronize (load)");
            cudaEventDestroy(l0);
            cudaEventDestroy(l1);
            break;
        }
        cudaEventElapsedTime(&g->stats.ms_load, l0, l1);
        g->stats.kernels_load = g->load_launches;
        cudaEventDestroy(l0);
        cudaEventDestroy(l1);
    } while (0);
    if (st != GG_OK) {
        gg_free_graph(g);
        return st;
    }
    *out = g;
    return GG_OK;
}

gg_status gg_sample_edges(gg_graph *g, double sample_ratio, uint64_t seed)
{
    if (!g) { set_error("gg_sample_edges: graph is NULL"); return GG_ERR_INVALID_ARG; }
    return sample_edges(g, sample_ratio, seed);
}

gg_status gg_run(gg_graph *g, gg_app app, double sample_ratio, gg_policy policy, const gg_params *p)
{
    if (!g) { set_error("gg_run: graph is NULL"); return GG_ERR_INVALID_ARG; }
    return run(g, app, sample_ratio, policy, p);
}

// Where a result lives and its size in bytes (0: it does not exist yet).
// The packed list's length is read back on the graph's stream.
static gg_status result_size(gg_graph *g, gg_result_kind kind, const void **src, size_t *bytes)
{
    *src = nullptr;
    *bytes = 0;
    const size_t n = (size_t)g->n, m = (size_t)g->m;
    switch (kind) {
    case GG_RESULT_VALUES:
        if (g->last_app < 0) break;
        *src = g->last_app == GG_APP_PAGERANK ? (const void *)g->rank[g->cur] : (const void *)g->val[g->cur];
        *bytes = 4 * n;
        break;
    case GG_RESULT_MASK:
        if (!g->sampled) break;
        *src = g->mask;
        *bytes = 4 * g->mask_words;
        break;
    case GG_RESULT_STATS: *bytes = sizeof(gg_stats); break;
    case GG_RESULT_ITER_STATS: *src = g->iter_stats; *bytes = sizeof(gg_iter_stats) * g->iterations; break;
    case GG_RESULT_CSC_PTR: *src = g->in_ptr; *bytes = 4 * (n + 1); break;
    case GG_RESULT_CSC_SRC: *src = g->in_src; *bytes = 4 * m; break;
    case GG_RESULT_CSC_W:
        if (!g->has_w) break;
        *src = g->in_w;
        *bytes = 4 * m;
        break;
    case GG_RESULT_SPARSE_PTR:
        if (!g->sampled) break;
        if (ensure_packed(g, false, PACK_ANY) != GG_OK) return GG_ERR_CUDA;
        *src = g->sp_ptr;
        *bytes = 4 * (n + 1);
        break;
    case GG_RESULT_SPARSE_SRC:
        if (!g->sampled) break;
        if (ensure_packed(g, false, PACK_ANY) != GG_OK) return GG_ERR_CUDA;
        GG_CUDA(cudaMemcpyAsync(&g->sp_nnz_host, g->sp_nnz, 4, cudaMemcpyDeviceToHost, g->stream));
        GG_CUDA(cudaStreamSynchronize(g->stream));
        *src = g->sp_src;
        *bytes = 4 * (size_t)g->sp_nnz_host;
        break;
    case GG_RESULT_OUT_TO_IN: *src = g->out_to_in; *bytes = 4 * m; break;
    case GG_RESULT_SCORES:
        if (!g->logits_valid) break;
        *src = g->logits;
        *bytes = 4 * n;
        break;
    }
    return GG_OK;
}

size_t gg_result_size(gg_graph *g, gg_result_kind kind)
{
    if (!g) { set_error("gg_result_size: graph is NULL"); return GG_RESULT_SIZE_ERROR; }
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) { cuda_fail(e, "cudaStreamSynchronize"); return GG_RESULT_SIZE_ERROR; }
    const void *src;
    size_t bytes = 0;
    if (result_size(g, kind, &src, &bytes) != GG_OK) return GG_RESULT_SIZE_ERROR;
    return bytes;
}

static gg_status fill_stats(gg_graph *g)
{
    gg_stats &s = g->stats;
    if (g->iterations > 0) {
        gg_iter_stats *h = new (std::nothrow) gg_iter_stats[g->iterations];
        if (!h) { set_error("host allocation failed"); return GG_ERR_OOM; }
        cudaError_t e = cudaMemcpyAsync(h, g->iter_stats, sizeof(gg_iter_stats) * g->iterations,
                                        cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) { delete[] h; return cuda_fail(e, "cudaMemcpyAsync (iteration stats)"); }
        uint64_t arcs = 0;
        for (uint32_t i = 0; i < g->iterations; ++i) arcs += (h[i].mode & 0xFFu) == MODE_SKIPPED ? 0 : h[i].arcs;
        s.arcs_processed = arcs;
        s.changed_last = h[g->iterations - 1].changed;
        delete[] h;
    }
    uint32_t nnz = (uint32_t)g->m;
    if (g->sampled) GG_CUDA(cudaMemcpyAsync(&nnz, g->sp_nnz, 4, cudaMemcpyDeviceToHost, g->stream));
    uint32_t err = 0;
    GG_CUDA(cudaMemcpyAsync(&err, g->dev_err, 4, cudaMemcpyDeviceToHost, g->stream));
    GG_CUDA(cudaStreamSynchronize(g->stream));
    s.active_arcs = nnz;
    s.trace_rows = g->trace_rows;
    s.device_error = err;
    if (g->run_timed) GG_CUDA(cudaEventElapsedTime(&s.ms_run, g->ev_run0, g->ev_run1));
    if (g->sample_timed) GG_CUDA(cudaEventElapsedTime(&s.ms_sample, g->ev_s0, g->ev_s1));
    s.ms_gather = s.ms_correct = s.ms_push = 0.0f;
    s.n_gather = s.n_correct = s.n_push = 0;
    for (size_t i = 0; i < g->timed_used; ++i) {
        float ms = 0.0f;
        GG_CUDA(cudaEventElapsedTime(&ms, g->timed[i].start, g->timed[i].stop));
        if (g->timed[i].cls == 0) { s.ms_gather += ms; s.n_gather++; }
        else if (g->timed[i].cls == 1) { s.ms_correct += ms; s.n_correct++; }
        else { s.ms_push += ms; s.n_push++; }
    }
    return GG_OK;
}

gg_status gg_result(gg_graph *g, gg_result_kind kind, void *dst, size_t bytes, int dst_is_device)
{
    if (!g || !dst) { set_error("gg_result: graph or dst is NULL"); return GG_ERR_INVALID_ARG; }
    GG_CUDA(cudaStreamSynchronize(g->stream));
    if ((int)kind < GG_RESULT_VALUES || (int)kind > GG_RESULT_SCORES) {
        set_error("gg_result: unknown kind %d", (int)kind);
        return GG_ERR_INVALID_ARG;
    }
    if (kind == GG_RESULT_STATS) {
        if (bytes < sizeof(gg_stats)) { set_error("gg_result: buffer too small"); return GG_ERR_INVALID_ARG; }
        gg_status st = fill_stats(g);
        if (st != GG_OK) return st;
        if (dst_is_device) {
            GG_CUDA(cudaMemcpyAsync(dst, &g->stats, sizeof(gg_stats), cudaMemcpyHostToDevice, g->stream));
            GG_CUDA(cudaStreamSynchronize(g->stream));
        } else {
            memcpy(dst, &g->stats, sizeof(gg_stats));
        }
        return GG_OK;
    }
    const void *src;
    size_t need = 0;
    gg_status rs = result_size(g, kind, &src, &need);
    if (rs != GG_OK) return rs;
    if (!src && need == 0 && kind != GG_RESULT_SPARSE_SRC && kind != GG_RESULT_ITER_STATS) {
        set_error("gg_result: result %d does not exist yet", (int)kind);
        return GG_ERR_STATE;
    }
    if (bytes < need) {
        set_error("gg_result: buffer of %zu bytes, result needs %zu", bytes, need);
        return GG_ERR_INVALID_ARG;
    }
    if (kind == GG_RESULT_SPARSE_SRC && need) {   // hub-coded sources back to vertex ids
        GG_CUDA(launch_decode_src(g->sp_src, g->sp_nnz, (uint32_t)(need / 4), g->hub_ids, (int32_t *)g->stash,
                                  g->num_sms, g->stream));
        GG_CUDA(cudaStreamSynchronize(g->stream));
        src = (const void *)g->stash;
    }
    if (need) {
        GG_CUDA(cudaMemcpyAsync(dst, src, need, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                g->stream));
        GG_CUDA(cudaStreamSynchronize(g->stream));
    }
    return GG_OK;
}

gg_status gg_set_stream(gg_graph *g, void *cuda_stream)
{
    if (!g) { set_error("gg_set_stream: graph is NULL"); return GG_ERR_INVALID_ARG; }
    g->stream = (cudaStream_t)cuda_stream;
    return GG_OK;
}

void gg_free_graph(gg_graph *g)
{
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    for (auto &t : g->timed) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    if (g->ev_run0) cudaEventDestroy(g->ev_run0);
    if (g->ev_run1) cudaEventDestroy(g->ev_run1);
    if (g->ev_s0) cudaEventDestroy(g->ev_s0);
    if (g->ev_s1) cudaEventDestroy(g->ev_s1);
    delete g;
}

const char *gg_last_error(void) { return g_err; }

gg_status gg_set_scorer(gg_graph *g, const float *params)
{
    if (!g || !params) { set_error("gg_set_scorer: graph or params is NULL"); return GG_ERR_INVALID_ARG; }
    if (!g->mlp) {
        GG_ALLOC_BUF(g->b_mlp, 4 * (size_t)GG_MLP_NPARAM);
        g->mlp = g->b_mlp.f32();
    }
    GG_CUDA(cudaMemcpyAsync(g->mlp, params, 4 * (size_t)GG_MLP_NPARAM, cudaMemcpyHostToDevice, g->stream));
    GG_CUDA(cudaStreamSynchronize(g->stream));
    g->has_scorer = true;
    return GG_OK;
}

gg_status gg_set_trace(gg_graph *g, float *features, uint8_t *labels, uint64_t cap_rows, float label_tol)
{
    if (!g) { set_error("gg_set_trace: graph is NULL"); return GG_ERR_INVALID_ARG; }
    if (features && !labels) { set_error("gg_set_trace: labels is NULL"); return GG_ERR_INVALID_ARG; }
    if (!(label_tol >= 0.0f && label_tol <= 3.0e38f)) {
        set_error("gg_set_trace: label_tol must be finite and >= 0");
        return GG_ERR_INVALID_ARG;
    }
    if (features && (((uintptr_t)features) & 7u)) { set_error("gg_set_trace: features must be 8-byte aligned"); return GG_ERR_INVALID_ARG; }
    g->trace_x = features;
    g->trace_y = features ? labels : nullptr;
    g->trace_cap = features ? cap_rows : 0;
    g->trace_rows = 0;
    g->label_tol = label_tol;
    return GG_OK;
}

gg_status gg_mlp_score(const float *features, uint64_t rows, const float *params, float *logits, void *stream)
{
    if (rows == 0) return GG_OK;
    if (!features || !params || !logits) { set_error("gg_mlp_score: NULL argument"); return GG_ERR_INVALID_ARG; }
    if (((uintptr_t)features) & 7u) { set_error("gg_mlp_score: features must be 8-byte aligned"); return GG_ERR_INVALID_ARG; }
    if (rows > ((uint64_t)1 << 40)) { set_error("gg_mlp_score: too many rows"); return GG_ERR_INVALID_ARG; }
    int dev = 0, sms = 0;
    GG_CUDA(cudaGetDevice(&dev));
    GG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GG_CUDA(launch_mlp_score(features, (long long)rows, params, logits, sms, (cudaStream_t)stream));
    return GG_OK;
}

gg_status gg_mlp_train(const float *features, const uint8_t *labels, uint64_t rows, float *params, uint32_t batch,
                       uint32_t steps, float lr, uint64_t stride, uint64_t start, float *losses, float *grad_last,
                       void *stream)
{
    if (!features || !labels || !params) { set_error("gg_mlp_train: NULL argument"); return GG_ERR_INVALID_ARG; }
    if (rows < 1 || rows > 0xFFFFFFFFull) { set_error("gg_mlp_train: rows must be in [1, 2^32)"); return GG_ERR_INVALID_ARG; }
    if (batch < 1 || batch > 16384) { set_error("gg_mlp_train: batch must be in [1, 16384]"); return GG_ERR_INVALID_ARG; }
    if (stride >= rows && rows > 1) { set_error("gg_mlp_train: stride must be < rows"); return GG_ERR_INVALID_ARG; }
    if (!(lr == lr)) { set_error("gg_mlp_train: lr is NaN"); return GG_ERR_INVALID_ARG; }
    if (((uintptr_t)features) & 7u) { set_error("gg_mlp_train: features must be 8-byte aligned"); return GG_ERR_INVALID_ARG; }
    if (steps == 0) return GG_OK;
    DevBuf scratch;   // partial gradients of the blocks, released in stream order
    gg_status st = scratch.alloc(4 * mlp_train_scratch((int)batch), (cudaStream_t)stream);
    if (st != GG_OK) return st;
    GG_CUDA(launch_mlp_train(features, labels, rows, params, (int)batch, (int)steps, lr, rows > 1 ? stride : 0,
                             start, losses, grad_last, scratch.f32(), (cudaStream_t)stream));
    return GG_OK;
}

}  // extern "C"

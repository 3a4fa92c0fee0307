/*
 * graphgen.c - seeded synthetic graph inputs shared by the tests, the bench
 * and the smoke check: R-MAT and Erdos-Renyi edge lists turned into CSR,
 * arc weights and source vertices.
 *
 * This module holds input generation only. It contains none of GraphGuess's
 * own arithmetic (sampling, gathering, influence, correction); its random
 * stream is Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC 2011), a generator the method itself never
 * uses.
 *
 * R-MAT follows Chakrabarti, Zhan, Faloutsos (SDM 2004): every arc descends
 * `scale` levels of the adjacency matrix, picking quadrant a (src bit 0, dst
 * bit 0), b (0, 1), c (1, 0) or d (1, 1) at each level. Vertex ids are then
 * relabelled by a seeded bijection so that hubs do not cluster at low ids.
 * Self-loops and duplicate arcs are kept, so the arc count is exact.
 *
 * Output CSR: rowptr int32[n+1], colidx int32[m], every row sorted by
 * destination ascending. All entry points return a negative value on error.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

/* Philox4x32 with 10 rounds: a counter (4 words) and a key (2 words) map to
 * 4 random words. */
void graphgen_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static inline void draw4(uint64_t i, uint32_t stream, uint32_t sub, uint64_t seed, uint32_t out[4])
{
    uint32_t c[4] = {(uint32_t)i, (uint32_t)(i >> 32), sub, stream};
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    graphgen_philox(c, k, out);
}

/* Seeded bijection on [0, 2^s): four rounds of (odd multiply + add) mod 2^s
 * followed by an xor-shift; each step is invertible on s bits. */
typedef struct { uint64_t mask, mul[4], add[4]; int shift; } relabel_t;

static void relabel_init(relabel_t *r, int s, uint64_t seed)
{
    r->mask = (s >= 64) ? ~0ull : ((1ull << s) - 1);
    r->shift = (s + 1) / 2;
    for (int i = 0; i < 4; ++i) {
        uint32_t o[4];
        draw4((uint64_t)i, 0x7E1Au, 0, seed, o);
        r->mul[i] = (((uint64_t)o[0] << 32) | o[1]) | 1ull;
        r->add[i] = ((uint64_t)o[2] << 32) | o[3];
    }
}

static inline uint64_t relabel_apply(const relabel_t *r, uint64_t x)
{
    for (int i = 0; i < 4; ++i) {
        x = (x * r->mul[i] + r->add[i]) & r->mask;
        x ^= x >> r->shift;
    }
    return x;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Arc list -> CSR with rows sorted by destination. */
static int arcs_to_csr(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                       int32_t *rowptr, int32_t *colidx)
{
    int32_t *fill = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    if (!fill) return -1;
    memset(rowptr, 0, ((size_t)n + 1) * sizeof(int32_t));
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e)
        __atomic_fetch_add(&rowptr[src[e] + 1], 1, __ATOMIC_RELAXED);
    for (int32_t v = 0; v < n; ++v) rowptr[v + 1] += rowptr[v];
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        int32_t s = src[e];
        int32_t k = __atomic_fetch_add(&fill[s], 1, __ATOMIC_RELAXED);
        colidx[rowptr[s] + k] = dst[e];
    }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t v = 0; v < n; ++v) {
        int32_t len = rowptr[v + 1] - rowptr[v];
        if (len > 1) qsort(colidx + rowptr[v], (size_t)len, sizeof(int32_t), cmp_i32);
    }
    free(fill);
    return 0;
}

/* R-MAT graph with 2^scale vertices from npairs generated pairs. Directed:
 * m = npairs arcs. Symmetric: every pair (u, v) gives arcs u->v and v->u, so
 * m = 2 * npairs. Returns m, or -1. */
int64_t graphgen_rmat_csr(int scale, int64_t npairs, double a, double b, double c,
                          uint64_t seed, int symmetric, int permute,
                          int32_t *rowptr, int32_t *colidx)
{
    if (scale < 1 || scale > 30 || npairs < 0) return -1;
    if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
    int32_t n = (int32_t)1 << scale;
    int64_t m = symmetric ? 2 * npairs : npairs;
    if (m >= ((int64_t)1 << 31)) return -1;
    int32_t *src = (int32_t *)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    int32_t *dst = (int32_t *)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    if (!src || !dst) { free(src); free(dst); return -1; }
    const double two32 = 4294967296.0;
    const uint64_t ta = (uint64_t)(a * two32);
    const uint64_t tab = (uint64_t)((a + b) * two32);
    const uint64_t tabc = (uint64_t)((a + b + c) * two32);
    relabel_t rl;
    relabel_init(&rl, scale, seed ^ 0x5CA1AB1Eull);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npairs; ++i) {
        uint64_t s = 0, d = 0;
        uint32_t r[4];
        for (int l = 0; l < scale; ++l) {
            if ((l & 3) == 0) draw4((uint64_t)i, 0x0A11u, (uint32_t)(l >> 2), seed, r);
            uint64_t u = r[l & 3];
            uint32_t sb, db;
            if (u < ta) { sb = 0; db = 0; }
            else if (u < tab) { sb = 0; db = 1; }
            else if (u < tabc) { sb = 1; db = 0; }
            else { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        if (permute) { s = relabel_apply(&rl, s); d = relabel_apply(&rl, d); }
        if (symmetric) {
            src[2 * i] = (int32_t)s; dst[2 * i] = (int32_t)d;
            src[2 * i + 1] = (int32_t)d; dst[2 * i + 1] = (int32_t)s;
        } else {
            src[i] = (int32_t)s; dst[i] = (int32_t)d;
        }
    }
    int rc = arcs_to_csr(n, m, src, dst, rowptr, colidx);
    free(src); free(dst);
    return rc < 0 ? -1 : m;
}

/* Erdos-Renyi-style multigraph: npairs pairs with independent uniform
 * endpoints in [0, n). Directed or symmetric as above. Returns m, or -1. */
int64_t graphgen_er_csr(int32_t n, int64_t npairs, uint64_t seed, int symmetric,
                        int32_t *rowptr, int32_t *colidx)
{
    if (n < 1 || npairs < 0) return -1;
    int64_t m = symmetric ? 2 * npairs : npairs;
    if (m >= ((int64_t)1 << 31)) return -1;
    int32_t *src = (int32_t *)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    int32_t *dst = (int32_t *)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    if (!src || !dst) { free(src); free(dst); return -1; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npairs; ++i) {
        uint32_t r[4];
        draw4((uint64_t)i, 0x0E70u, 0, seed, r);
        int32_t s = (int32_t)(((uint64_t)r[0] * (uint64_t)n) >> 32);
        int32_t d = (int32_t)(((uint64_t)r[1] * (uint64_t)n) >> 32);
        if (symmetric) {
            src[2 * i] = s; dst[2 * i] = d;
            src[2 * i + 1] = d; dst[2 * i + 1] = s;
        } else {
            src[i] = s; dst[i] = d;
        }
    }
    int rc = arcs_to_csr(n, m, src, dst, rowptr, colidx);
    free(src); free(dst);
    return rc < 0 ? -1 : m;
}

/* Arc weights uniform in [lo, hi], keyed on the unordered pair {src, dst} so
 * that both directions of an undirected edge, and duplicates, agree. */
int graphgen_weights(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                     uint64_t seed, uint32_t lo, uint32_t hi, uint32_t *w)
{
    if (n < 0 || hi < lo) return -1;
    const uint64_t span = (uint64_t)hi - lo + 1;
#pragma omp parallel for schedule(dynamic, 4096)
    for (int32_t s = 0; s < n; ++s) {
        for (int32_t e = rowptr[s]; e < rowptr[s + 1]; ++e) {
            int32_t d = colidx[e];
            uint32_t x = (uint32_t)(s < d ? s : d), y = (uint32_t)(s < d ? d : s);
            uint32_t c[4] = {x, y, 0x3E16u, 0};
            uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
            uint32_t r[4];
            graphgen_philox(c, k, r);
            w[e] = lo + (uint32_t)((((uint64_t)r[0] << 32 | r[1]) % span));
        }
    }
    return 0;
}

/* k distinct uniform-random vertices with out-degree > 0. Returns how many
 * were found (fewer than k only if the graph has fewer such vertices). */
int graphgen_sources(int32_t n, const int32_t *rowptr, uint64_t seed, int k, int32_t *out)
{
    int found = 0;
    int64_t nonempty = 0;
    for (int32_t v = 0; v < n; ++v) nonempty += rowptr[v + 1] > rowptr[v];
    if (k > nonempty) k = (int)nonempty;
    for (uint64_t t = 0; found < k && t < (uint64_t)1 << 40; ++t) {
        uint32_t r[4];
        draw4(t, 0x50C5u, 0, seed, r);
        int32_t v = (int32_t)(((uint64_t)r[0] * (uint64_t)n) >> 32);
        if (rowptr[v + 1] == rowptr[v]) continue;
        int dup = 0;
        for (int j = 0; j < found; ++j) dup |= (out[j] == v);
        if (!dup) out[found++] = v;
    }
    return found;
}

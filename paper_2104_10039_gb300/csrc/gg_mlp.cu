// gg_mlp.cu - the learned correction's scorer (beyond the paper, which only
// notes that the correction points could be chosen differently, Sec. 3.4): a
// per-vertex MLP 8 -> 64 -> 64 -> 1 with ReLU after both hidden layers.
//
// Arithmetic: weights and each layer's inputs in bfloat16 (round to nearest
// even), products accumulated in FP32 on the tensor cores (mma.sync
// m16n8k16, one warp per 16 rows), FP32 biases. Training runs its forward and
// backward contractions on the tensor cores too (k_train_grad). A layer's FP32 output
// fragment is, element for element, the next layer's input fragment, so the
// activations never leave registers.
//
// Parameters (FP32, row-major): W1[64][8], b1[64], W2[64][64], b2[64],
// w3[64], b3 - 4801 floats.
#include <cuda_bf16.h>

#include "gg_internal.cuh"

namespace gg {

namespace {

constexpr int kOffW1 = 0, kOffB1 = 512, kOffW2 = 576, kOffB2 = 4672, kOffW3 = 4736, kOffB3 = 4800;

// B-operand fragments of the three layers, per lane, plus the biases.
struct MlpFrag {
    uint32_t w1[8][32];      // layer 1: n-tile j (8 outputs), lane -> k = 2t, 2t+1 (k >= 8 is padding)
    uint2 w2[4][8][32];      // layer 2: k-chunk kc (16 inputs), n-tile j, lane -> k = 16kc+2t(+1), +8
    uint2 w3[4][32];         // layer 3: k-chunk kc, lane (only output column 0 is nonzero)
    float b1[64], b2[64], b3;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float2 unpack_bf16(uint32_t v)
{
    return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xFFFF0000u));
}

// D (16x8, FP32) += A (16x16, bf16, row-major) * B (16x8, bf16, column-major)
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Fragment layout of mma.m16n8k16 (bf16): with g = lane / 4 and t = lane % 4,
// A register 0 holds row g, columns 2t, 2t+1; register 1 row g+8; registers 2
// and 3 the same rows at columns 8+2t, 9+2t. B register 0 holds rows 2t, 2t+1
// of column g, register 1 rows 8+2t, 9+2t. D element 0/1 is row g, columns
// 2t, 2t+1; elements 2/3 row g+8.
__device__ void mlp_build(const float *P, MlpFrag &f)
{
    for (int i = threadIdx.x; i < 8 * 32; i += blockDim.x) {
        const int j = i >> 5, l = i & 31, g = l >> 2, t = l & 3;
        const float *w = P + kOffW1 + (8 * j + g) * 8 + 2 * t;
        f.w1[j][l] = pack_bf16(w[0], w[1]);
    }
    for (int i = threadIdx.x; i < 4 * 8 * 32; i += blockDim.x) {
        const int kc = i >> 8, j = (i >> 5) & 7, l = i & 31, g = l >> 2, t = l & 3;
        const float *w = P + kOffW2 + (8 * j + g) * 64 + 16 * kc + 2 * t;
        f.w2[kc][j][l] = make_uint2(pack_bf16(w[0], w[1]), pack_bf16(w[8], w[9]));
    }
    for (int i = threadIdx.x; i < 4 * 32; i += blockDim.x) {
        const int kc = i >> 5, l = i & 31, g = l >> 2, t = l & 3;
        const float *w = P + kOffW3 + 16 * kc + 2 * t;
        f.w3[kc][l] = g == 0 ? make_uint2(pack_bf16(w[0], w[1]), pack_bf16(w[8], w[9])) : make_uint2(0u, 0u);
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        f.b1[i] = P[kOffB1 + i];
        f.b2[i] = P[kOffB2 + i];
    }
    if (threadIdx.x == 0) f.b3 = P[kOffB3];
}

// One warp, 16 rows: xg = features (2t, 2t+1) of row g, xg8 of row g+8.
// Returns the logits of rows g and g+8 (valid in lanes with t == 0). With
// h1 / h2 (row-major [16][64] in shared memory) the rounded activations are
// kept for the backward pass.
__device__ __forceinline__ float2 mlp_forward16(const MlpFrag &f, float2 xg, float2 xg8, float *h1 = nullptr,
                                               float *h2 = nullptr)
{
    const int l = (int)lane_id(), g = l >> 2, t = l & 3;
    const uint32_t a0 = pack_bf16(xg.x, xg.y), a1 = pack_bf16(xg8.x, xg8.y);
    uint32_t A[4][4];
    {
        float d[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float c0 = f.b1[8 * j + 2 * t], c1 = f.b1[8 * j + 2 * t + 1];
            d[j][0] = c0;
            d[j][1] = c1;
            d[j][2] = c0;
            d[j][3] = c1;
            mma_bf16(d[j], a0, a1, 0u, 0u, f.w1[j][l], 0u);
        }
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            A[kc][0] = pack_bf16(fmaxf(d[2 * kc][0], 0.0f), fmaxf(d[2 * kc][1], 0.0f));
            A[kc][1] = pack_bf16(fmaxf(d[2 * kc][2], 0.0f), fmaxf(d[2 * kc][3], 0.0f));
            A[kc][2] = pack_bf16(fmaxf(d[2 * kc + 1][0], 0.0f), fmaxf(d[2 * kc + 1][1], 0.0f));
            A[kc][3] = pack_bf16(fmaxf(d[2 * kc + 1][2], 0.0f), fmaxf(d[2 * kc + 1][3], 0.0f));
        }
    }
    if (h1) {
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 v = unpack_bf16(A[kc][q]);
                const int row = g + ((q & 1) ? 8 : 0), col = 16 * kc + ((q & 2) ? 8 : 0) + 2 * t;
                h1[row * 64 + col] = v.x;
                h1[row * 64 + col + 1] = v.y;
            }
        }
    }
    uint32_t B[4][4];
    {
        float d[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float c0 = f.b2[8 * j + 2 * t], c1 = f.b2[8 * j + 2 * t + 1];
            d[j][0] = c0;
            d[j][1] = c1;
            d[j][2] = c0;
            d[j][3] = c1;
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {
                const uint2 w = f.w2[kc][j][l];
                mma_bf16(d[j], A[kc][0], A[kc][1], A[kc][2], A[kc][3], w.x, w.y);
            }
        }
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            B[kc][0] = pack_bf16(fmaxf(d[2 * kc][0], 0.0f), fmaxf(d[2 * kc][1], 0.0f));
            B[kc][1] = pack_bf16(fmaxf(d[2 * kc][2], 0.0f), fmaxf(d[2 * kc][3], 0.0f));
            B[kc][2] = pack_bf16(fmaxf(d[2 * kc + 1][0], 0.0f), fmaxf(d[2 * kc + 1][1], 0.0f));
            B[kc][3] = pack_bf16(fmaxf(d[2 * kc + 1][2], 0.0f), fmaxf(d[2 * kc + 1][3], 0.0f));
        }
    }
    if (h2) {
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 v = unpack_bf16(B[kc][q]);
                const int row = g + ((q & 1) ? 8 : 0), col = 16 * kc + ((q & 2) ? 8 : 0) + 2 * t;
                h2[row * 64 + col] = v.x;
                h2[row * 64 + col + 1] = v.y;
            }
        }
    }
    float d[4] = {f.b3, 0.0f, f.b3, 0.0f};
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
        const uint2 w = f.w3[kc][l];
        mma_bf16(d, B[kc][0], B[kc][1], B[kc][2], B[kc][3], w.x, w.y);
    }
    return make_float2(d[0], d[2]);
}

__device__ __forceinline__ float2 ld_pair(const float *x, long long row, long long rows, int t)
{
    if (row >= rows) return make_float2(0.0f, 0.0f);
    return *reinterpret_cast<const float2 *>(x + row * 8 + 2 * t);
}

__global__ void __launch_bounds__(256) k_mlp_score(const float *__restrict__ x, long long rows,
                                                   const float *__restrict__ P, float *__restrict__ logits)
{
    __shared__ MlpFrag f;
    mlp_build(P, f);
    __syncthreads();
    const int l = (int)lane_id(), g = l >> 2, t = l & 3;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long grp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); grp * 16 < rows;
         grp += nwarps) {
        const long long r0 = grp * 16 + g, r1 = r0 + 8;
        const float2 z = mlp_forward16(f, ld_pair(x, r0, rows, t), ld_pair(x, r1, rows, t));
        if (t == 0) {
            if (r0 < rows) logits[r0] = z.x;
            if (r1 < rows) logits[r1] = z.y;
        }
    }
}

// Features (2t, 2t+1) of vertex u (Sec. 3.4 gives the signals a correction
// could look at; the choice is this project's): sqrt(in-degree)/64,
// sqrt(out-degree)/64 | change features of the last two executed iterations |
// of the third, active fraction of the in-edges | iteration/64, app id.
__device__ __forceinline__ float2 feature_pair(const FeatArgs &fa, int32_t u, int t, int32_t *indeg)
{
    if (u >= fa.n) return make_float2(0.0f, 0.0f);
    switch (t) {
    case 0: {
        const int32_t di = fa.in_ptr[u + 1] - fa.in_ptr[u];
        const int32_t dout = fa.out_ptr[u + 1] - fa.out_ptr[u];
        *indeg = di;
        return make_float2(__fmul_rn(__fsqrt_rn((float)di), 0.015625f), __fmul_rn(__fsqrt_rn((float)dout), 0.015625f));
    }
    case 1: return make_float2(fa.hist1[u], fa.hist2[u]);
    case 2: {
        const int32_t di = fa.in_ptr[u + 1] - fa.in_ptr[u];
        const int32_t act = fa.sp_ptr[u + 1] - fa.sp_ptr[u];
        return make_float2(fa.hist3[u], di > 0 ? __fdiv_rn((float)act, (float)di) : 1.0f);
    }
    default: return make_float2(fa.iter_f, fa.app_f);
    }
}

// Learned correction, step 1: score every vertex; select those whose logit
// exceeds fmaf(cost, L(d), tau), L(d) the bit length of the in-degree d.
__global__ void __launch_bounds__(256) k_mlp_select(FeatArgs fa, const float *__restrict__ P, float tau, float cost,
                                                    uint32_t *__restrict__ sel_flag, uint32_t *__restrict__ sel_deg,
                                                    float *__restrict__ logits)
{
    __shared__ MlpFrag f;
    mlp_build(P, f);
    __syncthreads();
    const int l = (int)lane_id(), g = l >> 2, t = l & 3;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    // the next group's features are loaded while this group runs the MLP
    long long grp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int32_t nd0 = 0, nd1 = 0;
    float2 nx0 = feature_pair(fa, (int32_t)(grp * 16 + g), t, &nd0);
    float2 nx1 = feature_pair(fa, (int32_t)(grp * 16 + g + 8), t, &nd1);
    for (; grp * 16 < fa.n; grp += nwarps) {
        const int32_t u0 = (int32_t)(grp * 16 + g), u1 = u0 + 8;
        const int32_t d0 = nd0, d1 = nd1;
        const float2 x0 = nx0, x1 = nx1;
        const long long ng = grp + nwarps;
        nd0 = nd1 = 0;
        nx0 = feature_pair(fa, ng * 16 < fa.n ? (int32_t)(ng * 16 + g) : fa.n, t, &nd0);
        nx1 = feature_pair(fa, ng * 16 < fa.n ? (int32_t)(ng * 16 + g + 8) : fa.n, t, &nd1);
        const float2 z = mlp_forward16(f, x0, x1);
        if (t == 0) {
            if (u0 < fa.n) {
                const bool s = z.x > __fmaf_rn(cost, (float)(32 - __clz(d0)), tau);
                sel_flag[u0] = s;
                sel_deg[u0] = s ? (uint32_t)d0 : 0u;
                if (logits) logits[u0] = z.x;
            }
            if (u1 < fa.n) {
                const bool s = z.y > __fmaf_rn(cost, (float)(32 - __clz(d1)), tau);
                sel_flag[u1] = s;
                sel_deg[u1] = s ? (uint32_t)d1 : 0u;
                if (logits) logits[u1] = z.y;
            }
        }
    }
}

// Trace: the features of every vertex, rows out[u * 8 ...].
__global__ void __launch_bounds__(256) k_trace_features(FeatArgs fa, float *__restrict__ out)
{
    const int t = (int)(threadIdx.x & 3);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 4LL * fa.n;
         i += (long long)gridDim.x * blockDim.x) {
        const int32_t u = (int32_t)(i >> 2);
        int32_t d = 0;
        *reinterpret_cast<float2 *>(out + (long long)u * 8 + 2 * t) = feature_pair(fa, u, t, &d);
    }
}

// Trace labels after a full correction: PageRank |new - old| > tol |new|
// (FP32), the min applications new < old.
__global__ void k_trace_labels(int32_t n, const float *__restrict__ rc, const float *__restrict__ rn,
                               const uint32_t *__restrict__ vc, const uint32_t *__restrict__ vn, float tol,
                               uint8_t *__restrict__ y)
{
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        bool lab;
        if (rc) {
            const float nw = rn[u];
            lab = fabsf(__fsub_rn(nw, rc[u])) > __fmul_rn(tol, fabsf(nw));
        } else {
            lab = vn[u] < vc[u];
        }
        y[u] = lab ? 1 : 0;
    }
}

// ---------------------------------------------------------------- training ---
// One SGD step on the mean logistic loss over a minibatch of B rows, in two
// launches: k_train_grad (one block per 128 rows) runs the forward pass and
// the backward contractions on the tensor cores and writes the block's
// partial gradient; k_train_update sums the blocks' partials in block order
// and updates the parameters (deterministic). The backward contractions
//   dH1 = (dH2 W2) .* [H1 > 0],   gW2 = dH2^T H1,   gW1 = dH1^T X
// run as mma.sync m16n8k16 (bfloat16 operands, FP32 accumulation). H1 and X
// are bfloat16 values already; the FP32 gradients dH2 and dH1 enter as two
// bfloat16 parts (hi = bf16(v), lo = bf16(v - hi)) in two products, so the
// operands lose almost nothing to the rounding. Biases and w3: FP32 column
// sums in row order.
constexpr int kTrainRows = 128;   // rows per block (8 warps x 16)

struct GradSmem {
    MlpFrag f;                    // forward fragments
    uint2 w2b[4][8][32];          // backward B fragments: B[k = j][n = i] = W2[j][i], k-chunk, n-tile, lane
    float w3r[64];                // bfloat16 values of w3
    float X[kTrainRows][8];       // bfloat16 values of the inputs
    float H1[kTrainRows][64];
    float H2[kTrainRows][64];
    float DH2[kTrainRows][64];
    float DH1[kTrainRows][64];
    float Z[kTrainRows];
    float DZ[kTrainRows];
    float red[8];
    unsigned long long idx[kTrainRows];
};

// hi / lo bfloat16 parts of two FP32 values, packed
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    hi = pack_bf16(a, b);
    const float2 h = unpack_bf16(hi);
    lo = pack_bf16(a - h.x, b - h.y);
}

__global__ void __launch_bounds__(256) k_train_grad(const float *__restrict__ x, const uint8_t *__restrict__ y,
                                                    unsigned long long rows, const float *__restrict__ params, int B,
                                                    unsigned long long first, unsigned long long stride,
                                                    float *__restrict__ part, float *__restrict__ loss_part)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GradSmem &s = *reinterpret_cast<GradSmem *>(smem_raw);
    const int tid = threadIdx.x, w = tid >> 5;
    const int l = (int)lane_id(), g = l >> 2, t = l & 3;
    const int row0 = kTrainRows * (int)blockIdx.x;
    mlp_build(params, s.f);
    for (int i = tid; i < 4 * 8 * 32; i += blockDim.x) {
        const int kc = i >> 8, j = (i >> 5) & 7, ln = i & 31, gg_ = ln >> 2, tt = ln & 3;
        const float *p0 = params + kOffW2 + (16 * kc + 2 * tt) * 64 + 8 * j + gg_;
        s.w2b[kc][j][ln] = make_uint2(pack_bf16(p0[0], p0[64]), pack_bf16(p0[8 * 64], p0[9 * 64]));
    }
    if (tid < 64) s.w3r[tid] = bf16r(params[kOffW3 + tid]);
    if (tid < kTrainRows) {
        const unsigned long long j = (first + (unsigned long long)(row0 + tid)) % rows;
        s.idx[tid] = (j * stride) % rows;
    }
    __syncthreads();
    // ---- forward (16 rows per warp), activations kept -----------------------
    {
        const int r0 = 16 * w + g, r1 = r0 + 8;
        const bool v0 = row0 + r0 < B, v1 = row0 + r1 < B;
        const float2 xa = v0 ? *reinterpret_cast<const float2 *>(x + s.idx[r0] * 8 + 2 * t) : make_float2(0.0f, 0.0f);
        const float2 xb = v1 ? *reinterpret_cast<const float2 *>(x + s.idx[r1] * 8 + 2 * t) : make_float2(0.0f, 0.0f);
        s.X[r0][2 * t] = bf16r(xa.x);
        s.X[r0][2 * t + 1] = bf16r(xa.y);
        s.X[r1][2 * t] = bf16r(xb.x);
        s.X[r1][2 * t + 1] = bf16r(xb.y);
        const float2 z = mlp_forward16(s.f, xa, xb, &s.H1[16 * w][0], &s.H2[16 * w][0]);
        if (t == 0) {
            s.Z[r0] = z.x;
            s.Z[r1] = z.y;
        }
    }
    __syncthreads();
    // ---- loss and dL/dz (rows past the batch contribute nothing) -------------
    float lpart = 0.0f;
    if (tid < kTrainRows) {
        float dz = 0.0f;
        if (row0 + tid < B) {
            const float z = s.Z[tid];
            const float lab = y[s.idx[tid]] ? 1.0f : 0.0f;
            dz = (1.0f / (1.0f + expf(-z)) - lab) / (float)B;
            lpart = fmaxf(z, 0.0f) - z * lab + log1pf(expf(-fabsf(z)));
        }
        s.DZ[tid] = dz;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lpart += __shfl_xor_sync(0xFFFFFFFFu, lpart, o);
    if (l == 0) s.red[w] = lpart;
    __syncthreads();
    if (tid == 0) {
        float sum = 0.0f;
        for (int i = 0; i < 8; ++i) sum += s.red[i];
        loss_part[blockIdx.x] = sum;
    }
    for (int i = tid; i < kTrainRows * 64; i += blockDim.x) {
        const int r = i >> 6, j = i & 63;
        s.DH2[r][j] = s.H2[r][j] > 0.0f ? s.DZ[r] * s.w3r[j] : 0.0f;
    }
    __syncthreads();
    // ---- dH1 = (dH2 W2) .* [H1 > 0]: warp w, rows 16w .. 16w + 15 -----------
    {
        const int ra = 16 * w + g, rb = ra + 8;
        uint32_t ah[4][4], al[4][4];
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            const int c = 16 * kc + 2 * t;
            split2(s.DH2[ra][c], s.DH2[ra][c + 1], ah[kc][0], al[kc][0]);
            split2(s.DH2[rb][c], s.DH2[rb][c + 1], ah[kc][1], al[kc][1]);
            split2(s.DH2[ra][c + 8], s.DH2[ra][c + 9], ah[kc][2], al[kc][2]);
            split2(s.DH2[rb][c + 8], s.DH2[rb][c + 9], ah[kc][3], al[kc][3]);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {
                const uint2 b = s.w2b[kc][nt][l];
                mma_bf16(d, ah[kc][0], ah[kc][1], ah[kc][2], ah[kc][3], b.x, b.y);
                mma_bf16(d, al[kc][0], al[kc][1], al[kc][2], al[kc][3], b.x, b.y);
            }
            const int c = 8 * nt + 2 * t;
            s.DH1[ra][c] = s.H1[ra][c] > 0.0f ? d[0] : 0.0f;
            s.DH1[ra][c + 1] = s.H1[ra][c + 1] > 0.0f ? d[1] : 0.0f;
            s.DH1[rb][c] = s.H1[rb][c] > 0.0f ? d[2] : 0.0f;
            s.DH1[rb][c + 1] = s.H1[rb][c + 1] > 0.0f ? d[3] : 0.0f;
        }
    }
    __syncthreads();
    float *pb = part + (size_t)blockIdx.x * GG_MLP_NPARAM;
    // ---- gW2[j][i] = sum_r dH2[r][j] H1[r][i]: warp w, j-tile w & 3, i-tiles 4 (w >> 2) .. +3
    {
        const int mt = w & 3, nt0 = 4 * (w >> 2);
        float d[4][4] = {};
#pragma unroll 2
        for (int kc = 0; kc < kTrainRows / 16; ++kc) {
            const int r = 16 * kc + 2 * t, jr = 16 * mt + g;
            uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
            split2(s.DH2[r][jr], s.DH2[r + 1][jr], h0, l0);
            split2(s.DH2[r][jr + 8], s.DH2[r + 1][jr + 8], h1, l1);
            split2(s.DH2[r + 8][jr], s.DH2[r + 9][jr], h2, l2);
            split2(s.DH2[r + 8][jr + 8], s.DH2[r + 9][jr + 8], h3, l3);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int ic = 8 * (nt0 + q) + g;
                const uint32_t b0 = pack_bf16(s.H1[r][ic], s.H1[r + 1][ic]);
                const uint32_t b1 = pack_bf16(s.H1[r + 8][ic], s.H1[r + 9][ic]);
                mma_bf16(d[q], h0, h1, h2, h3, b0, b1);
                mma_bf16(d[q], l0, l1, l2, l3, b0, b1);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j0 = 16 * mt + g, i0 = 8 * (nt0 + q) + 2 * t;
            pb[kOffW2 + j0 * 64 + i0] = d[q][0];
            pb[kOffW2 + j0 * 64 + i0 + 1] = d[q][1];
            pb[kOffW2 + (j0 + 8) * 64 + i0] = d[q][2];
            pb[kOffW2 + (j0 + 8) * 64 + i0 + 1] = d[q][3];
        }
    }
    if (w < 4) {
        // ---- gW1[k][f] = sum_r dH1[r][k] X[r][f]: warp w, k-tile w ----------
        float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 2
        for (int kc = 0; kc < kTrainRows / 16; ++kc) {
            const int r = 16 * kc + 2 * t, kr = 16 * w + g;
            uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
            split2(s.DH1[r][kr], s.DH1[r + 1][kr], h0, l0);
            split2(s.DH1[r][kr + 8], s.DH1[r + 1][kr + 8], h1, l1);
            split2(s.DH1[r + 8][kr], s.DH1[r + 9][kr], h2, l2);
            split2(s.DH1[r + 8][kr + 8], s.DH1[r + 9][kr + 8], h3, l3);
            const uint32_t b0 = pack_bf16(s.X[r][g], s.X[r + 1][g]);
            const uint32_t b1 = pack_bf16(s.X[r + 8][g], s.X[r + 9][g]);
            mma_bf16(d, h0, h1, h2, h3, b0, b1);
            mma_bf16(d, l0, l1, l2, l3, b0, b1);
        }
        const int k0 = 16 * w + g, f0 = 2 * t;
        pb[kOffW1 + k0 * 8 + f0] = d[0];
        pb[kOffW1 + k0 * 8 + f0 + 1] = d[1];
        pb[kOffW1 + (k0 + 8) * 8 + f0] = d[2];
        pb[kOffW1 + (k0 + 8) * 8 + f0 + 1] = d[3];
    } else {
        // ---- biases and w3: column sums in row order --------------------------
        for (int c = tid - 128; c < 193; c += 128) {
            float acc = 0.0f;
            if (c < 64) {
                for (int r = 0; r < kTrainRows; ++r) acc += s.DH1[r][c];
                pb[kOffB1 + c] = acc;
            } else if (c < 128) {
                for (int r = 0; r < kTrainRows; ++r) acc += s.DH2[r][c - 64];
                pb[kOffB2 + c - 64] = acc;
            } else if (c < 192) {
                for (int r = 0; r < kTrainRows; ++r) acc = fmaf(s.DZ[r], s.H2[r][c - 128], acc);
                pb[kOffW3 + c - 128] = acc;
            } else {
                for (int r = 0; r < kTrainRows; ++r) acc += s.DZ[r];
                pb[kOffB3] = acc;
            }
        }
    }
}

// Sum of the blocks' partial gradients in block order; parameters updated.
__global__ void __launch_bounds__(256) k_train_update(const float *__restrict__ part, int nb,
                                                      const float *__restrict__ loss_part, float *__restrict__ params,
                                                      float lr, float inv_b, float *__restrict__ loss_out,
                                                      float *__restrict__ grad_out)
{
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < GG_MLP_NPARAM; o += gridDim.x * blockDim.x) {
        float gsum = 0.0f;
        for (int b = 0; b < nb; ++b) gsum += part[(size_t)b * GG_MLP_NPARAM + o];
        if (grad_out) grad_out[o] = gsum;
        params[o] = params[o] - lr * gsum;
    }
    if (loss_out && blockIdx.x == 0 && threadIdx.x == 0) {
        float sum = 0.0f;
        for (int b = 0; b < nb; ++b) sum += loss_part[b];
        *loss_out = sum * inv_b;
    }
}

}  // namespace

// ------------------------------------------------------------- launchers ---
cudaError_t launch_mlp_score(const float *x, long long rows, const float *P, float *logits, int num_sms,
                             cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    long long blocks = (rows + 127) / 128;   // 8 warps x 16 rows
    if (blocks > (long long)num_sms * 4) blocks = (long long)num_sms * 4;
    k_mlp_score<<<(unsigned)blocks, 256, 0, s>>>(x, rows, P, logits);
    return cudaGetLastError();
}

cudaError_t launch_mlp_select(const FeatArgs &fa, const float *P, float tau, float cost, uint32_t *sel_flag,
                              uint32_t *sel_deg,
                              float *logits, int num_sms, cudaStream_t s)
{
    long long blocks = ((long long)fa.n + 127) / 128;
    if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
    if (blocks < 1) blocks = 1;
    k_mlp_select<<<(unsigned)blocks, 256, 0, s>>>(fa, P, tau, cost, sel_flag, sel_deg, logits);
    return cudaGetLastError();
}

cudaError_t launch_trace_features(const FeatArgs &fa, float *out, int num_sms, cudaStream_t s)
{
    long long blocks = (4LL * fa.n + 255) / 256;
    if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
    if (blocks < 1) blocks = 1;
    k_trace_features<<<(unsigned)blocks, 256, 0, s>>>(fa, out);
    return cudaGetLastError();
}

cudaError_t launch_trace_labels(int32_t n, const float *rc, const float *rn, const uint32_t *vc, const uint32_t *vn,
                                float tol, uint8_t *y, int num_sms, cudaStream_t s)
{
    k_trace_labels<<<num_sms * 8, 256, 0, s>>>(n, rc, rn, vc, vn, tol, y);
    return cudaGetLastError();
}

size_t mlp_train_smem() { return sizeof(GradSmem); }

cudaError_t launch_mlp_train(const float *x, const uint8_t *y, unsigned long long rows, float *params, int B,
                             int steps, float lr, unsigned long long stride, unsigned long long start, float *losses,
                             float *grad_last, float *scratch, cudaStream_t s)
{
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_train_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(GradSmem));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int nb = (B + kTrainRows - 1) / kTrainRows;
    float *part = scratch, *loss_part = scratch + (size_t)nb * GG_MLP_NPARAM;
    for (int step = 0; step < steps; ++step) {
        const unsigned long long first = start + (unsigned long long)step * (unsigned long long)B;
        k_train_grad<<<nb, 256, sizeof(GradSmem), s>>>(x, y, rows, params, B, first, stride, part, loss_part);
        k_train_update<<<(GG_MLP_NPARAM + 255) / 256, 256, 0, s>>>(part, nb, loss_part, params, lr, 1.0f / (float)B,
                                                                   losses ? losses + step : nullptr,
                                                                   step == steps - 1 ? grad_last : nullptr);
    }
    return cudaGetLastError();
}

// Scratch (floats) of launch_mlp_train: the blocks' partial gradients and losses.
size_t mlp_train_scratch(int B)
{
    const size_t nb = (size_t)(B + kTrainRows - 1) / kTrainRows;
    return nb * GG_MLP_NPARAM + nb;
}

}  // namespace gg

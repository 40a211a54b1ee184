// mlp.cu - the learned ring filter: ring features, an MLP 16 -> 128 -> 128 ->
// 128 -> 2 (ReLU) whose outputs are a source/background logit z and the log v
// of a predicted ring width, its loss and gradients, Adam, and the filter that
// applies it to rings before the sweep.
//
// The forward pass (k_mlp_forward_tc, below) runs the whole network in one
// persistent kernel on the tcgen05 tensor cores, for inference and for
// training (which keeps the activations).  The backward pass runs its matrix
// products through one BF16 GEMM kernel on the warp-level tensor-core path
// (mma.sync m16n8k16, FP32 accumulation, operands staged through shared
// memory and loaded with ldmatrix): strided operand addressing lets the same
// kernel do both products of the backward pass, dP x W (through a layer) and
// dP^T x A (weight gradient, reduced over the batch in fixed-order split-K
// partials, so results are deterministic).  Weights, layer inputs and
// backward signals are BF16; biases, accumulators, losses, gradients and the
// Adam state are FP32.
#include <cuda_bf16.h>

#include "cc_math.cuh"
#include "cc_pipe.cuh"

namespace cc {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kH = 128;                   // hidden width
constexpr int kF = CC_MLP_FEATURES;       // 16 input features
constexpr int kP = CC_MLP_PARAMS;         // 35,458 parameters
constexpr int kChunk = 65536;             // rows per forward/backward pass

// offsets of the flat parameter vector
constexpr int oW1 = 0, ob1 = oW1 + kH * kF, oW2 = ob1 + kH, ob2 = oW2 + kH * kH,
              oW3 = ob2 + kH, ob3 = oW3 + kH * kH, oW4 = ob3 + kH, ob4 = oW4 + 2 * kH;
static_assert(ob4 + 2 == kP, "parameter layout");

// ---------------------------------------------------------------------------
// BF16 tensor-core GEMM:  C[M,N] = A[M,K] B[K,N]  (+ bias, ReLU, mask)
// ---------------------------------------------------------------------------
constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;

struct GemmArgs {
    int M, N, K;
    const bf16 *A;
    int64_t lda_m, lda_k;       // A(m, k) = A[m * lda_m + k * lda_k]
    const bf16 *B;
    int64_t ldb_k, ldb_n;       // B(k, n) = B[k * ldb_k + n * ldb_n]
    const float *bias;          // [N] or null
    int relu;
    const bf16 *mask;           // keep C(m, n) only where mask[m * ldmask + n] > 0
    int64_t ldmask;
    void *C;                    // output, row stride ldc
    int64_t ldc;
    int c_bf16;
    float *part;                // split-K partials [gridDim.z][M][N] when gridDim.z > 1
    int ksplit;                 // K per split, multiple of BK
};

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void *p) {
    unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ void ldmatrix_x2(uint32_t (&r)[2], const void *p) {
    unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) k_gemm(GemmArgs g) {
    __shared__ __align__(16) bf16 As[BM][BK + PAD];   // [m][k]
    __shared__ __align__(16) bf16 Bs[BN][BK + PAD];   // [n][k]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * g.ksplit;
    const int kend = min(g.K, kbeg + g.ksplit);
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const bf16 zero = __float2bfloat16(0.0f);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int r = 0; r < 4; r++) acc[i][j][r] = 0.0f;

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        // stage the tiles; consecutive threads walk the unit-stride index
        for (int e = tid; e < BM * BK; e += 128) {
            int mm, kk;
            if (g.lda_m == 1) { mm = e % BM; kk = e / BM; } else { mm = e / BK; kk = e % BK; }
            const int m = m0 + mm, k = k0 + kk;
            As[mm][kk] = (m < g.M && k < kend) ? g.A[m * g.lda_m + k * g.lda_k] : zero;
        }
        for (int e = tid; e < BN * BK; e += 128) {
            int nn, kk;
            if (g.ldb_n == 1) { nn = e % BN; kk = e / BN; } else { nn = e / BK; kk = e % BK; }
            const int n = n0 + nn, k = k0 + kk;
            Bs[nn][kk] = (n < g.N && k < kend) ? g.B[k * g.ldb_k + n * g.ldb_n] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; i++)
                ldmatrix_x4(a[i], &As[wm + i * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
            for (int j = 0; j < 4; j++)
                ldmatrix_x2(b[j], &Bs[wn + j * 8 + (lane & 7)][kk + ((lane >> 3) & 1) * 8]);
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) mma_bf16(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int row = m0 + wm + i * 16 + (lane >> 2) + ((r & 2) ? 8 : 0);
                const int col = n0 + wn + j * 8 + 2 * (lane & 3) + (r & 1);
                if (row >= g.M || col >= g.N ||
                    !CC_IN_BOUNDS(CC_SITE_MLP_GEMM_OUT, (int64_t)row * g.N + col, (int64_t)g.M * g.N))
                    continue;
                float v = acc[i][j][r];
                if (gridDim.z > 1) {
                    g.part[((int64_t)blockIdx.z * g.M + row) * g.N + col] = v;
                    continue;
                }
                if (g.bias) v += g.bias[col];
                if (g.relu) v = fmaxf(v, 0.0f);
                if (g.mask && !(__bfloat162float(g.mask[row * g.ldmask + col]) > 0.0f)) v = 0.0f;
                if (g.c_bf16)
                    static_cast<bf16 *>(g.C)[row * g.ldc + col] = __float2bfloat16(v);
                else
                    static_cast<float *>(g.C)[row * g.ldc + col] = v;
            }
}

// out[i] = sum over splits of part[s][i], in split order
__global__ void k_sum_splits(const float *__restrict__ part, int S, int64_t n,
                             float *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int z = 0; z < S; z++) s += part[z * n + i];
    out[i] = s;
}

cudaError_t gemm(const GemmArgs &g0, cudaStream_t s) {
    GemmArgs g = g0;
    int S = 1;
    if (g.part) {
        g.ksplit = ((g.ksplit + BK - 1) / BK) * BK;
        S = (g.K + g.ksplit - 1) / g.ksplit;
    } else {
        g.ksplit = ((g.K + BK - 1) / BK) * BK;
    }
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, S);
    k_gemm<<<grid, 128, 0, s>>>(g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || S == 1) return e;
    int64_t n = (int64_t)g.M * g.N;
    k_sum_splits<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g.part, S, n,
                                                             static_cast<float *>(g.C));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// element-wise kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ void perm_of_rank(int k, int rank, int (&o)[4]) {
    int avail[4] = {0, 1, 2, 3};
    int f = k == 4 ? 6 : (k == 3 ? 2 : 1);
    for (int p = 0; p < k; p++) {
        int q = rank / f;
        rank %= f;
        o[p] = avail[q];
        for (int j = q; j < 3; j++) avail[j] = avail[j + 1];
        if (k - 1 - p > 0) f /= (k - 1 - p);
    }
}

__global__ void k_features(const uint8_t *__restrict__ n, const float *__restrict__ xs,
                           const float *__restrict__ ys, const float *__restrict__ zs,
                           const float *__restrict__ es, int64_t count, int64_t stride,
                           const float *__restrict__ az, const float *__restrict__ eta,
                           const float *__restrict__ deta, const uint8_t *__restrict__ valid,
                           const uint8_t *__restrict__ perm, float sig_pos,
                           bf16 *__restrict__ F) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    float f[kF];
#pragma unroll
    for (int q = 0; q < kF; q++) f[q] = 0.0f;
    const int k = n[i];
    if (valid[i] && k >= 2 && k <= 4) {
        int o[4];
        perm_of_rank(k, perm[i], o);
        float x[4], y[4], z[4], e[4], e0 = 0.0f;
        for (int s = 0; s < k; s++) {
            x[s] = xs[s * stride + i];
            y[s] = ys[s * stride + i];
            z[s] = zs[s * stride + i];
            e[s] = es[s * stride + i];
            e0 += e[s];
        }
        const int a = o[0], b = o[1], l = o[k - 1];
        float dx = x[a] - x[b], dy = y[a] - y[b], dz = z[a] - z[b];
        float L = sqrtf(dx * dx + dy * dy + dz * dz);
        float th = eta[i], de = deta[i];
        f[0] = th * (1.0f / kPiF);
        f[1] = cosf(th);
        f[2] = sinf(th);
        f[3] = 0.25f * logf(de);
        f[4] = k == 2;
        f[5] = k == 3;
        f[6] = k == 4;
        f[7] = logf(e0 * (1.0f / 500.0f));
        f[8] = e[a] / e0;
        f[9] = e[b] / e0;
        f[10] = e[l] / e0;
        f[11] = logf(L * 0.2f);
        f[12] = az[i];
        f[13] = z[a] * (1.0f / 30.0f);
        f[14] = z[b] * (1.0f / 30.0f);
        f[15] = 1.41421356237f * sig_pos / (L * de);
    }
#pragma unroll
    for (int q = 0; q < kF; q++) F[i * kF + q] = __float2bfloat16(f[q]);
}

// d(loss)/d(out) for a batch, as BF16 [B, 2]; per-block loss partial sums.
__global__ void k_loss_grad(const float *__restrict__ out, const uint8_t *__restrict__ y,
                            const float *__restrict__ res, const uint8_t *__restrict__ w,
                            int64_t B, float inv_total, bf16 *__restrict__ dout,
                            float *__restrict__ loss_part) {
    __shared__ float red[256];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (i < B) {
        float z = out[2 * i], v = out[2 * i + 1];
        float yy = y[i] ? 1.0f : 0.0f, ww = w[i] ? 1.0f : 0.0f, r = res[i];
        float sg = 1.0f / (1.0f + expf(-z));
        float e2v = expf(-2.0f * v);
        dout[2 * i] = __float2bfloat16(ww * (sg - yy) * inv_total);
        dout[2 * i + 1] = __float2bfloat16(ww * yy * (1.0f - r * r * e2v) * inv_total);
        float bce = fmaxf(z, 0.0f) - z * yy + log1pf(expf(-fabsf(z)));
        l = ww * (bce + yy * (v + 0.5f * r * r * e2v)) * inv_total;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// Column sums of a BF16 [B, N] matrix (bias gradients), one block per column,
// fixed order.
__global__ void k_col_sums(const bf16 *__restrict__ X, int64_t B, int N, float *__restrict__ out) {
    __shared__ float red[256];
    const int col = blockIdx.x;
    float s = 0.0f;
    for (int64_t r = threadIdx.x; r < B; r += blockDim.x) s += __bfloat162float(X[r * N + col]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[col] = red[0];
}

__global__ void k_sum_small(const float *__restrict__ x, int n, float *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.0f;
        for (int i = 0; i < n; i++) s += x[i];
        *out = s;
    }
}

__global__ void k_to_bf16(const float *__restrict__ x, int64_t n, bf16 *__restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16(x[i]);
}

__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, bf16 *__restrict__ wb, int64_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    p[i] = pi;
    wb[i] = __float2bfloat16(pi);
}

__global__ void k_apply_filter(const float *__restrict__ out, int64_t R, float tau, float dmin,
                               float dmax, uint8_t *__restrict__ valid, float *__restrict__ deta) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= R || !valid[i]) return;
    float z = out[2 * i], v = out[2 * i + 1];
    float p = 1.0f / (1.0f + expf(-z));
    if (!(p >= tau)) {
        valid[i] = 0;
        return;
    }
    deta[i] = fminf(fmaxf(expf(v), dmin), dmax);
}

// ---------------------------------------------------------------------------
// network passes (host side)
// ---------------------------------------------------------------------------
struct Work {
    bf16 *H[3];        // layer outputs H1..H3, [rows, 128]
    float *out;        // [rows, 2]
    bf16 *dout;        // [rows, 2]
    bf16 *dP[2];       // backward signals, [rows, 128], ping-pong
    float *part;       // split-K partials
    float *loss_part;  // per-block loss sums
    int64_t rows;
};

// Rows per weight-gradient split: about 64 splits (a 128 x 128 gradient is
// only 4 CTA tiles, so the batch dimension supplies the parallelism), at
// least 128 rows and a multiple of the GEMM's K step.
constexpr int kWgSplits = 64;
__host__ __device__ inline int64_t wg_split_rows(int64_t rows) {
    const int64_t r = (rows + kWgSplits - 1) / kWgSplits;
    const int64_t r32 = (r + BK - 1) / BK * BK;
    return r32 < 128 ? 128 : r32;
}

size_t work_layout(int64_t rows, Work *w, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off = align256(off + bytes);
        return p;
    };
    for (int l = 0; l < 3; l++) w->H[l] = (bf16 *)take(rows * kH * sizeof(bf16));
    w->out = (float *)take(rows * 2 * sizeof(float));
    w->dout = (bf16 *)take(rows * 2 * sizeof(bf16));
    for (int l = 0; l < 2; l++) w->dP[l] = (bf16 *)take(rows * kH * sizeof(bf16));
    const int64_t S = (rows + wg_split_rows(rows) - 1) / wg_split_rows(rows);
    w->part = (float *)take((size_t)S * kH * kH * sizeof(float));
    w->loss_part = (float *)take(((rows + 255) / 256) * sizeof(float));
    w->rows = rows;
    return off;
}

// ---------------------------------------------------------------------------
// Inference on the fifth-generation tensor cores (tcgen05, tensor memory).
// One persistent CTA per SM takes 128-row tiles of the features; its warps
// have fixed roles:
//   warp 0      TMA producer: feature tiles [128][16] into a 4-stage ring
//               (32-byte swizzle, zero rows past the end); owns the TMEM
//               allocation (all 512 columns).
//   warp 1      MMA issuer (one elected lane of a converged warp, operand
//               descriptors built once): per tile and layer the product
//               D[128][N] = A[128][K] W^T, W K-major in shared memory, D in
//               the tile's TMEM slot.  Layer 1 reads A (the features) from
//               shared memory; layers 2-4 read A (the activations) from
//               TMEM, so the tensor cores stream only W from shared memory.
//               tcgen05.commit signals the epilogue.
//   warps 2..17 epilogue: a thread owns one row (its warp's TMEM lane
//               quarter) and one quarter of the columns; it loads the row's
//               accumulators, applies ReLU, rounds to BF16 and stores the
//               packed values back into TMEM as the next layer's A - or,
//               after the last layer, writes the two outputs.
// The bias rides on the tensor cores: one more K = 16 product per layer
// multiplies a constant TMEM block whose row is (1, 1, 1, 0, ...) by a block
// holding each bias as the sum of three BF16 pieces (hi, mid, lo: 24
// significant bits, the FP32 bias to within its last bit), so the
// accumulator already holds x W^T + b and the epilogue does no arithmetic
// but ReLU and rounding.
// TMEM columns: accumulators of slot 0 / 1 at 0 / 128, activations (BF16
// pairs) of slot 0 / 1 at 256 / 320, the constant block at 384.  Two tiles
// are in flight, issued pairwise by layer (L1 a, L1 b, L2 a, ...), so the
// epilogue of one tile overlaps the products of the other.  Weights (72 KB,
// swizzled) are staged once per CTA.  Rounding points: FP32 accumulation
// (bias included), ReLU, BF16 activations.  For training the same kernel
// also writes the three hidden layers' activations out.
// Every wait is bounded; a CTA that gives up writes NaN to the rows it still
// owes, so a failure cannot pass for a result.
// ---------------------------------------------------------------------------
constexpr int kTM = 128;                  // rows per tile = MMA M
constexpr int kXStages = 4;
constexpr int kEpiWarps = 16;
constexpr int kTcWarps = 2 + kEpiWarps;
constexpr int kTmemCols = 512;
constexpr unsigned kActCol = 256;         // activations of slot j at kActCol + 64 j
constexpr unsigned kOnesCol = 384;        // the constant (1, 1, 1, 0, ...) block: K = 16

struct TcSmem {                           // every operand block 1024-byte aligned
    bf16 w2[2][kH * 64];                  // [k block][n][64 k], 128B swizzle
    bf16 w3[2][kH * 64];
    bf16 w4[2][16 * 64];                  // rows 2..15 zero (MMA N = 16)
    bf16 w1[kH * kF];                     // [n][16 k], 32B swizzle
    bf16 x[kXStages][kTM * kF];           // feature tiles, 32B swizzle
    bf16 bias[3][kH * 16];                // [n][16 k]: hi, mid, lo, 0...; 32B swizzle
    bf16 bias4[16 * 16];
    unsigned long long x_full[kXStages], x_empty[kXStages], acc_full[2], h_done[2], fin;
    unsigned tmem;
    int err;
};
constexpr size_t kTcSmemBytes = sizeof(TcSmem) + 1024;

// byte offset of 16-byte chunk `c` of row `r` in the two swizzled layouts
__device__ __forceinline__ int sw128(int r, int c) { return r * 128 + ((c ^ (r & 7)) << 4); }
__device__ __forceinline__ int sw32(int r, int c) { return r * 32 + ((c ^ ((r >> 2) & 1)) << 4); }

// shared-memory matrix descriptor: start address, leading byte offset 16
// (unused by the swizzled K-major layouts), stride byte offset between 8-row
// groups, descriptor version 1, swizzle mode (2 = 128B, 6 = 32B)
constexpr uint64_t kSw128 = 2, kSw32 = 6;
__device__ __forceinline__ uint64_t sdesc(unsigned addr, unsigned sbo, uint64_t mode) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
           ((uint64_t)(sbo >> 4) << 32) | ((uint64_t)1 << 46) | (mode << 61);
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr unsigned idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) |
           ((unsigned)(M >> 4) << 24);
}

// The issuing helpers are executed by a whole converged warp with uniform
// operands; elect.sync picks the one lane that issues.

// D (+)= A B^T with A and B in shared memory
__device__ __forceinline__ void umma_ss(unsigned d, uint64_t a, uint64_t b, unsigned id, int acc) {
    asm volatile(
        "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

// D (+)= A B^T with A in tensor memory (row m in lane m, BF16 pairs per column)
__device__ __forceinline__ void umma_ts(unsigned d, unsigned a, uint64_t b, unsigned id, int acc) {
    asm volatile(
        "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}

// arrive on `bar` once every product issued so far by this warp has completed
__device__ __forceinline__ void umma_commit(unsigned long long *bar) {
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane; the
// wait is in the same statement, so the registers are valid on return
__device__ __forceinline__ void tmem_ld32(unsigned addr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(addr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld2(unsigned addr, uint32_t (&r)[2]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1])
        : "r"(addr)
        : "memory");
}

// 16 consecutive columns of this thread's TMEM lane; returns once written
__device__ __forceinline__ void tmem_st16(unsigned addr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16};\n"
        "tcgen05.wait::st.sync.aligned;" ::"r"(addr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15])
        : "memory");
}

// BF16x2 of (max(lo, 0), max(hi, 0)), round to nearest even; lo in the low half
__device__ __forceinline__ uint32_t relu_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Bounded wait on an mbarrier phase by polling test_wait, which never
// suspends the thread: the MMA warp waits for the epilogue's arrivals this
// way (measured 42.3 -> 41.6 us per 500k-ring forward against try_wait;
// polling in the 16 epilogue warps as well was slower, 43.5 us)
__device__ __forceinline__ bool mbar_spin(unsigned long long *bar, unsigned parity) {
    const unsigned b = smem_u32(bar);
    unsigned long long t0 = 0;
    for (unsigned it = 0; it < (1u << 30); ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(b), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255) == 255) {
            const unsigned long long now = globaltimer_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > kWaitLimitNs) return false;
        }
    }
    return false;
}

// kKeep: also write the three hidden activations out (training); inference
// is compiled without those stores.
template <bool kKeep>
__global__ void __launch_bounds__(kTcWarps * 32, 1)
k_mlp_forward_tc(const __grid_constant__ CUtensorMap xmap, const bf16 *__restrict__ wb,
                 const float *__restrict__ pf, int64_t R, float *__restrict__ out,
                 bf16 *__restrict__ h1, bf16 *__restrict__ h2, bf16 *__restrict__ h3) {
    extern __shared__ unsigned char smem_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t T = (R + kTM - 1) / kTM;
    const int nt = (int)((T - blockIdx.x + gridDim.x - 1) / gridDim.x);   // this CTA's tiles
    auto tile_of = [&](int k) { return (int64_t)blockIdx.x + (int64_t)k * gridDim.x; };

    // weights (16-byte chunks into their swizzled places) and biases
    const uint4 *wg = reinterpret_cast<const uint4 *>(wb);
    for (int i = tid; i < kH * 2; i += blockDim.x)
        *reinterpret_cast<uint4 *>(reinterpret_cast<char *>(S.w1) + sw32(i >> 1, i & 1)) =
            wg[oW1 / 8 + i];
    for (int i = tid; i < kH * 16; i += blockDim.x) {
        const int n = i >> 4, kb = (i >> 3) & 1, c = i & 7;
        *reinterpret_cast<uint4 *>(reinterpret_cast<char *>(S.w2[kb]) + sw128(n, c)) =
            wg[oW2 / 8 + i];
        *reinterpret_cast<uint4 *>(reinterpret_cast<char *>(S.w3[kb]) + sw128(n, c)) =
            wg[oW3 / 8 + i];
    }
    for (int i = tid; i < 16 * 16; i += blockDim.x) {
        const int n = i >> 4, kb = (i >> 3) & 1, c = i & 7;
        *reinterpret_cast<uint4 *>(reinterpret_cast<char *>(S.w4[kb]) + sw128(n, c)) =
            n < 2 ? wg[oW4 / 8 + i] : make_uint4(0u, 0u, 0u, 0u);
    }
    for (int i = tid; i < 4 * kH; i += blockDim.x) {   // bias rows: 3 x 128, then 16 (2 real)
        const int l = i / kH, n = i % kH;
        if (l == 3 && n >= 16) continue;
        const float b = l < 3 ? pf[(l == 0 ? ob1 : l == 1 ? ob2 : ob3) + n]
                              : (n < 2 ? pf[ob4 + n] : 0.0f);
        const bf16 hi = __float2bfloat16_rn(b);
        const float r1 = b - __bfloat162float(hi);             // exact
        const bf16 mid = __float2bfloat16_rn(r1);
        const bf16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
        __align__(16) bf16 row[8] = {hi, mid, lo, __float2bfloat16_rn(0.0f),
                                     __float2bfloat16_rn(0.0f), __float2bfloat16_rn(0.0f),
                                     __float2bfloat16_rn(0.0f), __float2bfloat16_rn(0.0f)};
        char *blk = reinterpret_cast<char *>(l < 3 ? S.bias[l] : S.bias4);
        *reinterpret_cast<uint4 *>(blk + sw32(n, 0)) = *reinterpret_cast<const uint4 *>(row);
        *reinterpret_cast<uint4 *>(blk + sw32(n, 1)) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int i = 0; i < kXStages; i++) {
            mbar_init(&S.x_full[i], 1);
            mbar_init(&S.x_empty[i], 1);
        }
        for (int i = 0; i < 2; i++) {
            mbar_init(&S.acc_full[i], 1);
            mbar_init(&S.h_done[i], kEpiWarps);
        }
        mbar_init(&S.fin, 1);
        S.err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");    // weights -> tensor cores
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&S.tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = S.tmem;
    volatile int *err = &S.err;
    if (warp >= 2 && warp < 6) {          // the constant block, one row per thread
        const uint32_t one2 = 0x3F803F80u, one1 = 0x00003F80u;   // BF16 pairs (1, 1), (1, 0)
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n"
            "tcgen05.wait::st.sync.aligned;" ::"r"(tmem + ((unsigned)(32 * (warp & 3)) << 16) +
                                                   kOnesCol),
            "r"(one2), "r"(one1), "r"(0u), "r"(0u), "r"(0u), "r"(0u), "r"(0u), "r"(0u)
            : "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 0) {
        if (lane == 0) {                  // producer
            int uses[kXStages] = {};
            for (int k = 0; k < nt && !*err; k++) {
                const int st = k % kXStages;
                if (uses[st] > 0 && !mbar_wait(&S.x_empty[st], (uses[st] - 1) & 1)) {
                    *err = 1;
                    break;
                }
                expect_tx(&S.x_full[st], kTM * kF * 2);
                tma_load_2d(S.x[st], &xmap, 0, (int)(tile_of(k) * kTM), &S.x_full[st]);
                uses[st]++;
            }
            for (int st = 0; st < kXStages; st++)    // no copy may outlive the CTA
                if (uses[st] > 0 && !mbar_wait(&S.x_full[st], (uses[st] - 1) & 1)) *err = 1;
        }
    } else if (warp == 1) {
        // MMA issuer.  The whole warp runs the loop, so descriptors and
        // addresses are warp-uniform; one elected lane issues each product.
        // Operand descriptors are built once and advanced by adding to their
        // address field (16-byte units).
        const uint64_t dx = sdesc(smem_u32(S.x[0]), 256, kSw32);
        const uint64_t dw1 = sdesc(smem_u32(S.w1), 256, kSw32);
        const uint64_t dw2 = sdesc(smem_u32(S.w2[0]), 1024, kSw128);
        const uint64_t dw3 = sdesc(smem_u32(S.w3[0]), 1024, kSw128);
        const uint64_t dw4 = sdesc(smem_u32(S.w4[0]), 1024, kSw128);
        const uint64_t db[4] = {sdesc(smem_u32(S.bias[0]), 256, kSw32),
                                sdesc(smem_u32(S.bias[1]), 256, kSw32),
                                sdesc(smem_u32(S.bias[2]), 256, kSw32),
                                sdesc(smem_u32(S.bias4), 256, kSw32)};
        int hd[2] = {0, 0};
        bool ok = true;
        for (int p = 0; p < nt && ok; p += 2) {
            const int q = nt - p < 2 ? nt - p : 2;
            for (int l = 0; l < 4 && ok; l++) {
                for (int j = 0; j < q; j++) {
                    const int k = p + j;
                    const unsigned d = tmem + (unsigned)(j * 128);
                    if (l == 0) {
                        const int st = k % kXStages;
                        ok = !*err && mbar_wait(&S.x_full[st], (k / kXStages) & 1) &&
                             (k < 2 || mbar_spin(&S.h_done[j], hd[j]++ & 1));
                        if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
                        tc_fence_after();
                        umma_ss(d, dx + (uint64_t)(st * (kTM * kF * 2 / 16)), dw1, idesc(kTM, kH), 0);
                        umma_ts(d, tmem + kOnesCol, db[0], idesc(kTM, kH), 1);
                        umma_commit(&S.acc_full[j]);
                        umma_commit(&S.x_empty[st]);
                    } else {
                        ok = !*err && mbar_spin(&S.h_done[j], hd[j]++ & 1);
                        if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
                        tc_fence_after();
                        const unsigned a0 = tmem + kActCol + (unsigned)(j * 64);
                        const uint64_t b0 = l == 1 ? dw2 : l == 2 ? dw3 : dw4;
                        const uint64_t bblk = l == 3 ? (16 * 128) / 16 : (kH * 128) / 16;
                        const unsigned id = l == 3 ? idesc(kTM, 16) : idesc(kTM, kH);
#pragma unroll
                        for (int kk = 0; kk < 8; kk++)        // K = 16: 8 TMEM columns of A
                            umma_ts(d, a0 + (unsigned)(kk * 8),
                                    b0 + (uint64_t)(kk >> 2) * bblk + (uint64_t)((kk & 3) * 2), id,
                                    kk > 0);
                        umma_ts(d, tmem + kOnesCol, db[l], id, 1);
                        umma_commit(&S.acc_full[j]);
                    }
                }
            }
        }
        if (!ok && lane == 0) *err = 1;
        umma_commit(&S.fin);              // every product issued has completed
        if (!__all_sync(0xffffffffu, mbar_wait(&S.fin, 0)) && lane == 0) *err = 1;
    } else {                              // epilogue: one row, one column quarter per thread
        const int qd = warp & 3, cq = (warp - 2) >> 2, row = 32 * qd + lane;
        const unsigned lanes = (unsigned)(32 * qd) << 16;
        int af[2] = {0, 0};
        int p = 0;
        for (p = 0; p < nt; p += 2) {
            const int q = nt - p < 2 ? nt - p : 2;
            for (int l = 0; l < 4; l++) {
                for (int j = 0; j < q; j++) {
                    const bool ok = !*err && mbar_wait(&S.acc_full[j], af[j]++ & 1);
                    if (!__all_sync(0xffffffffu, ok)) {    // warp-uniform: the loads are .aligned
                        *err = 1;
                        goto fail;
                    }
                    tc_fence_after();
                    const unsigned t = tmem + lanes + (unsigned)(j * 128);
                    if (l < 3) {
                        uint32_t r[32], w[16];
                        tmem_ld32(t + (unsigned)(cq * 32), r);
#pragma unroll
                        for (int c = 0; c < 16; c++)
                            w[c] = relu_bf16x2(__uint_as_float(r[2 * c]),
                                               __uint_as_float(r[2 * c + 1]));
                        tmem_st16(tmem + lanes + kActCol + (unsigned)(j * 64 + cq * 16), w);
                        bf16 *hl = l == 0 ? h1 : l == 1 ? h2 : h3;
                        const int64_t g = tile_of(p + j) * kTM + row;
                        if (kKeep && g < R) {
                            uint4 *dst = reinterpret_cast<uint4 *>(hl + g * kH + cq * 32);
#pragma unroll
                            for (int c = 0; c < 4; c++)
                                dst[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
                        }
                    } else if (cq == 0) {
                        uint32_t r[2];
                        tmem_ld2(t, r);
                        const int64_t g = tile_of(p + j) * kTM + row;
                        if (g < R)
                            *reinterpret_cast<float2 *>(out + 2 * g) =
                                make_float2(__uint_as_float(r[0]), __uint_as_float(r[1]));
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&S.h_done[j]);
                }
            }
        }
    fail:
        if (p < nt && cq == 0) {          // gave up: NaN for every row still owed
            const float nan = __int_as_float(0x7fc00000);
            for (int k = p; k < nt; k++) {
                const int64_t g = tile_of(k) * kTM + row;
                if (g < R) *reinterpret_cast<float2 *>(out + 2 * g) = make_float2(nan, nan);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
}

// dW[out, in] = dP^T A over the rows (split-K, fixed order); db = column sums of dP
cudaError_t weight_grad(const bf16 *dP, int out, const bf16 *A, int in, int rows, float *gW,
                        float *gb, Work &w, cudaStream_t s) {
    GemmArgs g{};
    g.M = out;
    g.N = in;
    g.K = rows;
    g.A = dP;            // A(m = output, k = row) = dP[row][m]
    g.lda_m = 1;
    g.lda_k = out;
    g.B = A;             // B(k = row, n = input) = A[row][n]
    g.ldb_k = in;
    g.ldb_n = 1;
    g.C = gW;
    g.ldc = in;
    g.part = w.part;
    g.ksplit = (int)wg_split_rows(rows);
    cudaError_t e = gemm(g, s);
    if (e != cudaSuccess) return e;
    k_col_sums<<<out, 256, 0, s>>>(dP, rows, out, gb);
    return cudaGetLastError();
}

// dP_prev[rows, in] = (dP[rows, out] W[out, in]) where Hprev > 0
GemmArgs back_data(const bf16 *dP, int out, const bf16 *W, int in, int rows, const bf16 *Hprev,
                   bf16 *dPprev) {
    GemmArgs g{};
    g.M = rows;
    g.N = in;
    g.K = out;
    g.A = dP;
    g.lda_m = out;
    g.lda_k = 1;
    g.B = W;             // B(k = output, n = input) = W[k][n]
    g.ldb_k = in;
    g.ldb_n = 1;
    g.mask = Hprev;
    g.ldmask = in;
    g.C = dPprev;
    g.ldc = in;
    g.c_bf16 = 1;
    return g;
}

// The network on the tcgen05 kernel for R rows of features; with H (the
// three hidden layers' [R][128] BF16 outputs, for training) the activations
// are also written out.
cudaError_t forward_tc(const float *params, const uint16_t *wb, const uint16_t *F, int64_t R,
                       float *out, bf16 *const *H, cudaStream_t s) {
    if (R == 0) return cudaSuccess;
    TmapEncodeFn enc = encode_fn();
    if (enc == nullptr) return cudaErrorNotSupported;
    auto kern = H ? k_mlp_forward_tc<true> : k_mlp_forward_tc<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmemBytes);
    if (e != cudaSuccess) return e;
    const int64_t sms = device_sm_count();
    constexpr int64_t kRowsPerLaunch = (int64_t)1 << 30;   // TMA row coordinates stay int32
    for (int64_t r0 = 0; r0 < R; r0 += kRowsPerLaunch) {
        const int64_t n = R - r0 < kRowsPerLaunch ? R - r0 : kRowsPerLaunch;
        CUtensorMap xmap;
        const cuuint64_t dims[2] = {(cuuint64_t)kF, (cuuint64_t)n};
        const cuuint64_t strides[1] = {(cuuint64_t)kF * 2};
        const cuuint32_t box[2] = {(cuuint32_t)kF, (cuuint32_t)kTM};
        const cuuint32_t es[2] = {1, 1};
        if (enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(F + r0 * kF),
                dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        const int64_t tiles = (n + kTM - 1) / kTM;
        kern<<<(unsigned)(tiles < sms ? tiles : sms), kTcWarps * 32, kTcSmemBytes, s>>>(
            xmap, reinterpret_cast<const bf16 *>(wb), params, n, out + 2 * r0,
            H ? H[0] + r0 * kH : nullptr, H ? H[1] + r0 * kH : nullptr,
            H ? H[2] + r0 * kH : nullptr);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// dZ[l] receives the backward signal of hidden layer l + 1 (the gradient at
// its pre-activation, BF16); without a trace the signals ping-pong through
// two workspace buffers.
cudaError_t grad_rows(const bf16 *wb, const float *pf, const bf16 *X, const uint8_t *y,
                      const float *res, const uint8_t *wv, int rows, float inv_total,
                      float *grad, Work &w, bf16 *const *dZ, cudaStream_t s) {
    cudaError_t e = forward_tc(pf, reinterpret_cast<const uint16_t *>(wb),
                               reinterpret_cast<const uint16_t *>(X), rows, w.out, w.H, s);
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)((rows + 255) / 256);
    k_loss_grad<<<nb, 256, 0, s>>>(w.out, y, res, wv, rows, inv_total, w.dout, w.loss_part);
    if ((e = cudaGetLastError())) return e;
    // layer 4
    if ((e = weight_grad(w.dout, 2, w.H[2], kH, rows, grad + oW4, grad + ob4, w, s))) return e;
    if ((e = gemm(back_data(w.dout, 2, wb + oW4, kH, rows, w.H[2], dZ[2]), s))) return e;
    // layer 3
    if ((e = weight_grad(dZ[2], kH, w.H[1], kH, rows, grad + oW3, grad + ob3, w, s))) return e;
    if ((e = gemm(back_data(dZ[2], kH, wb + oW3, kH, rows, w.H[1], dZ[1]), s))) return e;
    // layer 2
    if ((e = weight_grad(dZ[1], kH, w.H[0], kH, rows, grad + oW2, grad + ob2, w, s))) return e;
    if ((e = gemm(back_data(dZ[1], kH, wb + oW2, kH, rows, w.H[0], dZ[0]), s))) return e;
    // layer 1
    return weight_grad(dZ[0], kH, X, kF, rows, grad + oW1, grad + ob1, w, s);
}

}  // namespace

size_t mlp_workspace_bytes(int64_t rows) {
    Work w;
    int64_t r = rows < kChunk ? rows : kChunk;
    if (r < 1) r = 1;
    return work_layout(r, &w, nullptr) + 256;
}

cudaError_t mlp_features(const cc_events &ev, const cc_rings &r, float sig_pos, uint16_t *F,
                         cudaStream_t s) {
    if (ev.count == 0) return cudaSuccess;
    TraceScope ts(CC_STAGE_MLP, s);
    k_features<<<(unsigned)((ev.count + 255) / 256), 256, 0, s>>>(
        ev.n, ev.x, ev.y, ev.z, ev.e, ev.count, ev.stride, r.az, r.eta, r.deta, r.valid, r.perm,
        sig_pos, reinterpret_cast<bf16 *>(F));
    return cudaGetLastError();
}

cudaError_t mlp_forward(const float *params, const uint16_t *wb, const uint16_t *F, int64_t R,
                        float *out, char *ws, cudaStream_t s) {
    (void)ws;                                  // activations stay on chip
    TraceScope ts(CC_STAGE_MLP, s);
    return forward_tc(params, wb, F, R, out, nullptr, s);
}

cudaError_t mlp_grad(const float *params, const uint16_t *wb, const uint16_t *F,
                     const uint8_t *y, const float *res, const uint8_t *wv, int64_t B,
                     float *grad, float *loss, char *ws, const MlpTrace *trace,
                     cudaStream_t s) {
    Work w;
    work_layout(B, &w, ws);
    bf16 *dZ[3] = {w.dP[0], w.dP[1], w.dP[0]};
    if (trace) {
        bf16 *hid = reinterpret_cast<bf16 *>(trace->hidden);
        bf16 *sig = reinterpret_cast<bf16 *>(trace->signals);
        for (int l = 0; l < 3; l++) {
            if (hid) w.H[l] = hid + (size_t)l * B * kH;
            if (sig) dZ[l] = sig + (size_t)l * B * kH;
        }
        if (trace->out) w.out = trace->out;
        if (trace->dout) w.dout = reinterpret_cast<bf16 *>(trace->dout);
    }
    TraceScope ts(CC_STAGE_MLP, s);
    cudaError_t e = grad_rows(reinterpret_cast<const bf16 *>(wb), params,
                              reinterpret_cast<const bf16 *>(F), y, res, wv, (int)B,
                              1.0f / (float)B, grad, w, dZ, s);
    if (e != cudaSuccess) return e;
    k_sum_small<<<1, 32, 0, s>>>(w.loss_part, (int)((B + 255) / 256), loss);
    return cudaGetLastError();
}

cudaError_t mlp_adam(float *p, float *m, float *v, const float *g, uint16_t *wb, int32_t t,
                     float lr, float b1, float b2, float eps, cudaStream_t s) {
    TraceScope ts(CC_STAGE_MLP, s);
    float c1 = 1.0f / (1.0f - powf(b1, (float)t)), c2 = 1.0f / (1.0f - powf(b2, (float)t));
    k_adam<<<(kP + 255) / 256, 256, 0, s>>>(p, m, v, g, reinterpret_cast<bf16 *>(wb), kP, lr, b1,
                                            b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t mlp_params_to_bf16(const float *p, uint16_t *wb, cudaStream_t s) {
    k_to_bf16<<<(kP + 255) / 256, 256, 0, s>>>(p, kP, reinterpret_cast<bf16 *>(wb));
    return cudaGetLastError();
}

cudaError_t mlp_apply_filter(const float *out, const cc_rings &r, float tau, float dmin,
                             float dmax, cudaStream_t s) {
    if (r.count == 0) return cudaSuccess;
    TraceScope ts(CC_STAGE_MLP, s);
    k_apply_filter<<<(unsigned)((r.count + 255) / 256), 256, 0, s>>>(out, r.count, tau, dmin, dmax,
                                                                     r.valid, r.deta);
    return cudaGetLastError();
}

}  // namespace cc

// mlp.cu - the learned ring filter: ring features, an MLP 16 -> 128 -> 128 ->
// 128 -> 2 (ReLU) whose outputs are a source/background logit z and the log v
// of a predicted ring width, its loss and gradients, Adam, and the filter that
// applies it to rings before the sweep.
//
// All matrix products run on the tensor cores through one BF16 GEMM kernel
// (mma.sync m16n8k16, FP32 accumulation, operands staged through shared memory
// and loaded with ldmatrix).  Strided operand addressing lets the same kernel
// do the three products of training: activations x W^T (forward), dP x W
// (backward through a layer) and dP^T x A (weight gradient, reduced over the
// batch in fixed-order split-K partials, so results are deterministic).
// Weights, layer inputs and backward signals are BF16; biases, accumulators,
// losses, gradients and the Adam state are FP32.
#include <cuda_bf16.h>

#include "cc_math.cuh"

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
                if (row >= g.M || col >= g.N) continue;
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

constexpr int kWgSplitRows = 512;                         // rows per weight-gradient split

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
    int64_t S = (rows + kWgSplitRows - 1) / kWgSplitRows;
    w->part = (float *)take((size_t)S * kH * kH * sizeof(float));
    w->loss_part = (float *)take(((rows + 255) / 256) * sizeof(float));
    w->rows = rows;
    return off;
}

GemmArgs layer_fwd(const bf16 *A, int in, const bf16 *W, const float *b, int out, int rows,
                   void *C, bool relu, bool c_bf16) {
    GemmArgs g{};
    g.M = rows;
    g.N = out;
    g.K = in;
    g.A = A;
    g.lda_m = in;
    g.lda_k = 1;
    g.B = W;             // B(k = input, n = output) = W[n][k]
    g.ldb_k = 1;
    g.ldb_n = in;
    g.bias = b;
    g.relu = relu;
    g.C = C;
    g.ldc = out;
    g.c_bf16 = c_bf16;
    return g;
}

// ---------------------------------------------------------------------------
// Inference: the whole network in one kernel.  A CTA stages the BF16 weights
// (rows padded so that ldmatrix reads are conflict-free) and the FP32 biases
// in shared memory once, then its warps take 16-row slices of the input.  A
// warp keeps its slice's activations in registers: the FP32 accumulators of
// a layer (16 n8 tiles of m16n8k16) become, after bias, ReLU and rounding to
// BF16, the A fragments of the next layer directly - the C fragment pair of
// columns 16c .. 16c + 15 is exactly the A fragment of k-chunk c - so no
// activation leaves the SM.  Rounding points are those of forward_rows.
// ---------------------------------------------------------------------------
constexpr int kW1S = kF + 8;        // padded row strides (bf16 elements)
constexpr int kWHS = kH + 8;

struct FusedSmem {
    bf16 w1[kH][kW1S];
    bf16 w2[kH][kWHS];
    bf16 w3[kH][kWHS];
    bf16 w4[8][kWHS];               // rows 2..7 zero
    float b[3][kH];
    float b4[2];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// acc (16 n8 tiles) + bias, ReLU, BF16 -> A fragments of the 8 k-chunks
__device__ __forceinline__ void to_afrag(const float (&acc)[16][4], const float *bias, int t,
                                         uint32_t (&A)[8][4]) {
#pragma unroll
    for (int c = 0; c < 8; c++) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int j = 2 * c + h, col = 8 * j + 2 * t;
            const float b0 = bias[col], b1 = bias[col + 1];
            A[c][2 * h] = pack_bf16(fmaxf(acc[j][0] + b0, 0.0f), fmaxf(acc[j][1] + b1, 0.0f));
            A[c][2 * h + 1] = pack_bf16(fmaxf(acc[j][2] + b0, 0.0f), fmaxf(acc[j][3] + b1, 0.0f));
        }
    }
}

// acc[j] = A (16 x 128) W^T for the 16 n8 tiles of a 128-wide layer
__device__ __forceinline__ void layer128(const uint32_t (&A)[8][4], const bf16 (*W)[kWHS],
                                         int lane, float (&acc)[16][4]) {
#pragma unroll
    for (int j = 0; j < 16; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
    const int r = lane & 7, kh = (lane >> 3) & 1;     // ldmatrix row / k half of this lane
#pragma unroll
    for (int c = 0; c < 8; c++) {
#pragma unroll
        for (int j = 0; j < 16; j++) {
            uint32_t bfr[2];
            ldmatrix_x2(bfr, &W[8 * j + r][16 * c + 8 * kh]);
            mma_bf16(acc[j], A[c], bfr);
        }
    }
}

constexpr int kFusedWarps = 8;

__global__ void __launch_bounds__(kFusedWarps * 32)
k_mlp_forward_fused(const bf16 *__restrict__ wb, const float *__restrict__ pf,
                    const bf16 *__restrict__ X, int64_t R, float *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FusedSmem &S = *reinterpret_cast<FusedSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kH * kF; i += blockDim.x) S.w1[i / kF][i % kF] = wb[oW1 + i];
    for (int i = tid; i < kH * kH; i += blockDim.x) {
        S.w2[i / kH][i % kH] = wb[oW2 + i];
        S.w3[i / kH][i % kH] = wb[oW3 + i];
    }
    for (int i = tid; i < 8 * kH; i += blockDim.x)
        S.w4[i / kH][i % kH] = i < 2 * kH ? wb[oW4 + i] : __float2bfloat16(0.0f);
    for (int i = tid; i < kH; i += blockDim.x) {
        S.b[0][i] = pf[ob1 + i];
        S.b[1][i] = pf[ob2 + i];
        S.b[2][i] = pf[ob3 + i];
    }
    if (tid < 2) S.b4[tid] = pf[ob4 + tid];
    __syncthreads();

    const int g = lane >> 2, t = lane & 3;
    const int64_t nslices = (R + 15) / 16;
    for (int64_t sl = (int64_t)blockIdx.x * kFusedWarps + warp; sl < nslices;
         sl += (int64_t)gridDim.x * kFusedWarps) {
        const int64_t r0 = sl * 16, ra = r0 + g, rb = ra + 8;
        // layer 1: the A fragment straight from the feature rows (16 features)
        uint32_t a1[4];
        const uint32_t *xa = reinterpret_cast<const uint32_t *>(X + ra * kF);
        const uint32_t *xb = reinterpret_cast<const uint32_t *>(X + rb * kF);
        a1[0] = ra < R ? xa[t] : 0u;
        a1[1] = rb < R ? xb[t] : 0u;
        a1[2] = ra < R ? xa[4 + t] : 0u;
        a1[3] = rb < R ? xb[4 + t] : 0u;
        float acc[16][4];
        {
            const int r = lane & 7, kh = (lane >> 3) & 1;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
                uint32_t bfr[2];
                ldmatrix_x2(bfr, &S.w1[8 * j + r][8 * kh]);
                mma_bf16(acc[j], a1, bfr);
            }
        }
        uint32_t A[8][4];
        to_afrag(acc, S.b[0], t, A);
        layer128(A, S.w2, lane, acc);
        to_afrag(acc, S.b[1], t, A);
        layer128(A, S.w3, lane, acc);
        to_afrag(acc, S.b[2], t, A);
        // layer 4: one n8 tile, columns 0 and 1 real
        float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        {
            const int r = lane & 7, kh = (lane >> 3) & 1;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                uint32_t bfr[2];
                ldmatrix_x2(bfr, &S.w4[r][16 * c + 8 * kh]);
                mma_bf16(o, A[c], bfr);
            }
        }
        if (t == 0) {                                     // columns 0, 1 of rows g, g + 8
            if (ra < R) {
                out[2 * ra] = o[0] + S.b4[0];
                out[2 * ra + 1] = o[1] + S.b4[1];
            }
            if (rb < R) {
                out[2 * rb] = o[2] + S.b4[0];
                out[2 * rb + 1] = o[3] + S.b4[1];
            }
        }
    }
}

cudaError_t forward_rows(const bf16 *wb, const float *pf, const bf16 *X, int rows, Work &w,
                         cudaStream_t s) {
    cudaError_t e;
    if ((e = gemm(layer_fwd(X, kF, wb + oW1, pf + ob1, kH, rows, w.H[0], true, true), s))) return e;
    if ((e = gemm(layer_fwd(w.H[0], kH, wb + oW2, pf + ob2, kH, rows, w.H[1], true, true), s)))
        return e;
    if ((e = gemm(layer_fwd(w.H[1], kH, wb + oW3, pf + ob3, kH, rows, w.H[2], true, true), s)))
        return e;
    return gemm(layer_fwd(w.H[2], kH, wb + oW4, pf + ob4, 2, rows, w.out, false, false), s);
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
    g.ksplit = kWgSplitRows;
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

cudaError_t grad_rows(const bf16 *wb, const float *pf, const bf16 *X, const uint8_t *y,
                      const float *res, const uint8_t *wv, int rows, float inv_total,
                      float *grad, Work &w, cudaStream_t s) {
    cudaError_t e = forward_rows(wb, pf, X, rows, w, s);
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)((rows + 255) / 256);
    k_loss_grad<<<nb, 256, 0, s>>>(w.out, y, res, wv, rows, inv_total, w.dout, w.loss_part);
    if ((e = cudaGetLastError())) return e;
    // layer 4
    if ((e = weight_grad(w.dout, 2, w.H[2], kH, rows, grad + oW4, grad + ob4, w, s))) return e;
    if ((e = gemm(back_data(w.dout, 2, wb + oW4, kH, rows, w.H[2], w.dP[0]), s))) return e;
    // layer 3
    if ((e = weight_grad(w.dP[0], kH, w.H[1], kH, rows, grad + oW3, grad + ob3, w, s))) return e;
    if ((e = gemm(back_data(w.dP[0], kH, wb + oW3, kH, rows, w.H[1], w.dP[1]), s))) return e;
    // layer 2
    if ((e = weight_grad(w.dP[1], kH, w.H[0], kH, rows, grad + oW2, grad + ob2, w, s))) return e;
    if ((e = gemm(back_data(w.dP[1], kH, wb + oW2, kH, rows, w.H[0], w.dP[0]), s))) return e;
    // layer 1
    return weight_grad(w.dP[0], kH, X, kF, rows, grad + oW1, grad + ob1, w, s);
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
    (void)ws;                                  // the fused forward keeps activations on chip
    if (R == 0) return cudaSuccess;
    const size_t smem = sizeof(FusedSmem);     // > 48 KB: opt in (per device, so every call)
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward_fused,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mlp_forward_fused, kFusedWarps * 32, smem);
    if (occ < 1) occ = 1;
    int64_t ctas = (int64_t)device_sm_count() * occ;
    const int64_t need = ((R + 15) / 16 + kFusedWarps - 1) / kFusedWarps;
    if (ctas > need) ctas = need;
    TraceScope ts(CC_STAGE_MLP, s);
    k_mlp_forward_fused<<<(unsigned)ctas, kFusedWarps * 32, smem, s>>>(
        reinterpret_cast<const bf16 *>(wb), params, reinterpret_cast<const bf16 *>(F), R, out);
    return cudaGetLastError();
}

cudaError_t mlp_grad(const float *params, const uint16_t *wb, const uint16_t *F,
                     const uint8_t *y, const float *res, const uint8_t *wv, int64_t B,
                     float *grad, float *loss, char *ws, cudaStream_t s) {
    Work w;
    work_layout(B, &w, ws);
    TraceScope ts(CC_STAGE_MLP, s);
    cudaError_t e = grad_rows(reinterpret_cast<const bf16 *>(wb), params,
                              reinterpret_cast<const bf16 *>(F), y, res, wv, (int)B,
                              1.0f / (float)B, grad, w, s);
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

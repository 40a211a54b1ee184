// mlp.cu - the learned ring filter: ring features, an MLP 16 -> 128 -> 128 ->
// 128 -> 2 (ReLU) whose outputs are a source/background logit z and the log v
// of a predicted ring width, its loss and gradients, Adam, and the filter that
// applies it to rings before the sweep.
//
// The forward pass (k_mlp_forward_tc, below) runs the whole network in one
// persistent kernel on the tcgen05 tensor cores, for inference and for
// training (which keeps the activations).  The backward pass runs on the
// tcgen05 tensor cores too (k_mlp_bwd_tc, one launch per hidden layer: the
// signal through the layer, and the weight and bias gradients read from the
// same TMA tiles as MN-major operands), with the output layer's K = 2
// products on CUDA cores (k_bwd_out); per-CTA partial gradients are summed in
// a fixed order, so results are deterministic.  Weights, layer inputs and
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
constexpr int64_t kFwdRows = (int64_t)1 << 30;   // rows per forward launch (TMA rows stay int32)

// offsets of the flat parameter vector
constexpr int oW1 = 0, ob1 = oW1 + kH * kF, oW2 = ob1 + kH, ob2 = oW2 + kH * kH,
              oW3 = ob2 + kH, ob3 = oW3 + kH * kH, oW4 = ob3 + kH, ob4 = oW4 + 2 * kH;
static_assert(ob4 + 2 == kP, "parameter layout");

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
    float *part;       // per-CTA partial gradients of the backward kernels
    float *loss_part;  // per-block loss sums
    int64_t rows;
};

// The CTA plan of the backward kernels for `rows` rows on `sms` SMs: the
// 128-row tiles spread over at most min(sms, 256) CTAs, tpc consecutive
// tiles each (a batch of at most one tile per SM gets one tile per CTA);
// every CTA has at least one tile.
constexpr int kRowTile = 128, kBwMaxCtas = 256;
struct BwPlan {
    int64_t tiles;
    int tpc, ncta;
};
inline BwPlan bw_plan(int64_t rows, int sms) {
    BwPlan p;
    p.tiles = (rows + kRowTile - 1) / kRowTile;
    if (p.tiles < 1) p.tiles = 1;
    const int64_t cap = sms < 1 ? 1 : (sms < kBwMaxCtas ? sms : kBwMaxCtas);
    p.tpc = (int)((p.tiles + cap - 1) / cap);
    p.ncta = (int)((p.tiles + p.tpc - 1) / p.tpc);
    return p;
}
// partial gradients of the four layers: [ncta][outputs][inputs + 1]
inline size_t bw_part_floats(int ncta) {
    return (size_t)ncta * ((size_t)kH * (kF + 1) + 2 * (size_t)kH * (kH + 1) + 2 * (kH + 1));
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
    const int64_t tiles = (rows + kRowTile - 1) / kRowTile;     // the most CTAs any plan has
    w->part = (float *)take(bw_part_floats((int)(tiles < kBwMaxCtas ? (tiles < 1 ? 1 : tiles)
                                                                     : kBwMaxCtas)) *
                            sizeof(float));
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
//   warps 2..17 epilogue, in two groups of 8, one per TMEM slot, so that
//               the two tiles in flight are finished concurrently: a thread
//               owns one row (its warp's TMEM lane quarter) and one half of
//               the columns of its group's slot; it loads the row's
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
            mbar_init(&S.h_done[i], kEpiWarps / 2);
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
    } else {                              // epilogue: slot j = grp; one row, one column half
        const int grp = (warp - 2) >> 3, ch = ((warp - 2) >> 2) & 1, qd = warp & 3,
                  row = 32 * qd + lane;
        const unsigned lanes = (unsigned)(32 * qd) << 16;
        int af = 0;
        int p = 0;
        for (p = 0; p < nt; p += 2) {
            const int q = nt - p < 2 ? nt - p : 2;
            if (grp >= q) continue;       // the last odd tile is slot 0's
            const int j = grp;
            for (int l = 0; l < 4; l++) {
                const bool ok = !*err && mbar_wait(&S.acc_full[j], af++ & 1);
                if (!__all_sync(0xffffffffu, ok)) {        // warp-uniform: the loads are .aligned
                    *err = 1;
                    goto fail;
                }
                tc_fence_after();
                const unsigned t = tmem + lanes + (unsigned)(j * 128);
                if (l < 3) {
                    bf16 *hl = l == 0 ? h1 : l == 1 ? h2 : h3;
                    const int64_t g = tile_of(p + j) * kTM + row;
#pragma unroll
                    for (int hh = 0; hh < 2; hh++) {
                        const int c0 = ch * 64 + hh * 32;          // accumulator columns
                        uint32_t r[32], w[16];
                        tmem_ld32(t + (unsigned)c0, r);
#pragma unroll
                        for (int c = 0; c < 16; c++)
                            w[c] = relu_bf16x2(__uint_as_float(r[2 * c]),
                                               __uint_as_float(r[2 * c + 1]));
                        tmem_st16(tmem + lanes + kActCol + (unsigned)(j * 64 + c0 / 2), w);
                        if (kKeep && g < R) {
                            uint4 *dst = reinterpret_cast<uint4 *>(hl + g * kH + c0);
#pragma unroll
                            for (int c = 0; c < 4; c++)
                                dst[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
                        }
                    }
                } else if (ch == 0) {
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
    fail:
        if (p < nt && ch == 0) {          // gave up: NaN for every row of this slot still owed
            const float nan = __int_as_float(0x7fc00000);
            for (int k = p + grp; k < nt; k += 2) {
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

// ---------------------------------------------------------------------------
// Backward pass on the fifth-generation tensor cores.  One launch per hidden
// layer l (3, 2, 1) takes 128-row tiles of the layer's backward signal dZ_l
// ([rows][128] BF16) and of its input H_(l-1) (the previous layer's
// activations, or the features for l = 1) by TMA, and computes with
// tcgen05.mma, FP32 accumulators in TMEM:
//   D1 = dZ_l W_l               the signal through the layer (l = 3, 2):
//                               A = the dZ tile (K-major, K = 128 outputs),
//                               B = W_l as stored, [output][input], staged
//                               once per CTA as an MN-major operand;
//   D2 += dZ_l^T H_(l-1)        the weight gradient over the CTA's rows:
//                               both operands are the same tiles read
//                               MN-major (the row is K), so nothing is
//                               transposed: the 128B-swizzled [row][64]
//                               blocks a TMA load leaves are an MN-major
//                               operand (LBO = block stride, SBO = 8 rows);
//   D3 += dZ_l^T 1              the bias gradient, against a constant
//                               block whose first column is 1.
// The epilogue gates D1 by H_(l-1) > 0 (the ReLU of the layer below), rounds
// it to BF16 into a swizzled tile and stores it with TMA as dZ_(l-1); after
// the CTA's last tile it writes D2 and D3 as the CTA's partial gradients,
// which k_reduce_grad sums over the CTAs in a fixed order (deterministic).
// Warps: 0 TMA producer (2-stage ring) and TMEM owner, 1 MMA issuer (one
// elected lane of a converged warp), 2..5 epilogue (one row each).  Every
// wait is bounded; a CTA that gives up writes NaN partials.
// ---------------------------------------------------------------------------
constexpr int kBwStages = 2;
constexpr int kBwEpiWarps = 4;
constexpr int kBwWarps = 2 + kBwEpiWarps;
constexpr unsigned kD1Col = 0, kD2Col = 128, kD3Col = 256;
static_assert(kTM == kRowTile, "backward tiles are the forward's");

struct BwSmem {                           // every operand block 1024-byte aligned
    bf16 dz[kBwStages][2][kTM * 64];      // signal tile: 2 blocks [row][64], 128B swizzle
    bf16 hp[kBwStages][2][kTM * 64];      // layer input tile (features: [row][16], 32B swizzle)
    bf16 wt[2][kH * 64];                  // W: [o = output][64 n = input], 2 n blocks
    bf16 out[2][kTM * 64];                // the gated signal before its TMA store
    bf16 ones[kTM * 16];                  // [row][16] = (1, 0, ..., 0), 32B swizzle
    unsigned long long full[kBwStages], empty[kBwStages], d1_full, d1_free, fin;
    unsigned tmem;
    int err;
};
constexpr size_t kBwSmemBytes = sizeof(BwSmem) + 1024;

// Shared-memory descriptor of an MN-major operand: `lbo` the byte stride
// between atoms along M/N, `sbo` between 8-row groups along K.
__device__ __forceinline__ uint64_t sdesc_mn(unsigned addr, unsigned lbo, unsigned sbo,
                                             uint64_t mode) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | ((uint64_t)1 << 46) | (mode << 61);
}

// instruction descriptor with both operands MN-major (transpose bits 15, 16)
__host__ __device__ constexpr unsigned idesc_mn(int M, int N) {
    return idesc(M, N) | (1u << 15) | (1u << 16);
}

__device__ __forceinline__ void tmem_ld16(unsigned addr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr)
        : "memory");
}

__device__ __forceinline__ void epi_sync() {   // the epilogue warps only
    asm volatile("bar.sync 1, %0;" ::"r"(kBwEpiWarps * 32) : "memory");
}

// BF16x2 of (lo, hi), round to nearest even; lo in the low half
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

struct BwArgs {
    int64_t rows, tiles;
    int tpc;              // tiles per CTA: CTA c takes tiles [c tpc, (c + 1) tpc)
    int nin;              // inputs of the layer: 128, or 16 for the first layer
    const bf16 *w;        // W_l [128 outputs][128 inputs] (signal through the layer)
    float *part;          // [CTA][128 outputs][nin + 1]: weight then bias partials
};

template <bool kData>
__global__ void __launch_bounds__(kBwWarps * 32, 1)
k_mlp_bwd_tc(const __grid_constant__ CUtensorMap dzmap, const __grid_constant__ CUtensorMap hpmap,
             const __grid_constant__ CUtensorMap outmap, const BwArgs a) {
    extern __shared__ unsigned char smem_raw[];
    BwSmem &S = *reinterpret_cast<BwSmem *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * a.tpc;
    const int nt = (int)(a.tiles - t0 < a.tpc ? a.tiles - t0 : a.tpc);
    const bool wide = a.nin == kH;

    if (kData) {       // W as it is stored, [o][n], is the MN-major B operand of D1
        const uint4 *wg = reinterpret_cast<const uint4 *>(a.w);
        constexpr int kChunks = kH * kH / 8;      // 16-byte chunks: row o, columns 8 c..
        for (int i0 = tid; i0 < kChunks; i0 += 4 * kBwWarps * 32) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int i = i0 + u * kBwWarps * 32;
                v[u] = i < kChunks ? wg[i] : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int i = i0 + u * kBwWarps * 32;
                if (i < kChunks) {
                    const int o = i >> 4, c = i & 15;
                    *reinterpret_cast<uint4 *>(reinterpret_cast<char *>(S.wt[c >> 3]) +
                                               sw128(o, c & 7)) = v[u];
                }
            }
        }
    }
    for (int r = tid; r < kTM; r += blockDim.x) {     // the constant block
        char *row = reinterpret_cast<char *>(S.ones);
        *reinterpret_cast<uint4 *>(row + sw32(r, 0)) = make_uint4(0x3F80u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(row + sw32(r, 1)) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int i = 0; i < kBwStages; i++) {
            mbar_init(&S.full[i], 1);
            mbar_init(&S.empty[i], kData ? 1 + kBwEpiWarps : 1);
        }
        mbar_init(&S.d1_full, 1);
        mbar_init(&S.d1_free, kBwEpiWarps);
        mbar_init(&S.fin, 1);
        S.err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");    // staged blocks -> tensor cores
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

    if (warp == 0) {
        if (lane == 0) {                  // producer
            const unsigned bytes = 2 * kTM * 64 * 2 + (wide ? 2 * kTM * 64 * 2 : kTM * kF * 2);
            int k = 0;
            for (; k < nt && !*err; k++) {
                const int st = k % kBwStages;
                if (k >= kBwStages && !mbar_wait(&S.empty[st], ((k / kBwStages) - 1) & 1)) {
                    *err = 1;
                    break;
                }
                const int y = (int)((t0 + k) * kTM);
                expect_tx(&S.full[st], bytes);
                tma_load_2d(S.dz[st][0], &dzmap, 0, y, &S.full[st]);
                tma_load_2d(S.dz[st][1], &dzmap, 64, y, &S.full[st]);
                tma_load_2d(S.hp[st][0], &hpmap, 0, y, &S.full[st]);
                if (wide) tma_load_2d(S.hp[st][1], &hpmap, 64, y, &S.full[st]);
            }
            for (int j = k - kBwStages < 0 ? 0 : k - kBwStages; j < k; j++)   // no copy outlives the CTA
                if (!mbar_wait(&S.full[j % kBwStages], (j / kBwStages) & 1)) *err = 1;
        }
    } else if (warp == 1) {               // MMA issuer (whole warp, one elected lane issues)
        const uint64_t dw = sdesc_mn(smem_u32(S.wt[0]), kH * 128, 1024, kSw128);
        const uint64_t d1s = sdesc_mn(smem_u32(S.ones), 4096, 256, kSw32);
        bool ok = true;
        for (int k = 0; k < nt && ok; k++) {
            const int st = k % kBwStages;
            ok = !*err && mbar_wait(&S.full[st], (k / kBwStages) & 1) &&
                 (!kData || k == 0 || mbar_spin(&S.d1_free, (k - 1) & 1));
            if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
            tc_fence_after();
            const unsigned dz0 = smem_u32(S.dz[st][0]), hp0 = smem_u32(S.hp[st][0]);
            if (kData) {                  // D1 = dZ W: K = 128 outputs in 8 steps of 16
                const uint64_t da = sdesc(dz0, 1024, kSw128);
#pragma unroll
                for (int kk = 0; kk < 8; kk++) {
                    const uint64_t off = (uint64_t)(kk >> 2) * (kTM * 128 / 16) + (uint64_t)((kk & 3) * 2);
                    umma_ss(tmem + kD1Col, da + off, dw + (uint64_t)(kk * 2048 / 16),
                            idesc(kTM, kH) | (1u << 16), kk > 0);   // B MN-major
                }
                umma_commit(&S.d1_full);
            }
            // D2 += dZ^T H and D3 += dZ^T 1: K = the tile's 128 rows in 8 steps of 16
            const uint64_t am = sdesc_mn(dz0, kTM * 128, 1024, kSw128);
            const uint64_t bm = wide ? sdesc_mn(hp0, kTM * 128, 1024, kSw128)
                                     : sdesc_mn(hp0, 4096, 256, kSw32);
#pragma unroll
            for (int kk = 0; kk < 8; kk++) {
                const int acc = (k > 0 || kk > 0) ? 1 : 0;
                umma_ss(tmem + kD2Col, am + (uint64_t)(kk * 2048 / 16),
                        bm + (uint64_t)(kk * (wide ? 2048 : 512) / 16), idesc_mn(kTM, a.nin), acc);
                umma_ss(tmem + kD3Col, am + (uint64_t)(kk * 2048 / 16),
                        d1s + (uint64_t)(kk * 512 / 16), idesc_mn(kTM, 16), acc);
            }
            umma_commit(&S.empty[st]);
        }
        if (!ok && lane == 0) *err = 1;
        umma_commit(&S.fin);              // every product issued has completed
        if (!__all_sync(0xffffffffu, mbar_wait(&S.fin, 0)) && lane == 0) *err = 1;
    } else {                              // epilogue: one row per thread
        const int qd = warp & 3, row = 32 * qd + lane;
        const unsigned lanes = (unsigned)(32 * qd) << 16;
        const bool leader = warp == 2 && lane == 0;
        if (kData) {
            for (int k = 0; k < nt; k++) {
                const int st = k % kBwStages;
                const bool ok = !*err && mbar_wait(&S.d1_full, k & 1);
                if (!__all_sync(0xffffffffu, ok)) {      // warp-uniform: the loads are .aligned
                    *err = 1;
                    break;
                }
                tc_fence_after();
                uint32_t r[4][32];
#pragma unroll
                for (int q = 0; q < 4; q++) tmem_ld32(tmem + lanes + kD1Col + 32 * q, r[q]);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.d1_free);
                // gate by the layer input > 0, round, into the swizzled out tile
#pragma unroll
                for (int c8 = 0; c8 < 16; c8++) {
                    const char *hb = reinterpret_cast<const char *>(S.hp[st][c8 >> 3]);
                    const uint4 h = *reinterpret_cast<const uint4 *>(hb + sw128(row, c8 & 7));
                    const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
                    uint32_t o[4];
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const int c = 8 * c8 + 2 * j;
                        const float v0 = __uint_as_float(r[c >> 5][c & 31]);
                        const float v1 = __uint_as_float(r[(c + 1) >> 5][(c + 1) & 31]);
                        const float g0 = __uint_as_float(hw[j] << 16);
                        const float g1 = __uint_as_float(hw[j] & 0xFFFF0000u);
                        o[j] = bf16x2(g0 > 0.0f ? v0 : 0.0f, g1 > 0.0f ? v1 : 0.0f);
                    }
                    char *ob = reinterpret_cast<char *>(S.out[c8 >> 3]);
                    *reinterpret_cast<uint4 *>(ob + sw128(row, c8 & 7)) =
                        make_uint4(o[0], o[1], o[2], o[3]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.empty[st]);   // the mask is read
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                epi_sync();
                if (leader) {
                    const int y = (int)((t0 + k) * kTM);
                    tma_store_2d(&outmap, 0, y, S.out[0]);
                    tma_store_2d(&outmap, 64, y, S.out[1]);
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                }
                epi_sync();                   // the out tile may be written again
            }
            if (leader) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        }
        // the CTA's partial gradients: row `row` of D2 (weights) and D3 (bias)
        const bool ok = !*err && mbar_wait(&S.fin, 0);
        float *dst = a.part + ((int64_t)blockIdx.x * kTM + row) * (a.nin + 1);
        if (__all_sync(0xffffffffu, ok) && !*err) {
            tc_fence_after();
            uint32_t b[2];
            tmem_ld2(tmem + lanes + kD3Col, b);
            if (wide) {
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    uint32_t r[32];
                    tmem_ld32(tmem + lanes + kD2Col + 32 * q, r);
#pragma unroll
                    for (int c = 0; c < 32; c++) dst[32 * q + c] = __uint_as_float(r[c]);
                }
            } else {
                uint32_t r[16];
                tmem_ld16(tmem + lanes + kD2Col, r);
#pragma unroll
                for (int c = 0; c < 16; c++) dst[c] = __uint_as_float(r[c]);
            }
            dst[a.nin] = __uint_as_float(b[0]);
        } else {                          // gave up: a failure cannot pass for a gradient
            for (int c = 0; c <= a.nin; c++) dst[c] = __int_as_float(0x7fc00000);
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

// Layer 4 on CUDA cores (its products have K = 2 or M = 2, below one
// tensor-core tile): dZ3 = bf16((dout W4) gated by H3 > 0), and the CTA's
// partial gradients of layer 4 over its rows, part[cta][o][n] =
// sum_r dout[r][o] H3[r][n] and part[cta][o][128] = sum_r dout[r][o].
// kOutGroups row groups of 128 threads (one per column n) take every
// kOutGroups-th row; their sums are added in group order.
constexpr int kOutGroups = 4;
__global__ void __launch_bounds__(kOutGroups * kH)
k_bwd_out(const bf16 *__restrict__ dout, const bf16 *__restrict__ h3,
          const bf16 *__restrict__ w4, int64_t rows, int tpc, bf16 *__restrict__ dz3,
          float *__restrict__ part) {
    __shared__ float red[kOutGroups][4][kH];
    const int n = threadIdx.x % kH, grp = threadIdx.x / kH;
    const float w0 = __bfloat162float(w4[n]), w1 = __bfloat162float(w4[kH + n]);
    const int64_t r0 = (int64_t)blockIdx.x * tpc * kTM;
    const int64_t r1 = rows < r0 + (int64_t)tpc * kTM ? rows : r0 + (int64_t)tpc * kTM;
    float g0 = 0.0f, g1 = 0.0f, b0 = 0.0f, b1 = 0.0f;
#pragma unroll 4
    for (int64_t r = r0 + grp; r < r1; r += kOutGroups) {
        const __nv_bfloat162 d = reinterpret_cast<const __nv_bfloat162 *>(dout)[r];
        const float d0 = __low2float(d), d1 = __high2float(d);
        const float h = __bfloat162float(h3[r * kH + n]);
        const float v = d0 * w0 + d1 * w1;
        if (CC_IN_BOUNDS(CC_SITE_MLP_ROWS, r, rows))
            dz3[r * kH + n] = __float2bfloat16(h > 0.0f ? v : 0.0f);
        g0 = fmaf(d0, h, g0);
        g1 = fmaf(d1, h, g1);
        b0 += d0;
        b1 += d1;
    }
    red[grp][0][n] = g0;
    red[grp][1][n] = g1;
    red[grp][2][n] = b0;
    red[grp][3][n] = b1;
    __syncthreads();
    if (grp == 0) {
        float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int g = 0; g < kOutGroups; g++)
#pragma unroll
            for (int q = 0; q < 4; q++) s[q] += red[g][q][n];
        float *p = part + (int64_t)blockIdx.x * 2 * (kH + 1);
        p[n] = s[0];
        p[kH + 1 + n] = s[1];
        if (n == 0) {
            p[kH] = s[2];
            p[2 * kH + 1] = s[3];
        }
    }
}

// grad = the sum over the CTAs of each layer's partials, CTA 0 first
// (deterministic).  Layer l's partials: [ncta][outputs][inputs + 1], the
// bias last.
struct GradParts {
    const float *part[4];
    int ncta;
};

__global__ void k_reduce_grad(const GradParts g, float *__restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kP) return;
    int l, o, n, nin, nout;
    if (i < ob1) { l = 0; o = i / kF; n = i % kF; }
    else if (i < oW2) { l = 0; o = i - ob1; n = kF; }
    else if (i < ob2) { l = 1; o = (i - oW2) / kH; n = (i - oW2) % kH; }
    else if (i < oW3) { l = 1; o = i - ob2; n = kH; }
    else if (i < ob3) { l = 2; o = (i - oW3) / kH; n = (i - oW3) % kH; }
    else if (i < oW4) { l = 2; o = i - ob3; n = kH; }
    else if (i < ob4) { l = 3; o = (i - oW4) / kH; n = (i - oW4) % kH; }
    else { l = 3; o = i - ob4; n = kH; }
    nin = l == 0 ? kF : kH;
    nout = l == 3 ? 2 : kH;
    const int64_t per = (int64_t)nout * (nin + 1);
    const float *p = g.part[l] + (int64_t)o * (nin + 1) + n;
    float s = 0.0f;
    for (int c = 0; c < g.ncta; c++) s += p[c * per];
    grad[i] = s;
}

// [rows][inner] BF16, row-major, as a TMA map with boxes of `box` columns x
// 128 rows
bool bf16_map(CUtensorMap *m, const void *p, int inner, int64_t rows, int box,
              CUtensorMapSwizzle sw) {
    TmapEncodeFn enc = encode_fn();
    if (enc == nullptr) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)inner * 2};
    const cuuint32_t boxd[2] = {(cuuint32_t)box, (cuuint32_t)kTM};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(p), dims, strides, boxd,
               es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One hidden layer's backward launch: dz [rows][128] the layer's signal, hp
// its input ([rows][128], or the features [rows][16] when nin = 16), out
// [rows][128] the gated signal of the layer below (nin = 128 only).
cudaError_t bwd_layer(const bf16 *dz, const bf16 *hp, int nin, const bf16 *w, bf16 *out,
                      int64_t rows, const BwPlan &pl, float *part, cudaStream_t s) {
    CUtensorMap mdz, mhp, mout;
    if (!bf16_map(&mdz, dz, kH, rows, 64, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !bf16_map(&mhp, hp, nin, rows, nin == kH ? 64 : kF,
                  nin == kH ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B) ||
        !bf16_map(&mout, out ? (const void *)out : (const void *)dz, kH, rows, 64,
                  CU_TENSOR_MAP_SWIZZLE_128B))
        return cudaErrorInvalidValue;
    auto kern = out ? k_mlp_bwd_tc<true> : k_mlp_bwd_tc<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kBwSmemBytes);
    if (e != cudaSuccess) return e;
    BwArgs a{rows, pl.tiles, pl.tpc, nin, w, part};
    kern<<<(unsigned)pl.ncta, kBwWarps * 32, kBwSmemBytes, s>>>(mdz, mhp, mout, a);
    return cudaGetLastError();
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
    for (int64_t r0 = 0; r0 < R; r0 += kFwdRows) {
        const int64_t n = R - r0 < kFwdRows ? R - r0 : kFwdRows;
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
    const BwPlan pl = bw_plan(rows, device_sm_count());
    GradParts gp;
    gp.ncta = pl.ncta;
    gp.part[0] = w.part;                                           // layer 1: [.][128][17]
    gp.part[1] = gp.part[0] + (size_t)pl.ncta * kH * (kF + 1);      // layers 2, 3: [.][128][129]
    gp.part[2] = gp.part[1] + (size_t)pl.ncta * kH * (kH + 1);
    gp.part[3] = gp.part[2] + (size_t)pl.ncta * kH * (kH + 1);      // layer 4: [.][2][129]
    // layer 4 (CUDA cores), then layers 3, 2, 1 on the tensor cores
    k_bwd_out<<<(unsigned)pl.ncta, kOutGroups * kH, 0, s>>>(w.dout, w.H[2], wb + oW4, rows,
                                                            pl.tpc, dZ[2],
                                                            const_cast<float *>(gp.part[3]));
    if ((e = cudaGetLastError())) return e;
    if ((e = bwd_layer(dZ[2], w.H[1], kH, wb + oW3, dZ[1], rows, pl,
                       const_cast<float *>(gp.part[2]), s)))
        return e;
    if ((e = bwd_layer(dZ[1], w.H[0], kH, wb + oW2, dZ[0], rows, pl,
                       const_cast<float *>(gp.part[1]), s)))
        return e;
    if ((e = bwd_layer(dZ[0], X, kF, nullptr, nullptr, rows, pl,
                       const_cast<float *>(gp.part[0]), s)))
        return e;
    k_reduce_grad<<<(kP + 255) / 256, 256, 0, s>>>(gp, grad);
    return cudaGetLastError();
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
    TraceScope ts(CC_STAGE_MLP, s, (int)((R + kFwdRows - 1) / kFwdRows));
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
    // forward, loss gradient, four backward layers, reduction, loss sum
    TraceScope ts(CC_STAGE_MLP, s, (int)((B + kFwdRows - 1) / kFwdRows) + 7);
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

// refine.cu - Gauss-Newton refinement of the best direction on the tangent
// plane, all seeds at once, in one persistent cooperative kernel.
//
// Each pass evaluates, for every active seed, the objective L and the 2x2
// normal-equation sums at that seed's current candidate point: per ring in
// FP32 (angle from the chord, Gaussian weight, Jacobian); within the CTA and
// across CTAs the sums are carried as double-float pairs (two FP32 values,
// ~48-bit significand, error-free TwoSum additions), because FP64 arithmetic
// on GB300 runs at 1/64 of the FP32 rate.  One bounded grid barrier per pass;
// then every CTA reduces all CTA partials in the same fixed order and runs the
// same update (accept / halve / solve / stop), so every CTA holds identical
// state without a second barrier.  FP64 is used only in the 2x2 normal-
// equation solve and the final normalisation of the result.  No host round trip per
// iteration; the step and stopping rules are those of the C header.
#include <float.h>

#include "cc_math.cuh"
#include "cc_pipe.cuh"

namespace cc {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxSeeds = 64;
constexpr int kGroup = 4;          // seeds evaluated per pass over the rings
constexpr int kMaxHalvings = 10;
constexpr int kSums = 9;           // L, n11, n12, n22, a11, a12, a22, g1, g2
constexpr int kCache = 8;          // rings per thread kept in registers across passes

// ---------------------------------------------------------------------------
// double-float arithmetic (pairs hi + lo of FP32 values)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return make_float2(s, e);
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float2 s = two_sum(a.x, b.x);
    float e = s.y + (a.y + b.y);
    float h = s.x + e;
    return make_float2(h, e - (h - s.x));
}

__device__ __forceinline__ bool df_ge(float2 a, float2 b) {   // a >= b, both normalised
    return a.x > b.x || (a.x == b.x && a.y >= b.y);
}

__device__ __forceinline__ float2 df_from_double(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

__device__ __forceinline__ double df_to_double(float2 v) { return (double)v.x + (double)v.y; }

__device__ __forceinline__ float2 df_shfl_xor(float2 v, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o),
                       __shfl_xor_sync(0xffffffffu, v.y, o));
}

// ---------------------------------------------------------------------------
// seed state (identical in every CTA)
// ---------------------------------------------------------------------------
struct SeedState {
    float2 s[3], c[3];             // accepted point, candidate (double-float)
    float e1[3], e2[3];            // tangent basis at s
    float ce1[3], ce2[3];          // tangent basis at c
    float2 cur[kSums];             // sums at s (double-float)
    float d1, d2;                  // the step in the tangent basis of s
    int h, iter, phase, st;        // phase 0: first evaluation, 1: trial, 2: done
};

// Tangent basis at c (FP32: it only orients the step and the FP32 per-ring
// Jacobian): e1 = unit(c x z) (c x x when |c_z| > 0.9), e2 = c x e1.
__device__ __forceinline__ void basis(const float2 *c, float *e1, float *e2) {
    float s0 = c[0].x, s1 = c[1].x, s2 = c[2].x;
    float r0 = 0.0f, r1 = 0.0f, r2 = 1.0f;
    if (fabsf(s2) > 0.9f) { r0 = 1.0f; r2 = 0.0f; }
    float a0 = s1 * r2 - s2 * r1, a1 = s2 * r0 - s0 * r2, a2 = s0 * r1 - s1 * r0;
    float inv = rsqrtf(a0 * a0 + a1 * a1 + a2 * a2);
    a0 *= inv; a1 *= inv; a2 *= inv;
    e1[0] = a0; e1[1] = a1; e1[2] = a2;
    e2[0] = s1 * a2 - s2 * a1;
    e2[1] = s2 * a0 - s0 * a2;
    e2[2] = s0 * a1 - s1 * a0;
}

// FP64 arithmetic is slow on GB300 (1/64 of the FP32 rate; the update below
// is one dependent chain on one thread, and every FP64 operation or
// conversion on it costs ~100 clocks), so FP64 is kept to the places that
// need it - the 2x2 normal-equation solve and the final normalisation of the
// result - and the rest of the update runs in FP32: the accepted point and
// the candidate are double-float pairs (~48 bits), the step t a small FP32
// tangent vector, the slope test FP32.
__device__ __forceinline__ void unit3(double *a) {
    double inv = rsqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    a[0] *= inv;
    a[1] *= inv;
    a[2] *= inv;
}

// x^2 as a double-float pair (FMA gives the product's rounding error exactly)
__device__ __forceinline__ float2 df_sq(float2 x) {
    const float p = x.x * x.x;
    const float e = fmaf(x.x, x.x, -p);
    return two_sum(p, fmaf(2.0f * x.x, x.y, e));
}

// c / |c| for a double-float vector near the unit sphere: |c|^2 = 1 + e is
// summed in double-float, so the norm never drifts; 1 / sqrt(1 + e) =
// 1 + delta with delta = -e/2 + 3 e^2 / 8 (truncation below 1e-13) for
// |e| < 1e-4, else the FP32 reciprocal square root with one Newton step (the
// norm is then within ~1e-7 of 1 and the next renormalisation corrects it).
__device__ __forceinline__ void df_unit3(float2 *c) {
    float2 n2 = make_float2(-1.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < 3; k++) n2 = df_add(n2, df_sq(c[k]));
    const float e = n2.x;                                   // |c|^2 - 1
    float delta;
    if (fabsf(e) < 1e-4f) {
        delta = e * fmaf(0.375f, e, -0.5f);
    } else {
        const float x = 1.0f + e, y = rsqrt_approx(x);
        delta = y * fmaf(-0.5f * x * y, y, 1.5f) - 1.0f;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) c[k] = df_add(c[k], make_float2(c[k].x * delta, 0.0f));
}

// Candidate (s + t) / |s + t| with t = f (d1 e1 + d2 e2), and its tangent basis.
__device__ void set_candidate(SeedState &S, float f) {
#pragma unroll
    for (int c = 0; c < 3; c++)
        S.c[c] = df_add(S.s[c], make_float2(f * fmaf(S.d1, S.e1[c], S.d2 * S.e2[c]), 0.0f));
    df_unit3(S.c);
    basis(S.c, S.ce1, S.ce2);
}

// Normal equations at the accepted point -> next candidate or stop, solved in
// FP64.  The Gauss-Newton matrix N = sum w (1 - r^2) J J^T is used when
// positive definite, else the IRLS matrix A = sum w J J^T.
__device__ void next_step(SeedState &S, int max_iter, double tol) {
    if (S.iter >= max_iter) { S.phase = 2; S.st = CC_ENOCONV; return; }
    double a11 = df_to_double(S.cur[1]), a12 = df_to_double(S.cur[2]),
           a22 = df_to_double(S.cur[3]);
    const double g1 = df_to_double(S.cur[7]), g2 = df_to_double(S.cur[8]);
    double det = a11 * a22 - a12 * a12;
    if (!(a11 > 0.0) || !(det > 0.0) || !isfinite(det)) {
        a11 = df_to_double(S.cur[4]);
        a12 = df_to_double(S.cur[5]);
        a22 = df_to_double(S.cur[6]);
        det = a11 * a22 - a12 * a12;
    }
    if (!(det > 0.0) || !isfinite(det)) { S.phase = 2; S.st = CC_ENOCONV; return; }
    const double idet = 1.0 / det;
    const double d1 = (-g1 * a22 + g2 * a12) * idet;
    const double d2 = (-g2 * a11 + g1 * a12) * idet;
    if (!isfinite(d1) || !isfinite(d2)) { S.phase = 2; S.st = CC_ENOCONV; return; }
    S.iter++;
    if (d1 * d1 + d2 * d2 < tol * tol) { S.phase = 2; S.st = CC_OK; return; }
    S.d1 = (float)d1;
    S.d2 = (float)d2;
    S.h = 0;
    S.phase = 1;
    set_candidate(S, 1.0f);
}

// Consume the sums evaluated at the candidate.
__device__ void update(SeedState &S, const float2 *sums, int max_iter, double tol) {
    if (S.phase == 0) {
#pragma unroll
        for (int c = 0; c < 3; c++) { S.s[c] = S.c[c]; S.e1[c] = S.ce1[c]; S.e2[c] = S.ce2[c]; }
#pragma unroll
        for (int q = 0; q < kSums; q++) S.cur[q] = sums[q];
        next_step(S, max_iter, tol);
    } else if (S.phase == 1) {
        // acceptable: L not lower, or the slope of L along the step is still
        // >= 0 at the trial (before the maximum on the step's great circle)
        float slope = 0.0f;
        const float s7 = sums[7].x, s8 = sums[8].x;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float Dc = fmaf(S.d1, S.e1[c], S.d2 * S.e2[c]);
            slope -= Dc * fmaf(s7, S.ce1[c], s8 * S.ce2[c]);
        }
        if (df_ge(sums[0], S.cur[0]) || slope >= 0.0f) {
#pragma unroll
            for (int c = 0; c < 3; c++) { S.s[c] = S.c[c]; S.e1[c] = S.ce1[c]; S.e2[c] = S.ce2[c]; }
#pragma unroll
            for (int q = 0; q < kSums; q++) S.cur[q] = sums[q];
            next_step(S, max_iter, tol);
        } else if (++S.h > kMaxHalvings) {
            S.phase = 2;                 // no acceptable trial: stationary
            S.st = CC_OK;
        } else {
            set_candidate(S, ldexpf(1.0f, -S.h));
        }
    }
}

// Bounded grid barrier (all CTAs co-resident: cooperative launch) on one
// counter that only grows: pass n ends when it reaches (n + 1) G.
__device__ bool grid_sync(unsigned *count, unsigned target) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        __threadfence();
        atomicAdd(count, 1u);
        ok = spin_until_ge(count, target);
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// One ring's FP32 terms at a candidate point C = (s, e1, e2): the weight w
// (into the double-float L) and the normal-equation terms.  The angle comes
// from the chord as in the sweep; sin(theta) = sqrt(h (2 - h)).  Branch-free
// (a ring outside the angular selection, or keep = 0, adds exact zeros; a
// ring with sin(theta) < 1e-6 adds its weight only), so the rings of a thread
// overlap in the pipeline.
__device__ __forceinline__ void ring_terms(float a0, float a1, float a2, float eta, float inv_de,
                                           const float *C, float kcut, bool keep, float2 &L,
                                           float *acc) {
    float dx = a0 - C[0], dy = a1 - C[1], dz = a2 - C[2];
    float h = 0.5f * fmaf(dx, dx, fmaf(dy, dy, dz * dz));   // 1 - cos(theta)
    float th = angle_from_half_chord2(h);
    float r = (th - eta) * inv_de;
    keep = keep && !(kcut > 0.0f && fabsf(r) > kcut);
    float w = keep ? ex2_approx(-0.72134752f * r * r) : 0.0f;   // exp(-r^2 / 2)
    L = df_add(L, make_float2(w, 0.0f));
    float st2 = h * (2.0f - h);                              // sin^2(theta)
    float f = st2 < 1e-12f ? 0.0f : -inv_de * rsqrt_approx(st2);   // -1 / (sin(theta) deta)
    float j1 = f * fmaf(a0, C[3], fmaf(a1, C[4], a2 * C[5]));
    float j2 = f * fmaf(a0, C[6], fmaf(a1, C[7], a2 * C[8]));
    float wj1 = w * j1, wj2 = w * j2;
    float nf = fmaf(-r, r, 1.0f);
    acc[1] = fmaf(nf * wj1, j1, acc[1]);
    acc[2] = fmaf(nf * wj1, j2, acc[2]);
    acc[3] = fmaf(nf * wj2, j2, acc[3]);
    acc[4] = fmaf(wj1, j1, acc[4]);
    acc[5] = fmaf(wj1, j2, acc[5]);
    acc[6] = fmaf(wj2, j2, acc[6]);
    acc[7] = fmaf(wj1, r, acc[7]);
    acc[8] = fmaf(wj2, r, acc[8]);
}

// Ring i as the per-pass terms use it: unit axis, eta, 1 / deta.
__device__ __forceinline__ void load_ring(const float *__restrict__ ax,
                                          const float *__restrict__ ay,
                                          const float *__restrict__ az,
                                          const float *__restrict__ eta,
                                          const float *__restrict__ deta, int64_t i, float &a0,
                                          float &a1, float &a2, float &et, float &inv_de) {
    a0 = ax[i];
    a1 = ay[i];
    a2 = az[i];
    const float inv = rsqrt_approx(fmaf(a0, a0, fmaf(a1, a1, a2 * a2)));
    a0 *= inv;
    a1 *= inv;
    a2 *= inv;
    et = eta[i];
    inv_de = __frcp_rn(deta[i]);
}

__global__ void __launch_bounds__(kThreads)
k_refine(const float *__restrict__ ax, const float *__restrict__ ay,
         const float *__restrict__ az, const float *__restrict__ eta,
         const float *__restrict__ deta, const uint8_t *__restrict__ valid, int64_t R,
         const double *__restrict__ seeds, int k, float k_cut, int max_iter, double tol,
         unsigned *bar, float2 *partials, double *out_dir, double *out_obj,
         int32_t *out_iters, int32_t *status) {
    __shared__ SeedState S[kMaxSeeds];
    __shared__ float cf[kMaxSeeds][9];                  // FP32 candidate + basis
    __shared__ float2 red[kThreads / 32][kGroup * kSums];
    __shared__ float2 sums[kMaxSeeds * kSums];
    __shared__ int active_any;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned G = gridDim.x;
    const int P = k * kSums;                            // partial sums per CTA
    if (tid < k) {
        SeedState &T = S[tid];
        for (int c = 0; c < 3; c++) T.c[c] = df_from_double(seeds[3 * tid + c]);
        df_unit3(T.c);
        basis(T.c, T.ce1, T.ce2);
        T.phase = 0;
        T.iter = 0;
        T.h = 0;
        T.st = CC_ENOCONV;
        T.d1 = T.d2 = 0.0f;
        for (int q = 0; q < kSums; q++) T.cur[q] = make_float2(0.0f, 0.0f);
    }
    __syncthreads();

    // The first kCache rings of this thread (unit axis, eta, 1/deta) stay in
    // registers for every pass; rings beyond them are re-read per pass.  The
    // order in which a thread visits its rings is the same either way.
    const int64_t stride = (int64_t)G * kThreads;
    const int64_t i0 = blockIdx.x * (int64_t)kThreads + tid;
    float ca0[kCache], ca1[kCache], ca2[kCache], cet[kCache], cid[kCache];
    unsigned cok = 0;
#pragma unroll
    for (int j = 0; j < kCache; j++) {
        const int64_t i = i0 + j * stride;
        ca0[j] = ca1[j] = ca2[j] = cet[j] = cid[j] = 0.0f;
        if (i < R && CC_IN_BOUNDS(CC_SITE_REFINE_RING, i, R) && (valid == nullptr || valid[i])) {
            load_ring(ax, ay, az, eta, deta, i, ca0[j], ca1[j], ca2[j], cet[j], cid[j]);
            cok |= 1u << j;
        }
    }

    for (int pass = 0;; pass++) {
        if (tid < k) {
            for (int c = 0; c < 3; c++) {
                cf[tid][c] = S[tid].c[c].x;
                cf[tid][3 + c] = S[tid].ce1[c];
                cf[tid][6 + c] = S[tid].ce2[c];
            }
        }
        __syncthreads();
        float2 *slot = partials + (size_t)(pass & 1) * G * P;

        // this CTA's sums, seeds in groups of kGroup
        for (int g0 = 0; g0 < k; g0 += kGroup) {
            bool act[kGroup];
            bool any = false;
#pragma unroll
            for (int g = 0; g < kGroup; g++) {
                act[g] = (g0 + g < k) && S[g0 + g].phase != 2;
                any = any || act[g];
            }
            if (!any) continue;                         // uniform across the CTA
            float acc[kGroup][kSums];
            float2 L[kGroup];
#pragma unroll
            for (int g = 0; g < kGroup; g++) {
                L[g] = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int q = 0; q < kSums; q++) acc[g][q] = 0.0f;
            }
#pragma unroll
            for (int g = 0; g < kGroup; g++) {
                if (!act[g]) continue;              // uniform across the CTA
#pragma unroll
                for (int j = 0; j < kCache; j++)
                    ring_terms(ca0[j], ca1[j], ca2[j], cet[j], cid[j], cf[g0 + g], k_cut,
                               (cok >> j) & 1u, L[g], acc[g]);
            }
            for (int64_t i = i0 + kCache * stride; i < R; i += stride) {
                if (!CC_IN_BOUNDS(CC_SITE_REFINE_RING, i, R)) break;
                if (valid != nullptr && !valid[i]) continue;
                float a0, a1, a2, et, inv_de;
                load_ring(ax, ay, az, eta, deta, i, a0, a1, a2, et, inv_de);
#pragma unroll
                for (int g = 0; g < kGroup; g++)
                    if (act[g])
                        ring_terms(a0, a1, a2, et, inv_de, cf[g0 + g], k_cut, true, L[g], acc[g]);
            }
            // warp and CTA sums in double-float
#pragma unroll
            for (int g = 0; g < kGroup; g++) {
                if (!act[g]) continue;
                float2 v[kSums];                        // the 9 trees advance level by level
#pragma unroll
                for (int q = 0; q < kSums; q++) v[q] = q == 0 ? L[g] : make_float2(acc[g][q], 0.0f);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int q = 0; q < kSums; q++) v[q] = df_add(v[q], df_shfl_xor(v[q], o));
                if (lane == 0)
#pragma unroll
                    for (int q = 0; q < kSums; q++) red[wid][g * kSums + q] = v[q];
            }
            __syncthreads();
            if (tid < kGroup * kSums && g0 + tid / kSums < k) {
                float2 v = make_float2(0.0f, 0.0f);
                if (act[tid / kSums])
                    for (int ww = 0; ww < kThreads / 32; ww++) v = df_add(v, red[ww][tid]);
                if (CC_IN_BOUNDS(CC_SITE_REFINE_SLOT, (int64_t)blockIdx.x * P + g0 * kSums + tid,
                                 (int64_t)G * P))
                    slot[(size_t)blockIdx.x * P + g0 * kSums + tid] = v;
            }
            __syncthreads();
        }
        if (!grid_sync(bar, (unsigned)(pass + 1) * G)) {
            if (tid == 0) atomicExch(status, (int32_t)CC_ETIMEOUT);
            return;
        }
        // every CTA reduces all CTA partials in one fixed order: 16 lanes (a
        // half warp) per sum, each adding the CTAs b = v, v + 16, ... in turn,
        // then a fixed shuffle tree over the 16.  The first kBatch partials
        // of a lane are loaded before any is added, so that their L2 round
        // trips overlap (adding the zeros of absent CTAs changes nothing:
        // (0, 0) is an exact identity of df_add on normalised pairs)
        for (int u0 = 0; u0 < P; u0 += kThreads / 16) {
            const int u = u0 + (tid >> 4), v = tid & 15;
            float2 a = make_float2(0.0f, 0.0f);
            if (u < P && S[u / kSums].phase != 2) {
                constexpr int kBatch = 8;
                float2 pv[kBatch];
#pragma unroll
                for (int j = 0; j < kBatch; j++) {
                    const unsigned b = v + 16u * j;
                    pv[j] = b < G ? __ldcg(slot + (size_t)b * P + u) : make_float2(0.0f, 0.0f);
                }
#pragma unroll
                for (int j = 0; j < kBatch; j++) a = df_add(a, pv[j]);
                for (unsigned b = v + 16u * kBatch; b < G; b += 16)
                    a = df_add(a, __ldcg(slot + (size_t)b * P + u));
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) a = df_add(a, df_shfl_xor(a, o));
            if (v == 0 && u < P) sums[u] = a;
        }
        __syncthreads();
        if (tid < k && S[tid].phase != 2) update(S[tid], sums + tid * kSums, max_iter, tol);
        if (tid == 0) active_any = 0;
        __syncthreads();
        if (tid < k && S[tid].phase != 2) active_any = 1;
        __syncthreads();
        if (!active_any) break;
    }

    if (blockIdx.x == 0 && tid == 0) {
        int best = 0;
        for (int t = 1; t < k; t++)
            if (!df_ge(S[best].cur[0], S[t].cur[0])) best = t;
        double d[3] = {df_to_double(S[best].s[0]), df_to_double(S[best].s[1]),
                       df_to_double(S[best].s[2])};
        unit3(d);
        out_dir[0] = d[0];
        out_dir[1] = d[1];
        out_dir[2] = d[2];
        *out_obj = df_to_double(S[best].cur[0]);
        *out_iters = S[best].iter;
        *status = S[best].st;
    }
}

int refine_grid(int64_t R) {
    const int sms = device_sm_count();
    if (sms <= 0) return 0;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_refine, kThreads, 0);
    if (occ < 1) occ = 1;
    int64_t cap = (int64_t)sms * occ;
    int64_t want = (R + 2047) / 2048;                  // ~8 rings per thread per seed
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

}  // namespace

size_t refine_workspace_bytes(int64_t R, int k) {
    if (R < 0 || k < 1 || k > kMaxSeeds) return 0;
    int G = refine_grid(R);
    if (G <= 0) return 0;
    return 256 + align256((size_t)2 * G * k * kSums * sizeof(float2));
}

cudaError_t launch_refine(const cc_rings &rings, const double *seeds, int k,
                          const cc_params &p, double *out_dir, double *out_obj,
                          int32_t *out_iters, int32_t *status, char *ws, size_t ws_bytes,
                          cudaStream_t s) {
    (void)ws_bytes;
    cudaError_t e = cudaMemsetAsync(ws, 0, 256, s);   // barrier counter
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    int G = refine_grid(rings.count);
    unsigned *bar = reinterpret_cast<unsigned *>(ws);
    float2 *partials = reinterpret_cast<float2 *>(ws + 256);
    int64_t R = rings.count;
    float kc = p.k_cut;
    int mi = p.max_iter;
    double tol = p.tol_rad;
    void *args[] = {(void *)&rings.ax, (void *)&rings.ay, (void *)&rings.az,
                    (void *)&rings.eta, (void *)&rings.deta, (void *)&rings.valid,
                    (void *)&R,        (void *)&seeds,    (void *)&k,
                    (void *)&kc,       (void *)&mi,       (void *)&tol,
                    (void *)&bar,      (void *)&partials, (void *)&out_dir,
                    (void *)&out_obj,  (void *)&out_iters, (void *)&status};
    TraceScope ts(CC_STAGE_REFINE, s);
    return cudaLaunchCooperativeKernel((void *)k_refine, dim3(G), dim3(kThreads), args, 0, s);
}

}  // namespace cc

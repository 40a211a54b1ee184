// refine.cu - Gauss-Newton (iteratively reweighted least squares) refinement
// of the best direction on the tangent plane, all seeds at once, in one
// persistent cooperative kernel.
//
// Each pass evaluates, for every active seed, the objective L and the 2x2
// normal-equation sums at that seed's current candidate point: per ring in
// FP32 (angle from the chord, Gaussian weight, Jacobian), per CTA summed in
// FP64 and written to a double-buffered workspace slot; one bounded grid
// barrier; then every CTA reduces all CTA partials in the same fixed order and
// runs the same FP64 update (accept / halve / solve / stop), so every CTA
// holds identical state without a second barrier.  No host round trip per
// iteration; the step rule and stopping rule are those of the header.
#include <float.h>

#include "cc_internal.cuh"

namespace cc {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxSeeds = 64;
constexpr int kGroup = 4;          // seeds evaluated per pass over the rings
constexpr int kMaxHalvings = 10;
constexpr int kSums = 9;           // L, n11, n12, n22, a11, a12, a22, g1, g2

struct SeedState {
    double s[3], e1[3], e2[3];     // accepted point and tangent basis
    double c[3], ce1[3], ce2[3];   // candidate under evaluation
    double cur[kSums];             // sums at s (see kSums)
    double d1, d2;
    int h, iter, phase, st;        // phase 0: first evaluation, 1: trial, 2: done
};

__device__ __forceinline__ void unit3(double *a) {
    double n = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    a[0] /= n;
    a[1] /= n;
    a[2] /= n;
}

__device__ __forceinline__ void basis(const double *s, double *e1, double *e2) {
    double r0 = 0.0, r1 = 0.0, r2 = 1.0;
    if (fabs(s[2]) > 0.9) { r0 = 1.0; r2 = 0.0; }
    e1[0] = s[1] * r2 - s[2] * r1;
    e1[1] = s[2] * r0 - s[0] * r2;
    e1[2] = s[0] * r1 - s[1] * r0;
    unit3(e1);
    e2[0] = s[1] * e1[2] - s[2] * e1[1];
    e2[1] = s[2] * e1[0] - s[0] * e1[2];
    e2[2] = s[0] * e1[1] - s[1] * e1[0];
}

// Candidate s + f (d1 e1 + d2 e2), renormalised, with its tangent basis.
__device__ void set_candidate(SeedState &S, double f) {
    for (int c = 0; c < 3; c++) S.c[c] = S.s[c] + f * (S.d1 * S.e1[c] + S.d2 * S.e2[c]);
    unit3(S.c);
    basis(S.c, S.ce1, S.ce2);
}

// Normal equations at the accepted point -> next candidate or stop.  The
// Gauss-Newton matrix N = sum w (1 - r^2) J J^T is used when positive
// definite, else the IRLS matrix A = sum w J J^T.
__device__ void next_step(SeedState &S, int max_iter, double tol) {
    if (S.iter >= max_iter) { S.phase = 2; S.st = CC_ENOCONV; return; }
    double a11 = S.cur[1], a12 = S.cur[2], a22 = S.cur[3], g1 = S.cur[7], g2 = S.cur[8];
    double det = a11 * a22 - a12 * a12;
    if (!(a11 > 0.0) || !(det > 0.0) || !isfinite(det)) {
        a11 = S.cur[4];
        a12 = S.cur[5];
        a22 = S.cur[6];
        det = a11 * a22 - a12 * a12;
    }
    if (!(det > 0.0) || !isfinite(det)) { S.phase = 2; S.st = CC_ENOCONV; return; }
    double d1 = (-g1 * a22 + g2 * a12) / det;
    double d2 = (-g2 * a11 + g1 * a12) / det;
    if (!isfinite(d1) || !isfinite(d2)) { S.phase = 2; S.st = CC_ENOCONV; return; }
    S.iter++;
    if (sqrt(d1 * d1 + d2 * d2) < tol) { S.phase = 2; S.st = CC_OK; return; }
    S.d1 = d1;
    S.d2 = d2;
    S.h = 0;
    S.phase = 1;
    set_candidate(S, 1.0);
}

// Consume the sums evaluated at the candidate.
__device__ void update(SeedState &S, const double *sums, int max_iter, double tol) {
    if (S.phase == 0) {
        for (int c = 0; c < 3; c++) { S.s[c] = S.c[c]; S.e1[c] = S.ce1[c]; S.e2[c] = S.ce2[c]; }
        for (int q = 0; q < kSums; q++) S.cur[q] = sums[q];
        next_step(S, max_iter, tol);
    } else if (S.phase == 1) {
        if (sums[0] >= S.cur[0]) {       // first trial that does not lower L
            for (int c = 0; c < 3; c++) { S.s[c] = S.c[c]; S.e1[c] = S.ce1[c]; S.e2[c] = S.ce2[c]; }
            for (int q = 0; q < kSums; q++) S.cur[q] = sums[q];
            next_step(S, max_iter, tol);
        } else if (++S.h > kMaxHalvings) {
            S.phase = 2;                 // every trial lowers L: stationary
            S.st = CC_OK;
        } else {
            set_candidate(S, ldexp(1.0, -S.h));
        }
    }
}

// Bounded grid barrier (all CTAs co-resident: cooperative launch).
__device__ bool grid_sync(unsigned *count, unsigned *gen, unsigned nblocks) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *vgen = gen;
        unsigned g = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(count, 1u) + 1u;
        if (arrived == nblocks) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            unsigned long long t0 = globaltimer_ns();
            unsigned it = 0;
            while (*vgen == g) {
                __nanosleep(64);
                if ((++it & 255) == 0 && globaltimer_ns() - t0 > kWaitLimitNs) {
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

__global__ void __launch_bounds__(kThreads)
k_refine(const float *__restrict__ ax, const float *__restrict__ ay,
         const float *__restrict__ az, const float *__restrict__ eta,
         const float *__restrict__ deta, const uint8_t *__restrict__ valid, int64_t R,
         const double *__restrict__ seeds, int k, float k_cut, int max_iter, double tol,
         unsigned *bar, double *partials, double *out_dir, double *out_obj,
         int32_t *out_iters, int32_t *status) {
    __shared__ SeedState S[kMaxSeeds];
    __shared__ float cf[kMaxSeeds][9];      // FP32 copy of candidate + basis
    __shared__ double red[kThreads / 32][kGroup * kSums];
    __shared__ int active_any;

    const int tid = threadIdx.x;
    const unsigned G = gridDim.x;
    if (tid < k) {
        SeedState &T = S[tid];
        for (int c = 0; c < 3; c++) T.c[c] = seeds[3 * tid + c];
        unit3(T.c);
        basis(T.c, T.ce1, T.ce2);
        T.phase = 0;
        T.iter = 0;
        T.h = 0;
        T.st = CC_ENOCONV;
        T.d1 = T.d2 = 0.0;
        for (int q = 0; q < kSums; q++) T.cur[q] = 0.0;
    }
    __syncthreads();

    const float kcut = k_cut;
    for (int pass = 0;; pass++) {
        // FP32 copies of the candidates
        if (tid < k) {
            for (int c = 0; c < 3; c++) {
                cf[tid][c] = (float)S[tid].c[c];
                cf[tid][3 + c] = (float)S[tid].ce1[c];
                cf[tid][6 + c] = (float)S[tid].ce2[c];
            }
        }
        __syncthreads();
        double *slot = partials + (size_t)(pass & 1) * G * k * kSums;
        for (int g0 = 0; g0 < k; g0 += kGroup) {
            float acc[kGroup][kSums];
#pragma unroll
            for (int g = 0; g < kGroup; g++)
#pragma unroll
                for (int q = 0; q < kSums; q++) acc[g][q] = 0.0f;
            bool act[kGroup];
#pragma unroll
            for (int g = 0; g < kGroup; g++) act[g] = (g0 + g < k) && S[g0 + g].phase != 2;
            for (int64_t i = blockIdx.x * (int64_t)kThreads + tid; i < R;
                 i += (int64_t)G * kThreads) {
                if (valid != nullptr && !valid[i]) continue;
                float a0 = ax[i], a1 = ay[i], a2 = az[i];
                float inv = rsqrtf(a0 * a0 + a1 * a1 + a2 * a2);
                a0 *= inv; a1 *= inv; a2 *= inv;
                const float et = eta[i], de = deta[i];
#pragma unroll
                for (int g = 0; g < kGroup; g++) {
                    if (!act[g]) continue;
                    const float *C = cf[g0 + g];
                    float dx = a0 - C[0], dy = a1 - C[1], dz = a2 - C[2];
                    float sx = a0 + C[0], sy = a1 + C[1], sz = a2 + C[2];
                    float qm = dx * dx + dy * dy + dz * dz;   // |a - s|^2
                    float qp = sx * sx + sy * sy + sz * sz;   // |a + s|^2
                    float th = qm <= qp ? 2.0f * asinf(0.5f * sqrtf(qm))
                                        : kPiF - 2.0f * asinf(0.5f * sqrtf(qp));
                    float r = (th - et) / de;
                    if (kcut > 0.0f && fabsf(r) > kcut) continue;
                    float w = expf(-0.5f * r * r);
                    acc[g][0] += w;
                    float st = 0.5f * sqrtf(qm * qp);          // sin(theta)
                    if (st < 1e-6f) continue;
                    float f = -1.0f / (st * de);
                    float j1 = f * (a0 * C[3] + a1 * C[4] + a2 * C[5]);
                    float j2 = f * (a0 * C[6] + a1 * C[7] + a2 * C[8]);
                    float wj1 = w * j1, wj2 = w * j2;
                    float nf = 1.0f - r * r;
                    acc[g][1] += nf * wj1 * j1;
                    acc[g][2] += nf * wj1 * j2;
                    acc[g][3] += nf * wj2 * j2;
                    acc[g][4] += wj1 * j1;
                    acc[g][5] += wj1 * j2;
                    acc[g][6] += wj2 * j2;
                    acc[g][7] += wj1 * r;
                    acc[g][8] += wj2 * r;
                }
            }
            // block sums in FP64
            const int w = tid >> 5, l = tid & 31;
#pragma unroll
            for (int g = 0; g < kGroup; g++)
#pragma unroll
                for (int q = 0; q < kSums; q++) {
                    double v = (double)acc[g][q];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (l == 0) red[w][g * kSums + q] = v;
                }
            __syncthreads();
            if (tid < kGroup * kSums) {
                int g = tid / kSums;
                if (g0 + g < k) {
                    double v = 0.0;
                    for (int ww = 0; ww < kThreads / 32; ww++) v += red[ww][tid];
                    slot[((size_t)blockIdx.x * k + g0 + g) * kSums + (tid % kSums)] = v;
                }
            }
            __syncthreads();
        }
        if (!grid_sync(bar, bar + 1, G)) {
            if (tid == 0) atomicExch(status, (int32_t)CC_ETIMEOUT);
            return;
        }
        // every CTA: reduce all partials (fixed order) and update the seeds
        if (tid < k && S[tid].phase != 2) {
            double sums[kSums];
            for (int q = 0; q < kSums; q++) sums[q] = 0.0;
            for (unsigned b = 0; b < G; b++)
                for (int q = 0; q < kSums; q++)
                    sums[q] += __ldcg(slot + ((size_t)b * k + tid) * kSums + q);
            update(S[tid], sums, max_iter, tol);
        }
        if (tid == 0) active_any = 0;
        __syncthreads();
        if (tid < k && S[tid].phase != 2) active_any = 1;
        __syncthreads();
        if (!active_any) break;
    }

    if (blockIdx.x == 0 && tid == 0) {
        int best = 0;
        for (int t = 1; t < k; t++)
            if (S[t].cur[0] > S[best].cur[0]) best = t;
        double d[3] = {S[best].s[0], S[best].s[1], S[best].s[2]};
        unit3(d);
        out_dir[0] = d[0];
        out_dir[1] = d[1];
        out_dir[2] = d[2];
        *out_obj = S[best].cur[0];
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
    int64_t want = (R + kThreads * 4 - 1) / (kThreads * 4);
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

}  // namespace

size_t refine_workspace_bytes(int64_t R, int k) {
    if (R < 0 || k < 1 || k > kMaxSeeds) return 0;
    int G = refine_grid(R);
    if (G <= 0) return 0;
    return 256 + align256((size_t)2 * G * k * kSums * sizeof(double));
}

cudaError_t launch_refine(const cc_rings &rings, const double *seeds, int k,
                          const cc_params &p, double *out_dir, double *out_obj,
                          int32_t *out_iters, int32_t *status, char *ws, size_t ws_bytes,
                          cudaStream_t s) {
    (void)ws_bytes;
    cudaError_t e = cudaMemsetAsync(ws, 0, 256, s);   // barrier counter + generation
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    int G = refine_grid(rings.count);
    unsigned *bar = reinterpret_cast<unsigned *>(ws);
    double *partials = reinterpret_cast<double *>(ws + 256);
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

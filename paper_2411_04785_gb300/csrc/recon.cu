// recon.cu - rings from detector events: site ordering, cone axis, opening
// angle and width (Sec. 1.1 of the paper: the Compton formula and the cone of
// two interactions; the ordering of 3-4 sites and the width are readings).
//
// One thread per event.  The ORDER is an integer decided by floating point,
// so it is decided in IEEE binary32 with every operation rounded once
// (__fadd_rn / __fmul_rn / __frcp_rn / __fdiv_rn / __fsqrt_rn: no
// contraction into FMA), in a fixed sequence:
//   E(S)        = deposits of the slots in set S added in increasing slot order
//   cos(Ea, Eb) = 1 - m_e c^2 * (1/Ea - 1/Eb)
//   |x_q - x_p|^2 = ((dx*dx) + (dy*dy)) + (dz*dz), d = x_q - x_p
//   cos_G(p,q,r)  = dot(x_q - x_p, x_r - x_q) / sqrt(|x_q-x_p|^2 * |x_r-x_q|^2)
//   chi2        = sum over intermediate positions (ascending) of (cos_E - cos_G)^2
// so any implementation of the same rule in binary32 picks the same order.
// The ring itself (axis, eta, width) is computed in FP32 with
// better-conditioned but mathematically equal formulas.
#include "cc_internal.cuh"

namespace cc {
namespace {

constexpr float kInf = __builtin_huge_valf();

template <int K>
__device__ __forceinline__ float set_energy(const float (&e)[4], unsigned mask) {
    float s = 0.0f;
#pragma unroll
    for (int m = 0; m < K; m++)
        if (mask & (1u << m)) s = __fadd_rn(s, e[m]);
    return s;
}

__device__ __forceinline__ float compton_cos(float e_after, float e_before) {
    float ia = __frcp_rn(e_after);
    float ib = __frcp_rn(e_before);
    return __fsub_rn(1.0f, __fmul_rn(kMeKeV, __fsub_rn(ia, ib)));
}

__device__ __forceinline__ float sqdist(const float (&x)[4], const float (&y)[4],
                                        const float (&z)[4], int p, int q) {
    float dx = __fsub_rn(x[q], x[p]);
    float dy = __fsub_rn(y[q], y[p]);
    float dz = __fsub_rn(z[q], z[p]);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)),
                     __fmul_rn(dz, dz));
}

__device__ __forceinline__ bool in_unit(float c) { return c >= -1.0f && c <= 1.0f; }

// Compton chi2 of the order o[0..K) (compile-time indices after unrolling);
// +inf when the order is kinematically invalid.
template <int K>
__device__ __forceinline__ float order_chi2(const float (&x)[4], const float (&y)[4],
                                            const float (&z)[4], const float (&e)[4],
                                            const int (&o)[K]) {
    constexpr unsigned all = (1u << K) - 1u;
    float e0 = set_energy<K>(e, all);
    float e2 = set_energy<K>(e, all & ~(1u << o[0]));
    float c1 = compton_cos(e2, e0);
    bool ok = (e0 > 0.0f) && (e2 > 0.0f) && in_unit(c1) &&
              (sqdist(x, y, z, o[0], o[1]) > 1e-12f);
    float chi2 = 0.0f;
#pragma unroll
    for (int j = 1; j + 1 < K; j++) {
        unsigned before = 0;
#pragma unroll
        for (int m = j; m < K; m++) before |= 1u << o[m];
        unsigned after = before & ~(1u << o[j]);
        float eb = set_energy<K>(e, before);
        float ea = set_energy<K>(e, after);
        float ce = compton_cos(ea, eb);
        int p = o[j - 1], q = o[j], r = o[j + 1];
        float ux = __fsub_rn(x[q], x[p]), uy = __fsub_rn(y[q], y[p]),
              uz = __fsub_rn(z[q], z[p]);
        float vx = __fsub_rn(x[r], x[q]), vy = __fsub_rn(y[r], y[q]),
              vz = __fsub_rn(z[r], z[q]);
        float dot = __fadd_rn(__fadd_rn(__fmul_rn(ux, vx), __fmul_rn(uy, vy)),
                              __fmul_rn(uz, vz));
        float nn = __fmul_rn(sqdist(x, y, z, p, q), sqdist(x, y, z, q, r));
        float cg = __fdiv_rn(dot, __fsqrt_rn(nn));
        float d = __fsub_rn(ce, cg);
        chi2 = __fadd_rn(chi2, __fmul_rn(d, d));
        ok = ok && (ea > 0.0f) && in_unit(ce) && (nn > 0.0f);
    }
    return ok ? chi2 : kInf;
}

// Klein-Nishina angular weight P^2 (P + 1/P - sin^2 eta), binary32 sequence.
__device__ __forceinline__ float kn_weight(float P, float c) {
    float s2 = __fsub_rn(1.0f, __fmul_rn(c, c));
    float t = __fsub_rn(__fadd_rn(P, __frcp_rn(P)), s2);
    return __fmul_rn(__fmul_rn(P, P), t);
}

__device__ __forceinline__ float pick(const float (&v)[4], int i) {
    float r = v[0];
    r = (i == 1) ? v[1] : r;
    r = (i == 2) ? v[2] : r;
    r = (i == 3) ? v[3] : r;
    return r;
}

// Ordering rule: returns the rank (or -1) and the first two slots.
template <int K>
__device__ __forceinline__ int choose_order(const float (&x)[4], const float (&y)[4],
                                            const float (&z)[4], const float (&e)[4],
                                            int &f0, int &f1) {
    if constexpr (K == 2) {
        const int o01[2] = {0, 1}, o10[2] = {1, 0};
        bool ok0 = order_chi2<2>(x, y, z, e, o01) == 0.0f;
        bool ok1 = order_chi2<2>(x, y, z, e, o10) == 0.0f;
        float e0 = set_energy<2>(e, 3u);
        float w0 = kn_weight(__fdiv_rn(e[1], e0), compton_cos(e[1], e0));
        float w1 = kn_weight(__fdiv_rn(e[0], e0), compton_cos(e[0], e0));
        // set_energy of a single slot is the deposit itself (0 + e = e)
        if (ok1 && (!ok0 || w1 > w0)) { f0 = 1; f1 = 0; return 1; }
        if (ok0) { f0 = 0; f1 = 1; return 0; }
        return -1;
    } else {
        float best = kInf;
        int best_rank = -1, rank = 0;
#pragma unroll
        for (int p0 = 0; p0 < K; p0++)
#pragma unroll
            for (int p1 = 0; p1 < K; p1++) {
                if (p1 == p0) continue;
                if constexpr (K == 3) {
                    const int o[3] = {p0, p1, 3 - p0 - p1};
                    float c = order_chi2<3>(x, y, z, e, o);
                    if (c < best) { best = c; best_rank = rank; f0 = p0; f1 = p1; }
                    rank++;
                } else {
#pragma unroll
                    for (int p2 = 0; p2 < 4; p2++) {
                        if (p2 == p0 || p2 == p1) continue;
                        const int o[4] = {p0, p1, p2, 6 - p0 - p1 - p2};
                        float c = order_chi2<4>(x, y, z, e, o);
                        if (c < best) { best = c; best_rank = rank; f0 = p0; f1 = p1; }
                        rank++;
                    }
                }
            }
        return best_rank;
    }
}

__global__ void __launch_bounds__(128)
k_rings_from_events(const uint8_t *__restrict__ n, const float *__restrict__ xs,
                    const float *__restrict__ ys, const float *__restrict__ zs,
                    const float *__restrict__ es, int64_t count, int64_t stride,
                    float sig_e, float sig_pos, float deta_min, float deta_max,
                    float *__restrict__ ax, float *__restrict__ ay,
                    float *__restrict__ az, float *__restrict__ eta,
                    float *__restrict__ deta, uint8_t *__restrict__ valid,
                    uint8_t *__restrict__ perm) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int k = n[i];
    float x[4], y[4], z[4], e[4];
#pragma unroll
    for (int s = 0; s < 4; s++) {
        bool used = s < k;
        int64_t o = s * stride + i;
        x[s] = used ? __ldg(xs + o) : 0.0f;
        y[s] = used ? __ldg(ys + o) : 0.0f;
        z[s] = used ? __ldg(zs + o) : 0.0f;
        e[s] = used ? __ldg(es + o) : 0.0f;
    }
    int f0 = 0, f1 = 1, rank = -1;
    if (k == 2) rank = choose_order<2>(x, y, z, e, f0, f1);
    else if (k == 3) rank = choose_order<3>(x, y, z, e, f0, f1);
    else if (k == 4) rank = choose_order<4>(x, y, z, e, f0, f1);

    if (rank < 0) {
        ax[i] = ay[i] = az[i] = eta[i] = deta[i] = 0.0f;
        valid[i] = 0;
        perm[i] = 255;
        return;
    }
    // ring of the chosen order: E1 first deposit, E2 the rest, E0 = E1 + E2
    float e1 = pick(e, f0);
    float e2 = 0.0f, var2 = 0.0f;
#pragma unroll
    for (int s = 0; s < 4; s++)
        if (s < k && s != f0) {
            e2 += e[s];
            float sd = sig_e * e[s];
            var2 = fmaf(sd, sd, var2);
        }
    float e0 = e1 + e2;
    // 1/E2 - 1/E0 = E1 / (E2 E0): no cancellation for small E1
    float u = kMeKeV * e1 / (e2 * e0);
    float c = fminf(fmaxf(1.0f - u, -1.0f), 1.0f);
    float th = acosf(c);
    float sin_eta = sqrtf(fmaxf(u * (2.0f - u), 0.0f));   // sqrt((1-c)(1+c))

    float dx = pick(x, f0) - pick(x, f1);
    float dy = pick(y, f0) - pick(y, f1);
    float dz = pick(z, f0) - pick(z, f1);
    float len = sqrtf(dx * dx + dy * dy + dz * dz);
    float inv_len = 1.0f / len;

    float s1 = sig_e * e1;
    // 1/E2^2 - 1/E0^2 = E1 (E0 + E2) / (E2^2 E0^2)
    float q = e1 * (e0 + e2) / ((e2 * e2) * (e0 * e0));
    float t1 = s1 / (e0 * e0);
    float var_cos = kMeKeV * kMeKeV * (t1 * t1 + var2 * q * q);
    float w_e = sqrtf(var_cos) / fmaxf(sin_eta, 1e-3f);
    float w_g = 1.41421356237f * sig_pos * inv_len;
    float w = sqrtf(w_e * w_e + w_g * w_g);

    ax[i] = dx * inv_len;
    ay[i] = dy * inv_len;
    az[i] = dz * inv_len;
    eta[i] = th;
    deta[i] = fminf(fmaxf(w, deta_min), deta_max);
    valid[i] = 1;
    perm[i] = (uint8_t)rank;
}

}  // namespace

cudaError_t launch_rings_from_events(const cc_events &ev, const cc_rings &out,
                                     const cc_params &p, cudaStream_t s) {
    if (ev.count == 0) return cudaSuccess;
    const int threads = 128;
    int64_t blocks = (ev.count + threads - 1) / threads;
    TraceScope ts(CC_STAGE_RECON, s);
    k_rings_from_events<<<(unsigned)blocks, threads, 0, s>>>(
        ev.n, ev.x, ev.y, ev.z, ev.e, ev.count, ev.stride, p.sigma_e_frac,
        p.sigma_pos_cm, p.deta_min, p.deta_max, out.ax, out.ay, out.az, out.eta,
        out.deta, out.valid, out.perm);
    return cudaGetLastError();
}

}  // namespace cc

// recon.cu - rings from detector events: site ordering, cone axis, opening
// angle and width (Sec. 1.1 of the paper: the Compton formula and the cone of
// two interactions; the ordering of 3-4 sites and the width are readings).
//
// One thread per event, events grouped by site count within each CTA (see
// k_rings_from_events).  The ORDER is an integer decided by floating point,
// so it is decided in IEEE binary32 with every operation rounded once
// (__fadd_rn / __fmul_rn / __fdiv_rn and the correctly rounded reciprocal,
// root and quotient of cc_math.cuh: no contraction into FMA), in a fixed
// sequence:
//   E(S)        = deposits of the slots in set S added in increasing slot order
//   cos(Ea, Eb) = 1 - m_e c^2 * (1/Ea - 1/Eb)
//   |x_q - x_p|^2 = ((dx*dx) + (dy*dy)) + (dz*dz), d = x_q - x_p
//   il(p,q)     = 1 / sqrt(|x_q - x_p|^2)       (one per site pair)
//   cos_G(p,q,r)  = dot(x_q - x_p, x_r - x_q) * (il(p,q) * il(q,r))
//   chi2        = sum over intermediate positions (ascending) of (cos_E - cos_G)^2
// so any implementation of the same rule in binary32 picks the same order.
// The ring itself (axis, eta, width) is not a decision: it is computed in
// FP32 with better-conditioned but mathematically equal formulas, using the
// MUFU approximations.
#include "cc_math.cuh"
#include "cc_pipe.cuh"

namespace cc {
namespace {

constexpr float kInf = __builtin_huge_valf();
constexpr float kPosEps2 = 1e-12f;   // |x1 - x2|^2 below (1e-6 cm)^2: no axis

__device__ __forceinline__ float sqdist(const float (&x)[4], const float (&y)[4],
                                        const float (&z)[4], int p, int q) {
    float dx = __fsub_rn(x[q], x[p]);
    float dy = __fsub_rn(y[q], y[p]);
    float dz = __fsub_rn(z[q], z[p]);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)),
                     __fmul_rn(dz, dz));
}

// -1 <= c <= 1 (false for NaN)
__device__ __forceinline__ bool in_unit(float c) { return fabsf(c) <= 1.0f; }

template <bool kFast>
__device__ __forceinline__ float rcp_k(float x) {
    if constexpr (kFast) return rcp_core(x);
    else return rcp_exact(x);
}

template <bool kFast>
__device__ __forceinline__ float sqrt_k(float x) {
    if constexpr (kFast) return sqrt_core(x);
    else return sqrt_exact(x);
}

__host__ __device__ constexpr int high_slot(unsigned m) { return m >= 8u ? 3 : m >= 4u ? 2 : m >= 2u ? 1 : 0; }

// Rank (in lexicographic order of the K! orders) of the best order of a
// K-site event, K = 3 or 4, under the binary32 sequence above; -1 if no
// order is valid.  Every quantity an order uses is a table entry built once
// per event: subset energies E[S] (each the previous subset plus its highest
// slot, which is the increasing-slot sum) and their reciprocals, inverse
// lengths, geometric cosines cg(p -> q -> r) (bitwise symmetric in p, r),
// the first step's cosine c1[o0][o1] and, for K = 4, the second step's
// c2[o2][o3].  An order's validity conditions are folded into those entries
// as NaN (unphysical first cone or energy cosine, a non-positive energy, a
// coincident pair), so an invalid order's chi2 is NaN and loses every strict
// comparison, exactly as the +inf of an invalid order does in the rule (a
// chi2 that is NaN for a valid order, from an overflow, loses in both).
// kFast: every deposit is in [2^-100, 2^98] and every squared distance is 0
// or in [2^-100, 2^100].  Then every subset energy is positive and in
// [2^-100, 2^100], every reciprocal and root argument is in the range of the
// one-FMA corrections, and a zero distance's root is NaN, which makes both of
// its geometric cosines NaN, as the rule's validity wants.
template <int K, bool kFast>
__device__ __forceinline__ int order_rank(const float (&x)[4], const float (&y)[4],
                                          const float (&z)[4], const float (&e)[4],
                                          const float (&nsq)[4][4]) {
    constexpr unsigned all = (1u << K) - 1u;
    const float nan = __int_as_float(0x7fc00000);
    float E[1 << K], inv[1 << K];
    E[0] = 0.0f;
#pragma unroll
    for (unsigned m = 1; m <= all; m++) {
        const int h = high_slot(m);
        E[m] = (kFast && m == (1u << h)) ? e[h] : __fadd_rn(E[m & ~(1u << h)], e[h]);
        inv[m] = rcp_k<kFast>(E[m]);
    }
    auto pos = [&](unsigned m) { return kFast || E[m] > 0.0f; };
    auto ccos = [&](unsigned after, unsigned before) {
        return __fsub_rn(1.0f, __fmul_rn(kMeKeV, __fsub_rn(inv[after], inv[before])));
    };
    float il[4][4];
#pragma unroll
    for (int p = 0; p < K; p++)
#pragma unroll
        for (int q = p + 1; q < K; q++) il[p][q] = il[q][p] = rcp_k<kFast>(sqrt_k<kFast>(nsq[p][q]));
    float cg[4][4][4];
#pragma unroll
    for (int q = 0; q < K; q++)
#pragma unroll
        for (int p = 0; p < K; p++)
#pragma unroll
            for (int r = p + 1; r < K; r++) {
                if (p == q || r == q) continue;
                const float ux = __fsub_rn(x[q], x[p]), uy = __fsub_rn(y[q], y[p]),
                            uz = __fsub_rn(z[q], z[p]);
                const float vx = __fsub_rn(x[r], x[q]), vy = __fsub_rn(y[r], y[q]),
                            vz = __fsub_rn(z[r], z[q]);
                const float dot = __fadd_rn(__fadd_rn(__fmul_rn(ux, vx), __fmul_rn(uy, vy)),
                                            __fmul_rn(uz, vz));
                const float c = __fmul_rn(dot, __fmul_rn(il[p][q], il[q][r]));
                // a zero-length segment makes c NaN by itself on the fast path
                // (the uncorrected root of 0 is NaN, so is the inverse
                // length); the checked path selects it
                cg[p][q][r] = cg[r][q][p] = (kFast || (nsq[p][q] > 0.0f && nsq[q][r] > 0.0f)) ? c : nan;
            }
    // o0 -> o1: the first cone (o0 first) and the cosine at o1
    float c1[4][4];
#pragma unroll
    for (int o0 = 0; o0 < K; o0++) {
        const unsigned m0 = all & ~(1u << o0);
        const bool first = pos(all) && pos(m0) && in_unit(ccos(m0, all));
#pragma unroll
        for (int o1 = 0; o1 < K; o1++) {
            if (o1 == o0) continue;
            const unsigned after = m0 & ~(1u << o1);
            const float ce = ccos(after, m0);
            c1[o0][o1] = (first && nsq[o0][o1] > kPosEps2 && pos(after) && in_unit(ce)) ? ce : nan;
        }
    }
    float best = kInf;
    int best_rank = -1, rank = 0;
    if constexpr (K == 3) {
#pragma unroll
        for (int p0 = 0; p0 < 3; p0++)
#pragma unroll
            for (int p1 = 0; p1 < 3; p1++) {
                if (p1 == p0) continue;
                const float d = __fsub_rn(c1[p0][p1], cg[p0][p1][3 - p0 - p1]);
                const float c = __fmul_rn(d, d);           // 0 + d^2 = d^2 (d^2 is +0 or more)
                if (c < best) { best = c; best_rank = rank; }
                rank++;
            }
    } else {
        // o2 -> o3: the cosine at o2 with o3 last
        float c2[4][4];
#pragma unroll
        for (int o2 = 0; o2 < 4; o2++)
#pragma unroll
            for (int o3 = 0; o3 < 4; o3++) {
                if (o3 == o2) continue;
                const float ce = ccos(1u << o3, (1u << o2) | (1u << o3));
                c2[o2][o3] = (pos(1u << o3) && in_unit(ce)) ? ce : nan;
            }
#pragma unroll
        for (int p0 = 0; p0 < 4; p0++)
#pragma unroll
            for (int p1 = 0; p1 < 4; p1++) {
                if (p1 == p0) continue;
#pragma unroll
                for (int p2 = 0; p2 < 4; p2++) {
                    if (p2 == p0 || p2 == p1) continue;
                    const int p3 = 6 - p0 - p1 - p2;
                    const float d1 = __fsub_rn(c1[p0][p1], cg[p0][p1][p2]);
                    const float d2 = __fsub_rn(c2[p2][p3], cg[p1][p2][p3]);
                    const float c = __fadd_rn(__fmul_rn(d1, d1), __fmul_rn(d2, d2));
                    if (c < best) { best = c; best_rank = rank; }
                    rank++;
                }
            }
    }
    return best_rank;
}

template <int K>
static __device__ __noinline__ int order_rank_slow(const float (&x)[4], const float (&y)[4],
                                                   const float (&z)[4], const float (&e)[4],
                                                   const float (&nsq)[4][4]) {
    return order_rank<K, false>(x, y, z, e, nsq);
}

// Klein-Nishina angular weight P^2 (P + 1/P - sin^2 eta), binary32 sequence.
__device__ __forceinline__ float kn_weight(float P, float c) {
    float s2 = __fsub_rn(1.0f, __fmul_rn(c, c));
    float t = __fsub_rn(__fadd_rn(P, rcp_exact(P)), s2);
    return __fmul_rn(__fmul_rn(P, P), t);
}

template <int K>
__device__ __forceinline__ float pick(const float (&v)[4], int i) {
    float r = v[0];
#pragma unroll
    for (int s = 1; s < K; s++) r = (i == s) ? v[s] : r;
    return r;
}

// Ordering rule: returns the rank (or -1) and the first two slots.
template <int K>
__device__ __forceinline__ int choose_order(const float (&x)[4], const float (&y)[4],
                                            const float (&z)[4], const float (&e)[4],
                                            int &f0, int &f1) {
    if constexpr (K == 2) {
        // two-site validity is the first-site cone alone; its cosine is
        // 1 - m_e c^2 (1/E2 - 1/E0) in the binary32 sequence above, each
        // shared quantity computed once.  A single slot's energy 0 + e is
        // used as e: they differ only for e = -0, which fails e > 0 on
        // both sides
        const float e0 = __fadd_rn(__fadd_rn(0.0f, e[0]), e[1]);
        const bool apart = sqdist(x, y, z, 0, 1) > kPosEps2;
        const bool fast = e[0] >= 0x1p-40f && e[0] <= 0x1p40f && e[1] >= 0x1p-40f &&
                          e[1] <= 0x1p40f;
        float c0, c1, w0, w1;
        bool ok0, ok1;
        if (fast) {   // every argument and quotient normal: the unchecked corrections
            const float ie0 = rcp_core(e0);
            c0 = __fsub_rn(1.0f, __fmul_rn(kMeKeV, __fsub_rn(rcp_core(e[1]), ie0)));
            c1 = __fsub_rn(1.0f, __fmul_rn(kMeKeV, __fsub_rn(rcp_core(e[0]), ie0)));
            ok0 = in_unit(c0) && apart;
            ok1 = in_unit(c1) && apart;
            const float P0 = div_core(e[1], e0, ie0), P1 = div_core(e[0], e0, ie0);
            w0 = __fmul_rn(__fmul_rn(P0, P0), __fsub_rn(__fadd_rn(P0, rcp_core(P0)),
                                                        __fsub_rn(1.0f, __fmul_rn(c0, c0))));
            w1 = __fmul_rn(__fmul_rn(P1, P1), __fsub_rn(__fadd_rn(P1, rcp_core(P1)),
                                                        __fsub_rn(1.0f, __fmul_rn(c1, c1))));
        } else {
            const float ie0 = rcp_exact(e0);
            c0 = __fsub_rn(1.0f, __fmul_rn(kMeKeV, __fsub_rn(rcp_exact(e[1]), ie0)));
            c1 = __fsub_rn(1.0f, __fmul_rn(kMeKeV, __fsub_rn(rcp_exact(e[0]), ie0)));
            ok0 = (e0 > 0.0f) && (e[1] > 0.0f) && in_unit(c0) && apart;
            ok1 = (e0 > 0.0f) && (e[0] > 0.0f) && in_unit(c1) && apart;
            w0 = kn_weight(__fdiv_rn(e[1], e0), c0);
            w1 = kn_weight(__fdiv_rn(e[0], e0), c1);
        }
        if (ok1 && (!ok0 || w1 > w0)) { f0 = 1; f1 = 0; return 1; }
        if (ok0) { f0 = 0; f1 = 1; return 0; }
        return -1;
    } else {
        float nsq[4][4];
        bool fast = true;
#pragma unroll
        for (int s = 0; s < K; s++) fast = fast && e[s] >= 0x1p-100f && e[s] <= 0x1p98f;
#pragma unroll
        for (int p = 0; p < K; p++)
#pragma unroll
            for (int q = p + 1; q < K; q++) {
                const float v = sqdist(x, y, z, p, q);
                nsq[p][q] = nsq[q][p] = v;
                fast = fast && v <= 0x1p100f && (v >= 0x1p-100f || v == 0.0f);
            }
        const int rk = fast ? order_rank<K, true>(x, y, z, e, nsq)
                            : order_rank_slow<K>(x, y, z, e, nsq);
        // the rank's first two slots (lexicographic: (K-1)! orders per first slot)
        constexpr int per0 = K == 4 ? 6 : 2;
        const int p0 = rk / per0, i1 = (rk % per0) / (per0 / (K - 1));
        f0 = p0;
        f1 = i1 + (i1 >= p0 ? 1 : 0);
        return rk;
    }
}

constexpr int kRThreads = 256;
constexpr int kWin = 768;             // events per CTA window (4 CTAs per SM)
constexpr int kChunks = kWin / 32;    // 32-event chunks, one warp each

// Once a thread has read an event's sites into registers, the event's ring
// goes to the same window position of rows that only that event's sites
// occupied: ax, ay, az, eta in the slot-0 rows of x, y, z, e and deta in the
// slot-1 row of x.
struct ReconSmem {
    float v[4][4][kWin];      // [x|y|z|e][slot][window position]
    uint16_t order[kWin];     // sorted position -> window position
    uint8_t k[kWin];          // site count by window position
    alignas(16) uint8_t ov[kWin];
    alignas(16) uint8_t op[kWin];
    int grp[kWin / 32][4];    // events of each class in each 32-event group
    int off[kWin / 32][4];    // sorted position of each group's first event of a class
    int next;
    unsigned long long bar;
    int load_failed;
};

__device__ __forceinline__ float *ring_row(ReconSmem &S, int a) {
    return a < 4 ? S.v[a][0] : S.v[0][1];
}

__device__ __forceinline__ void no_ring(ReconSmem &S, int w) {
#pragma unroll
    for (int a = 0; a < 5; a++) ring_row(S, a)[w] = 0.0f;
    S.ov[w] = 0;
    S.op[w] = 255;
}

// Ring of the K-site event at window position w (FP32) from its chosen order.
template <int K>
__device__ __forceinline__ void ring_of_event(ReconSmem &S, int w, float sig_e, float sig_pos,
                                              float deta_min, float deta_max) {
    float x[4] = {}, y[4] = {}, z[4] = {}, e[4] = {};
#pragma unroll
    for (int sl = 0; sl < K; sl++) {
        x[sl] = S.v[0][sl][w];
        y[sl] = S.v[1][sl][w];
        z[sl] = S.v[2][sl][w];
        e[sl] = S.v[3][sl][w];
    }
    int f0 = 0, f1 = 1;
    const int rk = choose_order<K>(x, y, z, e, f0, f1);
    if (rk < 0) {
        no_ring(S, w);
        return;
    }
    // E1 first deposit, E2 the rest, E0 = E1 + E2
    float e1 = pick<K>(e, f0);
    float e2 = 0.0f, var2 = 0.0f;
#pragma unroll
    for (int s = 0; s < K; s++)
        if (s != f0) {
            e2 += e[s];
            float sd = sig_e * e[s];
            var2 = fmaf(sd, sd, var2);
        }
    float e0 = e1 + e2;
    // 1/E2 - 1/E0 = E1 / (E2 E0): no cancellation for small E1
    // u = 1 - cos(eta) in [0, 2] for a valid order; eta from u directly (the
    // chord form of acos, no rounding of 1 - u)
    const float ie0 = rcp_approx(e0), ie2 = rcp_approx(e2);
    float u = fminf(fmaxf(kMeKeV * e1 * (ie2 * ie0), 0.0f), 2.0f);
    float th = angle_from_half_chord2(u);
    float sin_eta = sqrt_approx(fmaxf(u * (2.0f - u), 0.0f));   // sqrt((1-c)(1+c))

    float dx = pick<K>(x, f0) - pick<K>(x, f1);
    float dy = pick<K>(y, f0) - pick<K>(y, f1);
    float dz = pick<K>(z, f0) - pick<K>(z, f1);
    float inv_len = rsqrt_approx(dx * dx + dy * dy + dz * dz);

    float s1 = sig_e * e1;
    // 1/E2^2 - 1/E0^2 = E1 (E0 + E2) / (E2^2 E0^2)
    const float ie02 = ie0 * ie0;
    float q = e1 * (e0 + e2) * ((ie2 * ie2) * ie02);
    float t1 = s1 * ie02;
    float var_cos = kMeKeV * kMeKeV * (t1 * t1 + var2 * q * q);
    float w_e = sqrt_approx(var_cos) * rcp_approx(fmaxf(sin_eta, 1e-3f));
    float w_g = 1.41421356237f * sig_pos * inv_len;
    float wd = sqrt_approx(w_e * w_e + w_g * w_g);

    ring_row(S, 0)[w] = dx * inv_len;
    ring_row(S, 1)[w] = dy * inv_len;
    ring_row(S, 2)[w] = dz * inv_len;
    ring_row(S, 3)[w] = th;
    ring_row(S, 4)[w] = fminf(fmaxf(wd, deta_min), deta_max);
    S.ov[w] = 1;
    S.op[w] = (uint8_t)rk;
}

// One CTA takes a window of 768 consecutive events.  Their sites are staged
// in shared memory in window order, by 16 bulk copies (TMA: x, y, z, e of
// each slot, 3 KB each) on one mbarrier when the window is whole and the
// arrays are 16-byte aligned, by plain loads otherwise.  The events are
// grouped by site count (4, 3, 2, other) through an index, and the warps
// take 32-event chunks from a shared queue, the costly 4-site chunks first,
// so that a warp runs one code path at a time and the warps finish
// together; each event's ring is written over its own staged sites, and the
// rings go back in the original order with 16-byte stores (coalesced
// scalar stores for a ragged window or unaligned ring arrays).  Slots past
// an event's site count are staged too and never read.  Four CTAs share an
// SM (64 registers, 54 KB of shared memory each), so that while one waits
// for its window the others compute.
__global__ void __launch_bounds__(kRThreads, 4)
k_rings_from_events(const uint8_t *__restrict__ n, const float *__restrict__ xs,
                    const float *__restrict__ ys, const float *__restrict__ zs,
                    const float *__restrict__ es, int64_t count, int64_t stride, int bulk_ok,
                    int vec_ok,
                    float sig_e, float sig_pos, float deta_min, float deta_max,
                    float *__restrict__ ax, float *__restrict__ ay,
                    float *__restrict__ az, float *__restrict__ eta,
                    float *__restrict__ deta, uint8_t *__restrict__ valid,
                    uint8_t *__restrict__ perm) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ReconSmem &S = *reinterpret_cast<ReconSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t base = blockIdx.x * (int64_t)kWin;
    const bool bulk = bulk_ok && base + kWin <= count;
    if (tid == 0) {
        S.next = 0;
        S.load_failed = 0;
        if (bulk) {
            mbar_init(&S.bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                             smem_u32(&S.bar)), "r"((unsigned)(16 * kWin * sizeof(float)))
                         : "memory");
            const float *src[4] = {xs, ys, zs, es};
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int sl = 0; sl < 4; sl++)
                    if (CC_IN_BOUNDS(CC_SITE_RECON_BULK, base + kWin - 1, stride))
                        bulk_copy(S.v[a][sl], src[a] + sl * stride + base,
                                  (unsigned)(kWin * sizeof(float)), &S.bar);
        }
    }
    __syncthreads();

    // group the window by site count: 32-event groups g = w / 32 count their
    // classes by ballot, one warp scans the counts into positions
    constexpr int kPer = kWin / kRThreads;
    int kk[kPer], cls[kPer], rk[kPer];
#pragma unroll
    for (int j = 0; j < kPer; j++) {
        const int w = tid + j * kRThreads;
        const int64_t i = base + w;
        kk[j] = (i < count && CC_IN_BOUNDS(CC_SITE_RECON_N, i, count)) ? n[i] : 0;
        cls[j] = kk[j] == 4 ? 0 : kk[j] == 3 ? 1 : kk[j] == 2 ? 2 : 3;
        S.k[w] = (uint8_t)kk[j];
        unsigned mine = 0;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const unsigned m = __ballot_sync(0xffffffffu, cls[j] == c);
            if (lane == 0) S.grp[w >> 5][c] = __popc(m);
            mine = cls[j] == c ? m : mine;
        }
        rk[j] = __popc(mine & ((1u << lane) - 1u));
        if (!bulk) {
#pragma unroll
            for (int sl = 0; sl < 4; sl++) {
                const int64_t off = sl * stride + i;
                const bool used = sl < kk[j] &&   // kk = 0 past the end
                                  CC_IN_BOUNDS(CC_SITE_RECON_SITES, off, 4 * stride);
                S.v[0][sl][w] = used ? __ldg(xs + off) : 0.0f;
                S.v[1][sl][w] = used ? __ldg(ys + off) : 0.0f;
                S.v[2][sl][w] = used ? __ldg(zs + off) : 0.0f;
                S.v[3][sl][w] = used ? __ldg(es + off) : 0.0f;
            }
        }
    }
    __syncthreads();
    if (tid < 32) {                       // kWin / 32 = 24 groups: one lane each
        constexpr int G = kWin / 32;
        int before = 0;                   // events of earlier classes
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int v = tid < G ? S.grp[tid][c] : 0;
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (tid >= o) x += y;
            }
            if (tid < G) S.off[tid][c] = before + x - v;
            before += __shfl_sync(0xffffffffu, x, 31);
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPer; j++) {
        const int w = tid + j * kRThreads;
        S.order[S.off[w >> 5][cls[j]] + rk[j]] = (uint16_t)w;
    }
    if (bulk && tid == 0 && !mbar_wait(&S.bar, 0)) S.load_failed = 1;
    __syncthreads();

    if (!S.load_failed) {
        for (;;) {
            int c = 0;
            if (lane == 0) c = atomicAdd(&S.next, 1);
            c = __shfl_sync(0xffffffffu, c, 0);
            if (c >= kChunks) break;
            const int w = S.order[c * 32 + lane];
            const int kk = S.k[w];
            if (kk == 4) ring_of_event<4>(S, w, sig_e, sig_pos, deta_min, deta_max);
            else if (kk == 3) ring_of_event<3>(S, w, sig_e, sig_pos, deta_min, deta_max);
            else if (kk == 2) ring_of_event<2>(S, w, sig_e, sig_pos, deta_min, deta_max);
            else no_ring(S, w);
        }
    } else {   // a bounded wait gave up: the window's rings are left invalid
        for (int w = tid; w < kWin; w += kRThreads) no_ring(S, w);
    }
    __syncthreads();
    if (vec_ok && base + kWin <= count) {     // four events per thread, 16-byte stores
        static_assert(kWin / 4 <= kRThreads, "one pass of four-event stores");
        if (tid < kWin / 4 && CC_IN_BOUNDS(CC_SITE_RECON_RING, base + 4 * tid + 3, count)) {
            const int w = 4 * tid;
            const int64_t i = base + w;
            float *dst[5] = {ax, ay, az, eta, deta};
#pragma unroll
            for (int a = 0; a < 5; a++)
                *reinterpret_cast<float4 *>(dst[a] + i) = *reinterpret_cast<const float4 *>(ring_row(S, a) + w);
            *reinterpret_cast<uint32_t *>(valid + i) = *reinterpret_cast<const uint32_t *>(&S.ov[w]);
            *reinterpret_cast<uint32_t *>(perm + i) = *reinterpret_cast<const uint32_t *>(&S.op[w]);
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < kPer; j++) {
        const int w = tid + j * kRThreads;
        const int64_t i = base + w;
        if (i < count && CC_IN_BOUNDS(CC_SITE_RECON_RING, i, count)) {
            ax[i] = ring_row(S, 0)[w];
            ay[i] = ring_row(S, 1)[w];
            az[i] = ring_row(S, 2)[w];
            eta[i] = ring_row(S, 3)[w];
            deta[i] = ring_row(S, 4)[w];
            valid[i] = S.ov[w];
            perm[i] = S.op[w];
        }
    }
}

}  // namespace

// Every float of [1, 4) (all mantissas, both exponent parities): the
// correctly rounded rcp_exact / sqrt_exact against the CUDA intrinsics; and
// div_core on every float of [1, 2) against 64 divisor mantissas, each
// quotient taken both ways, against __fdiv_rn.
__global__ void k_selftest_exact(unsigned long long *__restrict__ bad) {
    const uint32_t lo = 0x3F800000u, hi = 0x40800000u;
    unsigned long long b0 = 0, b1 = 0, b2 = 0;
    for (uint32_t u = lo + blockIdx.x * blockDim.x + threadIdx.x; u < hi;
         u += gridDim.x * blockDim.x) {
        const float x = __uint_as_float(u);
        b0 += __float_as_uint(rcp_exact(x)) != __float_as_uint(__frcp_rn(x));
        b1 += __float_as_uint(sqrt_exact(x)) != __float_as_uint(__fsqrt_rn(x));
        if (u < 0x40000000u) {
            const float yx = rcp_core(x);
            uint32_t h = u * 2654435761u;
            for (int j = 0; j < 64; j++) {
                h = h * 1664525u + 1013904223u;           // divisor mantissas (LCG)
                const float d = __uint_as_float(0x3F800000u | (j == 0 ? 0u : h >> 9));
                b2 += __float_as_uint(div_core(x, d, rcp_core(d))) != __float_as_uint(__fdiv_rn(x, d));
                b2 += __float_as_uint(div_core(d, x, yx)) != __float_as_uint(__fdiv_rn(d, x));
            }
        }
    }
    if (b0) atomicAdd(bad, b0);
    if (b1) atomicAdd(bad + 1, b1);
    if (b2) atomicAdd(bad + 2, b2);
}

cudaError_t launch_selftest_exact(uint64_t *bad, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bad, 0, 3 * sizeof(uint64_t), s);
    if (e != cudaSuccess) return e;
    k_selftest_exact<<<(unsigned)device_sm_count() * 8, 256, 0, s>>>(
        reinterpret_cast<unsigned long long *>(bad));
    return cudaGetLastError();
}

cudaError_t launch_rings_from_events(const cc_events &ev, const cc_rings &out,
                                     const cc_params &p, cudaStream_t s) {
    if (ev.count == 0) return cudaSuccess;
    const size_t smem = sizeof(ReconSmem);   // > 48 KB: opt in (per device, so every call)
    cudaError_t e = cudaFuncSetAttribute(k_rings_from_events,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (ev.count + kWin - 1) / kWin;
    TraceScope ts(CC_STAGE_RECON, s);
    auto a16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    const int bulk_ok = a16(ev.x) && a16(ev.y) && a16(ev.z) && a16(ev.e) && (ev.stride % 4) == 0;
    auto a4 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 3u) == 0; };
    const int vec_ok = a16(out.ax) && a16(out.ay) && a16(out.az) && a16(out.eta) &&
                       a16(out.deta) && a4(out.valid) && a4(out.perm);
    k_rings_from_events<<<(unsigned)blocks, kRThreads, smem, s>>>(
        ev.n, ev.x, ev.y, ev.z, ev.e, ev.count, ev.stride, bulk_ok, vec_ok, p.sigma_e_frac,
        p.sigma_pos_cm, p.deta_min, p.deta_max, out.ax, out.ay, out.az, out.eta,
        out.deta, out.valid, out.perm);
    return cudaGetLastError();
}

}  // namespace cc

// sweep.cu - the ring x direction likelihood sweep with fused block argmax,
// the split-ring reduction, and argmax / top-k seed selection.
//
// Sec. 3 of the paper: every (event, probe) contribution is independent and
// the contributions are summed per probe; here probes are sky directions and
// the contribution of ring i to direction j is exp(-r^2/2),
// r = (angle(a_i, c_j) - eta_i) / deta_i, optionally dropped for |r| > k_cut
// (the paper's angular selection).
//
// Per pair the angle is evaluated from the chord, not from acos(a . c): with
// both vectors pre-scaled by 1/sqrt(2), h = |a' - c'|^2 = 1 - cos(theta) to
// relative (not absolute) FP32 accuracy, so small angles keep their precision.
// For theta <= pi/2, theta = sqrt(h) Q(h); for theta > pi/2 the mirror
// identity theta = pi - sqrt(2 - h) Q(2 - h) applies, with
// Q(s) = acos(1 - s) / sqrt(s) a degree-6 polynomial fitted on [0, 1]
// (fit_acos.py 6: |error| <= 8.8e-8 rad with exact coefficients, 2.7e-7 rad
// evaluated in FP32 against 2.3e-7 for degree 7 - the FP32 evaluation, not
// the fit, sets the error, so the seventh FMA per pair is not spent).  Rings with
// eta > pi/2 are mirrored (a -> -a, eta -> pi - eta; the map is unchanged)
// so that the ill-conditioned end theta -> pi only meets far tails.  The
// Gaussian is exp2(-t^2) with t = theta k - eta k, k = sqrt(log2(e)/2)/deta,
// on the MUFU ex2 unit.
//
// Layout: rings are repacked once per call into 48-byte records (axis', k,
// -b, -b2, duplicated where they meet a direction pair) in the workspace and
// streamed through shared memory by cp.async.bulk (TMA bulk copy) into a
// 4-stage mbarrier ring; every CTA owns 256 x D directions held in registers
// (D per thread) and a contiguous range of ring tiles.  The directions are
// taken in the grid's compact order (order.cu: HEALPix NESTED), so each warp
// owns a small patch of sky, and per tile each warp sorts the rings by where
// its patch lies from them.  Rings whose every angle to the patch lies
// within 33.4 degrees of pi/2 take the angle as pi/2 + asin of the dot product
// (an odd polynomial: no square root, no fold, no select); of the rest, those
// wholly on one side of the patch (every angle below pi/2, or every one
// above) skip the fold and the mirror select, and the wide ones far enough
// from both the axis and its opposite take h from the dot product.
// Directions are processed in pairs with the packed FP32x2 FMA / add /
// multiply of sm_100+ (one instruction issue per two lanes of FP32 work),
// which leaves the FP32 pipe, not instruction issue, as the limit.  Per
// direction the FP32 sum
// of a 128-ring tile is added into a Kahan-compensated accumulator.  When the
// grid has too few direction blocks to fill 152 SMs the rings are split over
// CTAs and the partial maps are summed in a fixed order (deterministic).
#include <float.h>

#include "cc_math.cuh"
#include "cc_pipe.cuh"

namespace cc {
namespace {

constexpr int kThreads = 256;
constexpr int kTile = 128;    // rings per shared-memory tile (4 KB)
constexpr int kStages = 4;
constexpr float kInvSqrt2 = 0.70710678118654752f;
constexpr float kGaussK = 0.84932180028801907f;   // sqrt(log2(e) / 2)
constexpr float kNullB = 1.0e4f;                  // ex2(-(1e4)^2) == 0
// The dot form of h (below) is used for rings at least this wide (k = kGaussK
// / deta <= kDotMaxK: deta >= 13.9 deg) whose every pair lies between
// kDotAngle and pi - kDotAngle from the axis.
constexpr float kDotAngle = 0.52359878f;          // pi / 6
constexpr float kDotMaxK = 3.5f;
// The equatorial form (below) is used for rings of any width whose every
// pair lies within kEquAngle of pi/2 from the axis (|cos(theta)| <= 0.55).
constexpr float kEquAngle = 0.58236424f;          // asin(0.55), 33.37 deg
// With the short polynomials the one-sided forms are used when every pair
// lies within kSideAngle of the axis or of its opposite (s <= 0.8: the
// degree-5 polynomial's range), or within kSide2Angle (s <= 0.55, degree 4).
constexpr float kSideAngle = 1.36943841f;         // acos(0.2), 78.46 deg
constexpr float kSide2Angle = 1.10403099f;        // acos(0.45), 63.26 deg

// Coefficients of acos_q (cc_math.cuh) as FP32x2 pairs.
__device__ __forceinline__ float2 pair(float v) { return make_float2(v, v); }

// ---------------------------------------------------------------------------
// ring repacking
// ---------------------------------------------------------------------------
// A ring enters the sweep when it is valid and its numbers are usable.
__device__ __forceinline__ bool ring_kept(const float *__restrict__ ax,
                                          const float *__restrict__ ay,
                                          const float *__restrict__ az,
                                          const float *__restrict__ eta,
                                          const float *__restrict__ deta,
                                          const uint8_t *__restrict__ valid, int64_t i,
                                          int64_t R) {
    if (i >= R || (valid != nullptr && !valid[i])) return false;
    float de = deta[i];
    return isfinite(ax[i]) && isfinite(ay[i]) && isfinite(az[i]) && isfinite(eta[i]) &&
           isfinite(de) && de > 0.0f;
}

__device__ __forceinline__ RingRec make_rec(float a0, float a1, float a2, float e, float de) {
    float k = kGaussK / de;
    float b = e * k, b2 = (kPiF - e) * k, ne = (0.5f * kPiF - e) * k;
    if (e > 0.5f * kPiF) {      // mirror: same ring, eta' <= pi/2
        a0 = -a0; a1 = -a1; a2 = -a2;
        float t = b; b = b2; b2 = t;
        ne = -ne;
    }
    float s0 = a0 * kInvSqrt2, s1 = a1 * kInvSqrt2, s2 = a2 * kInvSqrt2;
    return RingRec{s0, s0, s1, s1, s2, s2, k, k, -b, -b2, ne, ne};
}

// Kept rings are compacted, in index order, to the front of the record
// array, so the sweep's cost follows the rings that count (a filter that
// drops rings shortens the sweep).  Three passes: per-block counts, one scan
// of the counts, and the scatter.
__global__ void __launch_bounds__(256)
k_pack_count(const float *__restrict__ ax, const float *__restrict__ ay,
             const float *__restrict__ az, const float *__restrict__ eta,
             const float *__restrict__ deta, const uint8_t *__restrict__ valid, int64_t R,
             int32_t *__restrict__ blockcnt) {
    const int64_t base = blockIdx.x * (int64_t)kPackChunk;
    int n = 0;
    for (int r = 0; r < kPackChunk / 256; r++)
        n += __syncthreads_count(ring_kept(ax, ay, az, eta, deta, valid,
                                           base + r * 256 + threadIdx.x, R));
    if (threadIdx.x == 0) blockcnt[blockIdx.x] = n;
}

__global__ void __launch_bounds__(1024)
k_pack_scan(int32_t *__restrict__ blockcnt, int64_t nblk, int64_t *__restrict__ nkept) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t c = 0; c < nblk; c += 1024) {
        const int64_t i = c + threadIdx.x;
        int64_t v = i < nblk ? blockcnt[i] : 0, x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (l >= o) x += y;
        }
        if (l == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int64_t s = wsum[l], t = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (l >= o) t += y;
            }
            wsum[l] = t - s;                  // exclusive prefix of warp totals
        }
        __syncthreads();
        const int64_t excl = carry + wsum[w] + x - v;
        if (i < nblk) blockcnt[i] = (int32_t)excl;   // offsets fit: R < 2^31
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *nkept = carry;
}

__global__ void __launch_bounds__(256)
k_pack_scatter(const float *__restrict__ ax, const float *__restrict__ ay,
               const float *__restrict__ az, const float *__restrict__ eta,
               const float *__restrict__ deta, const uint8_t *__restrict__ valid, int64_t R,
               const int32_t *__restrict__ offs, const int64_t *__restrict__ nkept,
               RingRec *__restrict__ rec) {
    __shared__ int wcnt[8];
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = blockIdx.x * (int64_t)kPackChunk;
    int64_t pos = offs[blockIdx.x];
    for (int r = 0; r < kPackChunk / 256; r++) {
        const int64_t i = base + r * 256 + threadIdx.x;
        const bool keep = ring_kept(ax, ay, az, eta, deta, valid, i, R);
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (l == 0) wcnt[w] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            before += k < w ? wcnt[k] : 0;
            total += wcnt[k];
        }
        const int64_t at = pos + before + __popc(m & ((1u << l) - 1u));
        if (keep && CC_IN_BOUNDS(CC_SITE_PACK_REC, at, (R + kTile - 1) / kTile * kTile))
            rec[at] = make_rec(ax[i], ay[i], az[i], eta[i], deta[i]);
        pos += total;
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x < kTile) {   // null records up to the tile end
        const int64_t n = *nkept;
        const int64_t end = (n + kTile - 1) / kTile * kTile;
        if (n + threadIdx.x < end &&
            CC_IN_BOUNDS(CC_SITE_PACK_REC, n + threadIdx.x, (R + kTile - 1) / kTile * kTile))
            rec[n + threadIdx.x] =
                RingRec{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -kNullB, -kNullB, -kNullB, -kNullB};
    }
}

// ---------------------------------------------------------------------------
// the sweep
// ---------------------------------------------------------------------------
struct SweepSmem {
    RingRec tile[kStages][kTile];
    unsigned long long full[kStages];
    unsigned char lst[kThreads / 32][kTile];   // per warp: the tile's rings by side
    int abort_flag;
};

// The pair term for one ring and DP direction pairs (see the file header).
// SIDE 1: every pair is known to lie on the ring's near side (h <= 1), SIDE 2:
// on its far side; the fold and the select then have one outcome, and the
// result is the same as the general form's (SIDE 0) bit for bit.  SHORT = 1:
// every pair of SIDE 1 - 4 lies within kSideAngle of the axis or of its
// opposite (the folded s <= 0.8), and Q is the degree-5 fit on [0, 0.8]
// (fit_acos.py: 9.3e-8 rad, 2.6e-7 evaluated in FP32; as accurate as degree 6
// on [0, 1]: 8.8e-8 and 2.7e-7), one FMA fewer; SHORT = 2: within
// kSide2Angle (s <= 0.55), the degree-4 fit on [0, 0.55] (7.9e-8 and 2.4e-7),
// two FMAs fewer.  SIDE 3 / 4:
// near / far side, and every pair between kDotAngle and pi - kDotAngle from
// the axis: h from the dot product, h = 2 t with t = 1/2 + a'.(-c') (three
// FMAs instead of the chord's six operations).  Its absolute error (at most
// ~1.5e-7 in t) is harmless away from theta = 0 and pi: there it adds at
// most 6e-7 rad to the angle (the polynomial's own 2.7e-7 stays), which for
// rings of k <= kDotMaxK moves a term above the map rule's floor by at most
// ~1.3e-5 of its value with every rounding at its bound and the same sign,
// and by ~1e-6 typically; summed over many rings it averages out.
// SIDE 5 (equatorial): every pair within kEquAngle of pi/2 from the axis,
// any width: theta = pi/2 + asin(2 s), s = a'.(-c') = -cos(theta) / 2, with
// asin(2 s) = s P(s^2) (fit_asin.py 4 0.55: degree 4 in s^2, 1.4e-7 rad
// evaluated in FP32), so u = (theta - eta') k = s P(s^2) k + ne: twelve FP32
// operations and one MUFU per pair, no square root, no fold, no select.  The
// absolute error of s (~1e-7, as t above) moves the angle by at most 2.4e-7
// rad at |cos(theta)| <= 0.55, no more than the chord form's own error there
// (its h is ~1 with the same absolute rounding, and the acos polynomial adds
// 2.7e-7).
template <int DP, bool KCUT, int SIDE = 0, int SHORT = 0>
__device__ __forceinline__ void ring_pairs(const RingRec &R, const float2 (&ncx)[DP],
                                           const float2 (&ncy)[DP], const float2 (&ncz)[DP],
                                           float2 (&acc)[DP], float kc2) {
    const float4 P0 = *reinterpret_cast<const float4 *>(&R.ax);
    const float4 P1 = *reinterpret_cast<const float4 *>(&R.az);
    const float2 ax2 = make_float2(P0.x, P0.y), ay2 = make_float2(P0.z, P0.w);
    const float2 az2 = make_float2(P1.x, P1.y), k2 = make_float2(P1.z, P1.w);
    if constexpr (SIDE == 5) {
        const float2 ne2 = *reinterpret_cast<const float2 *>(&R.ne);
#pragma unroll
        for (int q = 0; q < DP; q++) {
            float2 sd = __fmul2_rn(az2, ncz[q]);      // s = -cos(theta) / 2
            sd = __ffma2_rn(ay2, ncy[q], sd);
            sd = __ffma2_rn(ax2, ncx[q], sd);
            const float2 w = __fmul2_rn(sd, sd);
            float2 p = pair(3.12643623e+01f);         // P(w), degree 4, FP32x2
            p = __ffma2_rn(p, w, pair(4.32808828e+00f));
            p = __ffma2_rn(p, w, pair(2.44986677e+00f));
            p = __ffma2_rn(p, w, pair(1.33261955e+00f));
            p = __ffma2_rn(p, w, pair(2.00000286e+00f));
            const float2 v = __fmul2_rn(sd, p);       // theta - pi/2
            const float2 u = __ffma2_rn(v, k2, ne2);
            const float2 u2 = __fmul2_rn(u, u);
            float2 e = make_float2(ex2_approx(-u2.x), ex2_approx(-u2.y));
            if (KCUT) {
                e.x = u2.x > kc2 ? 0.0f : e.x;
                e.y = u2.y > kc2 ? 0.0f : e.y;
            }
            acc[q] = __fadd2_rn(acc[q], e);
        }
    } else {
        const float2 P2 = *reinterpret_cast<const float2 *>(&R.nb);
        const float2 m1 = pair(-1.0f), two2 = pair(2.0f);
#pragma unroll
        for (int q = 0; q < DP; q++) {
            float2 h = pair(0.0f), sv;
            if (SIDE == 3 || SIDE == 4) {             // dot form: t = 1/2 + a'.nc = h / 2
                float2 t = __ffma2_rn(az2, ncz[q], pair(0.5f));
                t = __ffma2_rn(ay2, ncy[q], t);
                t = __ffma2_rn(ax2, ncx[q], t);
                sv = SIDE == 3 ? __fmul2_rn(t, two2) : __ffma2_rn(t, pair(-2.0f), two2);
            } else {
                float2 dx = __fadd2_rn(ax2, ncx[q]);
                float2 dy = __fadd2_rn(ay2, ncy[q]);
                float2 dz = __fadd2_rn(az2, ncz[q]);
                h = __fmul2_rn(dx, dx);
                h = __ffma2_rn(dy, dy, h);
                h = __ffma2_rn(dz, dz, h);                // 1 - cos(theta)
                if (SIDE == 1) {
                    sv = h;
                } else {
                    float2 g = __ffma2_rn(h, m1, two2);     // 2 - h
                    sv = SIDE == 2 ? make_float2(fabsf(g.x), fabsf(g.y))
                                   : make_float2(fminf(h.x, fabsf(g.x)), fminf(h.y, fabsf(g.y)));
                }
            }
            float2 p;
            if (SHORT == 0) {                                // Q(s) on [0, 1], degree 6
                p = pair(2.61164433e-03f);
                p = __ffma2_rn(p, sv, pair(-3.66667798e-03f));
                p = __ffma2_rn(p, sv, pair(6.92143012e-03f));
                p = __ffma2_rn(p, sv, pair(5.94551489e-03f));
                p = __ffma2_rn(p, sv, pair(2.69628558e-02f));
                p = __ffma2_rn(p, sv, pair(1.17806636e-01f));
                p = __ffma2_rn(p, sv, pair(1.41421485e+00f));
            } else if (SHORT == 1) {                         // Q(s) on [0, 0.8], degree 5
                p = pair(3.31251509e-03f);
                p = __ffma2_rn(p, sv, pair(-2.59509514e-04f));
                p = __ffma2_rn(p, sv, pair(9.49506927e-03f));
                p = __ffma2_rn(p, sv, pair(2.61093955e-02f));
                p = __ffma2_rn(p, sv, pair(1.17894620e-01f));
                p = __ffma2_rn(p, sv, pair(1.41421223e+00f));
            } else {                                         // Q(s) on [0, 0.55], degree 4
                p = pair(5.02272556e-03f);
                p = __ffma2_rn(p, sv, pair(6.41390355e-03f));
                p = __ffma2_rn(p, sv, pair(2.69000251e-02f));
                p = __ffma2_rn(p, sv, pair(1.17811434e-01f));
                p = __ffma2_rn(p, sv, pair(1.41421473e+00f));
            }
            float2 rt = make_float2(sqrt_approx(sv.x), sqrt_approx(sv.y));
            float2 th = __fmul2_rn(rt, p);
            float2 nbs = (SIDE == 1 || SIDE == 3)   ? make_float2(P2.x, P2.x)
                         : (SIDE == 2 || SIDE == 4) ? make_float2(P2.y, P2.y)
                                     : make_float2(h.x <= 1.0f ? P2.x : P2.y, h.y <= 1.0f ? P2.x : P2.y);
            float2 u = __ffma2_rn(th, k2, nbs);
            float2 u2 = __fmul2_rn(u, u);
            float2 e = make_float2(ex2_approx(-u2.x), ex2_approx(-u2.y));
            if (KCUT) {
                e.x = u2.x > kc2 ? 0.0f : e.x;
                e.y = u2.y > kc2 ? 0.0f : e.y;
            }
            acc[q] = __fadd2_rn(acc[q], e);
        }
    }
}

// Angular selection of a ring against a warp's cap (centre c' = c/sqrt(2),
// radius rho): false when every direction within rho of c lies more than
// k_cut widths from the ring, |theta - eta| > k_cut deta, so that all its
// terms there are 0.  |alpha - eta| k comes from the pair formula at the
// centre; by the triangle inequality no direction of the cap is closer to
// the ring than |alpha - eta| - rho.  rho carries a margin for the FP32
// error of both angles, so a skipped ring contributes exactly 0.
__device__ __forceinline__ bool ring_reaches(const RingRec &R, float cx, float cy, float cz,
                                             float rho, float kc) {
    const float dx = R.ax - cx, dy = R.ay - cy, dz = R.az - cz;
    const float h = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    const float sv = fminf(h, fabsf(2.0f - h));
    const float th = sqrt_approx(sv) * acos_q(sv);
    const float u = fmaf(th, R.k, h <= 1.0f ? R.nb : R.nb2);
    const float lim = fmaf(rho, R.k, kc);
    return fabsf(u) <= lim;
}

// The rings of a warp's list lst[b, e) of tile T, four at a time (eight made
// the list bodies too large for the instruction cache).
template <int DP, bool KCUT, int SIDE, int SHORT = 0>
__device__ __forceinline__ void side_run(const RingRec *T, const unsigned char *lst, int b, int e,
                                         const float2 (&ncx)[DP], const float2 (&ncy)[DP],
                                         const float2 (&ncz)[DP], float2 (&acc)[DP], float kc2) {
    int i = b;
    for (; i + 4 <= e; i += 4) {
#pragma unroll
        for (int k = 0; k < 4; k++)
            ring_pairs<DP, KCUT, SIDE, SHORT>(T[lst[i + k]], ncx, ncy, ncz, acc, kc2);
    }
    for (; i < e; i++) ring_pairs<DP, KCUT, SIDE, SHORT>(T[lst[i]], ncx, ncy, ncz, acc, kc2);
}

// One work unit of the sweep: the 256 x D directions of direction block db
// (warp w owns the 32 D consecutive ones from db 256 D + 32 D w; lane l the
// directions l, l + 32, ...; direction k of the sweep is perm[k] of the grid,
// or k without perm) against the ring tiles split, split + nsplit,
// split + 2 nsplit, ... of the *nkept packed rings.  Each warp sorts a
// tile's rings by side against its cap of directions: a ring whose axis is
// within L - rho - 1e-3 of the cap centre has every pair within L of it, one
// whose axis is that close to the opposite of the centre every pair within L
// of its opposite, and those rings skip the fold and the select (L = pi/2,
// or kSideAngle with the short polynomial when the cap is narrow enough for
// the equatorial form to take every ring between the two); a wide one whose
// axis is also more than kDotAngle + rho
// from the centre and from its opposite takes the dot form (ring_pairs).
// Before all of these, a ring whose axis lies within kEquAngle - rho - 1e-3
// of pi/2 from the centre takes the equatorial form.
// With the angular selection on, each warp skips, tile by
// tile, the rings that cannot reach its directions instead.  Writes the
// unit's partial (or full) map row (in grid order) and, when bb_slot is set,
// its block best.  Returns false when a bounded wait gave up (status set to
// CC_ETIMEOUT).
template <int D, bool KCUT, int SHORT>
__device__ __forceinline__ bool sweep_unit(SweepSmem &S, const RingRec *__restrict__ rec,
                                           const int64_t *__restrict__ nkept, int64_t nsplit,
                                           int64_t db, int64_t split,
                                           const float *__restrict__ cx,
                                           const float *__restrict__ cy,
                                           const float *__restrict__ cz,
                                           const int32_t *__restrict__ perm, int64_t M, float kc2,
                                           float *__restrict__ out, BlockBest *bb_slot,
                                           int32_t *__restrict__ status) {
    static_assert(D % 2 == 0, "directions are processed in FP32x2 pairs");
    constexpr int DP = D / 2;
    auto &tile = S.tile;
    auto &full = S.full;
    int &abort_flag = S.abort_flag;

    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t j0 = db * (int64_t)(kThreads * D) + (int64_t)(tid >> 5) * (32 * D) + lane;

    // direction d of this thread: j0 + 32 d; pair q holds d = 2q, 2q+1
    float2 ncx[DP], ncy[DP], ncz[DP], acc[DP], sum[DP], comp[DP];
#pragma unroll
    for (int q = 0; q < DP; q++) {
        int64_t ja = j0 + (int64_t)(64 * q), jb = ja + 32;
        ja = ja < M ? ja : M - 1;
        jb = jb < M ? jb : M - 1;
        if (perm != nullptr) {
            ja = __ldg(perm + ja);
            jb = __ldg(perm + jb);
        }
        ncx[q] = make_float2(-__ldg(cx + ja) * kInvSqrt2, -__ldg(cx + jb) * kInvSqrt2);
        ncy[q] = make_float2(-__ldg(cy + ja) * kInvSqrt2, -__ldg(cy + jb) * kInvSqrt2);
        ncz[q] = make_float2(-__ldg(cz + ja) * kInvSqrt2, -__ldg(cz + jb) * kInvSqrt2);
        acc[q] = sum[q] = comp[q] = make_float2(0.0f, 0.0f);
    }

    // the warp's cap: centre (scaled by 1/sqrt 2) and angular radius
    float capx = 0.f, capy = 0.f, capz = 0.f, rho = 0.f, kc = 0.f;
    {
        float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
        for (int q = 0; q < DP; q++) {
            sx -= ncx[q].x + ncx[q].y;
            sy -= ncy[q].x + ncy[q].y;
            sz -= ncz[q].x + ncz[q].y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
            sz += __shfl_xor_sync(0xffffffffu, sz, o);
        }
        const float inv = kInvSqrt2 * rsqrtf(fmaxf(fmaf(sz, sz, fmaf(sy, sy, sx * sx)), 1e-30f));
        capx = sx * inv;
        capy = sy * inv;
        capz = sz * inv;
        float h = 0.f;                                  // largest |c' - cap'|^2 = chord^2 / 2
#pragma unroll
        for (int q = 0; q < DP; q++) {
            const float ax = ncx[q].x + capx, ay = ncy[q].x + capy, az = ncz[q].x + capz;
            const float bx = ncx[q].y + capx, by = ncy[q].y + capy, bz = ncz[q].y + capz;
            h = fmaxf(h, fmaf(az, az, fmaf(ay, ay, ax * ax)));
            h = fmaxf(h, fmaf(bz, bz, fmaf(by, by, bx * bx)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) h = fmaxf(h, __shfl_xor_sync(0xffffffffu, h, o));
        // rho = 2 asin(chord / 2), chord = sqrt(2 h); plus 2e-5 rad for the
        // rounding of the centre, the chords and both angles
        rho = 2.0f * asinf(fminf(sqrtf(0.5f * h), 1.0f)) + 2.0e-5f;
        kc = sqrtf(kc2);
    }
    // side test: cos(angle(axis, centre)) = 2 a'.cap' against +-cos(L - rho -
    // 1e-3), L = kSideAngle / kSide2Angle with the short polynomials, else
    // pi/2 (no side decided when the cap reaches L)
    const float lside = SHORT == 2 ? kSide2Angle : kSideAngle;
    const float slim = SHORT ? (rho + 1.0e-3f < lside ? cosf(lside - rho - 1.0e-3f) : 2.0f)
                             : (rho + 1.0e-3f < 1.5707f ? sinf(rho + 1.0e-3f) : 2.0f);
    // ... and the dot form when cos(angle) also lies within +-cos(kDotAngle + rho)
    const float cdot = kDotAngle + rho < 1.5707f ? cosf(kDotAngle + rho) : -2.0f;
    // the equatorial form when |cos(angle)| <= sin(kEquAngle - rho - 1e-3)
    const float elim = rho + 1.0e-3f < kEquAngle ? sinf(kEquAngle - rho - 1.0e-3f) : -1.0f;
    const int w = tid >> 5;

    const int64_t ntk = (*nkept + kTile - 1) / kTile;
    const int64_t tiles = split < ntk ? (ntk - split + nsplit - 1) / nsplit : 0;
    const RingRec *src = rec + split * kTile;
    const int64_t stride = nsplit * kTile;
    if (tid == 0) {
        for (int s = 0; s < kStages; s++) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < kStages && s < tiles; s++)
            if (CC_IN_BOUNDS(CC_SITE_SWEEP_TILE, split + s * nsplit, ntk))
                tma_bulk_load(tile[s], src + (int64_t)s * stride, kTile * sizeof(RingRec),
                              &full[s]);
    }

    for (int64_t t = 0; t < tiles; t++) {
        const int stage = (int)(t % kStages);
        const unsigned parity = (unsigned)((t / kStages) & 1);
        if (!mbar_wait(&full[stage], parity)) {
            abort_flag = 1;
        } else {
            const RingRec *T = tile[stage];
            if constexpr (KCUT) {
                // with the angular selection: the rings that can reach the
                // warp's cap, by class as below
                unsigned m5s[kTile / 32], m1s[kTile / 32], m3s[kTile / 32], m4s[kTile / 32],
                    m2s[kTile / 32], mms[kTile / 32];
                int cnt[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
                for (int g = 0; g < kTile / 32; g++) {
                    const RingRec &R = T[32 * g + lane];
                    const bool reach = ring_reaches(R, capx, capy, capz, rho, kc);
                    const float c2 = 2.0f * fmaf(R.az, capz, fmaf(R.ay, capy, R.ax * capx));
                    const bool eq = reach && fabsf(c2) <= elim;
                    const bool wide = reach && R.k <= kDotMaxK && !eq;
                    const bool dn = wide && c2 >= slim && c2 <= cdot;
                    const bool df = wide && c2 <= -slim && c2 >= -cdot;
                    const bool n1 = reach && c2 >= slim && !dn && !eq;
                    const bool n2 = reach && c2 <= -slim && !df && !eq;
                    m5s[g] = __ballot_sync(0xffffffffu, eq);
                    m1s[g] = __ballot_sync(0xffffffffu, n1);
                    m3s[g] = __ballot_sync(0xffffffffu, dn);
                    m4s[g] = __ballot_sync(0xffffffffu, df);
                    m2s[g] = __ballot_sync(0xffffffffu, n2);
                    mms[g] = __ballot_sync(0xffffffffu, reach && !(eq || dn || df || n1 || n2));
                    cnt[0] += __popc(m5s[g]);
                    cnt[1] += __popc(m1s[g]);
                    cnt[2] += __popc(m3s[g]);
                    cnt[3] += __popc(m4s[g]);
                    cnt[4] += __popc(m2s[g]);
                    cnt[5] += __popc(mms[g]);
                }
                const unsigned lt = (1u << lane) - 1u;
                int b5 = 0, b1 = cnt[0], b3 = b1 + cnt[1], b4 = b3 + cnt[2], b2 = b4 + cnt[3],
                    bm = b2 + cnt[4];
                const int e5 = b1, e1 = b3, e3 = b4, e4 = b2, e2 = bm, em = bm + cnt[5];
#pragma unroll
                for (int g = 0; g < kTile / 32; g++) {
                    const unsigned bit = 1u << lane;
                    const int at = (m5s[g] & bit) ? b5 + __popc(m5s[g] & lt)
                                 : (m1s[g] & bit) ? b1 + __popc(m1s[g] & lt)
                                 : (m3s[g] & bit) ? b3 + __popc(m3s[g] & lt)
                                 : (m4s[g] & bit) ? b4 + __popc(m4s[g] & lt)
                                 : (m2s[g] & bit) ? b2 + __popc(m2s[g] & lt)
                                 : (mms[g] & bit) ? bm + __popc(mms[g] & lt) : -1;
                    if (at >= 0) S.lst[w][at] = (unsigned char)(32 * g + lane);
                    b5 += __popc(m5s[g]);
                    b1 += __popc(m1s[g]);
                    b3 += __popc(m3s[g]);
                    b4 += __popc(m4s[g]);
                    b2 += __popc(m2s[g]);
                    bm += __popc(mms[g]);
                }
                __syncwarp();
                const unsigned char *L = S.lst[w];
                side_run<DP, KCUT, 5>(T, L, 0, e5, ncx, ncy, ncz, acc, kc2);
                side_run<DP, KCUT, 1, SHORT>(T, L, e5, e1, ncx, ncy, ncz, acc, kc2);
                side_run<DP, KCUT, 3, SHORT>(T, L, e1, e3, ncx, ncy, ncz, acc, kc2);
                side_run<DP, KCUT, 4, SHORT>(T, L, e3, e4, ncx, ncy, ncz, acc, kc2);
                side_run<DP, KCUT, 2, SHORT>(T, L, e4, e2, ncx, ncy, ncz, acc, kc2);
                side_run<DP, KCUT, 0>(T, L, e2, em, ncx, ncy, ncz, acc, kc2);
            } else {
                // the tile's rings by class: equatorial, near side (chord
                // form, dot form), far side (dot, chord), then the rest, each
                // in tile order
                unsigned m5s[kTile / 32], m1s[kTile / 32], m3s[kTile / 32], m4s[kTile / 32],
                    m2s[kTile / 32];
                int cnt[5] = {0, 0, 0, 0, 0};
#pragma unroll
                for (int g = 0; g < kTile / 32; g++) {
                    const RingRec &R = T[32 * g + lane];
                    const float c2 = 2.0f * fmaf(R.az, capz, fmaf(R.ay, capy, R.ax * capx));
                    const bool eq = fabsf(c2) <= elim;
                    const bool wide = R.k <= kDotMaxK && !eq;
                    const bool dn = wide && c2 >= slim && c2 <= cdot;
                    const bool df = wide && c2 <= -slim && c2 >= -cdot;
                    m5s[g] = __ballot_sync(0xffffffffu, eq);
                    m1s[g] = __ballot_sync(0xffffffffu, c2 >= slim && !dn && !eq);
                    m3s[g] = __ballot_sync(0xffffffffu, dn);
                    m4s[g] = __ballot_sync(0xffffffffu, df);
                    m2s[g] = __ballot_sync(0xffffffffu, c2 <= -slim && !df && !eq);
                    cnt[0] += __popc(m5s[g]);
                    cnt[1] += __popc(m1s[g]);
                    cnt[2] += __popc(m3s[g]);
                    cnt[3] += __popc(m4s[g]);
                    cnt[4] += __popc(m2s[g]);
                }
                const unsigned lt = (1u << lane) - 1u;
                int b5 = 0, b1 = cnt[0], b3 = b1 + cnt[1], b4 = b3 + cnt[2], b2 = b4 + cnt[3],
                    bm = b2 + cnt[4];
                const int e5 = b1, e1 = b3, e3 = b4, e4 = b2, e2 = bm;
#pragma unroll
                for (int g = 0; g < kTile / 32; g++) {
                    const unsigned mm = ~(m5s[g] | m1s[g] | m3s[g] | m4s[g] | m2s[g]);
                    const unsigned bit = 1u << lane;
                    const int at = (m5s[g] & bit) ? b5 + __popc(m5s[g] & lt)
                                 : (m1s[g] & bit) ? b1 + __popc(m1s[g] & lt)
                                 : (m3s[g] & bit) ? b3 + __popc(m3s[g] & lt)
                                 : (m4s[g] & bit) ? b4 + __popc(m4s[g] & lt)
                                 : (m2s[g] & bit) ? b2 + __popc(m2s[g] & lt)
                                                  : bm + __popc(mm & lt);
                    S.lst[w][at] = (unsigned char)(32 * g + lane);
                    b5 += __popc(m5s[g]);
                    b1 += __popc(m1s[g]);
                    b3 += __popc(m3s[g]);
                    b4 += __popc(m4s[g]);
                    b2 += __popc(m2s[g]);
                    bm += __popc(mm);
                }
                __syncwarp();
                const unsigned char *L = S.lst[w];
                side_run<DP, false, 5>(T, L, 0, e5, ncx, ncy, ncz, acc, 0.0f);
                side_run<DP, false, 1, SHORT>(T, L, e5, e1, ncx, ncy, ncz, acc, 0.0f);
                side_run<DP, false, 3, SHORT>(T, L, e1, e3, ncx, ncy, ncz, acc, 0.0f);
                side_run<DP, false, 4, SHORT>(T, L, e3, e4, ncx, ncy, ncz, acc, 0.0f);
                side_run<DP, false, 2, SHORT>(T, L, e4, e2, ncx, ncy, ncz, acc, 0.0f);
                side_run<DP, false, 0>(T, L, e2, kTile, ncx, ncy, ncz, acc, 0.0f);
                __syncwarp();
            }
        }
        __syncthreads();
        if (abort_flag) break;
        if (tid == 0 && t + kStages < tiles &&
            CC_IN_BOUNDS(CC_SITE_SWEEP_TILE, split + (t + kStages) * nsplit, ntk))
            tma_bulk_load(tile[stage], src + (t + kStages) * stride, kTile * sizeof(RingRec),
                          &full[stage]);
#pragma unroll
        for (int q = 0; q < DP; q++) {   // Kahan-compensated tile sums
            float2 y = make_float2(acc[q].x - comp[q].x, acc[q].y - comp[q].y);
            float2 tt = make_float2(sum[q].x + y.x, sum[q].y + y.y);
            comp[q] = make_float2((tt.x - sum[q].x) - y.x, (tt.y - sum[q].y) - y.y);
            sum[q] = tt;
            acc[q] = make_float2(0.0f, 0.0f);
        }
    }
    if (abort_flag) {
        if (tid == 0) atomicExch(status, (int32_t)CC_ETIMEOUT);
        return false;
    }

    float bv = -__builtin_huge_valf();
    int bj = INT32_MAX;
#pragma unroll
    for (int q = 0; q < DP; q++) {
        const int64_t ka = j0 + (int64_t)(64 * q), kb = ka + 32;
        const float va = sum[q].x - comp[q].x, vb = sum[q].y - comp[q].y;
        if (ka < M) {
            const int64_t ja = perm != nullptr ? (int64_t)__ldg(perm + ka) : ka;
            if (CC_IN_BOUNDS(CC_SITE_SWEEP_OUT, split * M + ja, nsplit * M)) {
                out[split * M + ja] = va;
                better(bv, bj, va, (int)ja);
            }
        }
        if (kb < M) {
            const int64_t jb = perm != nullptr ? (int64_t)__ldg(perm + kb) : kb;
            if (CC_IN_BOUNDS(CC_SITE_SWEEP_OUT, split * M + jb, nsplit * M)) {
                out[split * M + jb] = vb;
                better(bv, bj, vb, (int)jb);
            }
        }
    }
    if (bb_slot != nullptr) {
        block_best(bv, bj);
        if (tid == 0) *bb_slot = BlockBest{bv, bj};
    }
    __syncthreads();   // the tiles and barriers may be reused by the next unit
    return true;
}


template <int D, bool KCUT, int SHORT>
__global__ void __launch_bounds__(kThreads)
k_sweep(const RingRec *__restrict__ rec, const int64_t *__restrict__ nkept, int64_t nsplit,
        int64_t ndb,
        const float *__restrict__ cx, const float *__restrict__ cy,
        const float *__restrict__ cz, const int32_t *__restrict__ perm, int64_t M, float kc2,
        float *__restrict__ out, BlockBest *__restrict__ bb, int32_t *__restrict__ status) {
    __shared__ __align__(128) SweepSmem S;
    sweep_unit<D, KCUT, SHORT>(S, rec, nkept, nsplit, blockIdx.x % ndb, blockIdx.x / ndb, cx, cy,
                               cz, perm, M, kc2, out, bb ? bb + blockIdx.x : nullptr, status);
}

// Several bursts in one launch: CTAs take work units of all the bursts from
// a shared counter until none is left (launched with one CTA per unit, so
// most CTAs take one).  A unit is computed exactly as in k_sweep, so each
// burst's map does not depend on the others.
struct BurstDesc {
    const RingRec *rec;
    const int64_t *nkept;
    int64_t nsplit, ndb;
    float *out;
    BlockBest *bb;
    int32_t *status;
};

struct MultiArgs {
    int n;
    BurstDesc b[CC_BATCH_MAX];
    int64_t unit_begin[CC_BATCH_MAX + 1];
    const float *cx, *cy, *cz;
    const int32_t *perm;
    int64_t M;
    float kc2;
    unsigned long long *counter;
};

template <int D, bool KCUT, int SHORT>
__global__ void __launch_bounds__(kThreads) k_sweep_multi(const __grid_constant__ MultiArgs a) {
    __shared__ __align__(128) SweepSmem S;
    __shared__ long long unit_s;
    const long long total = a.unit_begin[a.n];
    for (;;) {
        if (threadIdx.x == 0) unit_s = (long long)atomicAdd(a.counter, 1ull);
        __syncthreads();
        const long long u = unit_s;
        __syncthreads();
        if (u >= total) break;
        int b = 0;
        while (u >= a.unit_begin[b + 1]) b++;
        const BurstDesc &d = a.b[b];
        const int64_t lu = u - a.unit_begin[b];
        if (!sweep_unit<D, KCUT, SHORT>(S, d.rec, d.nkept, d.nsplit, lu % d.ndb, lu / d.ndb, a.cx,
                                        a.cy, a.cz, a.perm, a.M, a.kc2, d.out,
                                        d.bb ? d.bb + lu : nullptr, d.status))
            break;
    }
}

// Sum of the split partial maps, fixed order, Kahan; plus block argmax.
__global__ void __launch_bounds__(256)
k_reduce_splits(const float *__restrict__ part, int64_t nsplit, int64_t M,
                float *__restrict__ map, BlockBest *__restrict__ bb) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float bv = -__builtin_huge_valf();
    int bj = INT32_MAX;
    if (j < M) {
        float s = 0.0f, c = 0.0f;
        for (int64_t k = 0; k < nsplit; k++) {
            if (!CC_IN_BOUNDS(CC_SITE_REDUCE_PART, k * M + j, nsplit * M)) break;
            float y = part[k * M + j] - c;
            float t = s + y;
            c = (t - s) - y;
            s = t;
        }
        float v = s - c;
        map[j] = v;
        bv = v;
        bj = (int)j;
    }
    block_best(bv, bj);
    if (threadIdx.x == 0) bb[blockIdx.x] = BlockBest{bv, bj};
}

// Argmax from the block bests, then greedy top-k with angular suppression.
__global__ void __launch_bounds__(1024)
k_select(const float *__restrict__ map, const BlockBest *__restrict__ bb, int64_t nbb,
         const float *__restrict__ cx, const float *__restrict__ cy,
         const float *__restrict__ cz, int64_t M, int topk, float cos_nms,
         int32_t *__restrict__ argmax, int32_t *__restrict__ seeds) {
    __shared__ float sdir[64][3];
    __shared__ int sidx[64];
    __shared__ int nseed;
    float v = -__builtin_huge_valf();
    int j = INT32_MAX;
    for (int64_t b = threadIdx.x; b < nbb; b += blockDim.x)
        if (CC_IN_BOUNDS(CC_SITE_SELECT_BB, b, nbb)) better(v, j, bb[b].v, bb[b].j);
    block_best(v, j);
    if (threadIdx.x == 0) {
        if (j < 0 || j >= M) j = 0;   // empty or all-NaN map
        argmax[0] = j;
        nseed = 1;
        sidx[0] = j;
        sdir[0][0] = cx[j];
        sdir[0][1] = cy[j];
        sdir[0][2] = cz[j];
        if (seeds) {
            seeds[0] = j;
            for (int t = 1; t < topk; t++) seeds[t] = -1;
        }
    }
    __syncthreads();
    if (seeds == nullptr) return;
    for (int t = 1; t < topk; t++) {
        float bv = -__builtin_huge_valf();
        int bj = INT32_MAX;
        const int ns = nseed;
        for (int64_t jj = threadIdx.x; jj < M; jj += blockDim.x) {
            float c0 = cx[jj], c1 = cy[jj], c2 = cz[jj];
            bool sup = false;
            for (int s = 0; s < ns; s++) {
                float dot = c0 * sdir[s][0] + c1 * sdir[s][1] + c2 * sdir[s][2];
                sup = sup || (sidx[s] == (int)jj) || (dot > cos_nms);
            }
            if (!sup) better(bv, bj, map[jj], (int)jj);
        }
        block_best(bv, bj);
        if (threadIdx.x == 0) {
            if (bj >= 0 && bj < M) {
                seeds[t] = bj;
                sidx[t] = bj;
                sdir[t][0] = cx[bj];
                sdir[t][1] = cy[bj];
                sdir[t][2] = cz[bj];
                nseed = t + 1;
            }
        }
        __syncthreads();
        if (nseed != t + 1) break;
    }
}

template <int D>
void *sweep_fn(bool kcut, int shortq) {
    if (kcut)
        return shortq == 2 ? (void *)k_sweep<D, true, 2>
               : shortq == 1 ? (void *)k_sweep<D, true, 1> : (void *)k_sweep<D, true, 0>;
    return shortq == 2 ? (void *)k_sweep<D, false, 2>
           : shortq == 1 ? (void *)k_sweep<D, false, 1> : (void *)k_sweep<D, false, 0>;
}

void *pick_sweep_q(int d, bool kcut, int shortq) {
    switch (d) {
        case 8: return sweep_fn<8>(kcut, shortq);
        case 4: return sweep_fn<4>(kcut, shortq);
        default: return sweep_fn<2>(kcut, shortq);
    }
}

void *pick_sweep(int d, bool kcut) { return pick_sweep_q(d, kcut, 0); }

// Which short polynomial the caps of warps sweeping 32 d consecutive
// directions of the compact order (M directions on the sphere) allow: level L
// when every ring that a cap leaves between the one-sided limit (kSideAngle,
// kSide2Angle) and pi/2 from its axis takes the equatorial form, 2 rho +
// 2e-3 <= limit - (pi/2 - kEquAngle).  A patch is about a square of
// 4 pi 32 d / M sr, cap radius sqrt(2 pi 32 d / M) (HEALPix's elongated
// patches reach a quarter more).  A wider cap in a short-polynomial sweep is
// still exact: its rings beyond the limit take the general form (at nside 64
// and 256 directions per warp, the warps above the median cap put 2 % of the
// rings there and level 1 still pays: 90.2 % of the roofline against 88.1 %).
int short_level(int64_t M, int d) {
    if (M < 1) return 0;
    const double pi = 3.14159265358979, band = 0.5 * pi - (double)kEquAngle;
    const double rho = std::sqrt(2.0 * pi * 32.0 * d / (double)M);
    if (rho <= 0.5 * ((double)kSide2Angle - band) - 1e-3) return 2;
    if (rho <= 0.5 * ((double)kSideAngle - band) - 1e-3) return 1;
    return 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// launch planning
// ---------------------------------------------------------------------------
bool plan_sweep(int64_t R, int64_t M, const cc_params &p, SweepPlan *plan, int force_d,
                SweepPick pick, size_t rec_bytes, bool ordered) {
    if (pick == nullptr) pick = pick_sweep;
    if (R < 0 || M < 1 || M > INT32_MAX) return false;
    const int sms = device_sm_count();
    if (sms <= 0) return false;
    const bool kcut = p.k_cut > 0.0f;
    const int64_t ring_tiles = R > 0 ? (R + kTile - 1) / kTile : 1;
    const int64_t max_split = ring_tiles < 256 ? ring_tiles : 256;

    // D = 8 first: four independent direction pairs per ring record give
    // the FP32 pipe more to overlap than two, which outweighs the lower
    // occupancy (2 CTAs per SM against 4 at D = 4).  Measured on GB300: the
    // 200k-event sweep 63.9 -> 66.9 % of its roofline, the 1M-ring burst
    // 64.8 -> 67.5 %, the near-field image 66.7 -> 68.7 % (D = 6, at 3 CTAs
    // per SM, was slower than D = 4).  With the angular selection too, now
    // that the reaching rings take the class lists (the 1M-ring burst at
    // k_cut = 5: 108 ms against 126 at D = 4; with the general form for
    // every reaching ring D = 4 had won, 135 ms against 153, its caps of 128
    // directions skipping more rings).
    const int order[3] = {8, 4, 2};
    int d = 2;
    int64_t conc = 0;
    for (int ci = 0; ci < 3; ci++) {
        int cand = order[ci];
        if (force_d > 0) cand = force_d;
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pick(cand, kcut), kThreads, 0);
        if (occ < 1) occ = 1;
        int64_t c = (int64_t)sms * occ;
        int64_t ndb = (M + (int64_t)kThreads * cand - 1) / ((int64_t)kThreads * cand);
        d = cand;
        conc = c;
        if (force_d > 0 || ndb * max_split >= c) break;
    }
    const int64_t ndb = (M + (int64_t)kThreads * d - 1) / ((int64_t)kThreads * d);

    // ring splits: enough CTAs to fill the machine, whole waves (>= 97 % of
    // the last wave busy) when possible
    int64_t best_ns = 1;
    double best_eff = -1.0;
    for (int64_t ns = 1; ns <= max_split; ns++) {
        int64_t U = ndb * ns;
        double waves = (double)U / (double)conc;
        double eff = waves / std::ceil(waves);
        if (U < conc) eff = waves;      // machine not full
        if (eff > best_eff + 1e-9) { best_eff = eff; best_ns = ns; }
        if (U >= conc && eff >= 0.97) break;
    }
    const int64_t tiles = (ring_tiles + best_ns - 1) / best_ns;

    plan->d = d;
    plan->threads = kThreads;
    plan->tile = kTile;
    plan->tiles = tiles;
    plan->nsplit = best_ns;
    plan->ndb = ndb;
    plan->rpad = tiles * best_ns * kTile;
    plan->nbb = best_ns > 1 ? (M + 255) / 256 : ndb;
    size_t off = 0;
    plan->off_rec = off;
    off = align256(off + (size_t)plan->rpad * rec_bytes);
    plan->off_part = off;
    if (best_ns > 1) off = align256(off + (size_t)best_ns * (size_t)M * sizeof(float));
    plan->off_bb = off;
    off = align256(off + (size_t)plan->nbb * sizeof(BlockBest));
    plan->off_status = off;
    off = align256(off + sizeof(int32_t));
    plan->off_counter = off;
    off = align256(off + sizeof(unsigned long long));
    plan->off_nkept = off;
    off = align256(off + sizeof(int64_t));
    plan->npack = R > 0 ? (R + kPackChunk - 1) / kPackChunk : 1;
    plan->off_packcnt = off;
    off = align256(off + (size_t)plan->npack * sizeof(int32_t));
    // the directions' compact order: the single far-field sweep (and the
    // near-field one, which asks for it)
    plan->ordered = force_d == 0 && (pick == pick_sweep || ordered);
    plan->off_perm = off;
    plan->off_order = off;
    if (plan->ordered) {
        off = align256(off + (size_t)M * sizeof(int32_t));
        plan->off_order = off;
        off = align256(off + direction_order_bytes(M));
    }
    plan->bytes = off;
    return true;
}

cudaError_t launch_pack_scan(int32_t *blockcnt, int64_t nblk, int64_t *nkept, cudaStream_t s) {
    k_pack_scan<<<1, 1024, 0, s>>>(blockcnt, nblk, nkept);
    return cudaGetLastError();
}

// Pack one burst's rings into the plan's records (and zero its status).
cudaError_t pack_for_plan(const cc_rings &rings, const SweepPlan &plan, int32_t *status, char *ws,
                          cudaStream_t s) {
    RingRec *rec = reinterpret_cast<RingRec *>(ws + plan.off_rec);
    int32_t *st = status ? status : reinterpret_cast<int32_t *>(ws + plan.off_status);
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    int32_t *cnt = reinterpret_cast<int32_t *>(ws + plan.off_packcnt);
    int64_t *nkept = reinterpret_cast<int64_t *>(ws + plan.off_nkept);
    TraceScope ts(CC_STAGE_PACK, s, 3);   // count, scan, scatter
    const unsigned nb = (unsigned)plan.npack;
    k_pack_count<<<nb, 256, 0, s>>>(rings.ax, rings.ay, rings.az, rings.eta, rings.deta,
                                    rings.valid, rings.count, cnt);
    k_pack_scan<<<1, 1024, 0, s>>>(cnt, plan.npack, nkept);
    k_pack_scatter<<<nb, 256, 0, s>>>(rings.ax, rings.ay, rings.az, rings.eta, rings.deta,
                                      rings.valid, rings.count, cnt, nkept, rec);
    return cudaGetLastError();
}

// After the sweep of one burst: the split reduction and argmax / seeds.
cudaError_t finish_localize(const cc_grid &grid, const cc_params &p, const SweepPlan &plan,
                            float *map, int32_t *argmax, int32_t *seeds, char *ws,
                            cudaStream_t s) {
    float *part = reinterpret_cast<float *>(ws + plan.off_part);
    BlockBest *bb = reinterpret_cast<BlockBest *>(ws + plan.off_bb);
    cudaError_t e;
    if (plan.nsplit > 1) {
        {
            TraceScope ts(CC_STAGE_REDUCE, s);
            k_reduce_splits<<<(unsigned)plan.nbb, 256, 0, s>>>(part, plan.nsplit, grid.count,
                                                               map, bb);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    int topk = p.topk < 1 ? 1 : p.topk;
    TraceScope ts(CC_STAGE_SELECT, s);
    k_select<<<1, 1024, 0, s>>>(map, bb, plan.nbb, grid.x, grid.y, grid.z, grid.count, topk,
                                cosf(p.nms_rad), argmax, seeds);
    return cudaGetLastError();
}

cudaError_t launch_localize(const cc_rings &rings, const cc_grid &grid, const cc_params &p,
                            const SweepPlan &plan, float *map, int32_t *argmax,
                            int32_t *seeds, int32_t *status, char *ws, cudaStream_t s) {
    RingRec *rec = reinterpret_cast<RingRec *>(ws + plan.off_rec);
    float *part = reinterpret_cast<float *>(ws + plan.off_part);
    BlockBest *bb = reinterpret_cast<BlockBest *>(ws + plan.off_bb);
    int32_t *st = status ? status : reinterpret_cast<int32_t *>(ws + plan.off_status);
    cudaError_t e = pack_for_plan(rings, plan, status, ws, s);
    if (e != cudaSuccess) return e;
    const int64_t M = grid.count;
    const bool kcut = p.k_cut > 0.0f;
    const float kc = p.k_cut * kGaussK;
    const float kc2 = kcut ? kc * kc : 0.0f;
    float *out = plan.nsplit > 1 ? part : map;
    BlockBest *bbk = plan.nsplit > 1 ? nullptr : bb;
    const unsigned grid_ctas = (unsigned)(plan.ndb * plan.nsplit);
    void *fn = pick_sweep_q(plan.d, kcut, plan.ordered ? short_level(M, plan.d) : 0);
    const int64_t *nkept = reinterpret_cast<const int64_t *>(ws + plan.off_nkept);
    const int32_t *perm = nullptr;
    if (plan.ordered) {
        perm = grid.order;
        if (perm == nullptr) {        // not given with the grid: computed here
            int32_t *pm = reinterpret_cast<int32_t *>(ws + plan.off_perm);
            TraceScope ts(CC_STAGE_PACK, s, direction_order_kernels(M));
            if ((e = direction_order(grid, pm, ws + plan.off_order, s)) != cudaSuccess) return e;
            perm = pm;
        }
    }
    void *args[] = {(void *)&rec,    (void *)&nkept,  (void *)&plan.nsplit, (void *)&plan.ndb,
                    (void *)&grid.x, (void *)&grid.y, (void *)&grid.z,     (void *)&perm,
                    (void *)&M,      (void *)&kc2,    (void *)&out,         (void *)&bbk,
                    (void *)&st};
    {
        TraceScope ts(CC_STAGE_SWEEP, s);
        e = cudaLaunchKernel(fn, dim3(grid_ctas), dim3(kThreads), args, 0, s);
    }
    if (e != cudaSuccess) return e;
    return finish_localize(grid, p, plan, map, argmax, seeds, ws, s);
}

cudaError_t launch_localize_batch(int n, const cc_rings *rings, const cc_grid &grid,
                                  const cc_params &p, const SweepPlan *plans, float *const *maps,
                                  int32_t *const *argmax, int32_t *const *seeds,
                                  int32_t *const *status, char *const *ws, cudaStream_t s) {
    MultiArgs a{};
    a.n = n;
    a.cx = grid.x;
    a.cy = grid.y;
    a.cz = grid.z;
    a.perm = grid.order;     // the grid's order when the caller keeps one
    a.M = grid.count;
    const bool kcut = p.k_cut > 0.0f;
    const float kc = p.k_cut * kGaussK;
    a.kc2 = kcut ? kc * kc : 0.0f;
    a.counter = reinterpret_cast<unsigned long long *>(ws[0] + plans[0].off_counter);
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    a.unit_begin[0] = 0;
    for (int b = 0; b < n; b++) {
        const SweepPlan &pl = plans[b];
        if ((e = pack_for_plan(rings[b], pl, status ? status[b] : nullptr, ws[b], s))) return e;
        BurstDesc &d = a.b[b];
        d.rec = reinterpret_cast<const RingRec *>(ws[b] + pl.off_rec);
        d.nkept = reinterpret_cast<const int64_t *>(ws[b] + pl.off_nkept);
        d.nsplit = pl.nsplit;
        d.ndb = pl.ndb;
        d.out = pl.nsplit > 1 ? reinterpret_cast<float *>(ws[b] + pl.off_part) : maps[b];
        d.bb = pl.nsplit > 1 ? nullptr : reinterpret_cast<BlockBest *>(ws[b] + pl.off_bb);
        d.status = (status && status[b]) ? status[b]
                                         : reinterpret_cast<int32_t *>(ws[b] + pl.off_status);
        a.unit_begin[b + 1] = a.unit_begin[b] + pl.ndb * pl.nsplit;
    }
    // one CTA per work unit (a CTA still takes its unit from the counter): CTAs
    // retire as their units finish, so kernels of higher-priority streams
    // (the bursts' front ends) get SMs without waiting for the whole batch
    const int lvl = a.perm != nullptr ? short_level(a.M, kBatchD) : 0;
    void *fn = kcut ? (lvl == 2   ? (void *)k_sweep_multi<kBatchD, true, 2>
                       : lvl == 1 ? (void *)k_sweep_multi<kBatchD, true, 1>
                                  : (void *)k_sweep_multi<kBatchD, true, 0>)
                    : (lvl == 2   ? (void *)k_sweep_multi<kBatchD, false, 2>
                       : lvl == 1 ? (void *)k_sweep_multi<kBatchD, false, 1>
                                  : (void *)k_sweep_multi<kBatchD, false, 0>);
    int64_t ctas = a.unit_begin[n];
    if (ctas > (int64_t)INT32_MAX) ctas = INT32_MAX;
    if (ctas < 1) ctas = 1;
    void *args[] = {(void *)&a};
    {
        TraceScope ts(CC_STAGE_SWEEP, s);
        e = cudaLaunchKernel(fn, dim3((unsigned)ctas), dim3(kThreads), args, 0, s);
    }
    if (e != cudaSuccess) return e;
    for (int b = 0; b < n; b++)
        if ((e = finish_localize(grid, p, plans[b], maps[b], argmax[b], seeds ? seeds[b] : nullptr,
                                 ws[b], s)))
            return e;
    return cudaSuccess;
}

}  // namespace cc

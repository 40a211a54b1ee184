// voxel.cu - near-field 3D back projection (Sec. 3 of the paper): every
// (gamma-ray, voxel) pair contributes independently and the contributions
// are summed per voxel into the image.
//
// A gamma-ray is its Compton cone: apex p (the first interaction site), axis
// a, energetic half angle eta and width deta.  The geometric Compton angle of
// voxel centre v is theta = angle(v - p, a); the contribution is
// exp(-r^2/2), r = (theta - eta) / deta, dropped for |r| > k_cut when the
// angular selection is on.
//
// The paper precomputes the geometric angles in tables over discrete
// scatterer, absorber and voxel positions.  On GB300 the per-pair angle costs
// fewer cycles than reading it from a table, so nothing per pair is stored:
// per ring the record holds -p, -a/sqrt(2), k = sqrt(log2(e)/2)/deta and
// -eta k; per pair
//     d = v - p,  y' = rsqrt(2 |d|^2) (MUFU + one Newton step),
//     c = d y' - a/sqrt(2)  (the half chord between unit(d) and a),
//     h = |c|^2 = 1 - cos(theta)  (relative accuracy, also at small angles),
// and from h on it is the far-field pair: theta from the fitted
// acos(1 - h)/sqrt(h) polynomial (or its mirror for theta > pi/2), the
// Gaussian on the MUFU ex2 unit.  The voxels are swept in Morton order
// (order.cu), so each warp's 256 voxels are a compact block, and as in the
// far-field sweep each warp sorts a tile's rings by where its block's
// bounding sphere lies from them: every voxel within 33.4 deg of pi/2 from the
// axis, the equatorial form (cos(theta) from the dot product and the
// approximate rsqrt, theta = pi/2 + asin by an odd polynomial: no Newton
// step, no square root, no fold, no select); every voxel within 78.46 deg of
// the axis or of its opposite, the one-sided form (no fold, no select, a
// shorter polynomial: degree 4 within 63.26 deg, else degree 5); the rest,
// the general form.  Rings with eta > pi/2
// are mirrored (a -> -a, eta -> pi - eta).  The pipeline (TMA bulk tiles
// through a 4-stage mbarrier ring, ring splits over CTAs with a fixed-order
// Kahan reduction, block argmax) is the far-field sweep's, with 64-byte
// records.
//
// Image universes (Sec. 3, spatial optimisation): the n^3 voxels of a cube,
// or those whose centres lie in the inscribed cylinder (axis z) or sphere,
// decided by exact integer tests on the odd centre offsets 2i + 1 - n.
#include "cc_math.cuh"
#include "cc_pipe.cuh"

namespace cc {
namespace {

constexpr int kThreads = 256;   // as the plan
constexpr int kTile = 128;
constexpr int kStages = 4;
constexpr float kInvSqrt2 = 0.70710678118654752f;
constexpr float kGaussK = 0.84932180028801907f;   // sqrt(log2(e) / 2)
constexpr float kNullB = 1.0e4f;
// the equatorial form's band: within E = asin(0.55) = 33.37 deg of pi/2
constexpr float kEquSin = 0.54916456f;     // sin(E - 1e-3)
constexpr float kEquCos = 0.83571424f;     // cos(E - 1e-3)
// one-sided forms: every pair within acos(0.2) = 78.46 deg of the axis or of
// its opposite (s <= 0.8, the short polynomial's range); T = that - 1e-3
constexpr float kSideCos = 0.20097970f;    // cos(T)
constexpr float kSideSin = 0.97959541f;    // sin(T)
// and within acos(0.45) = 63.26 deg (s <= 0.55, degree 4); T2 = that - 1e-3
constexpr float kSide2Cos = 0.45089280f;    // cos(T2)
constexpr float kSide2Sin = 0.89257811f;    // sin(T2)

struct NearRec {   // 64 bytes; values met by a voxel pair are duplicated
    float mpx, mpx_, mpy, mpy_, mpz, mpz_;   // -p
    float msx, msx_, msy, msy_, msz, msz_;   // -a / sqrt(2)
    float k, k_;                             // sqrt(log2 e / 2) / deta
    float nb, nb2;                           // -eta k, -(pi - eta) k
};
static_assert(sizeof(NearRec) == 64, "record layout");

__device__ __forceinline__ float2 pair(float v) { return make_float2(v, v); }

// ---------------------------------------------------------------------------
// apex of each ring: the first site of its chosen order (rank perm = the
// perm-th permutation of the k slots in lexicographic order, whose first
// element is perm / (k-1)!)
// ---------------------------------------------------------------------------
__global__ void k_ring_apex(cc_events ev, const uint8_t *__restrict__ perm,
                            const uint8_t *__restrict__ valid, float *__restrict__ px,
                            float *__restrict__ py, float *__restrict__ pz) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ev.count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int k = ev.n[i];
        float x = 0.f, y = 0.f, z = 0.f;
        if (valid[i] && k >= 2 && k <= 4) {
            const int f = k == 2 ? 1 : (k == 3 ? 2 : 6);
            const int slot = perm[i] / f;
            x = ev.x[slot * ev.stride + i];
            y = ev.y[slot * ev.stride + i];
            z = ev.z[slot * ev.stride + i];
        }
        px[i] = x;
        py[i] = y;
        pz[i] = z;
    }
}

// ---------------------------------------------------------------------------
// universes
// ---------------------------------------------------------------------------
// exact floor(sqrt(v)) for 0 <= v < 2^62
__device__ __host__ __forceinline__ long long isqrt_ll(long long v) {
    long long r = (long long)sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

// voxels of row (k, j): the i with (2i + 1 - n)^2 <= lim form [lo, hi]
__device__ __host__ __forceinline__ void row_range(int shape, long long n, long long j,
                                                   long long k, long long *lo, long long *hi) {
    const long long oj = 2 * j + 1 - n, ok = 2 * k + 1 - n;
    long long lim = n * n;
    if (shape == 1) lim -= oj * oj;
    if (shape == 2) lim -= oj * oj + ok * ok;
    if (shape == 0) { *lo = 0; *hi = n - 1; return; }
    if (lim < 0) { *lo = 0; *hi = -1; return; }
    const long long m = isqrt_ll(lim);       // |2i + 1 - n| <= m
    long long a = n - 1 - m, b = n - 1 + m;  // 2i in [a, b]
    long long l = a <= 0 ? 0 : (a + 1) / 2, h = b / 2;
    if (h > n - 1) h = n - 1;
    *lo = l;
    *hi = h;
}

// One CTA per z slab: the slab's offset is the voxel count of the slabs
// below it (each thread sums its rows over them), rows are then placed by a
// block scan of their counts.
__global__ void __launch_bounds__(1024)
k_universe(int shape, int n, float pitch, float cx, float cy, float cz, float *__restrict__ x,
           float *__restrict__ y, float *__restrict__ z) {
    __shared__ long long part[32];
    __shared__ long long base_s;
    const int k = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long below = 0;
    for (int kk = 0; kk < k; kk++)
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            long long lo, hi;
            row_range(shape, n, j, kk, &lo, &hi);
            below += hi - lo + 1;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
    if (lane == 0) part[w] = below;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int q = 0; q < nw; q++) s += part[q];
        base_s = s;
    }
    __syncthreads();
    long long base = base_s;
    const double half = 0.5 * (double)pitch;
    const float zc = (float)((double)cz + half * (double)(2 * k + 1 - n));
    for (int j0 = 0; j0 < n; j0 += blockDim.x) {     // rows in chunks of blockDim
        const int j = j0 + threadIdx.x;
        long long lo = 0, hi = -1;
        if (j < n) row_range(shape, n, j, k, &lo, &hi);
        const long long c = hi - lo + 1;
        long long incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        __syncthreads();
        if (lane == 31) part[w] = incl;
        __syncthreads();
        long long wbase = 0, total = 0;
        for (int q = 0; q < nw; q++) {
            wbase += q < w ? part[q] : 0;
            total += part[q];
        }
        long long off = base + wbase + incl - c;
        if (j < n) {
            const float yc = (float)((double)cy + half * (double)(2 * j + 1 - n));
            for (long long i = lo; i <= hi; i++, off++) {
                x[off] = (float)((double)cx + half * (double)(2 * i + 1 - n));
                y[off] = yc;
                z[off] = zc;
            }
        }
        base += total;
    }
}

// ---------------------------------------------------------------------------
// ring records (compaction of the kept rings, as for the far-field sweep)
// ---------------------------------------------------------------------------
struct NearRings {
    const float *ax, *ay, *az, *eta, *deta, *px, *py, *pz;
    const uint8_t *valid;
    int64_t R;
};

__device__ __forceinline__ bool near_kept(const NearRings &g, int64_t i) {
    if (i >= g.R || (g.valid != nullptr && !g.valid[i])) return false;
    const float de = g.deta[i];
    return isfinite(g.ax[i]) && isfinite(g.ay[i]) && isfinite(g.az[i]) && isfinite(g.eta[i]) &&
           isfinite(de) && de > 0.0f && isfinite(g.px[i]) && isfinite(g.py[i]) &&
           isfinite(g.pz[i]);
}

__device__ __forceinline__ NearRec near_rec(const NearRings &g, int64_t i) {
    float a0 = g.ax[i], a1 = g.ay[i], a2 = g.az[i], e = g.eta[i];
    const float k = kGaussK / g.deta[i];
    float b = e * k, b2 = (kPiF - e) * k;
    if (e > 0.5f * kPiF) {        // mirror: same cone, eta' <= pi/2
        a0 = -a0; a1 = -a1; a2 = -a2;
        float t = b; b = b2; b2 = t;
    }
    const float s0 = -a0 * kInvSqrt2, s1 = -a1 * kInvSqrt2, s2 = -a2 * kInvSqrt2;
    const float p0 = -g.px[i], p1 = -g.py[i], p2 = -g.pz[i];
    return NearRec{p0, p0, p1, p1, p2, p2, s0, s0, s1, s1, s2, s2, k, k, -b, -b2};
}

__global__ void __launch_bounds__(256) k_near_count(NearRings g, int32_t *__restrict__ cnt) {
    const int64_t base = blockIdx.x * (int64_t)kPackChunk;
    int n = 0;
    for (int r = 0; r < kPackChunk / 256; r++)
        n += __syncthreads_count(near_kept(g, base + r * 256 + threadIdx.x));
    if (threadIdx.x == 0) cnt[blockIdx.x] = n;
}

__global__ void __launch_bounds__(256)
k_near_scatter(NearRings g, const int32_t *__restrict__ offs, const int64_t *__restrict__ nkept,
               NearRec *__restrict__ rec) {
    __shared__ int wcnt[8];
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = blockIdx.x * (int64_t)kPackChunk;
    int64_t pos = offs[blockIdx.x];
    for (int r = 0; r < kPackChunk / 256; r++) {
        const int64_t i = base + r * 256 + threadIdx.x;
        const bool keep = near_kept(g, i);
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (l == 0) wcnt[w] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            before += q < w ? wcnt[q] : 0;
            total += wcnt[q];
        }
        if (keep) rec[pos + before + __popc(m & ((1u << l) - 1u))] = near_rec(g, i);
        pos += total;
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x < kTile) {   // null records up to the tile end
        const int64_t n = *nkept;
        const int64_t end = (n + kTile - 1) / kTile * kTile;
        if (n + threadIdx.x < end)
            rec[n + threadIdx.x] = NearRec{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f,
                                           0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -kNullB, -kNullB};
    }
}

// ---------------------------------------------------------------------------
// the back-projection sweep
// ---------------------------------------------------------------------------
struct NearSmem {
    NearRec tile[kStages][kTile];
    unsigned long long full[kStages];
    unsigned char lst[kThreads / 32][kTile];   // per warp: the tile's rings by side
    int abort_flag;
};

// The pair terms of one ring for DP voxel pairs.  SIDE 1: every pair lies
// within acos(0.2) = 78.46 deg of the axis (h <= 0.8), SIDE 2: of its opposite
// (2 - h <= 0.8); the fold and the select then have one outcome, and the
// acos polynomial is the degree-5 fit on [0, 0.8] (fit_acos.py: 2.6e-7 rad
// evaluated in FP32, as accurate as the general form's degree 7 on [0, 1]:
// 2.3e-7).  SIDE 3 / 4: within acos(0.45) = 63.26 deg of the axis / of its
// opposite (s <= 0.55), the degree-4 fit on [0, 0.55] (2.4e-7).  SIDE 5: the
// equatorial form (below).
template <int DP, bool KCUT, int SIDE>
__device__ __forceinline__ void near_pairs(const NearRec &Rr, const float2 (&px2)[DP],
                                           const float2 (&py2)[DP], const float2 (&pz2)[DP],
                                           float2 (&acc)[DP], float kc2) {
    const float2 m1 = pair(-1.0f), two2 = pair(2.0f);
    const float2 nh = pair(-0.5f * kInvSqrt2), th2 = pair(1.5f * kInvSqrt2);
    const float4 R0 = *reinterpret_cast<const float4 *>(&Rr.mpx);
    const float4 R1 = *reinterpret_cast<const float4 *>(&Rr.mpz);
    const float4 R2 = *reinterpret_cast<const float4 *>(&Rr.msy);
    const float4 R3 = *reinterpret_cast<const float4 *>(&Rr.k);
    const float2 mpx = make_float2(R0.x, R0.y), mpy = make_float2(R0.z, R0.w);
    const float2 mpz = make_float2(R1.x, R1.y), msx = make_float2(R1.z, R1.w);
    const float2 msy = make_float2(R2.x, R2.y), msz = make_float2(R2.z, R2.w);
    const float2 k2 = make_float2(R3.x, R3.y);
    if constexpr (SIDE == 5) {
        // equatorial: every pair within E of pi/2 from the axis.
        // s = (-a/sqrt 2).d / |d| = -cos(theta) / sqrt(2), theta = pi/2 +
        // asin(sqrt(2) s) = pi/2 + s P(s^2) (fit_asin.py, sigma = sqrt(2):
        // 1.3e-7 rad evaluated in FP32); no Newton step (the approximate
        // rsqrt's relative error moves cos(theta) by at most 1e-7 of its
        // |value| <= 0.55), no square root, no fold, no select
        const float2 ne2 = __ffma2_rn(k2, pair(0.5f * kPiF), make_float2(R3.z, R3.z));
#pragma unroll
        for (int q = 0; q < DP; q++) {
            const float2 dx = __fadd2_rn(px2[q], mpx);
            const float2 dy = __fadd2_rn(py2[q], mpy);
            const float2 dz = __fadd2_rn(pz2[q], mpz);
            float2 n2 = __ffma2_rn(dx, dx, pair(1.0e-30f));
            n2 = __ffma2_rn(dy, dy, n2);
            n2 = __ffma2_rn(dz, dz, n2);
            const float2 y0 = make_float2(rsqrt_approx(n2.x), rsqrt_approx(n2.y));
            float2 t = __fmul2_rn(msz, dz);
            t = __ffma2_rn(msy, dy, t);
            t = __ffma2_rn(msx, dx, t);
            const float2 sd = __fmul2_rn(t, y0);
            const float2 w = __fmul2_rn(sd, sd);
            float2 p = pair(1.38170266e+00f);
            p = __ffma2_rn(p, w, pair(3.82552564e-01f));
            p = __ffma2_rn(p, w, pair(4.33079332e-01f));
            p = __ffma2_rn(p, w, pair(4.71152157e-01f));
            p = __ffma2_rn(p, w, pair(1.41421556e+00f));
            const float2 v = __fmul2_rn(sd, p);                    // theta - pi/2
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
#pragma unroll
        for (int q = 0; q < DP; q++) {
            const float2 dx = __fadd2_rn(px2[q], mpx);
            const float2 dy = __fadd2_rn(py2[q], mpy);
            const float2 dz = __fadd2_rn(pz2[q], mpz);
            // |d|^2 + 1e-30: a voxel centre on the apex stays finite
            float2 n2 = __ffma2_rn(dx, dx, pair(1.0e-30f));
            n2 = __ffma2_rn(dy, dy, n2);
            n2 = __ffma2_rn(dz, dz, n2);
            const float2 y0 = make_float2(rsqrt_approx(n2.x), rsqrt_approx(n2.y));
            float2 tt = __fmul2_rn(n2, y0);
            tt = __fmul2_rn(tt, y0);
            const float2 f = __ffma2_rn(tt, nh, th2);
            const float2 y1 = __fmul2_rn(y0, f);                // rsqrt(|d|^2)/sqrt(2)
            const float2 cx = __ffma2_rn(dx, y1, msx);
            const float2 cy = __ffma2_rn(dy, y1, msy);
            const float2 cz = __ffma2_rn(dz, y1, msz);
            float2 h = __fmul2_rn(cx, cx);
            h = __ffma2_rn(cy, cy, h);
            h = __ffma2_rn(cz, cz, h);                           // 1 - cos(theta)
            float2 sv;
            if (SIDE == 1 || SIDE == 3) {
                sv = h;
            } else {
                const float2 g = __ffma2_rn(h, m1, two2);
                sv = (SIDE == 2 || SIDE == 4) ? make_float2(fabsf(g.x), fabsf(g.y))
                               : make_float2(fminf(h.x, fabsf(g.x)), fminf(h.y, fabsf(g.y)));
            }
            float2 p;
            if (SIDE == 0) {                                     // acos_q on [0, 1], degree 7
                p = pair(1.4414361e-03f);
                p = __ffma2_rn(p, sv, pair(-2.8447455e-03f));
                p = __ffma2_rn(p, sv, pair(4.6071224e-03f));
                p = __ffma2_rn(p, sv, pair(5.2066805e-04f));
                p = __ffma2_rn(p, sv, pair(8.6035002e-03f));
                p = __ffma2_rn(p, sv, pair(2.6394552e-02f));
                p = __ffma2_rn(p, sv, pair(1.1786042e-01f));
                p = __ffma2_rn(p, sv, pair(1.4142133e+00f));
            } else if (SIDE == 1 || SIDE == 2) {                 // on [0, 0.8], degree 5
                p = pair(3.31251509e-03f);
                p = __ffma2_rn(p, sv, pair(-2.59509514e-04f));
                p = __ffma2_rn(p, sv, pair(9.49506927e-03f));
                p = __ffma2_rn(p, sv, pair(2.61093955e-02f));
                p = __ffma2_rn(p, sv, pair(1.17894620e-01f));
                p = __ffma2_rn(p, sv, pair(1.41421223e+00f));
            } else {                                             // on [0, 0.55], degree 4
                p = pair(5.02272556e-03f);
                p = __ffma2_rn(p, sv, pair(6.41390355e-03f));
                p = __ffma2_rn(p, sv, pair(2.69000251e-02f));
                p = __ffma2_rn(p, sv, pair(1.17811434e-01f));
                p = __ffma2_rn(p, sv, pair(1.41421473e+00f));
            }
            const float2 rt = make_float2(sqrt_approx(sv.x), sqrt_approx(sv.y));
            const float2 th = __fmul2_rn(rt, p);
            const float2 nbs = (SIDE == 1 || SIDE == 3)   ? make_float2(R3.z, R3.z)
                               : (SIDE == 2 || SIDE == 4) ? make_float2(R3.w, R3.w)
                                           : make_float2(h.x <= 1.0f ? R3.z : R3.w,
                                                         h.y <= 1.0f ? R3.z : R3.w);
            const float2 u = __ffma2_rn(th, k2, nbs);
            const float2 u2 = __fmul2_rn(u, u);
            float2 e = make_float2(ex2_approx(-u2.x), ex2_approx(-u2.y));
            if (KCUT) {
                e.x = u2.x > kc2 ? 0.0f : e.x;
                e.y = u2.y > kc2 ? 0.0f : e.y;
            }
            acc[q] = __fadd2_rn(acc[q], e);
        }
    }
}

template <int DP, bool KCUT, int SIDE>
__device__ __forceinline__ void near_run(const NearRec *T, const unsigned char *lst, int b, int e,
                                         const float2 (&px2)[DP], const float2 (&py2)[DP],
                                         const float2 (&pz2)[DP], float2 (&acc)[DP], float kc2) {
    int i = b;
    for (; i + 2 <= e; i += 2) {
        near_pairs<DP, KCUT, SIDE>(T[lst[i]], px2, py2, pz2, acc, kc2);
        near_pairs<DP, KCUT, SIDE>(T[lst[i + 1]], px2, py2, pz2, acc, kc2);
    }
    if (i < e) near_pairs<DP, KCUT, SIDE>(T[lst[i]], px2, py2, pz2, acc, kc2);
}

template <int D, bool KCUT>
__global__ void __launch_bounds__(kThreads, 2)
k_backproject(const NearRec *__restrict__ rec, const int64_t *__restrict__ nkept, int64_t nsplit,
              int64_t ndb, const float *__restrict__ vx, const float *__restrict__ vy,
              const float *__restrict__ vz, const int32_t *__restrict__ perm, int64_t V,
              float kc2, float *__restrict__ out,
              BlockBest *__restrict__ bb, int32_t *__restrict__ status) {
    static_assert(D % 2 == 0, "voxels are processed in FP32x2 pairs");
    constexpr int DP = D / 2;
    __shared__ __align__(128) NearSmem S;
    const int tid = threadIdx.x;
    const int64_t db = blockIdx.x % ndb, split = blockIdx.x / ndb;
    // warp w owns the 32 D consecutive voxels from db 256 D + 32 D w (lane l
    // the voxels l, l + 32, ...): a compact block when the list is
    const int64_t j0 = db * (int64_t)(kThreads * D) + (int64_t)(tid >> 5) * (32 * D) + (tid & 31);

    float2 px2[DP], py2[DP], pz2[DP], acc[DP], sum[DP], comp[DP];
#pragma unroll
    for (int q = 0; q < DP; q++) {
        int64_t ja = j0 + (int64_t)(64 * q), jb = ja + 32;
        ja = ja < V ? ja : V - 1;
        jb = jb < V ? jb : V - 1;
        if (perm != nullptr) {
            ja = __ldg(perm + ja);
            jb = __ldg(perm + jb);
        }
        px2[q] = make_float2(__ldg(vx + ja), __ldg(vx + jb));
        py2[q] = make_float2(__ldg(vy + ja), __ldg(vy + jb));
        pz2[q] = make_float2(__ldg(vz + ja), __ldg(vz + jb));
        acc[q] = sum[q] = comp[q] = make_float2(0.0f, 0.0f);
    }

    // the warp's voxels' bounding sphere: centre and radius (plus a margin for
    // the FP32 side test: 1e-3 of the distance to an apex is added below)
    const int lane = tid & 31, w = tid >> 5;
    float bcx = 0.f, bcy = 0.f, bcz = 0.f, brad = 0.f;
    {
#pragma unroll
        for (int q = 0; q < DP; q++) {
            bcx += px2[q].x + px2[q].y;
            bcy += py2[q].x + py2[q].y;
            bcz += pz2[q].x + pz2[q].y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bcx += __shfl_xor_sync(0xffffffffu, bcx, o);
            bcy += __shfl_xor_sync(0xffffffffu, bcy, o);
            bcz += __shfl_xor_sync(0xffffffffu, bcz, o);
        }
        const float inv = 1.0f / (32.0f * D);
        bcx *= inv;
        bcy *= inv;
        bcz *= inv;
        float r2 = 0.f;
#pragma unroll
        for (int q = 0; q < DP; q++) {
            const float ax_ = px2[q].x - bcx, ay_ = py2[q].x - bcy, az_ = pz2[q].x - bcz;
            const float bx_ = px2[q].y - bcx, by_ = py2[q].y - bcy, bz_ = pz2[q].y - bcz;
            r2 = fmaxf(r2, fmaf(az_, az_, fmaf(ay_, ay_, ax_ * ax_)));
            r2 = fmaxf(r2, fmaf(bz_, bz_, fmaf(by_, by_, bx_ * bx_)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
        brad = sqrtf(r2) * 1.0001f + 1.0e-6f;
    }

    const int64_t ntk = (*nkept + kTile - 1) / kTile;
    const int64_t tiles = split < ntk ? (ntk - split + nsplit - 1) / nsplit : 0;
    const NearRec *src = rec + split * kTile;
    const int64_t stride = nsplit * kTile;
    if (tid == 0) {
        for (int s = 0; s < kStages; s++) mbar_init(&S.full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.abort_flag = 0;
    }
    __syncthreads();
    if (tid == 0)
        for (int s = 0; s < kStages && s < tiles; s++)
            if (CC_IN_BOUNDS(CC_SITE_VOXEL_TILE, split + s * nsplit, ntk))
                tma_bulk_load(S.tile[s], src + (int64_t)s * stride, kTile * sizeof(NearRec),
                              &S.full[s]);

    for (int64_t t = 0; t < tiles; t++) {
        const int stage = (int)(t % kStages);
        const unsigned parity = (unsigned)((t / kStages) & 1);
        if (!mbar_wait(&S.full[stage], parity)) {
            S.abort_flag = 1;
        } else {
            const NearRec *T = S.tile[stage];
            // the tile's rings by class against the warp's sphere (centre C,
            // radius rad): alpha = angle(a, C - apex), beta = asin(rad /
            // dist) the sphere's half angle from the apex, so every voxel of
            // the sphere lies between alpha - beta and alpha + beta from the
            // axis.  Equatorial when |alpha - pi/2| <= A - beta, A =
            // E - 1e-3: |a . (C - apex)| <= sin(A) sqrt(dist^2 -
            // rad^2) - cos(A) rad.  Near side (far side) when alpha + beta
            // <= T (pi - alpha + beta <= T), T = acos(0.2) - 1e-3:
            // +-a . (C - apex) >= cos(T) sqrt(dist^2 - rad^2) + sin(T) rad,
            // with beta <= T; the same with T2 = acos(0.45) - 1e-3 for the
            // degree-4 polynomial.  The rest take the general form.
            unsigned em[kTile / 32], nm[kTile / 32], fm[kTile / 32], n2m[kTile / 32],
                f2m[kTile / 32];
            int ne = 0, nn = 0, nf = 0, nn2 = 0, nf2 = 0;
#pragma unroll
            for (int g = 0; g < kTile / 32; g++) {
                const NearRec &Rg = T[32 * g + lane];
                const float ex = bcx + Rg.mpx, ey = bcy + Rg.mpy, ez = bcz + Rg.mpz;   // centre - apex
                // a = -sqrt(2) ms
                const float sa = -1.41421356f * fmaf(Rg.msz, ez, fmaf(Rg.msy, ey, Rg.msx * ex));
                const float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                const float r2 = brad * brad;
                const float cb = d2 > r2 ? sqrtf(d2 - r2) : 0.0f;     // dist cos(beta)
                const float elim = d2 > r2 ? fmaf(kEquSin, cb, -kEquCos * brad) : -1.0f;
                const float lim2 = r2 < kSide2Sin * kSide2Sin * d2 ? fmaf(kSide2Cos, cb, kSide2Sin * brad)
                                                                   : __builtin_huge_valf();
                const float lim = r2 < kSideSin * kSideSin * d2 ? fmaf(kSideCos, cb, kSideSin * brad)
                                                                : __builtin_huge_valf();
                const bool live = Rg.k != 0.0f;
                const bool eq = live && fabsf(sa) <= elim;
                const bool n2 = live && !eq && sa >= lim2, f2 = live && !eq && -sa >= lim2;
                em[g] = __ballot_sync(0xffffffffu, eq);
                n2m[g] = __ballot_sync(0xffffffffu, n2);
                f2m[g] = __ballot_sync(0xffffffffu, f2);
                nm[g] = __ballot_sync(0xffffffffu, live && !eq && !n2 && sa >= lim);
                fm[g] = __ballot_sync(0xffffffffu, live && !eq && !f2 && -sa >= lim);
                nn2 += __popc(n2m[g]);
                nf2 += __popc(f2m[g]);
                ne += __popc(em[g]);
                nn += __popc(nm[g]);
                nf += __popc(fm[g]);
            }
            const unsigned lt = (1u << lane) - 1u;
            int be = 0, bn2 = ne, bf2 = bn2 + nn2, bn = bf2 + nf2, bf = bn + nn, bm = bf + nf;
            const int ee = bn2, en2 = bf2, ef2 = bn, en = bf, ef = bm;
#pragma unroll
            for (int g = 0; g < kTile / 32; g++) {
                const unsigned mm = ~(em[g] | n2m[g] | f2m[g] | nm[g] | fm[g]);
                const unsigned bit = 1u << lane;
                const int at = (em[g] & bit)    ? be + __popc(em[g] & lt)
                             : (n2m[g] & bit) ? bn2 + __popc(n2m[g] & lt)
                             : (f2m[g] & bit) ? bf2 + __popc(f2m[g] & lt)
                             : (nm[g] & bit)  ? bn + __popc(nm[g] & lt)
                             : (fm[g] & bit)  ? bf + __popc(fm[g] & lt)
                                              : bm + __popc(mm & lt);
                S.lst[w][at] = (unsigned char)(32 * g + lane);
                be += __popc(em[g]);
                bn2 += __popc(n2m[g]);
                bf2 += __popc(f2m[g]);
                bn += __popc(nm[g]);
                bf += __popc(fm[g]);
                bm += __popc(mm);
            }
            __syncwarp();
            const unsigned char *L = S.lst[w];
            near_run<DP, KCUT, 5>(T, L, 0, ee, px2, py2, pz2, acc, kc2);
            near_run<DP, KCUT, 3>(T, L, ee, en2, px2, py2, pz2, acc, kc2);
            near_run<DP, KCUT, 4>(T, L, en2, ef2, px2, py2, pz2, acc, kc2);
            near_run<DP, KCUT, 1>(T, L, ef2, en, px2, py2, pz2, acc, kc2);
            near_run<DP, KCUT, 2>(T, L, en, ef, px2, py2, pz2, acc, kc2);
            near_run<DP, KCUT, 0>(T, L, ef, kTile, px2, py2, pz2, acc, kc2);
            __syncwarp();
        }
        __syncthreads();
        if (S.abort_flag) break;
        if (tid == 0 && t + kStages < tiles &&
            CC_IN_BOUNDS(CC_SITE_VOXEL_TILE, split + (t + kStages) * nsplit, ntk))
            tma_bulk_load(S.tile[stage], src + (t + kStages) * stride, kTile * sizeof(NearRec),
                          &S.full[stage]);
#pragma unroll
        for (int q = 0; q < DP; q++) {   // Kahan-compensated tile sums
            float2 yv = make_float2(acc[q].x - comp[q].x, acc[q].y - comp[q].y);
            float2 tv = make_float2(sum[q].x + yv.x, sum[q].y + yv.y);
            comp[q] = make_float2((tv.x - sum[q].x) - yv.x, (tv.y - sum[q].y) - yv.y);
            sum[q] = tv;
            acc[q] = make_float2(0.0f, 0.0f);
        }
    }
    if (S.abort_flag) {
        if (tid == 0) atomicExch(status, (int32_t)CC_ETIMEOUT);
        return;
    }
    float bv = -__builtin_huge_valf();
    int bj = INT32_MAX;
#pragma unroll
    for (int q = 0; q < DP; q++) {
        const int64_t ka = j0 + (int64_t)(64 * q), kb = ka + 32;
        const float va = sum[q].x - comp[q].x, vb = sum[q].y - comp[q].y;
        if (ka < V) {
            const int64_t ja = perm != nullptr ? (int64_t)__ldg(perm + ka) : ka;
            if (CC_IN_BOUNDS(CC_SITE_VOXEL_OUT, split * V + ja, nsplit * V)) {
                out[split * V + ja] = va;
                better(bv, bj, va, (int)ja);
            }
        }
        if (kb < V) {
            const int64_t jb = perm != nullptr ? (int64_t)__ldg(perm + kb) : kb;
            if (CC_IN_BOUNDS(CC_SITE_VOXEL_OUT, split * V + jb, nsplit * V)) {
                out[split * V + jb] = vb;
                better(bv, bj, vb, (int)jb);
            }
        }
    }
    if (bb != nullptr) {
        block_best(bv, bj);
        if (tid == 0) bb[blockIdx.x] = BlockBest{bv, bj};
    }
}

template <int D, bool KCUT>
void *bp_fn() {
    return (void *)k_backproject<D, KCUT>;
}

void *pick_bp(int d, bool kcut) {
    switch (d) {
        case 8: return kcut ? bp_fn<8, true>() : bp_fn<8, false>();
        case 4: return kcut ? bp_fn<4, true>() : bp_fn<4, false>();
        default: return kcut ? bp_fn<2, true>() : bp_fn<2, false>();
    }
}

}  // namespace

bool plan_backproject(int64_t R, int64_t V, const cc_params &p, SweepPlan *plan) {
    return plan_sweep(R, V, p, plan, 0, pick_bp, sizeof(NearRec), true);
}

int64_t universe_count(int shape, int n) {
    int64_t total = 0;
    for (long long k = 0; k < n; k++)
        for (long long j = 0; j < n; j++) {
            long long lo, hi;
            row_range(shape, n, j, k, &lo, &hi);
            total += hi - lo + 1;
        }
    return total;
}

cudaError_t launch_ring_apex(const cc_events &ev, const cc_rings &r, float *px, float *py,
                             float *pz, cudaStream_t s) {
    if (ev.count == 0) return cudaSuccess;
    int64_t blocks = (ev.count + 255) / 256;
    if (blocks > (int64_t)device_sm_count() * 16) blocks = (int64_t)device_sm_count() * 16;
    TraceScope ts(CC_STAGE_RECON, s);
    k_ring_apex<<<(unsigned)blocks, 256, 0, s>>>(ev, r.perm, r.valid, px, py, pz);
    return cudaGetLastError();
}

cudaError_t launch_universe(int shape, int n, float pitch, float cx, float cy, float cz,
                            float *x, float *y, float *z, cudaStream_t s) {
    TraceScope ts(CC_STAGE_GRID, s);
    k_universe<<<(unsigned)n, 1024, 0, s>>>(shape, n, pitch, cx, cy, cz, x, y, z);
    return cudaGetLastError();
}

cudaError_t launch_backproject(const cc_rings &rings, const float *px, const float *py,
                               const float *pz, const cc_grid &vox, const cc_params &p,
                               const SweepPlan &plan, float *image, int32_t *argmax,
                               int32_t *status, char *ws, cudaStream_t s) {
    NearRec *rec = reinterpret_cast<NearRec *>(ws + plan.off_rec);
    int32_t *cnt = reinterpret_cast<int32_t *>(ws + plan.off_packcnt);
    int64_t *nkept = reinterpret_cast<int64_t *>(ws + plan.off_nkept);
    int32_t *st = status ? status : reinterpret_cast<int32_t *>(ws + plan.off_status);
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    NearRings g{rings.ax, rings.ay, rings.az, rings.eta, rings.deta, px, py, pz, rings.valid,
                rings.count};
    {
        TraceScope ts(CC_STAGE_PACK, s, 3);   // count, scan, scatter
        k_near_count<<<(unsigned)plan.npack, 256, 0, s>>>(g, cnt);
        if ((e = launch_pack_scan(cnt, plan.npack, nkept, s)) != cudaSuccess) return e;
        k_near_scatter<<<(unsigned)plan.npack, 256, 0, s>>>(g, cnt, nkept, rec);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const bool kcut = p.k_cut > 0.0f;
    const float kc = p.k_cut * kGaussK;
    const float kc2 = kcut ? kc * kc : 0.0f;
    float *out = plan.nsplit > 1 ? reinterpret_cast<float *>(ws + plan.off_part) : image;
    BlockBest *bbk = plan.nsplit > 1 ? nullptr : reinterpret_cast<BlockBest *>(ws + plan.off_bb);
    const int64_t V = vox.count;
    const unsigned ctas = (unsigned)(plan.ndb * plan.nsplit);
    void *fn = pick_bp(plan.d, kcut);
    const NearRec *crec = rec;
    const int64_t *cnk = nkept;
    const int32_t *perm = nullptr;
    if (plan.ordered) {             // the voxels in Morton order (order.cu)
        int32_t *pm = reinterpret_cast<int32_t *>(ws + plan.off_perm);
        TraceScope ts(CC_STAGE_PACK, s, point_order_kernels(V));
        if ((e = point_order(vox.x, vox.y, vox.z, V, pm, ws + plan.off_order, s)) != cudaSuccess)
            return e;
        perm = pm;
    }
    void *args[] = {(void *)&crec,  (void *)&cnk,   (void *)&plan.nsplit, (void *)&plan.ndb,
                    (void *)&vox.x, (void *)&vox.y, (void *)&vox.z,       (void *)&perm,
                    (void *)&V,     (void *)&kc2,   (void *)&out,         (void *)&bbk,
                    (void *)&st};
    {
        TraceScope ts(CC_STAGE_VOXEL, s);
        e = cudaLaunchKernel(fn, dim3(ctas), dim3(kThreads), args, 0, s);
    }
    if (e != cudaSuccess) return e;
    return finish_localize(vox, p, plan, image, argmax, nullptr, ws, s);
}

}  // namespace cc

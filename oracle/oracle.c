/*
 * oracle.c - plain, slow, obviously correct CPU oracle for the Compton
 * ring-localisation hot path (Gameiro et al., "Towards Real Time Compton
 * Imaging in Demanding Conditions", arXiv 2411.04785).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or constant generator with the CUDA library, and it never reads a
 * value the CUDA library produced.
 *
 * What follows the paper and what is a reading of it:
 *  - Compton formula (Sec. 1.1, the displayed equation): the scattered photon
 *    energy E' = E / (1 + (E / m_e c^2)(1 - cos theta)).  Solved for the cone
 *    half-angle with E' = E2 (energy left after the first site) and
 *    E = E0 = E1 + E2: cos eta = 1 - m_e c^2 (1/E2 - 1/E0).
 *  - Cone from two interactions (Sec. 1.1): the axis joins the first two
 *    sites; cones overlap at the source.  We point the axis from the second
 *    site back through the first, a = unit(x1 - x2), so that a . s = cos eta
 *    for the true source direction s.
 *  - Back projection (Sec. 3): every (event, probe) pair contributes
 *    independently a "probability the gamma-ray came from" the probe; the
 *    contributions are summed per probe.  Far-field reading: probes are sky
 *    directions c_j and the contribution is the unnormalised Gaussian of the
 *    angular residual, exp(-r^2/2), r = (angle(a_i, c_j) - eta_i) / deta_i.
 *  - Angular selection of voxels (Sec. 3, "Angular selection"): optional
 *    cut, terms with |r| > k_cut are dropped (k_cut = 0 keeps every term).
 *  - Site ordering for 3-4 sites, the ring width deta, the argmax/top-k seeds
 *    and the Gauss-Newton refinement are not in the paper; each function
 *    below states the reading it implements.
 *
 * Parity status of each function is listed in the design notes; every function
 * here is pinned by a CPU test except the physical correctness of the 2-site
 * ordering rule (parity unpinned: only its fraction correct is reported).
 *
 * Precision: FP64 throughout, except the site-ordering DECISION, which is an
 * integer result decided by floating point; it is taken in IEEE binary32 with
 * every operation rounded once (compile with -ffp-contract=off), the same
 * precision the GPU kernel decides in, so the chosen order is comparable bit
 * for bit.  That binary32 sequence is fixed; it is pinned to the rule's
 * definition evaluated plainly in FP64 (or_order_event_f64) by a rigorous
 * bound on its rounding (or_order_check): wherever the bound decides an
 * event, the binary32 choice must be the FP64 argmin.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ME_KEV 510.99895      /* electron rest energy m_e c^2, keV (CODATA) */
#define ME_KEV_F 510.99895f
#define POS_EPS2_F 1e-12f     /* |x1 - x2|^2 below (1e-6 cm)^2: no axis */
#define INF_F ((float)INFINITY)

/* ------------------------------------------------------------------------ */
/* Site ordering: binary32 decision.                                        */
/* ------------------------------------------------------------------------ */

/* Energy of a set of sites: the deposits of the set's slots added in
 * increasing slot order, starting from 0. */
static float set_energy_f32(int k, const float *e, unsigned mask)
{
    float s = 0.0f;
    for (int m = 0; m < k; m++)
        if (mask & (1u << m))
            s = s + e[m];
    return s;
}

/* Cosine of a Compton scatter from the photon energy before (e_before) and
 * after (e_after) the scatter, by the Sec. 1.1 formula solved for cos. */
static float compton_cos_f32(float e_after, float e_before)
{
    float inv_after = 1.0f / e_after;
    float inv_before = 1.0f / e_before;
    float d = inv_after - inv_before;
    float u = ME_KEV_F * d;
    return 1.0f - u;
}

/* Squared distance between sites p and q. */
static float sqdist_f32(const float *x, const float *y, const float *z, int p,
                        int q)
{
    float dx = x[q] - x[p];
    float dy = y[q] - y[p];
    float dz = z[q] - z[p];
    float a = dx * dx;
    float b = dy * dy;
    float c = dz * dz;
    return (a + b) + c;
}

/*
 * Compton chi-square of a site order (reading of the kinematic-consistency
 * ordering; the paper treats two sites only).  The photon deposits all of its
 * energy, so the energy entering site j is the sum of the deposits from j on.
 * At each intermediate site j (not first, not last) the scatter cosine from
 * energies, cos_E = 1 - m_e c^2 (1/E_after - 1/E_before), must agree with the
 * cosine of the angle between the incoming and outgoing segments,
 * cos_G = u(x_{j-1} -> x_j) . u(x_j -> x_{j+1}), in binary32 as
 * dot(d1, d2) * ((1/sqrt|d1|^2) * (1/sqrt|d2|^2)).
 * chi2 = sum_j (cos_E - cos_G)^2, unweighted.  The order is invalid (+inf)
 * when the first-site cone is invalid (E2 <= 0, |cos eta| > 1, or sites 1
 * and 2 closer than 1e-6 cm), or when some intermediate site has no energy
 * left after it, |cos_E| > 1, or a zero-length segment.
 */
float or_order_chi2(int k, const float *x, const float *y, const float *z,
                    const float *e, const int *ord)
{
    unsigned all = (1u << k) - 1u;
    float e0 = set_energy_f32(k, e, all);
    float e2 = set_energy_f32(k, e, all & ~(1u << ord[0]));
    if (!(e0 > 0.0f) || !(e2 > 0.0f))
        return INF_F;
    float c1 = compton_cos_f32(e2, e0);
    if (!(c1 >= -1.0f && c1 <= 1.0f))
        return INF_F;
    if (!(sqdist_f32(x, y, z, ord[0], ord[1]) > POS_EPS2_F))
        return INF_F;

    float chi2 = 0.0f;
    for (int j = 1; j + 1 < k; j++) {
        unsigned before = 0;
        for (int m = j; m < k; m++)
            before |= 1u << ord[m];
        unsigned after = before & ~(1u << ord[j]);
        float eb = set_energy_f32(k, e, before);
        float ea = set_energy_f32(k, e, after);
        if (!(ea > 0.0f))
            return INF_F;
        float ce = compton_cos_f32(ea, eb);
        if (!(ce >= -1.0f && ce <= 1.0f))
            return INF_F;

        int p = ord[j - 1], q = ord[j], r = ord[j + 1];
        float ux = x[q] - x[p], uy = y[q] - y[p], uz = z[q] - z[p];
        float vx = x[r] - x[q], vy = y[r] - y[q], vz = z[r] - z[q];
        float t0 = ux * vx;
        float t1 = uy * vy;
        float t2 = uz * vz;
        float dot = (t0 + t1) + t2;
        float npq = sqdist_f32(x, y, z, p, q), nqr = sqdist_f32(x, y, z, q, r);
        if (!(npq > 0.0f) || !(nqr > 0.0f))
            return INF_F;
        /* inverse segment lengths, each 1/sqrt rounded once per operation;
         * their product is the same in either direction of the path */
        float il_pq = 1.0f / sqrtf(npq), il_qr = 1.0f / sqrtf(nqr);
        float cg = dot * (il_pq * il_qr);
        float d = ce - cg;
        chi2 = chi2 + d * d;
    }
    return chi2;
}

/* Klein-Nishina angular weight: dsigma/dOmega is proportional to
 * P^2 (P + 1/P - sin^2 eta) with P = E'/E the energy ratio. */
float or_kn_weight_f32(float P, float cos_eta)
{
    float c2 = cos_eta * cos_eta;
    float s2 = 1.0f - c2;
    float ip = 1.0f / P;
    float t = P + ip;
    float u = t - s2;
    float pp = P * P;
    return pp * u;
}

/* Next permutation in lexicographic order; returns 0 after the last one. */
static int next_permutation(int *a, int k)
{
    int i = k - 2;
    while (i >= 0 && a[i] >= a[i + 1])
        i--;
    if (i < 0)
        return 0;
    int j = k - 1;
    while (a[j] <= a[i])
        j--;
    int t = a[i];
    a[i] = a[j];
    a[j] = t;
    for (int l = i + 1, r = k - 1; l < r; l++, r--) {
        t = a[l];
        a[l] = a[r];
        a[r] = t;
    }
    return 1;
}

/*
 * Ordering rule (reading).  k = 3, 4: every one of the k! orders of the
 * slots, ranked lexicographically; the valid order with the smallest chi2
 * wins, ties going to the lowest rank.  k = 2: no intermediate site, so among
 * the kinematically valid orders the one with the larger Klein-Nishina weight
 * at its own cone angle wins (P = E2 / E0), ties going to the input order.
 */
int or_order_event(int k, const float *x, const float *y, const float *z,
                   const float *e, int *order_out, int *rank_out,
                   float *chi2_out)
{
    if (k < 2 || k > 4)
        return 0;
    if (k == 2) {
        static const int ords[2][2] = {{0, 1}, {1, 0}};
        float e0 = set_energy_f32(2, e, 3u);
        int ok[2];
        float w[2];
        for (int o = 0; o < 2; o++) {
            ok[o] = or_order_chi2(2, x, y, z, e, ords[o]) == 0.0f;
            w[o] = 0.0f;
            if (ok[o]) {
                float e2 = set_energy_f32(2, e, 3u & ~(1u << ords[o][0]));
                float c1 = compton_cos_f32(e2, e0);
                float P = e2 / e0;
                w[o] = or_kn_weight_f32(P, c1);
            }
        }
        int pick;
        if (ok[1] && (!ok[0] || w[1] > w[0]))
            pick = 1;
        else if (ok[0])
            pick = 0;
        else
            return 0;
        order_out[0] = ords[pick][0];
        order_out[1] = ords[pick][1];
        *rank_out = pick;
        if (chi2_out)
            *chi2_out = 0.0f;
        return 1;
    }

    int a[4] = {0, 1, 2, 3};
    float best = INF_F;
    int best_rank = -1;
    int rank = 0;
    do {
        float c = or_order_chi2(k, x, y, z, e, a);
        if (c < best) {
            best = c;
            best_rank = rank;
            memcpy(order_out, a, sizeof(int) * (size_t)k);
        }
        rank++;
    } while (next_permutation(a, k));
    if (best_rank < 0)
        return 0;
    *rank_out = best_rank;
    if (chi2_out)
        *chi2_out = best;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Site ordering: the definition in FP64, and how far binary32 can stray.   */
/* ------------------------------------------------------------------------ */

/*
 * The decision above is taken in binary32.  What it decides is defined in
 * real arithmetic on the same (FP32) inputs: the chi2 of each order and, for
 * two sites, the Klein-Nishina weight.  or_order_chi2_f64 / or_kn_weight_f64
 * / or_order_event_f64 evaluate that definition plainly in FP64: energies
 * summed in FP64, cos_E = 1 - m_e c^2 (1/E_after - 1/E_before) with the
 * CODATA constant, cos_G = d1 . d2 / (|d1| |d2|).  Nothing is shared with the
 * binary32 sequence.
 */
#define ME_KEV_D 510.99895
#define POS_EPS2_D 1e-12      /* (1e-6 cm)^2 */

static double set_energy_f64(int k, const float *e, unsigned mask)
{
    double s = 0.0;
    for (int m = 0; m < k; m++)
        if (mask & (1u << m))
            s += (double)e[m];
    return s;
}

static double compton_cos_f64(double e_after, double e_before)
{
    return 1.0 - ME_KEV_D * (1.0 / e_after - 1.0 / e_before);
}

static double sqdist_f64(const float *x, const float *y, const float *z,
                         int p, int q)
{
    double dx = (double)x[q] - (double)x[p];
    double dy = (double)y[q] - (double)y[p];
    double dz = (double)z[q] - (double)z[p];
    return dx * dx + dy * dy + dz * dz;
}

double or_order_chi2_f64(int k, const float *x, const float *y,
                         const float *z, const float *e, const int *ord)
{
    unsigned all = (1u << k) - 1u;
    double e0 = set_energy_f64(k, e, all);
    double e2 = set_energy_f64(k, e, all & ~(1u << ord[0]));
    if (!(e0 > 0.0) || !(e2 > 0.0))
        return INFINITY;
    double c1 = compton_cos_f64(e2, e0);
    if (!(c1 >= -1.0 && c1 <= 1.0))
        return INFINITY;
    if (!(sqdist_f64(x, y, z, ord[0], ord[1]) > POS_EPS2_D))
        return INFINITY;
    double chi2 = 0.0;
    for (int j = 1; j + 1 < k; j++) {
        unsigned before = 0;
        for (int m = j; m < k; m++)
            before |= 1u << ord[m];
        double eb = set_energy_f64(k, e, before);
        double ea = set_energy_f64(k, e, before & ~(1u << ord[j]));
        if (!(ea > 0.0))
            return INFINITY;
        double ce = compton_cos_f64(ea, eb);
        if (!(ce >= -1.0 && ce <= 1.0))
            return INFINITY;
        int p = ord[j - 1], q = ord[j], r = ord[j + 1];
        double d1[3] = {(double)x[q] - x[p], (double)y[q] - y[p], (double)z[q] - z[p]};
        double d2[3] = {(double)x[r] - x[q], (double)y[r] - y[q], (double)z[r] - z[q]};
        double n1 = sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
        double n2 = sqrt(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
        if (!(n1 > 0.0) || !(n2 > 0.0))
            return INFINITY;
        double cg = (d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2]) / (n1 * n2);
        chi2 += (ce - cg) * (ce - cg);
    }
    return chi2;
}

double or_kn_weight_f64(double P, double cos_eta)
{
    return P * P * (P + 1.0 / P - (1.0 - cos_eta * cos_eta));
}

/* The ordering rule on the FP64 definition: smallest chi2 (ties: lowest
 * rank) for k = 3, 4; larger Klein-Nishina weight (ties: input order) for
 * k = 2.  Returns the rank, or -1 when no order is valid. */
int or_order_event_f64(int k, const float *x, const float *y, const float *z,
                       const float *e)
{
    if (k < 2 || k > 4)
        return -1;
    if (k == 2) {
        static const int ords[2][2] = {{0, 1}, {1, 0}};
        double e0 = set_energy_f64(2, e, 3u), w[2];
        int ok[2];
        for (int o = 0; o < 2; o++) {
            ok[o] = or_order_chi2_f64(2, x, y, z, e, ords[o]) == 0.0;
            double e2 = (double)e[ords[o][1]];
            w[o] = ok[o] ? or_kn_weight_f64(e2 / e0, compton_cos_f64(e2, e0)) : 0.0;
        }
        if (ok[1] && (!ok[0] || w[1] > w[0]))
            return 1;
        return ok[0] ? 0 : -1;
    }
    int a[4] = {0, 1, 2, 3}, rank = 0, best_rank = -1;
    double best = INFINITY;
    do {
        double c = or_order_chi2_f64(k, x, y, z, e, a);
        if (c < best) {
            best = c;
            best_rank = rank;
        }
        rank++;
    } while (next_permutation(a, k));
    return best_rank;
}

/*
 * How far the binary32 decision can stray from the definition.  Beside each
 * intermediate value v of the binary32 sequence (in the sequence's own order
 * of operations, but with v computed in FP64) a bound e on |v32 - v| is
 * carried, where v32 is the value binary32 computes.  An IEEE binary32
 * operation returns op(a32, b32)(1 + d) + t with |d| <= 2^-24, and t = 0 for
 * addition and subtraction (gradual underflow makes them exact below the
 * normal range) and |t| <= 2^-150 for multiplication, division and square
 * root; a32 = a + da with |da| <= e_a.  The bound of a result is the worst
 * case of op over the operand intervals, plus 2^-24 times the largest
 * magnitude it can take, plus 2^-150 where t applies.  A value that might
 * overflow, or a divisor or radicand whose interval holds 0, ends the
 * analysis (BND_OUT): the bound no longer holds.  The FP64 values themselves
 * err by about 2^-29 of these bounds, covered by a factor 1.001.
 */
#define U32 (1.0 / 16777216.0)
#define TINY32 7.006492321624085e-46      /* 2^-150 */
#define MAX32 3.4028234663852886e38

typedef struct {
    double v, e;
} bv_t;

typedef struct {
    int out;
} bctx_t;

static bv_t b_rnd(bctx_t *c, double v, double ep, int tiny)
{
    double mag = fabs(v) + ep;
    if (!(mag * (1.0 + U32) < MAX32))
        c->out = 1;
    bv_t r = {v, ep + U32 * mag + (tiny ? TINY32 : 0.0)};
    return r;
}

static bv_t b_exact(double v)
{
    bv_t r = {v, 0.0};
    return r;
}

static bv_t b_add(bctx_t *c, bv_t a, bv_t b)
{
    return b_rnd(c, a.v + b.v, a.e + b.e, 0);
}

static bv_t b_sub(bctx_t *c, bv_t a, bv_t b)
{
    return b_rnd(c, a.v - b.v, a.e + b.e, 0);
}

static bv_t b_mul(bctx_t *c, bv_t a, bv_t b)
{
    return b_rnd(c, a.v * b.v, fabs(a.v) * b.e + fabs(b.v) * a.e + a.e * b.e, 1);
}

/* |1/(a + da) - 1/a| <= e_a / (|a| (|a| - e_a)) while e_a < |a| */
static bv_t b_rcp(bctx_t *c, bv_t a)
{
    if (!(a.e < fabs(a.v))) {
        c->out = 1;
        return b_exact(0.0);
    }
    return b_rnd(c, 1.0 / a.v, a.e / (fabs(a.v) * (fabs(a.v) - a.e)), 1);
}

/* |(a + da)/(b + db) - a/b| <= (|a| e_b + |b| e_a) / (|b| (|b| - e_b)) */
static bv_t b_div(bctx_t *c, bv_t a, bv_t b)
{
    if (!(b.e < fabs(b.v))) {
        c->out = 1;
        return b_exact(0.0);
    }
    double ep = (fabs(a.v) * b.e + fabs(b.v) * a.e) / (fabs(b.v) * (fabs(b.v) - b.e));
    return b_rnd(c, a.v / b.v, ep, 1);
}

/* |sqrt(a + da) - sqrt(a)| = |da| / (sqrt(a + da) + sqrt(a)) <= e_a / sqrt(a) */
static bv_t b_sqrt(bctx_t *c, bv_t a)
{
    if (!(a.v > 0.0) || !(a.e < a.v)) {
        c->out = 1;
        return b_exact(0.0);
    }
    double s = sqrt(a.v);
    return b_rnd(c, s, a.e / s, 1);
}

/* The binary32 constant m_e c^2 times a: the constant's own representation
 * error counts like an operand error. */
static bv_t b_mul_me(bctx_t *c, bv_t a)
{
    bv_t m = {ME_KEV_D, fabs((double)ME_KEV_F - ME_KEV_D)};
    return b_mul(c, m, a);
}

/* Does binary32's `v32 > t32` agree with the definition's `v > t`?  Certain
 * when v lies farther from t than its bound plus the thresholds' gap.
 * Returns 1 (both true), 0 (both false) or -1 (undecided). */
static int b_gt(bv_t a, double t, double t32)
{
    double slack = a.e + fabs(t - t32);
    if (a.v - slack > t && a.v - slack > t32)
        return 1;
    if (a.v + slack <= t && a.v + slack <= t32)
        return 0;
    return -1;
}

static int b_ge(bv_t a, double t)
{
    if (a.v - a.e >= t)
        return 1;
    if (a.v + a.e < t)
        return 0;
    return -1;
}

static int b_le(bv_t a, double t)
{
    if (a.v + a.e <= t)
        return 1;
    if (a.v - a.e > t)
        return 0;
    return -1;
}

static bv_t b_energy(bctx_t *c, int k, const float *e, unsigned mask)
{
    bv_t s = b_exact(0.0);
    for (int m = 0; m < k; m++)
        if (mask & (1u << m))
            s = b_add(c, s, b_exact((double)e[m]));
    return s;
}

static bv_t b_compton_cos(bctx_t *c, bv_t ea, bv_t eb)
{
    bv_t d = b_sub(c, b_rcp(c, ea), b_rcp(c, eb));
    return b_sub(c, b_exact(1.0), b_mul_me(c, d));
}

static bv_t b_coord_diff(bctx_t *c, const float *v, int p, int q)
{
    return b_sub(c, b_exact((double)v[q]), b_exact((double)v[p]));
}

static bv_t b_sqdist(bctx_t *c, const float *x, const float *y, const float *z,
                     int p, int q)
{
    bv_t dx = b_coord_diff(c, x, p, q), dy = b_coord_diff(c, y, p, q),
         dz = b_coord_diff(c, z, p, q);
    return b_add(c, b_add(c, b_mul(c, dx, dx), b_mul(c, dy, dy)), b_mul(c, dz, dz));
}

enum { BND_VALID = 1, BND_INVALID = 0, BND_UNDECIDED = -1, BND_OUT = -2 };

/* Validity of one order as both precisions decide it, and for a valid order
 * the chi2 (k >= 3) or the Klein-Nishina weight (k = 2) with its bound. */
static int bound_order(int k, const float *x, const float *y, const float *z,
                       const float *e, const int *ord, bv_t *val)
{
    bctx_t c = {0};
    unsigned all = (1u << k) - 1u;
    bv_t e0 = b_energy(&c, k, e, all);
    bv_t e2 = b_energy(&c, k, e, all & ~(1u << ord[0]));
#define BND_CHECK(cond)                          \
    do {                                         \
        int t_ = (cond);                         \
        if (c.out)                               \
            return BND_OUT;                      \
        if (t_ != 1)                             \
            return t_ == 0 ? BND_INVALID : BND_UNDECIDED; \
    } while (0)
    BND_CHECK(b_gt(e0, 0.0, 0.0));
    BND_CHECK(b_gt(e2, 0.0, 0.0));
    bv_t c1 = b_compton_cos(&c, e2, e0);
    BND_CHECK(b_ge(c1, -1.0));
    BND_CHECK(b_le(c1, 1.0));
    BND_CHECK(b_gt(b_sqdist(&c, x, y, z, ord[0], ord[1]), POS_EPS2_D, (double)POS_EPS2_F));
    if (k == 2) {
        bv_t P = b_div(&c, e2, e0);
        bv_t s2 = b_sub(&c, b_exact(1.0), b_mul(&c, c1, c1));
        bv_t t = b_add(&c, P, b_rcp(&c, P));
        *val = b_mul(&c, b_mul(&c, P, P), b_sub(&c, t, s2));
        return c.out ? BND_OUT : BND_VALID;
    }
    bv_t chi2 = b_exact(0.0);
    for (int j = 1; j + 1 < k; j++) {
        unsigned before = 0;
        for (int m = j; m < k; m++)
            before |= 1u << ord[m];
        bv_t eb = b_energy(&c, k, e, before);
        bv_t ea = b_energy(&c, k, e, before & ~(1u << ord[j]));
        BND_CHECK(b_gt(ea, 0.0, 0.0));
        bv_t ce = b_compton_cos(&c, ea, eb);
        BND_CHECK(b_ge(ce, -1.0));
        BND_CHECK(b_le(ce, 1.0));
        int p = ord[j - 1], q = ord[j], r = ord[j + 1];
        bv_t u[3] = {b_coord_diff(&c, x, p, q), b_coord_diff(&c, y, p, q),
                     b_coord_diff(&c, z, p, q)};
        bv_t w[3] = {b_coord_diff(&c, x, q, r), b_coord_diff(&c, y, q, r),
                     b_coord_diff(&c, z, q, r)};
        bv_t dot = b_add(&c, b_add(&c, b_mul(&c, u[0], w[0]), b_mul(&c, u[1], w[1])),
                         b_mul(&c, u[2], w[2]));
        bv_t npq = b_sqdist(&c, x, y, z, p, q), nqr = b_sqdist(&c, x, y, z, q, r);
        BND_CHECK(b_gt(npq, 0.0, 0.0));
        BND_CHECK(b_gt(nqr, 0.0, 0.0));
        bv_t il = b_mul(&c, b_rcp(&c, b_sqrt(&c, npq)), b_rcp(&c, b_sqrt(&c, nqr)));
        bv_t d = b_sub(&c, ce, b_mul(&c, dot, il));
        chi2 = b_add(&c, chi2, b_mul(&c, d, d));
    }
#undef BND_CHECK
    *val = chi2;
    return c.out ? BND_OUT : BND_VALID;
}

/* One order: its validity as both precisions decide it (1 valid, 0
 * invalid, -1 undecided, -2 outside the model) and, when valid, the value
 * (chi2, or the Klein-Nishina weight for k = 2) with its binary32 bound. */
int or_order_bound(int k, const float *x, const float *y, const float *z,
                   const float *e, const int *ord, double *val, double *bnd)
{
    bv_t v = {0.0, 0.0};
    int b = bound_order(k, x, y, z, e, ord, &v);
    *val = v.v;
    *bnd = 1.001 * v.e;
    return b;
}

/*
 * Compare the binary32 decision with the FP64 definition on a batch of
 * events (layout as or_rings_from_events, FP32 inputs).  Per event:
 * rank32 / rank64 = the rank each chooses (-1: no valid order); status
 *   0  decided: every order's validity is the same in both precisions and
 *      the definition's winner beats every other valid order by more than
 *      the two bounds together, so binary32 must choose the same order;
 *   1  near tie: the winner's margin over some order is within the bounds;
 *   2  some order's validity is within its bound of a threshold;
 *   3  outside the model (non-finite input, or a value that might overflow
 *      binary32 or make a divisor or radicand vanish);
 * margin = the smallest (gap / sum of the two bounds) over the orders the
 * winner is compared with (+inf when it has no rival).
 */
void or_order_check(int64_t count, int64_t stride, const uint8_t *n,
                    const float *x, const float *y, const float *z,
                    const float *e, int32_t *rank32, int32_t *rank64,
                    uint8_t *status, double *margin)
{
    for (int64_t i = 0; i < count; i++) {
        int k = n[i];
        float xf[4], yf[4], zf[4], ef[4];
        int finite = 1;
        for (int s = 0; s < k && s < 4; s++) {
            xf[s] = x[s * stride + i];
            yf[s] = y[s * stride + i];
            zf[s] = z[s * stride + i];
            ef[s] = e[s * stride + i];
            finite &= isfinite(xf[s]) && isfinite(yf[s]) && isfinite(zf[s]) &&
                      isfinite(ef[s]);
        }
        int ord[4], r32;
        rank32[i] = or_order_event(k, xf, yf, zf, ef, ord, &r32, NULL) ? r32 : -1;
        rank64[i] = -1;
        status[i] = 0;
        margin[i] = INFINITY;
        if (k < 2 || k > 4)
            continue;
        if (!finite) {
            status[i] = 3;
            continue;
        }
        rank64[i] = or_order_event_f64(k, xf, yf, zf, ef);

        int a[4] = {0, 1, 2, 3}, rank = 0, nv = 0, st = 0;
        bv_t vals[24];
        int ok[24];
        do {
            int b = bound_order(k, xf, yf, zf, ef, a, &vals[rank]);
            if (b == BND_OUT)
                st = 3;
            else if (b == BND_UNDECIDED && st < 2)
                st = 2;
            ok[rank] = b == BND_VALID;
            nv += ok[rank];
            rank++;
        } while (next_permutation(a, k));
        if (st == 0 && rank64[i] >= 0) {
            int w = rank64[i];
            double m = INFINITY;
            for (int o = 0; o < rank; o++) {
                if (o == w || !ok[o])
                    continue;
                /* k = 2: the larger weight wins; k >= 3: the smaller chi2 */
                double gap = k == 2 ? vals[w].v - vals[o].v : vals[o].v - vals[w].v;
                double bnd = 1.001 * (vals[w].e + vals[o].e);
                double r = bnd > 0.0 ? gap / bnd : (gap > 0.0 ? INFINITY : 0.0);
                if (r < m)
                    m = r;
            }
            margin[i] = m;
            if (!(m > 1.0))
                st = 1;
        }
        status[i] = (uint8_t)st;
    }
}

/* ------------------------------------------------------------------------ */
/* Rings (FP64).                                                            */
/* ------------------------------------------------------------------------ */

static double clampd(double v, double lo, double hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/*
 * Ring of one event from its chosen order (Sec. 1.1 formula, reading of the
 * width).  E1 = first deposit, E2 = sum of the later deposits, E0 = E1 + E2.
 * Width (reading, first-order error propagation):
 *   sigma_cos^2 = (m_e c^2)^2 [ s1^2 / E0^4 + s2^2 (1/E2^2 - 1/E0^2)^2 ],
 *   s1 = f E1, s2^2 = sum over later sites of (f e_m)^2, f = sigma_e_frac;
 *   deta_E = sigma_cos / max(sin eta, 1e-3);
 *   deta_G = sqrt(2) sigma_pos / |x1 - x2|;
 *   deta = sqrt(deta_E^2 + deta_G^2) clamped to [deta_min, deta_max].
 */
void or_rings_from_events(int64_t count, int64_t stride, const uint8_t *n,
                          const double *x, const double *y, const double *z,
                          const double *e, double sigma_e_frac,
                          double sigma_pos_cm, double deta_min,
                          double deta_max, double *ax, double *ay, double *az,
                          double *eta, double *deta, uint8_t *valid,
                          uint8_t *perm)
{
    for (int64_t i = 0; i < count; i++) {
        int k = n[i];
        ax[i] = ay[i] = az[i] = eta[i] = deta[i] = 0.0;
        valid[i] = 0;
        perm[i] = 255;
        if (k < 2 || k > 4)
            continue;
        float xf[4], yf[4], zf[4], ef[4];
        double xd[4], yd[4], zd[4], ed[4];
        for (int s = 0; s < k; s++) {
            xd[s] = x[s * stride + i];
            yd[s] = y[s * stride + i];
            zd[s] = z[s * stride + i];
            ed[s] = e[s * stride + i];
            xf[s] = (float)xd[s];
            yf[s] = (float)yd[s];
            zf[s] = (float)zd[s];
            ef[s] = (float)ed[s];
        }
        int ord[4], rank;
        if (!or_order_event(k, xf, yf, zf, ef, ord, &rank, NULL))
            continue;

        double e1 = ed[ord[0]];
        double e2 = 0.0, var2 = 0.0;
        for (int j = 1; j < k; j++) {
            e2 += ed[ord[j]];
            double sj = sigma_e_frac * ed[ord[j]];
            var2 += sj * sj;
        }
        double e0 = e1 + e2;
        double ce = clampd(1.0 - ME_KEV * (1.0 / e2 - 1.0 / e0), -1.0, 1.0);
        double th = acos(ce);

        double d[3] = {xd[ord[0]] - xd[ord[1]], yd[ord[0]] - yd[ord[1]],
                       zd[ord[0]] - zd[ord[1]]};
        double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);

        double s1 = sigma_e_frac * e1;
        double q = 1.0 / (e2 * e2) - 1.0 / (e0 * e0);
        double var_cos =
            ME_KEV * ME_KEV * (s1 * s1 / (e0 * e0 * e0 * e0) + var2 * q * q);
        double sin_eta = sin(th);
        double w_e = sqrt(var_cos) / (sin_eta > 1e-3 ? sin_eta : 1e-3);
        double w_g = sqrt(2.0) * sigma_pos_cm / len;
        double w = sqrt(w_e * w_e + w_g * w_g);

        ax[i] = d[0] / len;
        ay[i] = d[1] / len;
        az[i] = d[2] / len;
        eta[i] = th;
        deta[i] = clampd(w, deta_min, deta_max);
        valid[i] = 1;
        perm[i] = (uint8_t)rank;
    }
}

/* ------------------------------------------------------------------------ */
/* Likelihood map (FP64).                                                   */
/* ------------------------------------------------------------------------ */

/* Angle between a and c, atan2(|a x c|, a . c): the plain definition of the
 * angle, equal to acos(a . c) for unit vectors and well conditioned near 0
 * and pi. */
double or_angle(const double *a, const double *c)
{
    double cr[3] = {a[1] * c[2] - a[2] * c[1], a[2] * c[0] - a[0] * c[2],
                    a[0] * c[1] - a[1] * c[0]};
    double sn = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    double cs = a[0] * c[0] + a[1] * c[1] + a[2] * c[2];
    return atan2(sn, cs);
}

/* One ring's contribution to one direction (Sec. 3 back projection, far-field
 * Gaussian reading, optional angular selection). */
static double ring_term(double ax, double ay, double az, double eta,
                        double deta, const double *c, double k_cut)
{
    double a[3] = {ax, ay, az};
    double r = (or_angle(a, c) - eta) / deta;
    if (k_cut > 0.0 && fabs(r) > k_cut)
        return 0.0;
    return exp(-0.5 * r * r);
}

double or_likelihood(int64_t R, const double *ax, const double *ay,
                     const double *az, const double *eta, const double *deta,
                     const uint8_t *valid, const double *s, double k_cut)
{
    double L = 0.0;
    for (int64_t i = 0; i < R; i++)
        if (valid[i])
            L += ring_term(ax[i], ay[i], az[i], eta[i], deta[i], s, k_cut);
    return L;
}

void or_map(int64_t R, const double *ax, const double *ay, const double *az,
            const double *eta, const double *deta, const uint8_t *valid,
            const double *cx, const double *cy, const double *cz,
            const int64_t *idx, int64_t nidx, double k_cut, int nthreads,
            double *out)
{
    if (nthreads < 1)
        nthreads = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
    for (int64_t t = 0; t < nidx; t++) {
        int64_t j = idx ? idx[t] : t;
        double c[3] = {cx[j], cy[j], cz[j]};
        out[t] = or_likelihood(R, ax, ay, az, eta, deta, valid, c, k_cut);
    }
}

/* ------------------------------------------------------------------------ */
/* Argmax and seeds.                                                        */
/* ------------------------------------------------------------------------ */

int64_t or_argmax(int64_t M, const double *map)
{
    int64_t best = 0;
    for (int64_t j = 1; j < M; j++)
        if (map[j] > map[best])
            best = j;
    return best;
}

typedef struct {
    double v;
    int64_t j;
} vj_t;

static int cmp_vj(const void *pa, const void *pb)
{
    const vj_t *a = (const vj_t *)pa, *b = (const vj_t *)pb;
    if (a->v > b->v)
        return -1;
    if (a->v < b->v)
        return 1;
    return (a->j > b->j) - (a->j < b->j);
}

/* Seeds (reading): directions sorted by (L descending, index ascending); a
 * direction is accepted unless it lies closer than nms_rad to a seed already
 * accepted; stop after topk. */
int or_seeds(int64_t M, const double *map, const double *cx, const double *cy,
             const double *cz, int topk, double nms_rad, int64_t *seeds)
{
    vj_t *v = (vj_t *)malloc(sizeof(vj_t) * (size_t)M);
    if (!v)
        return -1;
    for (int64_t j = 0; j < M; j++) {
        v[j].v = map[j];
        v[j].j = j;
    }
    qsort(v, (size_t)M, sizeof(vj_t), cmp_vj);
    int got = 0;
    for (int64_t t = 0; t < M && got < topk; t++) {
        int64_t j = v[t].j;
        double c[3] = {cx[j], cy[j], cz[j]};
        int near = 0;
        for (int s = 0; s < got && !near; s++) {
            double d[3] = {cx[seeds[s]], cy[seeds[s]], cz[seeds[s]]};
            near = or_angle(c, d) < nms_rad;
        }
        if (!near)
            seeds[got++] = j;
    }
    free(v);
    return got;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Newton (IRLS) refinement, FP64.                                    */
/* ------------------------------------------------------------------------ */

static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void unit3(double *a)
{
    double n = sqrt(dot3(a, a));
    a[0] /= n;
    a[1] /= n;
    a[2] /= n;
}

/* Tangent basis at s: e1 = unit(s x z) (s x x when |s . z| > 0.9),
 * e2 = s x e1. */
static void tangent_basis(const double *s, double *e1, double *e2)
{
    double ref[3] = {0.0, 0.0, 1.0};
    if (fabs(s[2]) > 0.9) {
        ref[0] = 1.0;
        ref[2] = 0.0;
    }
    cross3(s, ref, e1);
    unit3(e1);
    cross3(s, e1, e2);
}

typedef struct {
    double L, n11, n12, n22, a11, a12, a22, g1, g2;
} gn_sums_t;

/* Objective and normal-equation sums at s.  r_i = (theta_i - eta_i)/deta_i,
 * w_i = exp(-r_i^2/2) (0 beyond k_cut); the Jacobian of r_i with respect to a
 * tangent-plane step (u, v) at s is J_i = -[a.e1, a.e2] / (sin theta_i deta_i)
 * (rings with sin theta_i < 1e-6 give no Jacobian).
 *   gradient:            dL = -sum w r J            (g = sum w r J)
 *   Gauss-Newton matrix: N  = sum w (1 - r^2) J J^T  (minus the Hessian of L
 *                        without the second derivatives of r)
 *   IRLS matrix:         A  = sum w J J^T            (always positive)
 * Both steps d = -N^-1 g and d = -A^-1 g have the stationary points of L as
 * their fixed points. */
static void gn_sums(int64_t R, const double *ax, const double *ay,
                    const double *az, const double *eta, const double *deta,
                    const uint8_t *valid, const double *s, const double *e1,
                    const double *e2, double k_cut, gn_sums_t *o)
{
    memset(o, 0, sizeof(*o));
    for (int64_t i = 0; i < R; i++) {
        if (!valid[i])
            continue;
        double a[3] = {ax[i], ay[i], az[i]};
        unit3(a);
        double th = or_angle(a, s);
        double r = (th - eta[i]) / deta[i];
        if (k_cut > 0.0 && fabs(r) > k_cut)
            continue;
        double w = exp(-0.5 * r * r);
        o->L += w;
        double st = sin(th);
        if (st < 1e-6)
            continue;
        double j1 = -dot3(a, e1) / (st * deta[i]);
        double j2 = -dot3(a, e2) / (st * deta[i]);
        double wn = w * (1.0 - r * r);
        o->n11 += wn * j1 * j1;
        o->n12 += wn * j1 * j2;
        o->n22 += wn * j2 * j2;
        o->a11 += w * j1 * j1;
        o->a12 += w * j1 * j2;
        o->a22 += w * j2 * j2;
        o->g1 += w * r * j1;
        o->g2 += w * r * j2;
    }
}

/*
 * Refinement of one seed (reading of "Gauss-Newton refinement of the best
 * direction"): at each iteration solve the 2x2 normal equations N d = -g with
 * the Gauss-Newton matrix N when it is positive definite (n11 > 0 and
 * det N > 0), else with the IRLS matrix A (far from a maximum, where N is
 * indefinite, A still gives an ascent direction); stop converged when
 * |d| < tol_rad; otherwise try s + d, s + d/2, ..., s + d/1024 on the tangent
 * plane (renormalised) and move to the first acceptable trial, re-basing the
 * tangent plane there.  A trial t is acceptable when L(t) is not smaller than
 * L(s), or when the slope of L along the step is still >= 0 at t, i.e. t lies
 * before the maximum of L on the step's great circle, so that L(t) > L(s)
 * for a unimodal L along it.  (A sum of many terms near 1 cannot resolve L
 * differences close to a flat maximum; the slope comes from the gradient
 * sums and stays resolvable.)  When no trial is acceptable the point is
 * stationary to working precision (converged).  Singular or non-finite
 * normal equations, or max_iter iterations, end it unconverged.
 */
static int refine_one(int64_t R, const double *ax, const double *ay,
                      const double *az, const double *eta, const double *deta,
                      const uint8_t *valid, const double *seed, double k_cut,
                      int max_iter, double tol_rad, double *s_out,
                      double *L_out, int *iters_out)
{
    double s[3] = {seed[0], seed[1], seed[2]}, e1[3], e2[3];
    unit3(s);
    tangent_basis(s, e1, e2);
    gn_sums_t cur;
    gn_sums(R, ax, ay, az, eta, deta, valid, s, e1, e2, k_cut, &cur);
    int status = -5, it;
    for (it = 0; it < max_iter; it++) {
        double m11 = cur.n11, m12 = cur.n12, m22 = cur.n22;
        double det = m11 * m22 - m12 * m12;
        if (!(m11 > 0.0) || !(det > 0.0) || !isfinite(det)) {
            m11 = cur.a11;
            m12 = cur.a12;
            m22 = cur.a22;
            det = m11 * m22 - m12 * m12;
        }
        if (!(det > 0.0) || !isfinite(det))
            break;
        double d1 = (-cur.g1 * m22 + cur.g2 * m12) / det;
        double d2 = (-cur.g2 * m11 + cur.g1 * m12) / det;
        if (!isfinite(d1) || !isfinite(d2))
            break;
        if (sqrt(d1 * d1 + d2 * d2) < tol_rad) {
            status = 0;
            it++;
            break;
        }
        int moved = 0;
        for (int h = 0; h <= 10 && !moved; h++) {
            double f = ldexp(1.0, -h);
            double t[3], te1[3], te2[3];
            for (int c = 0; c < 3; c++)
                t[c] = s[c] + f * d1 * e1[c] + f * d2 * e2[c];
            unit3(t);
            tangent_basis(t, te1, te2);
            gn_sums_t trial;
            gn_sums(R, ax, ay, az, eta, deta, valid, t, te1, te2, k_cut,
                    &trial);
            /* slope of L along D = d1 e1 + d2 e2 at t, in t's tangent plane:
             * grad L = -(g1, g2) there */
            double D[3], slope;
            for (int c = 0; c < 3; c++)
                D[c] = d1 * e1[c] + d2 * e2[c];
            slope = -(trial.g1 * dot3(D, te1) + trial.g2 * dot3(D, te2));
            if (trial.L >= cur.L || slope >= 0.0) {
                memcpy(s, t, sizeof s);
                memcpy(e1, te1, sizeof e1);
                memcpy(e2, te2, sizeof e2);
                cur = trial;
                moved = 1;
            }
        }
        if (!moved) {
            status = 0;
            it++;
            break;
        }
    }
    memcpy(s_out, s, sizeof s);
    *L_out = cur.L;
    *iters_out = it;
    return status;
}

int or_refine(int64_t R, const double *ax, const double *ay, const double *az,
              const double *eta, const double *deta, const uint8_t *valid,
              const double *seeds, int k, double k_cut, int max_iter,
              double tol_rad, double *out_dir, double *out_obj,
              int *out_iters)
{
    double best_L = -INFINITY;
    int best_status = -5;
    for (int t = 0; t < k; t++) {
        double s[3], L;
        int iters;
        int st = refine_one(R, ax, ay, az, eta, deta, valid, seeds + 3 * t,
                            k_cut, max_iter, tol_rad, s, &L, &iters);
        if (L > best_L) {
            best_L = L;
            best_status = st;
            memcpy(out_dir, s, sizeof s);
            *out_obj = L;
            *out_iters = iters;
        }
    }
    return best_status;
}

/* ------------------------------------------------------------------------ */
/* Sky grids (FP64).                                                        */
/* ------------------------------------------------------------------------ */

/* Fibonacci sphere (reading): z_i = 1 - (2i+1)/n, phi_i = i * golden angle,
 * golden angle = pi (3 - sqrt 5). */
void or_grid_fibonacci(int64_t n, double *x, double *y, double *z)
{
    const double golden = M_PI * (3.0 - sqrt(5.0));
    for (int64_t i = 0; i < n; i++) {
        double zi = 1.0 - (2.0 * (double)i + 1.0) / (double)n;
        double phi = fmod((double)i * golden, 2.0 * M_PI);
        double rho = sqrt((1.0 - zi) * (1.0 + zi));
        x[i] = rho * cos(phi);
        y[i] = rho * sin(phi);
        z[i] = zi;
    }
}

/* HEALPix pixel centres in RING order (Gorski et al. 2005): 12 nside^2
 * equal-area pixels on 4 nside - 1 iso-latitude rings.  Polar-cap ring i
 * (1 <= i < nside) holds 4i pixels at z = +-(1 - i^2/(3 nside^2)),
 * phi = (j - 1/2) pi / (2i); equatorial ring i (nside <= i <= 3 nside) holds
 * 4 nside pixels at z = (2 nside - i) 2/(3 nside), phi = (j - f) pi/(2 nside)
 * with f = 1 when i + nside is odd and 1/2 when it is even. */
int or_grid_healpix_ring(int64_t nside, double *x, double *y, double *z)
{
    if (nside < 1)
        return -1;
    int64_t npix = 12 * nside * nside;
    int64_t ncap = 2 * nside * (nside - 1);
    double n2 = (double)nside * (double)nside;
    for (int64_t p = 0; p < npix; p++) {
        double zz, one_minus_abs_z, phi;
        if (p < ncap) {
            int64_t i = (int64_t)floor((1.0 + sqrt(1.0 + 2.0 * (double)p)) / 2.0);
            int64_t j = p + 1 - 2 * i * (i - 1);
            one_minus_abs_z = (double)(i * i) / (3.0 * n2);
            zz = 1.0 - one_minus_abs_z;
            phi = M_PI / (2.0 * (double)i) * ((double)j - 0.5);
        } else if (p < npix - ncap) {
            int64_t q = p - ncap;
            int64_t i = q / (4 * nside) + nside;
            int64_t j = q % (4 * nside) + 1;
            double f = ((i + nside) & 1) ? 1.0 : 0.5;
            zz = (double)(2 * nside - i) * 2.0 / (3.0 * (double)nside);
            one_minus_abs_z = 1.0 - fabs(zz);
            phi = M_PI / (2.0 * (double)nside) * ((double)j - f);
        } else {
            int64_t q = npix - p;
            int64_t i = (int64_t)floor((1.0 + sqrt(2.0 * (double)q - 1.0)) / 2.0);
            int64_t j = 4 * i + 1 - (q - 2 * i * (i - 1));
            one_minus_abs_z = (double)(i * i) / (3.0 * n2);
            zz = -(1.0 - one_minus_abs_z);
            phi = M_PI / (2.0 * (double)i) * ((double)j - 0.5);
        }
        double rho = sqrt(one_minus_abs_z * (2.0 - one_minus_abs_z));
        x[p] = rho * cos(phi);
        y[p] = rho * sin(phi);
        z[p] = zz;
    }
    return 0;
}

/*
 * HEALPix in NESTED order (Gorski et al. 2005): pixel p lies in base face
 * f = p / nside^2; the remaining index interleaves the bits of the face
 * coordinates (ix in the even bits, iy in the odd ones).  From (f, ix, iy):
 * ring number jr = jr0(f) nside - ix - iy - 1 counted from the north pole,
 * the pixel's place in its ring jp = (jp0(f) nr + ix - iy + 1 + shift) / 2
 * with nr pixels-per-quarter-ring and shift the equatorial half-pixel
 * offset, and from those z and phi as in the RING layout.  Consecutive
 * NESTED pixels form compact patches (4^k pixels = a 2^k x 2^k block).
 */
int or_grid_healpix_nest(int64_t nside, double *x, double *y, double *z)
{
    static const int jr0[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
    static const int jp0[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};
    if (nside < 1 || (nside & (nside - 1)) != 0)
        return -1;                                   /* a power of two */
    int64_t npface = nside * nside, npix = 12 * npface;
    double n2 = (double)nside * (double)nside;
    for (int64_t p = 0; p < npix; p++) {
        int64_t f = p / npface, q = p % npface, ix = 0, iy = 0;
        for (int b = 0; (int64_t)1 << (2 * b) < npface; b++) {
            ix |= ((q >> (2 * b)) & 1) << b;
            iy |= ((q >> (2 * b + 1)) & 1) << b;
        }
        int64_t jr = jr0[f] * nside - ix - iy - 1, nr, shift = 0;
        double zz, omz;
        if (jr < nside) {
            nr = jr;
            omz = (double)(nr * nr) / (3.0 * n2);
            zz = 1.0 - omz;
        } else if (jr > 3 * nside) {
            nr = 4 * nside - jr;
            omz = (double)(nr * nr) / (3.0 * n2);
            zz = omz - 1.0;
        } else {
            nr = nside;
            zz = (double)(2 * nside - jr) * 2.0 / (3.0 * (double)nside);
            omz = 1.0 - fabs(zz);
            shift = (jr - nside) & 1;
        }
        int64_t jp = (jp0[f] * nr + ix - iy + 1 + shift) / 2;
        if (jp > 4 * nside) jp -= 4 * nside;
        if (jp < 1) jp += 4 * nside;
        double phi = ((double)jp - 0.5 * (double)(shift + 1)) * M_PI / (2.0 * (double)nr);
        double rho = sqrt(omz * (2.0 - omz));
        x[p] = rho * cos(phi);
        y[p] = rho * sin(phi);
        z[p] = zz;
    }
    return 0;
}

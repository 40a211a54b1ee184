/*
 * nearfield.c - oracle of the near-field 3D back projection (Sec. 3 of the
 * paper): every (gamma-ray, voxel) pair contributes independently, and the
 * contributions are summed into a 3D image.
 *
 * TEST INFRASTRUCTURE ONLY (same rules as oracle.c).  FP64 throughout.
 *
 * Readings (the paper states the structure, not the formulas):
 *  - A gamma-ray is its Compton cone: apex p at the first interaction, axis
 *    a = unit(x1 - x2) (from the second site back through the first), half
 *    angle eta from the energies and width deta; these are the rings of the
 *    far-field path plus the apex.
 *  - The geometric Compton angle of a voxel is the angle between the
 *    incoming direction (voxel centre -> first site) and the outgoing one
 *    (first -> second site); equivalently theta = angle(v - p, a).  It is
 *    computed here as atan2(|d x a|, d . a), d = v - p, accurate at every
 *    angle.
 *  - The contribution of a gamma-ray to a voxel, "the probability it came
 *    from the voxel centre", is the unnormalised Gaussian of the difference
 *    between the geometric and the energetic angle, exp(-r^2/2),
 *    r = (theta - eta) / deta, the same reading as the far-field map.
 *  - Angular selection of voxels (Sec. 3): with k_cut > 0 the contribution
 *    is not computed (is 0) where |r| > k_cut.
 *  - Image universes (Sec. 3, spatial optimisation): an n x n x n cube of
 *    voxels of side `pitch`, or the voxels of that cube whose centre lies in
 *    the inscribed cylinder (axis along z) or the inscribed sphere.  In
 *    half-pitch units the centre offsets are the odd integers 2i + 1 - n, so
 *    "inside" is an exact integer test.  Voxels are listed z-major, then y,
 *    then x.
 */
#include <math.h>
#include <stdint.h>

#include "oracle.h"

void or_ring_apex(int64_t count, int64_t stride, const uint8_t *n, const double *x,
                  const double *y, const double *z, const uint8_t *perm, const uint8_t *valid,
                  double *px, double *py, double *pz) {
    for (int64_t i = 0; i < count; i++) {
        px[i] = py[i] = pz[i] = 0.0;
        int k = n[i];
        if (!valid[i] || k < 2 || k > 4) continue;
        /* the perm[i]-th permutation of the slots in lexicographic order */
        int a[4] = {0, 1, 2, 3};
        for (int r = 0; r < perm[i]; r++) {
            int j = k - 2;
            while (j >= 0 && a[j] > a[j + 1]) j--;
            if (j < 0) break;
            int l = k - 1;
            while (a[l] < a[j]) l--;
            int tmp = a[j]; a[j] = a[l]; a[l] = tmp;
            for (int u = j + 1, v = k - 1; u < v; u++, v--) {
                tmp = a[u]; a[u] = a[v]; a[v] = tmp;
            }
        }
        px[i] = x[a[0] * stride + i];
        py[i] = y[a[0] * stride + i];
        pz[i] = z[a[0] * stride + i];
    }
}

static double term(double px, double py, double pz, double ax, double ay, double az, double eta,
                   double deta, double vx, double vy, double vz, double k_cut) {
    double dx = vx - px, dy = vy - py, dz = vz - pz;
    double cx = dy * az - dz * ay, cy = dz * ax - dx * az, cz = dx * ay - dy * ax;
    double theta = atan2(sqrt(cx * cx + cy * cy + cz * cz), dx * ax + dy * ay + dz * az);
    double r = (theta - eta) / deta;
    if (k_cut > 0.0 && fabs(r) > k_cut) return 0.0;
    return exp(-0.5 * r * r);
}

void or_backproject(int64_t R, const double *px, const double *py, const double *pz,
                    const double *ax, const double *ay, const double *az, const double *eta,
                    const double *deta, const uint8_t *valid, const double *vx,
                    const double *vy, const double *vz, const int64_t *idx, int64_t nidx,
                    double k_cut, int nthreads, double *out) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t q = 0; q < nidx; q++) {
        int64_t j = idx[q];
        double s = 0.0;
        for (int64_t i = 0; i < R; i++) {
            if (valid && !valid[i]) continue;
            s += term(px[i], py[i], pz[i], ax[i], ay[i], az[i], eta[i], deta[i], vx[j], vy[j],
                      vz[j], k_cut);
        }
        out[q] = s;
    }
}

int64_t or_universe(int shape, int64_t n, double pitch, double cx, double cy, double cz,
                    double *x, double *y, double *z) {
    int64_t m = 0;
    for (int64_t k = 0; k < n; k++)
        for (int64_t j = 0; j < n; j++)
            for (int64_t i = 0; i < n; i++) {
                int64_t oi = 2 * i + 1 - n, oj = 2 * j + 1 - n, ok = 2 * k + 1 - n;
                int64_t rr = oi * oi + oj * oj;
                if (shape == 1 && rr > n * n) continue;             /* cylinder */
                if (shape == 2 && rr + ok * ok > n * n) continue;   /* sphere */
                if (x) {
                    x[m] = cx + 0.5 * pitch * (double)oi;
                    y[m] = cy + 0.5 * pitch * (double)oj;
                    z[m] = cz + 0.5 * pitch * (double)ok;
                }
                m++;
            }
    return m;
}

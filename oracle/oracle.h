/*
 * oracle.h - plain CPU oracle for the Compton ring-localisation hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header or constant table with the CUDA
 * library.
 *
 * Units: keV, cm, radians.  Every floating-point input is double; callers that
 * compare against the FP32 GPU path pass the FP32 arrays widened exactly.
 *
 * Event layout (one event i of `count`, site slot s < 4):
 *   n[i] in {2,3,4}; x[s*stride + i], y[...], z[...], e[...]
 * Ring layout: ax, ay, az, eta, deta, valid, perm (one entry per event).
 */
#ifndef COMPTON_ORACLE_H
#define COMPTON_ORACLE_H
#include <stdint.h>

/* Ordering decision for one event of k sites (slots 0..k-1), taken in IEEE
 * binary32 with every operation rounded once (see oracle.c).  Returns 1 and
 * writes the chosen order (slot indices) and its lexicographic rank when some
 * order is kinematically valid, else returns 0. */
int or_order_event(int k, const float *x, const float *y, const float *z,
                   const float *e, int *order_out, int *rank_out,
                   float *chi2_out);

/* Klein-Nishina angular weight P^2 (P + 1/P - sin^2 eta), evaluated in the
 * same binary32 sequence the k = 2 ordering rule uses. */
float or_kn_weight_f32(float P, float cos_eta);

/* Compton chi-square of one given order (binary32 sequence); +inf when the
 * order is kinematically invalid.  k = 2 orders return 0 when valid. */
float or_order_chi2(int k, const float *x, const float *y, const float *z,
                    const float *e, const int *order);

/* The ordering rule's definition evaluated plainly in FP64 on the same FP32
 * inputs (no shared subexpressions with the binary32 sequence): the chi2 of
 * one order (+inf when invalid; 0 for a valid 2-site order), the
 * Klein-Nishina weight, and the chosen rank (-1: no valid order). */
double or_order_chi2_f64(int k, const float *x, const float *y,
                         const float *z, const float *e, const int *order);
double or_kn_weight_f64(double P, double cos_eta);
int or_order_event_f64(int k, const float *x, const float *y, const float *z,
                       const float *e);

/* One order's validity in both precisions (1 valid, 0 invalid, -1 within a
 * bound of a threshold, -2 outside the model) and, when valid, its chi2 (the
 * Klein-Nishina weight for k = 2) in FP64 with the bound on binary32's
 * rounding of it. */
int or_order_bound(int k, const float *x, const float *y, const float *z,
                   const float *e, const int *order, double *val, double *bnd);

/* Binary32 decision against the FP64 definition on a batch of events (FP32
 * inputs, layout of or_rings_from_events), with a rigorous bound on the
 * binary32 rounding of every order's chi2 (see oracle.c).  status: 0 decided
 * (the two ranks must agree), 1 near tie within the bounds, 2 a validity
 * threshold within its bound, 3 outside the model (non-finite or overflow). */
void or_order_check(int64_t count, int64_t stride, const uint8_t *n,
                    const float *x, const float *y, const float *z,
                    const float *e, int32_t *rank32, int32_t *rank64,
                    uint8_t *status, double *margin);

/* Rings from events (ordering, cone axis, opening angle, width). */
void or_rings_from_events(int64_t count, int64_t stride, const uint8_t *n,
                          const double *x, const double *y, const double *z,
                          const double *e, double sigma_e_frac,
                          double sigma_pos_cm, double deta_min,
                          double deta_max, double *ax, double *ay, double *az,
                          double *eta, double *deta, uint8_t *valid,
                          uint8_t *perm);

/* Angle between two (not necessarily unit) vectors. */
double or_angle(const double *a, const double *c);

/* Likelihood map L_j = sum_i valid_i * exp(-r_ij^2 / 2) for the listed
 * directions j = idx[0..nidx) (all M directions when idx is NULL, then nidx
 * must equal M).  k_cut > 0 drops terms with |r| > k_cut. */
void or_map(int64_t R, const double *ax, const double *ay, const double *az,
            const double *eta, const double *deta, const uint8_t *valid,
            const double *cx, const double *cy, const double *cz,
            const int64_t *idx, int64_t nidx, double k_cut, int nthreads,
            double *out);

/* Likelihood at one arbitrary direction s (unit vector). */
double or_likelihood(int64_t R, const double *ax, const double *ay,
                     const double *az, const double *eta, const double *deta,
                     const uint8_t *valid, const double *s, double k_cut);

/* Argmax of a map (ties -> lowest index). */
int64_t or_argmax(int64_t M, const double *map);

/* Greedy top-k seeds with angular suppression. Returns the number found. */
int or_seeds(int64_t M, const double *map, const double *cx, const double *cy,
             const double *cz, int topk, double nms_rad, int64_t *seeds);

/* Gauss-Newton (IRLS) refinement from k seed directions (k x 3, row major).
 * Returns 0 when the chosen seed converged, -5 when it hit max_iter or the
 * normal equations were singular. */
int or_refine(int64_t R, const double *ax, const double *ay, const double *az,
              const double *eta, const double *deta, const uint8_t *valid,
              const double *seeds, int k, double k_cut, int max_iter,
              double tol_rad, double *out_dir, double *out_obj,
              int *out_iters);

/* Sky grids. */
void or_grid_fibonacci(int64_t n, double *x, double *y, double *z);
int or_grid_healpix_ring(int64_t nside, double *x, double *y, double *z);
int or_grid_healpix_nest(int64_t nside, double *x, double *y, double *z);

/* Event clustering of time-sorted detections (cluster.c, Sec. 2). */
void or_maxstep_edges(const int64_t *t, int64_t N, int64_t dt_max, uint8_t *edge);
int64_t or_events_from_edges(const uint8_t *edge, const uint32_t *adc, int64_t N,
                             int32_t *event_id, int64_t *first, int32_t *count,
                             uint64_t *adc_sum);
int64_t or_fixed_window(const int64_t *t, const uint32_t *adc, int64_t N, int64_t window,
                        int64_t n_min, uint64_t adc_min, int32_t *event_id, int64_t *first,
                        int32_t *count, uint64_t *adc_sum);
/* Histogram of event amplitudes: bin = adc / bin_width, the last bin also
 * takes everything above it. */
void or_spectrum(const uint64_t *adc_sum, int64_t K, uint64_t bin_width, int32_t nbins,
                 uint64_t *hist);

/* Near-field back projection (nearfield.c, Sec. 3). */
void or_ring_apex(int64_t count, int64_t stride, const uint8_t *n, const double *x,
                  const double *y, const double *z, const uint8_t *perm, const uint8_t *valid,
                  double *px, double *py, double *pz);
void or_backproject(int64_t R, const double *px, const double *py, const double *pz,
                    const double *ax, const double *ay, const double *az, const double *eta,
                    const double *deta, const uint8_t *valid, const double *vx,
                    const double *vy, const double *vz, const int64_t *idx, int64_t nidx,
                    double k_cut, int nthreads, double *out);
/* shape 0 cube, 1 cylinder (axis z), 2 sphere; x/y/z may be NULL (count
 * only).  Returns the number of voxels. */
int64_t or_universe(int shape, int64_t n, double pitch, double cx, double cy, double cz,
                    double *x, double *y, double *z);

#endif

/*
 * compton.h - C ABI of libcompton.so, the GB300 (sm_103a) hot path of
 * far-field Compton ring localisation.
 *
 * The method (Gameiro et al., "Towards Real Time Compton Imaging in Demanding
 * Conditions", arXiv 2411.04785):
 *   - Sec. 1.1: a gamma ray scattering by theta keeps E' = E / (1 + (E/m_e c^2)
 *     (1 - cos theta)); energies and positions of two interactions give a
 *     Compton cone, and overlapping cones localise the source.
 *   - Sec. 3: back projection - every (event, probe) pair contributes
 *     independently the probability that the event came from the probe; the
 *     contributions are summed per probe.  Angular selection drops pairs
 *     whose geometric and energetic angles differ by more than a cut.
 * Far-field restatement used here: probes are sky directions c_j, each event
 * gives a ring (axis a, opening angle eta, width deta), and the map is
 *   L_j = sum_i valid_i exp(-r_ij^2 / 2),  r_ij = (angle(a_i, c_j) - eta_i) / deta_i.
 *
 * Conventions (every entry point):
 *   - Array pointers are DEVICE pointers owned by the caller, unless a
 *     comment says otherwise; the library never allocates device memory.
 *     Scratch comes from a caller-provided workspace sized by the matching
 *     *_workspace_bytes() query.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream) and is asynchronous: outputs are valid once
 *     the caller synchronises the stream.
 *   - Argument errors return CC_EINVAL synchronously and launch nothing; the
 *     message is available from cc_last_error() (per host thread).  A failed
 *     CUDA launch returns CC_ECUDA.
 *   - Errors found on the device (a bounded wait that ran out, a refinement
 *     that did not converge) are written to the `status` device word of the
 *     call (CC_OK otherwise), readable after synchronisation.
 *   - An event the method cannot turn into a ring is not an error: its ring
 *     gets valid = 0 and is skipped by localisation and refinement.
 *   - Units: keV, cm, radians.
 */
#ifndef COMPTON_H
#define COMPTON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CC_ABI_VERSION 2

typedef enum {
    CC_OK = 0,
    CC_EINVAL = -1,   /* bad argument; nothing launched */
    CC_ECUDA = -2,    /* a CUDA call failed */
    CC_ENOMEM = -3,   /* workspace smaller than the *_workspace_bytes() query */
    CC_ETIMEOUT = -4, /* a device-side bounded wait gave up (device status) */
    CC_ENOCONV = -5   /* refinement stopped before converging (device status) */
} cc_status;

/* Detector events, structure of arrays.  Event i has n[i] interaction sites
 * (2..4 are reconstructed; any other count gives an invalid ring).  Site slot
 * s < 4 of event i is at index s * stride + i of x, y, z (cm) and e (keV).
 * Slots are in no particular order.  stride >= count. */
typedef struct {
    const uint8_t *n;
    const float *x, *y, *z, *e;
    int64_t count;
    int64_t stride;
} cc_events;

/* Rings, structure of arrays, `count` entries.  (ax, ay, az) is the unit cone
 * axis pointing from the second site through the first (so a . s = cos eta
 * for the source direction s), eta the opening angle, deta the width (both
 * radians).  valid = 1 for a usable ring.  perm is the lexicographic rank of
 * the chosen site order among the n! orders of the event's slots (255 for an
 * invalid event).  As an input, valid may be NULL (all rings valid) and perm
 * is ignored. */
typedef struct {
    float *ax, *ay, *az, *eta, *deta;
    uint8_t *valid;
    uint8_t *perm;
    int64_t count;
} cc_rings;

/* Sky grid: `count` unit direction vectors (x, y, z), structure of arrays.
 * order: NULL, or this grid's direction order from cc_grid_order (device
 * int32 [count]) for cc_localize and cc_localize_static to reuse instead of
 * computing it (in their workspace) on every call; it must belong to these
 * directions. */
typedef struct {
    const float *x, *y, *z;
    int64_t count;
    const int32_t *order;
} cc_grid;

/* Parameters.  cc_params_default() fills the documented defaults. */
typedef struct {
    float sigma_e_frac;   /* 1-sigma energy resolution, fraction of a deposit (0.05) */
    float sigma_pos_cm;   /* 1-sigma position resolution per axis, cm (1.0) */
    float deta_min;       /* ring width clamp, rad (0.5 deg) */
    float deta_max;       /* ring width clamp, rad (20 deg) */
    float k_cut;          /* angular selection: drop |r| > k_cut; 0 keeps every pair (0) */
    int32_t topk;         /* number of seeds returned by cc_localize, 1..64 (1) */
    float nms_rad;        /* seeds closer than this to an accepted seed are skipped (1 deg) */
    int32_t max_iter;     /* refinement iteration limit, 1..1000 (50) */
    double tol_rad;       /* refinement stops when its step is shorter (1e-7) */
} cc_params;

/* Library ABI version (CC_ABI_VERSION). */
int32_t cc_abi_version(void);

/* Message of the last error returned on this host thread ("" if none). */
const char *cc_last_error(void);

/* Fill `p` (host pointer) with the defaults listed in cc_params. */
void cc_params_default(cc_params *p);

/*
 * Copy `count` events between two event sets (host or device; pinned host
 * memory keeps the copy asynchronous): dst events [dst_offset, +count) get
 * src events [src_offset, +count), n and the 4 slot rows of x, y, z, e (one
 * 2D copy per array, each side with its own stride).  dst's arrays are
 * written through their (const-qualified) pointers.  Needs
 * dst_offset + count <= dst->stride, src_offset + count <= src->stride.
 * Plumbing for callers that stage events (e.g. a server filling a device
 * buffer from slices of a host pool); no counterpart in the paper.
 */
cc_status cc_events_copy(const cc_events *dst, int64_t dst_offset, const cc_events *src,
                         int64_t src_offset, int64_t count, void *stream);

/*
 * Rings from events (Sec. 1.1 formula and two-interaction cone).
 * Per event: the site order is chosen by Compton-kinematic consistency (for
 * 3-4 sites the order minimising sum over intermediate sites of
 * (cos_energy - cos_geometry)^2, for 2 sites the order of larger
 * Klein-Nishina weight; ties to the lowest permutation rank), decided in IEEE
 * binary32 with every operation rounded once.  Then
 *   a = unit(x1 - x2), cos eta = 1 - m_e c^2 (1/E2 - 1/(E1 + E2)),
 * E1 the first deposit and E2 the sum of the later ones, and the width
 *   deta = clamp(sqrt(deta_E^2 + deta_G^2), deta_min, deta_max),
 *   deta_E = sigma_cos / max(sin eta, 1e-3),
 *   sigma_cos^2 = (m_e c^2)^2 [s1^2/E0^4 + s2^2 (1/E2^2 - 1/E0^2)^2],
 *   deta_G = sqrt(2) sigma_pos / |x1 - x2|.
 * `ev`, `out` and `p` are host pointers to structs of device pointers;
 * out->count must equal ev->count.  count = 0 is valid (nothing launched).
 */
cc_status cc_rings_from_events(const cc_events *ev, const cc_rings *out,
                               const cc_params *p, void *stream);

/* Workspace bytes cc_localize needs for `rings` rings and `dirs` directions
 * (0 on invalid sizes). */
size_t cc_localize_workspace_bytes(int64_t rings, int64_t dirs,
                                   const cc_params *p);

/*
 * Likelihood map, argmax and seeds (Sec. 3 back projection, far field).
 *   map[j]   = sum over valid rings of exp(-r_ij^2/2) (FP32, Kahan-compensated
 *              tile sums), r_ij as in the file header; |r| > k_cut dropped
 *              when k_cut > 0;
 *   argmax[0] = index of the largest map value (ties: lowest index);
 *   seeds[0..topk) = greedy top-k: directions in (L desc, index asc) order,
 *              skipping those within nms_rad of a seed already taken
 *              (seeds[0] = argmax; unfilled slots are -1).
 * Only valid rings with finite values and deta > 0 are swept: they are
 * compacted (in index order) before the sweep, so the sweep's time follows
 * the number of such rings, not rings->count.  The directions are swept in
 * the grid's compact order (cc_grid_order; grid->order when given, else
 * computed in the workspace), which fixes the order of the FP32 sums: the
 * map is the same bit for bit for the same rings and directions.
 * 0 <= rings->count <= 2^31 - 1 (0 gives an all-zero map), grid->count >= 1.
 * `map` [grid->count] float, `argmax` [1] int32, `seeds` [p->topk] int32
 * (may be NULL), `status` [1] int32 (may be NULL), `workspace` device
 * memory of at least cc_localize_workspace_bytes() bytes, 256-byte aligned.
 * Host pointers: rings, grid, p.
 */
cc_status cc_localize(const cc_rings *rings, const cc_grid *grid,
                      const cc_params *p, float *map, int32_t *argmax,
                      int32_t *seeds, int32_t *status, void *workspace,
                      size_t ws_bytes, void *stream);

/*
 * cc_localize without a workspace, for callers that cannot allocate device
 * memory: a detector's real-time acquisition loop that must not allocate
 * once running, or a host application whose own pool owns all device memory
 * and hands out no scratch.  The paper has no counterpart; this is a
 * deployment variant of cc_localize.
 * Same arguments, results and status as cc_localize minus the workspace: the
 * scratch is one static device array of CC_LOCALIZE_STATIC_SCRATCH_BYTES
 * bytes inside libcompton.so, held on every GPU that loads the library until
 * the process exits.  Sizes whose scratch (cc_localize_workspace_bytes) does
 * not fit are rejected with CC_EINVAL and a message; nothing is launched.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is kept per device for the life
 * of the process: after the caller resets a device (cudaDeviceReset) the
 * kept address is stale and this entry point must not be called on that
 * device again.  Every call shares the one array: calls that
 * can overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller.  The call allocates nothing: no cudaMalloc,
 * no cudaFree, no allocating library routine.
 */
#define CC_LOCALIZE_STATIC_SCRATCH_BYTES ((size_t)32 << 20)

cc_status cc_localize_static(const cc_rings *rings, const cc_grid *grid,
                             const cc_params *p, float *map, int32_t *argmax,
                             int32_t *seeds, int32_t *status, void *stream);

/*
 * Several bursts in one call (continuous batching of a serving loop): the
 * sweep of all of them runs in one launch, one CTA per work unit, the units
 * of every burst taken from a shared counter; each burst keeps its own plan,
 * rings, map and outputs, and its results do not depend on the other bursts
 * of the batch (the same burst gives the same map alone or in any batch).
 * rings [n] is a host array of ring structs; maps, argmax, seeds (may be
 * NULL), status (may be NULL) and workspaces are host arrays of n device
 * pointers; ws_bytes [n] host.  Workspace i needs
 * cc_localize_batch_workspace_bytes(rings[i].count, grid->count, p) bytes.
 * The directions are swept in grid->order when given, else in grid order
 * (nothing is computed for the order here).  1 <= n <= CC_BATCH_MAX.
 */
#define CC_BATCH_MAX 64

size_t cc_localize_batch_workspace_bytes(int64_t rings, int64_t dirs,
                                         const cc_params *p);

cc_status cc_localize_batch(int32_t n, const cc_rings *rings,
                            const cc_grid *grid, const cc_params *p,
                            float *const *maps, int32_t *const *argmax,
                            int32_t *const *seeds, int32_t *const *status,
                            void *const *workspaces, const size_t *ws_bytes,
                            void *stream);

/* Workspace bytes cc_refine needs for `rings` rings and `k` seeds. */
size_t cc_refine_workspace_bytes(int64_t rings, int32_t k);

/*
 * Gauss-Newton refinement of the best direction on the tangent plane.  From
 * each of the k seeds (seed_dirs, device, k x 3 doubles, row major): weights
 * w_i = exp(-r_i^2/2), J_i = -[a_i.e1, a_i.e2] / (sin theta_i deta_i), step d
 * from N d = -sum w r J with N = sum w (1 - r^2) J J^T (the Gauss-Newton
 * Hessian of L) when positive definite, else sum w J J^T, solved in FP64; the
 * step is tried at full, half, ..., 1/1024 length and the first acceptable
 * trial is taken (L not lower, or the slope of L along the step still >= 0
 * there); stop when |d| < tol_rad or no trial is acceptable (converged), or
 * after max_iter iterations or on singular normal equations (CC_ENOCONV in
 * status).  Per-ring terms are FP32; the sums, the accepted point and the
 * candidate double-float (FP32 pairs, ~48 bits); the 2x2 solve FP64, the
 * step FP32; the result is normalised in FP64.  Of the refined seeds the
 * one with the largest L wins (ties: lower
 * seed index): out_dir [3] double (unit), out_obj [1] double (its L),
 * out_iters [1] int32, status [1] int32 (device pointers).  1 <= k <= 64.
 */
cc_status cc_refine(const cc_rings *rings, const double *seed_dirs, int32_t k,
                    const cc_params *p, double *out_dir, double *out_obj,
                    int32_t *out_iters, int32_t *status, void *workspace,
                    size_t ws_bytes, void *stream);

/* Fibonacci sphere grid, n >= 1 directions: z_i = 1 - (2i+1)/n,
 * phi_i = i pi (3 - sqrt 5) mod 2 pi.  x, y, z: [n] float device arrays. */
cc_status cc_grid_fibonacci(int64_t n, float *x, float *y, float *z,
                            void *stream);

/* HEALPix pixel centres in RING order (Gorski et al. 2005), 12 nside^2
 * directions, 1 <= nside <= 8192.  x, y, z: [12 nside^2] float device
 * arrays. */
cc_status cc_grid_healpix_ring(int32_t nside, float *x, float *y, float *z,
                               void *stream);

/* The same pixels in NESTED order (nside a power of two, 1..8192): pixel
 * p's centre is RING pixel nest_to_ring(p)'s, bit for bit.  Consecutive
 * NESTED pixels form compact patches, so sweep blocks of them can be skipped
 * by the angular selection (p->k_cut > 0) where no ring reaches them. */
cc_status cc_grid_healpix_nest(int32_t nside, float *x, float *y, float *z,
                               void *stream);

/* The order in which cc_localize sweeps a grid's directions: the grid sorted
 * by HEALPix NESTED pixel (Gorski et al. 2005) at the coarsest nside with at
 * least count pixels, ties in index order, so that each warp's directions
 * form a compact patch (a ring whose axis is far enough from the patch then
 * lies wholly on one side of it, and its pairs skip the fold of the angle
 * formula).  A HEALPix RING grid comes out in its NESTED order.  order
 * [count] int32 device array (a permutation of 0..count-1); workspace of
 * cc_grid_order_workspace_bytes(count) bytes (device, 256-byte aligned, else
 * CC_EINVAL); grid a host pointer to device arrays. */
size_t cc_grid_order_workspace_bytes(int64_t count);
cc_status cc_grid_order(const cc_grid *grid, int32_t *order, void *workspace,
                        size_t ws_bytes, void *stream);

/* Gather k grid directions as FP64 unit vectors (e.g. seeds for
 * cc_refine): out_dirs[3t..3t+2] = grid[idx[t]], renormalised.  Negative
 * indices give (0, 0, 0).  idx [k] int32 and out_dirs [3k] double are device
 * pointers, grid a host pointer.  1 <= k <= 64. */
cc_status cc_grid_gather(const cc_grid *grid, const int32_t *idx, int32_t k,
                         double *out_dirs, void *stream);

/*
 * Learned ring filter (an extension beyond the paper: the paper's imaging
 * has no learned part).  An MLP 16 -> 128 -> 128 -> 128 -> 2 with ReLU scores
 * each ring before the sweep: out[i] = (z, v), z the source/background logit
 * and v the log of a predicted ring width.  Weights, layer inputs and
 * backward signals are BF16 (tensor cores, FP32 accumulation); biases,
 * gradients and the Adam state are FP32.  Parameters are one flat FP32 vector
 * of CC_MLP_PARAMS values, W1[128][16] b1[128] W2[128][128] b2[128]
 * W3[128][128] b3[128] W4[2][128] b4[2], with a BF16 copy (uint16_t bit
 * patterns) that the products read.  Loss per ring, averaged over the batch
 * rows (rows with weight 0 contribute 0):
 *   BCE(z, is_source) + is_source (v + residual^2 exp(-2 v) / 2),
 * the residual being the ring's angular residual to the true source.
 */
#define CC_MLP_FEATURES 16
#define CC_MLP_PARAMS 35458
#define CC_MLP_MAX_BATCH 65536

/* 16 BF16 features per ring (row-major [count][16]) from its event and its
 * ring (valid, perm, eta, deta, az): eta/pi, cos eta, sin eta, log(deta)/4,
 * [k=2], [k=3], [k=4], log(E0/500 keV), E1/E0, E_2nd/E0, E_last/E0,
 * log(|x1-x2|/5 cm), a_z, z1/30 cm, z2/30 cm, sqrt(2) sigma_pos/|x1-x2|/deta.
 * Invalid rings get zeros.  rings->count == ev->count. */
cc_status cc_ring_features(const cc_events *ev, const cc_rings *rings,
                           const cc_params *p, uint16_t *features, void *stream);

/* Workspace bytes of cc_mlp_grad for `rows` rows. */
size_t cc_mlp_workspace_bytes(int64_t rows);

/* out [rows][2] = MLP(features); any number of rows.  features [rows][16]
 * BF16 and params_bf16 16-byte aligned, out 8-byte aligned (else
 * CC_EINVAL).  Runs on the tcgen05 tensor cores (FP32 accumulation, BF16
 * activations); a row whose computation could not finish reads NaN.  The
 * workspace is not used (may be NULL). */
cc_status cc_mlp_forward(const float *params, const uint16_t *params_bf16,
                         const uint16_t *features, int64_t rows, float *out,
                         void *workspace, size_t ws_bytes, void *stream);

/* Loss (device [1]) and its gradient (device [CC_MLP_PARAMS]) for one batch
 * of 1..CC_MLP_MAX_BATCH rows: is_source [rows] u8, residual [rows] f32 (rad),
 * weight [rows] u8 (0 excludes a row).  features and params_bf16 16-byte
 * aligned.  The forward pass runs on the tcgen05 kernel of cc_mlp_forward,
 * the backward pass on tcgen05 kernels as well.  Deterministic
 * (fixed-order sums). */
cc_status cc_mlp_grad(const float *params, const uint16_t *params_bf16,
                      const uint16_t *features, const uint8_t *is_source,
                      const float *residual, const uint8_t *weight,
                      int64_t rows, float *grad, float *loss, void *workspace,
                      size_t ws_bytes, void *stream);

/* cc_mlp_grad keeping the step's intermediate values, for inspecting a
 * training step and checking each of its stages on its own: hidden
 * [3][rows][128] BF16 the activations H1..H3 (each layer's ReLU output, the
 * next layer's input), out [rows][2] FP32 the network outputs, dout [rows][2]
 * BF16 the loss gradient at the outputs, signals [3][rows][128] BF16 the
 * backward signal at each hidden layer's pre-activation (dZ1..dZ3, the
 * ReLU-gated products that the weight gradients multiply).  Any of the four
 * may be NULL (not kept); hidden and signals 16-byte aligned, out 8, dout 4.
 * Same results as cc_mlp_grad, bit for bit. */
cc_status cc_mlp_grad_trace(const float *params, const uint16_t *params_bf16,
                            const uint16_t *features, const uint8_t *is_source,
                            const float *residual, const uint8_t *weight, int64_t rows,
                            float *grad, float *loss, void *workspace, size_t ws_bytes,
                            uint16_t *hidden, float *out, uint16_t *dout, uint16_t *signals,
                            void *stream);

/* One Adam step (step >= 1) on params with moments m, v; refreshes the BF16
 * copy. */
cc_status cc_mlp_adam(float *params, float *m, float *v, const float *grad,
                      uint16_t *params_bf16, int32_t step, float lr,
                      float beta1, float beta2, float eps, void *stream);

/* params_bf16 = bf16(params). */
cc_status cc_mlp_params_to_bf16(const float *params, uint16_t *params_bf16,
                                void *stream);

/* Filter rings in place with the MLP output: a valid ring stays valid when
 * sigmoid(z) >= tau, and its width becomes clamp(exp(v), deta_min,
 * deta_max). */
cc_status cc_mlp_apply_filter(const float *out, const cc_rings *rings,
                              float tau, float deta_min, float deta_max,
                              void *stream);

/*
 * Event clustering of monolithic-scintillator detections (Sec. 2 of the
 * paper: events delimited by a maximum step between consecutive detections).
 *
 * Detections, sorted by time (non-decreasing t): t [count] int64 time stamps
 * in any tick unit, 8-byte aligned; adc [count] uint32 amplitudes (ADC
 * channels), 4-byte aligned, may be NULL when no amplitude sums are asked for.
 * Device pointers, owned by the caller.
 */
typedef struct {
    const int64_t *t;
    const uint32_t *adc;
    int64_t count;
} cc_detections;

/* Workspace bytes of cc_cluster_maxstep for `count` detections. */
size_t cc_cluster_workspace_bytes(int64_t count);

/*
 * Max-step clustering (Sec. 2): with M_i = (t[i+1] - t[i] < dt_max) the mask
 * of the step after detection i (no step before the first or after the last
 * detection: false), the edge of detection i is
 *   edge[i] = M_{i-1} XOR M_i                      (uint8, the paper's E)
 * and a run of detections joined by masked steps is one event.  Events are
 * numbered 0, 1, ... in time order:
 *   event_id[i]  event of detection i, -1 for an isolated detection (int32)
 *   ev_first[k]  index of event k's first detection (int64)
 *   ev_count[k]  its number of detections, >= 2 (int32)
 *   ev_adc[k]    the sum of its amplitudes (uint64, exact)
 *   n_events[0]  the number of events (int64, written on the device)
 * Steps are taken in wrapping 64-bit arithmetic (meaningful for |step| <
 * 2^63); unsorted input is not an error, a negative step simply counts as
 * below dt_max.  Every output pointer may be NULL (not written); the per-event
 * arrays hold ev_capacity >= count / 2 entries (the most events count
 * detections can make).  status [1] int32 (may be NULL) receives
 * CC_ETIMEOUT if a bounded wait between CTAs gave up (no result is then
 * valid).  0 <= count <= 2^31 - 1; count = 0 writes n_events = 0.  Workspace:
 * cc_cluster_workspace_bytes(count) bytes, 256-byte aligned.  One kernel
 * launch; asynchronous on `stream`.
 */
cc_status cc_cluster_maxstep(const cc_detections *d, int64_t dt_max, uint8_t *edge,
                             int32_t *event_id, int64_t *ev_first, int32_t *ev_count,
                             uint64_t *ev_adc, int64_t ev_capacity, int64_t *n_events,
                             int32_t *status, void *workspace, size_t ws_bytes,
                             void *stream);

/*
 * Amplitude spectrum of the events (the validation of Sec. 2): hist[b]
 * (uint64 [nbins], device) counts the events with ev_adc / bin_width == b,
 * the last bin also those above it.  n_events is the device count written by
 * cc_cluster_maxstep.  bin_width >= 1, nbins >= 1.
 */
cc_status cc_cluster_spectrum(const uint64_t *ev_adc, const int64_t *n_events,
                              uint64_t bin_width, int32_t nbins, uint64_t *hist,
                              void *stream);

/*
 * Near-field 3D back projection (Sec. 3 of the paper): every (gamma-ray,
 * voxel) pair contributes "the probability the gamma-ray came from the voxel
 * centre", summed per voxel into an image.
 *
 * A gamma-ray is its ring (cone axis a, energetic half angle eta, width deta,
 * as cc_rings_from_events builds them) plus the cone's apex p, the first
 * interaction site of the chosen order.  For voxel centre v the geometric
 * Compton angle is theta = angle(v - p, a), the angle between the incoming
 * direction (voxel -> first site) and the outgoing one (first -> second
 * site), and the contribution is exp(-r^2/2), r = (theta - eta)/deta, left
 * out for |r| > k_cut when p->k_cut > 0 (the angular selection of voxels).
 */

/* Apex of every ring: (px, py, pz)[i] = position of the first site of ring
 * i's chosen order (rings->perm); 0 for invalid rings.  Device arrays of
 * ev->count floats; rings->count == ev->count. */
cc_status cc_ring_apex(const cc_events *ev, const cc_rings *rings, float *px,
                       float *py, float *pz, void *stream);

/* Image universes (Sec. 3, spatial optimisation): the n^3 voxels of side
 * `pitch` of a cube centred on (cx, cy, cz) (shape 0), or those whose centres
 * lie in the inscribed cylinder with axis along z (shape 1, about pi/4 of the
 * cube) or the inscribed sphere (shape 2, about pi/6).  Voxel (i, j, k) has
 * centre c + pitch/2 (2i+1-n, 2j+1-n, 2k+1-n), computed in FP64 and rounded
 * once to FP32; "inside" is the exact integer test on those odd offsets
 * (sum of squares <= n^2).  Voxels are listed z-major, then y, then x.
 * cc_voxel_count returns their number (host arithmetic, no GPU; -1 for bad
 * arguments); cc_voxel_universe writes them to device arrays x, y, z of that
 * length.  1 <= n <= CC_VOXEL_MAX_N. */
#define CC_VOXEL_MAX_N 1024
int64_t cc_voxel_count(int32_t shape, int32_t n);
cc_status cc_voxel_universe(int32_t shape, int32_t n, float pitch, float cx,
                            float cy, float cz, float *x, float *y, float *z,
                            void *stream);

/* Workspace bytes of cc_backproject (0 for bad arguments or no device). */
size_t cc_backproject_workspace_bytes(int64_t rings, int64_t voxels,
                                      const cc_params *p);

/*
 * The back projection: image[v] = sum over valid rings with finite values
 * and deta > 0 of exp(-r^2/2) (FP32, Kahan-compensated 128-ring tile sums,
 * fixed-order split reduction), r as above; argmax[0] = the voxel with the
 * largest value (ties: lowest index).  Rings are compacted before the sweep,
 * so its time follows the kept rings.  rings: as from cc_rings_from_events;
 * px, py, pz: apexes [rings->count]; voxels: centres (any layout, e.g. from
 * cc_voxel_universe), 1 <= voxels->count <= 2^31 - 1; image [voxels->count]
 * float, argmax [1] int32, status [1] int32 (may be NULL; CC_ETIMEOUT if a
 * bounded wait gave up).  A voxel centre that coincides with an apex is a
 * degenerate pair with a finite but unspecified contribution.  Workspace:
 * cc_backproject_workspace_bytes() bytes, 256-byte aligned.  All pointers
 * but rings, voxels and p are device pointers; asynchronous on `stream`.
 */
cc_status cc_backproject(const cc_rings *rings, const float *px, const float *py,
                         const float *pz, const cc_grid *voxels, const cc_params *p,
                         float *image, int32_t *argmax, int32_t *status,
                         void *workspace, size_t ws_bytes, void *stream);

/*
 * Self-check of the correctly rounded reciprocal, square root and quotient
 * that the ordering decision uses (no counterpart in the paper; it backs the
 * bit-exact ordering): on every float of [1, 4), mismatches[0] counts
 * results that differ from __frcp_rn, mismatches[1] from __fsqrt_rn; on
 * every float x of [1, 2) and 64 divisors d of [1, 2), mismatches[2] counts
 * quotients x/d and d/x that differ from __fdiv_rn.  mismatches: device
 * uint64 [3].  Asynchronous on `stream`.
 */
cc_status cc_selftest_exact_ops(uint64_t *mismatches, void *stream);

/*
 * Self-check of failure detection (no counterpart in the paper): runs one of
 * the library's bounded device waits against a signal that never comes and
 * writes the outcome to status (device int32 [1]): CC_ETIMEOUT once limit_ns
 * has passed.  which = 0: an mbarrier phase (the wait of the TMA and
 * tensor-core pipelines); which = 1: a global counter (the refinement's grid
 * barrier).  counter: device uint32 [1] of scratch.  limit_ns in
 * [1000, 10^10] (the library's own waits give up after 2 s).  The context
 * stays usable.  Asynchronous on `stream`; CC_EINVAL on bad arguments.
 */
cc_status cc_selftest_wait_timeout(int32_t which, int64_t limit_ns, uint32_t *counter,
                                   int32_t *status, void *stream);

/*
 * Index bounds checks of the debug build (no counterpart in the paper; a
 * stand-in for a memory checker).  The library built with
 * build(debug=True) (libcompton_debug.so) compares the index of each checked
 * global access - the reconstruction's event and ring arrays and bulk copies,
 * the ring records, tiles, partial and final maps of the sweeps, the block
 * bests, the refinement's rings and partial sums, the grids, the
 * clustering's outputs and the ring filter's GEMM outputs - with the bound of
 * its buffer.  Out of bounds, the first failure is recorded in one device
 * word, site << 48 | (index & (2^48 - 1)) with the sites of the CC_SITE_*
 * list in the library's internal header, and the access is skipped, so the
 * kernel runs on.
 * cc_debug_bounds: *word (host uint64) = the recorded word, 0 if no check
 * failed; reset != 0 clears it.  Synchronous (waits for the device).
 * cc_debug_selftest_bounds: launches a kernel whose one checked access asks
 * for element n of a device int32 buffer `buf` of n elements; the check
 * records (0x7fff, n) and skips the access.  Asynchronous on `stream`.
 * In the normal build both return CC_EINVAL ("not a debug build") and
 * launch nothing.
 */
cc_status cc_debug_bounds(uint64_t *word, int32_t reset);
cc_status cc_debug_selftest_bounds(int32_t *buf, int64_t n, void *stream);

/*
 * Stage tracing (CUDA events on the caller's stream).  Every kernel launch is
 * counted per stage; when tracing is enabled each launch is also bracketed by
 * two CUDA events recorded on the launching stream, and cc_trace_read()
 * waits for the recorded events and adds their elapsed time.  Host-side,
 * process-wide, thread-safe.
 */
typedef enum {
    CC_STAGE_RECON = 0,   /* rings from events */
    CC_STAGE_PACK = 1,    /* ring repacking for the sweep */
    CC_STAGE_SWEEP = 2,   /* ring x direction sweep (+ block argmax) */
    CC_STAGE_REDUCE = 3,  /* split-ring partial-map reduction */
    CC_STAGE_SELECT = 4,  /* argmax and seeds */
    CC_STAGE_GATHER = 5,  /* grid gather */
    CC_STAGE_REFINE = 6,  /* Gauss-Newton refinement */
    CC_STAGE_GRID = 7,    /* grid generation */
    CC_STAGE_MLP = 8,     /* learned ring filter (features, MLP, training, filter) */
    CC_STAGE_CLUSTER = 9, /* event clustering of detections and its spectrum */
    CC_STAGE_VOXEL = 10,  /* near-field back-projection sweep */
    CC_STAGE_COUNT = 11
} cc_stage;

typedef struct {
    int64_t launches; /* kernels launched in this stage */
    double ms;        /* summed event time (only while tracing is enabled) */
} cc_stage_time;

/* Enable (on != 0) or disable event timing. */
cc_status cc_trace_enable(int32_t on);

/* Copy min(n, CC_STAGE_COUNT) stage records into `out` (host array); with
 * reset != 0 clear them afterwards.  Synchronises on pending events. */
cc_status cc_trace_read(cc_stage_time *out, int32_t n, int32_t reset);

#ifdef __cplusplus
}
#endif

#endif /* COMPTON_H */

// cc_internal.cuh - declarations shared by the CUDA translation units of
// libcompton.so (kernels, launch planning, error state).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/compton.h"

namespace cc {

// electron rest energy m_e c^2, keV (CODATA)
constexpr float kMeKeV = 510.99895f;
constexpr float kPiF = 3.14159265358979323846f;

// ---------------------------------------------------------------------------
// error state (per host thread) - capi.cu
// ---------------------------------------------------------------------------
cc_status fail(cc_status st, const char *fmt, ...);
void clear_error();
cc_status cuda_fail(cudaError_t e, const char *what);
int device_sm_count();

// Bounded waits on the device give up after this long (ns) and report
// CC_ETIMEOUT instead of hanging.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// ---------------------------------------------------------------------------
// Index bounds checks of the debug build (build(debug=True): -DCC_DEBUG_BOUNDS,
// relocatable device code).  A checked access first compares its index with
// the bound of the buffer it touches; out of bounds, the first such failure is
// recorded in one device word (site << 48 | low 48 bits of the index) and the
// access is skipped, so the kernel runs on and the host reads the word
// (cc_debug_bounds) instead of meeting a fault.  The normal build compiles
// every check to `true`.
// ---------------------------------------------------------------------------
enum : int {
    CC_SITE_RECON_N = 1, CC_SITE_RECON_SITES, CC_SITE_RECON_BULK, CC_SITE_RECON_RING,
    CC_SITE_PACK_REC, CC_SITE_SWEEP_TILE, CC_SITE_SWEEP_OUT, CC_SITE_SWEEP_BB,
    CC_SITE_REDUCE_PART, CC_SITE_SELECT_BB, CC_SITE_SELECT_SEED, CC_SITE_REFINE_RING,
    CC_SITE_REFINE_SLOT, CC_SITE_GRID_OUT, CC_SITE_CLUSTER_IN, CC_SITE_CLUSTER_OUT,
    CC_SITE_CLUSTER_EVENT, CC_SITE_VOXEL_TILE, CC_SITE_VOXEL_OUT, CC_SITE_MLP_GEMM_OUT,
    CC_SITE_MLP_ROWS, CC_SITE_ORDER, CC_SITE_SELFTEST = 0x7fff
};

#ifdef CC_DEBUG_BOUNDS
extern __device__ unsigned long long cc_oob_word;
__device__ __forceinline__ bool in_bounds(int site, int64_t i, int64_t n) {
    if (i >= 0 && i < n) return true;
    const unsigned long long w = ((unsigned long long)(site & 0xffff) << 48) |
                                 ((unsigned long long)i & 0xffffffffffffull);
    atomicCAS(&cc_oob_word, 0ull, w);
    return false;
}
#define CC_IN_BOUNDS(site, i, n) (::cc::in_bounds((site), (int64_t)(i), (int64_t)(n)))
#else
#define CC_IN_BOUNDS(site, i, n) true
#endif

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// reconstruction - recon.cu
// ---------------------------------------------------------------------------
cudaError_t launch_rings_from_events(const cc_events &ev, const cc_rings &out,
                                     const cc_params &p, cudaStream_t s);

// ---------------------------------------------------------------------------
// sweep / argmax / seeds - sweep.cu
// ---------------------------------------------------------------------------
// Packed ring record of the sweep, 48 bytes: axis pre-scaled by 1/sqrt(2),
// k = sqrt(log2(e)/2)/deta, nb = -eta' k, nb2 = -(pi - eta') k,
// ne = (pi/2 - eta') k, where (axis, eta') is the ring mirrored to
// eta' <= pi/2 when needed.  Values that meet a pair of directions are stored
// twice so that they load as ready FP32x2 operands.
struct __align__(16) RingRec {
    float ax, ax_, ay, ay_;
    float az, az_, k, k_;
    float nb, nb2, ne, ne_;
};

struct BlockBest {
    float v;
    int32_t j;
};

struct SweepPlan {
    int d;             // directions per thread (1, 2, 4, 8)
    int threads;       // CTA size
    int64_t tile;      // rings per shared-memory tile
    int64_t tiles;     // tiles per split at most (split s takes tiles s, s + nsplit, ...)
    int64_t nsplit;    // ring splits (partial maps when > 1)
    int64_t ndb;       // direction blocks
    int64_t rpad;      // padded ring count = tiles * nsplit * tile
    int64_t nbb;       // block-best entries
    int64_t npack;     // blocks of the ring compaction
    bool ordered;      // directions swept in their compact order (order.cu)
    // workspace byte offsets
    size_t off_rec, off_part, off_bb, off_status, off_counter, off_nkept, off_packcnt, off_perm,
        off_order, bytes;
};

// force_d = 0 lets the planner pick the directions per thread and sweeps the
// directions in their compact order; the batched path fixes it so that
// bursts share one kernel instantiation, and keeps the grid's own order.
// `pick` returns the sweep kernel for (directions per thread, k_cut on) whose
// occupancy the plan sizes the grid for (NULL: the far-field sweep, which
// sweeps its directions in their compact order; `ordered` asks the same
// workspace for another sweep).
typedef void *(*SweepPick)(int d, bool kcut);
bool plan_sweep(int64_t R, int64_t M, const cc_params &p, SweepPlan *plan, int force_d = 0,
                SweepPick pick = nullptr, size_t rec_bytes = sizeof(RingRec),
                bool ordered = false);
// Ring compaction shared by the sweeps: blocks of kPackChunk rings are
// counted, the counts are scanned into block offsets (in place) and the total
// is written to *nkept; the plan's split reduction, argmax and seeds follow a
// sweep through finish_localize (probe coordinates in `grid`).
constexpr int kPackChunk = 512;
cudaError_t launch_pack_scan(int32_t *blockcnt, int64_t nblk, int64_t *nkept, cudaStream_t s);
// Compact traversal order of a grid's directions (order.cu): perm[k] is the
// k-th direction swept; scratch of direction_order_bytes(count) bytes.  The
// same for a set of points in space (Morton order: point_order, same scratch).
size_t direction_order_bytes(int64_t M);
cudaError_t direction_order(const cc_grid &g, int32_t *perm, char *scratch, cudaStream_t s);
cudaError_t point_order(const float *x, const float *y, const float *z, int64_t M, int32_t *perm,
                        char *scratch, cudaStream_t s);
int direction_order_kernels(int64_t M);   // kernels one call launches
int point_order_kernels(int64_t M);
cudaError_t finish_localize(const cc_grid &grid, const cc_params &p, const SweepPlan &plan,
                            float *map, int32_t *argmax, int32_t *seeds, char *ws,
                            cudaStream_t s);
cudaError_t launch_localize(const cc_rings &rings, const cc_grid &grid,
                            const cc_params &p, const SweepPlan &plan,
                            float *map, int32_t *argmax, int32_t *seeds,
                            int32_t *status, char *ws, cudaStream_t s);
constexpr int kBatchD = 8;   // directions per thread of the batched sweep
cudaError_t launch_localize_batch(int n, const cc_rings *rings, const cc_grid &grid,
                                  const cc_params &p, const SweepPlan *plans, float *const *maps,
                                  int32_t *const *argmax, int32_t *const *seeds,
                                  int32_t *const *status, char *const *ws, cudaStream_t s);

// ---------------------------------------------------------------------------
// refinement - refine.cu
// ---------------------------------------------------------------------------
size_t refine_workspace_bytes(int64_t R, int k);
cudaError_t launch_refine(const cc_rings &rings, const double *seeds, int k,
                          const cc_params &p, double *out_dir, double *out_obj,
                          int32_t *out_iters, int32_t *status, char *ws,
                          size_t ws_bytes, cudaStream_t s);

// ---------------------------------------------------------------------------
// grids - grid.cu
// ---------------------------------------------------------------------------
cudaError_t launch_grid_fibonacci(int64_t n, float *x, float *y, float *z,
                                  cudaStream_t s);
cudaError_t launch_grid_healpix(int32_t nside, float *x, float *y, float *z,
                                cudaStream_t s);
cudaError_t launch_grid_healpix_nest(int32_t nside, float *x, float *y, float *z,
                                     cudaStream_t s);
cudaError_t launch_grid_gather(const cc_grid &g, const int32_t *idx, int k,
                               double *out, cudaStream_t s);

// ---------------------------------------------------------------------------
// learned ring filter - mlp.cu
// ---------------------------------------------------------------------------
size_t mlp_workspace_bytes(int64_t rows);
cudaError_t mlp_features(const cc_events &ev, const cc_rings &r, float sig_pos, uint16_t *F,
                         cudaStream_t s);
cudaError_t mlp_forward(const float *params, const uint16_t *wb, const uint16_t *F, int64_t R,
                        float *out, char *ws, cudaStream_t s);
// Where a training step keeps its intermediate values (each may be null):
// the hidden activations H1..H3 [3][B][128], the outputs [B][2], their
// gradient d_out [B][2] and the backward signal of each hidden layer
// dZ1..dZ3 [3][B][128].
struct MlpTrace {
    uint16_t *hidden;
    float *out;
    uint16_t *dout;
    uint16_t *signals;
};
cudaError_t mlp_grad(const float *params, const uint16_t *wb, const uint16_t *F,
                     const uint8_t *y, const float *res, const uint8_t *wv, int64_t B,
                     float *grad, float *loss, char *ws, const MlpTrace *trace,
                     cudaStream_t s);
cudaError_t mlp_adam(float *p, float *m, float *v, const float *g, uint16_t *wb, int32_t t,
                     float lr, float b1, float b2, float eps, cudaStream_t s);
cudaError_t mlp_params_to_bf16(const float *p, uint16_t *wb, cudaStream_t s);
cudaError_t mlp_apply_filter(const float *out, const cc_rings &r, float tau, float dmin,
                             float dmax, cudaStream_t s);

cudaError_t launch_selftest_exact(uint64_t *bad, cudaStream_t s);   // recon.cu
cudaError_t launch_selftest_wait(int which, int64_t limit_ns, uint32_t *counter, int32_t *status,
                                 cudaStream_t s);                    // selftest.cu
#ifdef CC_DEBUG_BOUNDS
cudaError_t launch_selftest_bounds(int32_t *buf, int64_t n, cudaStream_t s);   // selftest.cu
#endif

// ---------------------------------------------------------------------------
// event clustering of detections - cluster.cu
// ---------------------------------------------------------------------------
size_t cluster_workspace_bytes(int64_t n);
cudaError_t launch_cluster(const int64_t *t, const uint32_t *adc, int64_t n, int64_t dt_max,
                           uint8_t *edge, int32_t *event_id, int64_t *ev_first, int32_t *ev_count,
                           uint64_t *ev_adc, int64_t *n_events, int32_t *status, char *ws,
                           cudaStream_t s);
cudaError_t launch_spectrum(const uint64_t *ev_adc, const int64_t *n_events, uint64_t bin_width,
                            int32_t nbins, uint64_t *hist, cudaStream_t s);

// ---------------------------------------------------------------------------
// near-field back projection - voxel.cu
// ---------------------------------------------------------------------------
bool plan_backproject(int64_t R, int64_t V, const cc_params &p, SweepPlan *plan);
int64_t universe_count(int shape, int n);
cudaError_t launch_ring_apex(const cc_events &ev, const cc_rings &r, float *px, float *py,
                             float *pz, cudaStream_t s);
cudaError_t launch_universe(int shape, int n, float pitch, float cx, float cy, float cz,
                            float *x, float *y, float *z, cudaStream_t s);
cudaError_t launch_backproject(const cc_rings &rings, const float *px, const float *py,
                               const float *pz, const cc_grid &vox, const cc_params &p,
                               const SweepPlan &plan, float *image, int32_t *argmax,
                               int32_t *status, char *ws, cudaStream_t s);

// ---------------------------------------------------------------------------
// stage tracing - trace.cu.  Construct before the scope's kernel launches
// (`kernels` of them), destroy after them.
// ---------------------------------------------------------------------------
class TraceScope {
  public:
    TraceScope(int stage, cudaStream_t s, int kernels = 1);
    ~TraceScope();

  private:
    int stage_;
    cudaStream_t s_;
    cudaEvent_t a_ = nullptr;
};

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace cc

// capi.cu - the extern "C" entry points of libcompton.so: argument checks,
// workspace planning, per-thread error messages.  Every entry point either
// returns CC_EINVAL before launching anything, or enqueues its kernels on the
// caller's stream and returns CC_OK / CC_ECUDA.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "cc_internal.cuh"

namespace cc {

static thread_local char g_err[512] = "";

cc_status fail(cc_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

void clear_error() { g_err[0] = 0; }

cc_status cuda_fail(cudaError_t e, const char *what) {
    return fail(CC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int device_sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

static bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

static cc_status check_params(const cc_params *p) {
    if (!p) return fail(CC_EINVAL, "params is NULL");
    if (!(p->k_cut >= 0.0f)) return fail(CC_EINVAL, "k_cut must be >= 0");
    if (p->topk < 1 || p->topk > 64) return fail(CC_EINVAL, "topk must be in 1..64");
    if (!(p->nms_rad >= 0.0f)) return fail(CC_EINVAL, "nms_rad must be >= 0");
    if (p->max_iter < 1 || p->max_iter > 1000)
        return fail(CC_EINVAL, "max_iter must be in 1..1000");
    if (!(p->tol_rad >= 0.0)) return fail(CC_EINVAL, "tol_rad must be >= 0");
    if (!(p->deta_min > 0.0f) || !(p->deta_max >= p->deta_min))
        return fail(CC_EINVAL, "need 0 < deta_min <= deta_max");
    if (!(p->sigma_e_frac >= 0.0f) || !(p->sigma_pos_cm >= 0.0f))
        return fail(CC_EINVAL, "resolutions must be >= 0");
    return CC_OK;
}

static cc_status check_rings_in(const cc_rings *r) {
    if (!r) return fail(CC_EINVAL, "rings is NULL");
    if (r->count < 0) return fail(CC_EINVAL, "rings->count < 0");
    if (r->count > INT32_MAX) return fail(CC_EINVAL, "rings->count > 2^31 - 1");
    if (r->count > 0 && (!r->ax || !r->ay || !r->az || !r->eta || !r->deta))
        return fail(CC_EINVAL, "ring arrays must be non-NULL");
    return CC_OK;
}

}  // namespace cc

using namespace cc;

extern "C" {

int32_t cc_abi_version(void) { return CC_ABI_VERSION; }

const char *cc_last_error(void) { return g_err; }

void cc_params_default(cc_params *p) {
    if (!p) return;
    const float deg = 3.14159265358979323846f / 180.0f;
    p->sigma_e_frac = 0.05f;
    p->sigma_pos_cm = 1.0f;
    p->deta_min = 0.5f * deg;
    p->deta_max = 20.0f * deg;
    p->k_cut = 0.0f;
    p->topk = 1;
    p->nms_rad = 1.0f * deg;
    p->max_iter = 50;
    p->tol_rad = 1e-7;
}

cc_status cc_rings_from_events(const cc_events *ev, const cc_rings *out, const cc_params *p,
                               void *stream) {
    g_err[0] = 0;
    cc_status st = check_params(p);
    if (st != CC_OK) return st;
    if (!ev || !out) return fail(CC_EINVAL, "events/rings is NULL");
    if (ev->count < 0) return fail(CC_EINVAL, "events->count < 0");
    if (ev->stride < ev->count) return fail(CC_EINVAL, "events->stride < count");
    if (out->count != ev->count) return fail(CC_EINVAL, "rings->count != events->count");
    if (ev->count == 0) return CC_OK;
    if (!ev->n || !ev->x || !ev->y || !ev->z || !ev->e)
        return fail(CC_EINVAL, "event arrays must be non-NULL");
    if (!out->ax || !out->ay || !out->az || !out->eta || !out->deta || !out->valid ||
        !out->perm)
        return fail(CC_EINVAL, "ring output arrays must be non-NULL");
    if (ev->stride > (INT64_MAX / 4)) return fail(CC_EINVAL, "events->stride too large");
    cudaError_t e = launch_rings_from_events(*ev, *out, *p, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "rings_from_events launch");
    return CC_OK;
}

cc_status cc_events_copy(const cc_events *dst, int64_t dst_offset, const cc_events *src,
                         int64_t src_offset, int64_t count, void *stream) {
    g_err[0] = 0;
    if (!dst || !src) return fail(CC_EINVAL, "events NULL");
    if (count < 0 || dst_offset < 0 || src_offset < 0 || dst_offset + count > dst->stride ||
        src_offset + count > src->stride)
        return fail(CC_EINVAL, "bad offsets or count for the strides");
    if (count == 0) return CC_OK;
    if (!dst->n || !dst->x || !dst->y || !dst->z || !dst->e || !src->n || !src->x || !src->y ||
        !src->z || !src->e)
        return fail(CC_EINVAL, "event arrays must be non-NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(const_cast<uint8_t *>(dst->n) + dst_offset, src->n + src_offset,
                                    (size_t)count, cudaMemcpyDefault, s);
    const float *sa[4] = {src->x, src->y, src->z, src->e};
    const float *da[4] = {dst->x, dst->y, dst->z, dst->e};
    for (int a = 0; a < 4 && e == cudaSuccess; a++)
        e = cudaMemcpy2DAsync(const_cast<float *>(da[a]) + dst_offset,
                              (size_t)dst->stride * sizeof(float), sa[a] + src_offset,
                              (size_t)src->stride * sizeof(float), (size_t)count * sizeof(float),
                              4, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(e, "events copy");
    return CC_OK;
}

size_t cc_localize_workspace_bytes(int64_t rings, int64_t dirs, const cc_params *p) {
    cc_params d;
    if (!p) { cc_params_default(&d); p = &d; }
    SweepPlan plan;
    if (!plan_sweep(rings, dirs, *p, &plan)) return 0;
    return plan.bytes;
}

cc_status cc_localize(const cc_rings *rings, const cc_grid *grid, const cc_params *p,
                      float *map, int32_t *argmax, int32_t *seeds, int32_t *status,
                      void *workspace, size_t ws_bytes, void *stream) {
    g_err[0] = 0;
    cc_status st = check_params(p);
    if (st != CC_OK) return st;
    if ((st = check_rings_in(rings)) != CC_OK) return st;
    if (!grid || grid->count < 1 || grid->count > INT32_MAX)
        return fail(CC_EINVAL, "grid->count must be in 1..2^31-1");
    if (!grid->x || !grid->y || !grid->z) return fail(CC_EINVAL, "grid arrays must be non-NULL");
    if (!map || !argmax) return fail(CC_EINVAL, "map and argmax must be non-NULL");
    if (!workspace || !aligned(workspace, 256))
        return fail(CC_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    SweepPlan plan;
    if (!plan_sweep(rings->count, grid->count, *p, &plan))
        return fail(CC_EINVAL, "cannot plan the sweep (sizes or device)");
    if (ws_bytes < plan.bytes)
        return fail(CC_ENOMEM, "workspace of %zu bytes < %zu needed", ws_bytes, plan.bytes);
    cudaError_t e = launch_localize(*rings, *grid, *p, plan, map, argmax, seeds, status,
                                    (char *)workspace, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "localize launch");
    return CC_OK;
}

size_t cc_localize_batch_workspace_bytes(int64_t rings, int64_t dirs, const cc_params *p) {
    cc_params d;
    if (!p) { cc_params_default(&d); p = &d; }
    SweepPlan plan;
    if (!plan_sweep(rings, dirs, *p, &plan, kBatchD)) return 0;
    return plan.bytes;
}

cc_status cc_localize_batch(int32_t n, const cc_rings *rings, const cc_grid *grid,
                            const cc_params *p, float *const *maps, int32_t *const *argmax,
                            int32_t *const *seeds, int32_t *const *status,
                            void *const *workspaces, const size_t *ws_bytes, void *stream) {
    g_err[0] = 0;
    cc_status st = check_params(p);
    if (st != CC_OK) return st;
    if (n < 1 || n > CC_BATCH_MAX) return fail(CC_EINVAL, "n must be in 1..%d", CC_BATCH_MAX);
    if (!rings || !maps || !argmax || !workspaces || !ws_bytes)
        return fail(CC_EINVAL, "rings, maps, argmax, workspaces, ws_bytes must be non-NULL");
    if (!grid || grid->count < 1 || grid->count > INT32_MAX || !grid->x || !grid->y || !grid->z)
        return fail(CC_EINVAL, "bad grid");
    SweepPlan plans[CC_BATCH_MAX];
    char *ws[CC_BATCH_MAX];
    for (int b = 0; b < n; b++) {
        if ((st = check_rings_in(&rings[b])) != CC_OK) return st;
        if (!maps[b] || !argmax[b]) return fail(CC_EINVAL, "burst %d: map/argmax NULL", b);
        if (!workspaces[b] || !aligned(workspaces[b], 256))
            return fail(CC_EINVAL, "burst %d: workspace NULL or not 256-byte aligned", b);
        if (!plan_sweep(rings[b].count, grid->count, *p, &plans[b], kBatchD))
            return fail(CC_EINVAL, "burst %d: cannot plan the sweep", b);
        if (ws_bytes[b] < plans[b].bytes)
            return fail(CC_ENOMEM, "burst %d: workspace of %zu bytes < %zu needed", b,
                        ws_bytes[b], plans[b].bytes);
        ws[b] = (char *)workspaces[b];
    }
    cudaError_t e = launch_localize_batch(n, rings, *grid, *p, plans, maps, argmax, seeds, status,
                                          ws, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "localize_batch launch");
    return CC_OK;
}

size_t cc_refine_workspace_bytes(int64_t rings, int32_t k) {
    return refine_workspace_bytes(rings, k);
}

cc_status cc_refine(const cc_rings *rings, const double *seed_dirs, int32_t k,
                    const cc_params *p, double *out_dir, double *out_obj, int32_t *out_iters,
                    int32_t *status, void *workspace, size_t ws_bytes, void *stream) {
    g_err[0] = 0;
    cc_status st = check_params(p);
    if (st != CC_OK) return st;
    if ((st = check_rings_in(rings)) != CC_OK) return st;
    if (k < 1 || k > 64) return fail(CC_EINVAL, "k must be in 1..64");
    if (!seed_dirs || !out_dir || !out_obj || !out_iters || !status)
        return fail(CC_EINVAL, "seed_dirs and outputs must be non-NULL");
    if (!workspace || !aligned(workspace, 256))
        return fail(CC_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    size_t need = refine_workspace_bytes(rings->count, k);
    if (need == 0) return fail(CC_EINVAL, "cannot size the refinement workspace");
    if (ws_bytes < need)
        return fail(CC_ENOMEM, "workspace of %zu bytes < %zu needed", ws_bytes, need);
    cudaError_t e = launch_refine(*rings, seed_dirs, k, *p, out_dir, out_obj, out_iters, status,
                                  (char *)workspace, ws_bytes, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "refine launch");
    return CC_OK;
}

cc_status cc_grid_fibonacci(int64_t n, float *x, float *y, float *z, void *stream) {
    g_err[0] = 0;
    if (n < 1 || n > ((int64_t)1 << 31)) return fail(CC_EINVAL, "n must be in 1..2^31");
    if (!x || !y || !z) return fail(CC_EINVAL, "output arrays must be non-NULL");
    cudaError_t e = launch_grid_fibonacci(n, x, y, z, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "grid_fibonacci launch");
    return CC_OK;
}

cc_status cc_grid_healpix_ring(int32_t nside, float *x, float *y, float *z, void *stream) {
    g_err[0] = 0;
    if (nside < 1 || nside > 8192) return fail(CC_EINVAL, "nside must be in 1..8192");
    if (!x || !y || !z) return fail(CC_EINVAL, "output arrays must be non-NULL");
    cudaError_t e = launch_grid_healpix(nside, x, y, z, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "grid_healpix_ring launch");
    return CC_OK;
}

cc_status cc_grid_healpix_nest(int32_t nside, float *x, float *y, float *z, void *stream) {
    g_err[0] = 0;
    if (nside < 1 || nside > 8192 || (nside & (nside - 1)) != 0)
        return fail(CC_EINVAL, "nside must be a power of two in 1..8192");
    if (!x || !y || !z) return fail(CC_EINVAL, "output arrays must be non-NULL");
    cudaError_t e = launch_grid_healpix_nest(nside, x, y, z, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "grid_healpix_nest launch");
    return CC_OK;
}

size_t cc_grid_order_workspace_bytes(int64_t count) {
    return count < 1 ? 0 : direction_order_bytes(count);
}

cc_status cc_grid_order(const cc_grid *grid, int32_t *order, void *workspace, size_t ws_bytes,
                        void *stream) {
    g_err[0] = 0;
    if (!grid || grid->count < 1 || grid->count > INT32_MAX || !grid->x || !grid->y || !grid->z)
        return fail(CC_EINVAL, "bad grid");
    if (!order) return fail(CC_EINVAL, "order must be non-NULL");
    if (ws_bytes < direction_order_bytes(grid->count) || !workspace ||
        (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
        return fail(CC_EINVAL, "workspace too small or not 256-byte aligned");
    cudaError_t e = direction_order(*grid, order, static_cast<char *>(workspace), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "grid_order launch");
    return CC_OK;
}

cc_status cc_grid_gather(const cc_grid *grid, const int32_t *idx, int32_t k, double *out_dirs,
                         void *stream) {
    g_err[0] = 0;
    if (!grid || grid->count < 1 || !grid->x || !grid->y || !grid->z)
        return fail(CC_EINVAL, "bad grid");
    if (k < 1 || k > 64) return fail(CC_EINVAL, "k must be in 1..64");
    if (!idx || !out_dirs) return fail(CC_EINVAL, "idx/out_dirs must be non-NULL");
    cudaError_t e = launch_grid_gather(*grid, idx, k, out_dirs, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "grid_gather launch");
    return CC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// learned ring filter
// ---------------------------------------------------------------------------
extern "C" {

cc_status cc_ring_features(const cc_events *ev, const cc_rings *rings, const cc_params *p,
                           uint16_t *features, void *stream) {
    g_err[0] = 0;
    cc_status st = check_params(p);
    if (st != CC_OK) return st;
    if (!ev || !rings || !features) return fail(CC_EINVAL, "events/rings/features is NULL");
    if (ev->count < 0 || ev->stride < ev->count || rings->count != ev->count)
        return fail(CC_EINVAL, "bad counts (need 0 <= count <= stride, rings->count == count)");
    if (ev->count == 0) return CC_OK;
    if (!ev->n || !ev->x || !ev->y || !ev->z || !ev->e || !rings->az || !rings->eta ||
        !rings->deta || !rings->valid || !rings->perm)
        return fail(CC_EINVAL, "event and ring arrays must be non-NULL");
    cudaError_t e = mlp_features(*ev, *rings, p->sigma_pos_cm, features, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ring_features launch");
    return CC_OK;
}

size_t cc_mlp_workspace_bytes(int64_t rows) {
    if (rows < 0) return 0;
    return mlp_workspace_bytes(rows);
}

cc_status cc_mlp_forward(const float *params, const uint16_t *params_bf16,
                         const uint16_t *features, int64_t rows, float *out, void *workspace,
                         size_t ws_bytes, void *stream) {
    g_err[0] = 0;
    if (rows < 0) return fail(CC_EINVAL, "rows < 0");
    if (rows == 0) return CC_OK;
    if (!params || !params_bf16 || !features || !out)
        return fail(CC_EINVAL, "params/features/out must be non-NULL");
    if (!aligned(features, 16) || !aligned(params_bf16, 16) || !aligned(out, 8))
        return fail(CC_EINVAL, "features and params_bf16 must be 16-byte aligned, out 8-byte");
    (void)workspace;                       // the forward keeps its activations on chip
    (void)ws_bytes;
    cudaError_t e = mlp_forward(params, params_bf16, features, rows, out, nullptr,
                                (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mlp_forward launch");
    return CC_OK;
}

static cc_status mlp_grad_checked(const float *params, const uint16_t *params_bf16,
                                  const uint16_t *features, const uint8_t *is_source,
                                  const float *residual, const uint8_t *weight, int64_t rows,
                                  float *grad, float *loss, void *workspace, size_t ws_bytes,
                                  const MlpTrace *trace, void *stream);

cc_status cc_mlp_grad(const float *params, const uint16_t *params_bf16, const uint16_t *features,
                      const uint8_t *is_source, const float *residual, const uint8_t *weight,
                      int64_t rows, float *grad, float *loss, void *workspace, size_t ws_bytes,
                      void *stream) {
    return mlp_grad_checked(params, params_bf16, features, is_source, residual, weight, rows,
                            grad, loss, workspace, ws_bytes, nullptr, stream);
}

cc_status cc_mlp_grad_trace(const float *params, const uint16_t *params_bf16,
                            const uint16_t *features, const uint8_t *is_source,
                            const float *residual, const uint8_t *weight, int64_t rows,
                            float *grad, float *loss, void *workspace, size_t ws_bytes,
                            uint16_t *hidden, float *out, uint16_t *dout, uint16_t *signals,
                            void *stream) {
    if ((hidden && !aligned(hidden, 16)) || (signals && !aligned(signals, 16)) ||
        (out && !aligned(out, 8)) || (dout && !aligned(dout, 4))) {
        g_err[0] = 0;
        return fail(CC_EINVAL, "hidden/signals must be 16-byte aligned, out 8, dout 4");
    }
    MlpTrace t{hidden, out, dout, signals};
    return mlp_grad_checked(params, params_bf16, features, is_source, residual, weight, rows,
                            grad, loss, workspace, ws_bytes, &t, stream);
}

static cc_status mlp_grad_checked(const float *params, const uint16_t *params_bf16,
                                  const uint16_t *features, const uint8_t *is_source,
                                  const float *residual, const uint8_t *weight, int64_t rows,
                                  float *grad, float *loss, void *workspace, size_t ws_bytes,
                                  const MlpTrace *trace, void *stream) {
    g_err[0] = 0;
    if (rows < 1 || rows > CC_MLP_MAX_BATCH)
        return fail(CC_EINVAL, "rows must be in 1..%d", CC_MLP_MAX_BATCH);
    if (!params || !params_bf16 || !features || !is_source || !residual || !weight || !grad ||
        !loss)
        return fail(CC_EINVAL, "arguments must be non-NULL");
    if (!aligned(features, 16) || !aligned(params_bf16, 16))
        return fail(CC_EINVAL, "features and params_bf16 must be 16-byte aligned");
    if (!workspace || !aligned(workspace, 256))
        return fail(CC_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    size_t need = mlp_workspace_bytes(rows);
    if (ws_bytes < need) return fail(CC_ENOMEM, "workspace of %zu bytes < %zu needed", ws_bytes, need);
    cudaError_t e = mlp_grad(params, params_bf16, features, is_source, residual, weight, rows,
                             grad, loss, (char *)workspace, trace, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mlp_grad launch");
    return CC_OK;
}

cc_status cc_mlp_adam(float *params, float *m, float *v, const float *grad, uint16_t *params_bf16,
                      int32_t step, float lr, float beta1, float beta2, float eps, void *stream) {
    g_err[0] = 0;
    if (!params || !m || !v || !grad || !params_bf16) return fail(CC_EINVAL, "NULL argument");
    if (step < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return fail(CC_EINVAL, "need step >= 1, lr > 0, 0 <= beta < 1, eps > 0");
    cudaError_t e = mlp_adam(params, m, v, grad, params_bf16, step, lr, beta1, beta2, eps,
                             (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mlp_adam launch");
    return CC_OK;
}

cc_status cc_mlp_params_to_bf16(const float *params, uint16_t *params_bf16, void *stream) {
    g_err[0] = 0;
    if (!params || !params_bf16) return fail(CC_EINVAL, "NULL argument");
    cudaError_t e = mlp_params_to_bf16(params, params_bf16, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mlp_params_to_bf16 launch");
    return CC_OK;
}

cc_status cc_mlp_apply_filter(const float *out, const cc_rings *rings, float tau, float deta_min,
                              float deta_max, void *stream) {
    g_err[0] = 0;
    if (!out || !rings || rings->count < 0) return fail(CC_EINVAL, "bad arguments");
    if (rings->count > 0 && (!rings->valid || !rings->deta))
        return fail(CC_EINVAL, "rings->valid and rings->deta must be non-NULL");
    if (!(deta_min > 0.0f) || !(deta_max >= deta_min)) return fail(CC_EINVAL, "bad deta clamp");
    cudaError_t e = mlp_apply_filter(out, *rings, tau, deta_min, deta_max, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mlp_apply_filter launch");
    return CC_OK;
}

// ---------------------------------------------------------------------------
// event clustering of detections (Sec. 2)
// ---------------------------------------------------------------------------
size_t cc_cluster_workspace_bytes(int64_t count) {
    return count < 0 ? 0 : cluster_workspace_bytes(count);
}

cc_status cc_cluster_maxstep(const cc_detections *d, int64_t dt_max, uint8_t *edge,
                             int32_t *event_id, int64_t *ev_first, int32_t *ev_count,
                             uint64_t *ev_adc, int64_t ev_capacity, int64_t *n_events,
                             int32_t *status, void *workspace, size_t ws_bytes, void *stream) {
    g_err[0] = 0;
    if (!d) return fail(CC_EINVAL, "detections is NULL");
    if (d->count < 0 || d->count > INT32_MAX)
        return fail(CC_EINVAL, "need 0 <= detections->count <= 2^31 - 1");
    if (d->count > 0 && !d->t) return fail(CC_EINVAL, "detections->t is NULL");
    if (ev_adc && d->count > 0 && !d->adc) return fail(CC_EINVAL, "ev_adc needs detections->adc");
    if ((ev_first || ev_count || ev_adc) && ev_capacity < d->count / 2)
        return fail(CC_EINVAL, "ev_capacity < count / 2 (the most events count detections make)");
    if (!workspace || ws_bytes < cluster_workspace_bytes(d->count))
        return fail(CC_EINVAL, "workspace too small (cc_cluster_workspace_bytes)");
    if (((uintptr_t)workspace & 255u) != 0) return fail(CC_EINVAL, "workspace not 256-byte aligned");
    if (((uintptr_t)d->t & 7u) != 0 || ((uintptr_t)d->adc & 3u) != 0)
        return fail(CC_EINVAL, "misaligned detection arrays");
    cudaError_t e = launch_cluster(d->t, d->adc, d->count, dt_max, edge, event_id, ev_first,
                                   ev_count, ev_adc, n_events, status, (char *)workspace,
                                   (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cluster launch");
    return CC_OK;
}

cc_status cc_cluster_spectrum(const uint64_t *ev_adc, const int64_t *n_events, uint64_t bin_width,
                              int32_t nbins, uint64_t *hist, void *stream) {
    g_err[0] = 0;
    if (!ev_adc || !n_events || !hist) return fail(CC_EINVAL, "NULL argument");
    if (bin_width < 1 || nbins < 1) return fail(CC_EINVAL, "need bin_width >= 1 and nbins >= 1");
    cudaError_t e = launch_spectrum(ev_adc, n_events, bin_width, nbins, hist, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "spectrum launch");
    return CC_OK;
}

cc_status cc_selftest_exact_ops(uint64_t *mismatches, void *stream) {
    g_err[0] = 0;
    if (!mismatches) return fail(CC_EINVAL, "mismatches is NULL");
    cudaError_t e = launch_selftest_exact(mismatches, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "selftest launch");
    return CC_OK;
}

cc_status cc_selftest_wait_timeout(int32_t which, int64_t limit_ns, uint32_t *counter,
                                   int32_t *status, void *stream) {
    g_err[0] = 0;
    if (which != 0 && which != 1) return fail(CC_EINVAL, "which must be 0 or 1");
    if (limit_ns < 1000 || limit_ns > 10000000000LL)
        return fail(CC_EINVAL, "limit_ns must be in [1000, 1e10]");
    if (!counter || !status) return fail(CC_EINVAL, "counter and status must be non-NULL");
    cudaError_t e = launch_selftest_wait(which, limit_ns, counter, status, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "selftest launch");
    return CC_OK;
}

cc_status cc_debug_bounds(uint64_t *word, int32_t reset) {
    g_err[0] = 0;
    if (!word) return fail(CC_EINVAL, "word is NULL");
    *word = 0;
#ifdef CC_DEBUG_BOUNDS
    unsigned long long w = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&w, cc::cc_oob_word, sizeof(w));
    if (e != cudaSuccess) return cuda_fail(e, "reading the bounds word");
    *word = w;
    if (reset) {
        const unsigned long long z = 0;
        if ((e = cudaMemcpyToSymbol(cc::cc_oob_word, &z, sizeof(z))) != cudaSuccess)
            return cuda_fail(e, "clearing the bounds word");
    }
    return CC_OK;
#else
    (void)reset;
    return fail(CC_EINVAL, "not a debug build");
#endif
}

cc_status cc_debug_selftest_bounds(int32_t *buf, int64_t n, void *stream) {
    g_err[0] = 0;
#ifdef CC_DEBUG_BOUNDS
    if (!buf || n < 1) return fail(CC_EINVAL, "need a buffer of n >= 1 elements");
    cudaError_t e = launch_selftest_bounds(buf, n, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "selftest launch");
    return CC_OK;
#else
    (void)buf;
    (void)n;
    (void)stream;
    return fail(CC_EINVAL, "not a debug build");
#endif
}

// ---------------------------------------------------------------------------
// near-field back projection (Sec. 3)
// ---------------------------------------------------------------------------
cc_status cc_ring_apex(const cc_events *ev, const cc_rings *rings, float *px, float *py,
                       float *pz, void *stream) {
    g_err[0] = 0;
    if (!ev || !rings) return fail(CC_EINVAL, "events/rings is NULL");
    if (ev->count < 0 || ev->stride < ev->count || rings->count != ev->count)
        return fail(CC_EINVAL, "bad counts (need 0 <= count <= stride, rings->count == count)");
    if (ev->stride > (INT64_MAX / 4)) return fail(CC_EINVAL, "events->stride too large");
    if (ev->count == 0) return CC_OK;
    if (!ev->n || !ev->x || !ev->y || !ev->z || !rings->perm || !rings->valid || !px || !py ||
        !pz)
        return fail(CC_EINVAL, "event, ring and apex arrays must be non-NULL");
    cudaError_t e = launch_ring_apex(*ev, *rings, px, py, pz, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "ring_apex launch");
    return CC_OK;
}

int64_t cc_voxel_count(int32_t shape, int32_t n) {
    if (shape < 0 || shape > 2 || n < 1 || n > CC_VOXEL_MAX_N) return -1;
    return universe_count(shape, n);
}

cc_status cc_voxel_universe(int32_t shape, int32_t n, float pitch, float cx, float cy, float cz,
                            float *x, float *y, float *z, void *stream) {
    g_err[0] = 0;
    if (shape < 0 || shape > 2) return fail(CC_EINVAL, "shape must be 0 (cube), 1 (cylinder) or 2 (sphere)");
    if (n < 1 || n > CC_VOXEL_MAX_N) return fail(CC_EINVAL, "need 1 <= n <= CC_VOXEL_MAX_N");
    if (!(pitch > 0.0f) || !isfinite(cx) || !isfinite(cy) || !isfinite(cz))
        return fail(CC_EINVAL, "need pitch > 0 and a finite centre");
    if (!x || !y || !z) return fail(CC_EINVAL, "x, y, z must be non-NULL");
    cudaError_t e = launch_universe(shape, n, pitch, cx, cy, cz, x, y, z, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "universe launch");
    return CC_OK;
}

size_t cc_backproject_workspace_bytes(int64_t rings, int64_t voxels, const cc_params *p) {
    if (!p || rings < 0 || voxels < 1 || voxels > INT32_MAX) return 0;
    SweepPlan plan;
    if (!plan_backproject(rings, voxels, *p, &plan)) return 0;
    return plan.bytes;
}

cc_status cc_backproject(const cc_rings *rings, const float *px, const float *py, const float *pz,
                         const cc_grid *voxels, const cc_params *p, float *image, int32_t *argmax,
                         int32_t *status, void *workspace, size_t ws_bytes, void *stream) {
    g_err[0] = 0;
    cc_status st;
    if ((st = check_rings_in(rings)) != CC_OK) return st;
    if (rings->count > 0 && (!px || !py || !pz)) return fail(CC_EINVAL, "apex arrays must be non-NULL");
    if (!voxels || voxels->count < 1 || voxels->count > INT32_MAX || !voxels->x || !voxels->y ||
        !voxels->z)
        return fail(CC_EINVAL, "need 1 <= voxels->count <= 2^31 - 1 and voxel arrays");
    if ((st = check_params(p)) != CC_OK) return st;
    if (!image || !argmax) return fail(CC_EINVAL, "image and argmax must be non-NULL");
    SweepPlan plan;
    if (!plan_backproject(rings->count, voxels->count, *p, &plan))
        return fail(CC_ECUDA, "no CUDA device for planning");
    if (!workspace || ws_bytes < plan.bytes)
        return fail(CC_EINVAL, "workspace too small (cc_backproject_workspace_bytes)");
    if (((uintptr_t)workspace & 255u) != 0) return fail(CC_EINVAL, "workspace not 256-byte aligned");
    cudaError_t e = launch_backproject(*rings, px, py, pz, *voxels, *p, plan, image, argmax, status,
                                       (char *)workspace, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "backproject launch");
    return CC_OK;
}

}  // extern "C"

// noalloc.cu - cc_localize_static: the same localisation as cc_localize
// (same plan, same kernels), with its scratch in a file-scope device array
// instead of a caller workspace, for callers that cannot allocate device
// memory.  It calls no cudaMalloc / cudaFree and no allocating routine.
//
// g_scratch below is a device array.  In host code its name is only a
// host-side stand-in for the symbol, not a device address, so the device
// address is looked up once per device with cudaGetSymbolAddress (the first
// call made on that device, with it current) and cached; kernels get that
// address.
#include <mutex>

#include "cc_internal.cuh"

namespace cc {
namespace {

constexpr size_t kStaticScratchBytes = CC_LOCALIZE_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices];   // device address of g_scratch, per device

}  // namespace
}  // namespace cc

using namespace cc;

extern "C" cc_status cc_localize_static(const cc_rings *rings, const cc_grid *grid,
                                        const cc_params *p, float *map, int32_t *argmax,
                                        int32_t *seeds, int32_t *status, void *stream) {
    clear_error();
    if (!p) return fail(CC_EINVAL, "params is NULL");
    if (!(p->k_cut >= 0.0f)) return fail(CC_EINVAL, "k_cut must be >= 0");
    if (p->topk < 1 || p->topk > 64) return fail(CC_EINVAL, "topk must be in 1..64");
    if (!(p->nms_rad >= 0.0f)) return fail(CC_EINVAL, "nms_rad must be >= 0");
    if (!rings || rings->count < 0) return fail(CC_EINVAL, "rings is NULL or count < 0");
    if (rings->count > 0 &&
        (!rings->ax || !rings->ay || !rings->az || !rings->eta || !rings->deta))
        return fail(CC_EINVAL, "ring arrays must be non-NULL");
    if (!grid || grid->count < 1 || grid->count > INT32_MAX)
        return fail(CC_EINVAL, "grid->count must be in 1..2^31-1");
    if (!grid->x || !grid->y || !grid->z) return fail(CC_EINVAL, "grid arrays must be non-NULL");
    if (!map || !argmax) return fail(CC_EINVAL, "map and argmax must be non-NULL");

    SweepPlan plan;
    if (!plan_sweep(rings->count, grid->count, *p, &plan))
        return fail(CC_EINVAL, "cannot plan the sweep (sizes or device)");
    if (plan.bytes > kStaticScratchBytes)
        return fail(CC_EINVAL,
                    "%lld rings x %lld directions need %zu bytes of scratch; the static "
                    "scratch of cc_localize_static holds %zu (use cc_localize with a "
                    "workspace)",
                    (long long)rings->count, (long long)grid->count, plan.bytes,
                    kStaticScratchBytes);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(CC_EINVAL, "device index %d too large", dev);
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_scratch);
            if (e != cudaSuccess) {
                g_scratch_addr[dev] = nullptr;
                return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
            }
        }
        scratch = g_scratch_addr[dev];
    }
    e = launch_localize(*rings, *grid, *p, plan, map, argmax, seeds, status, (char *)scratch,
                        (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "localize_static launch");
    return CC_OK;
}

// selftest.cu - device self-tests exposed through the C ABI: the bounded
// waits of the pipelines run out on a signal that never comes and report
// CC_ETIMEOUT, leaving the context usable.
#include "cc_internal.cuh"
#include "cc_pipe.cuh"

namespace cc {
namespace {

// which = 0: an mbarrier phase that never completes (the TMA / tensor-core
// pipelines' wait); which = 1: a global counter that nothing raises (the
// refinement's grid barrier).  status = CC_ETIMEOUT when the wait gave up.
__global__ void k_selftest_wait(int which, unsigned long long limit_ns, unsigned *counter,
                                int32_t *status) {
    __shared__ unsigned long long bar;
    if (threadIdx.x != 0) return;
    bool ok;
    if (which == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        ok = mbar_wait(&bar, 0, limit_ns);
    } else {
        ok = spin_until_ge(counter, 1u, limit_ns);
    }
    *status = ok ? (int32_t)CC_OK : (int32_t)CC_ETIMEOUT;
}

}  // namespace

cudaError_t launch_selftest_wait(int which, int64_t limit_ns, uint32_t *counter, int32_t *status,
                                 cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_selftest_wait<<<1, 32, 0, s>>>(which, (unsigned long long)limit_ns,
                                     reinterpret_cast<unsigned *>(counter), status);
    return cudaGetLastError();
}

}  // namespace cc

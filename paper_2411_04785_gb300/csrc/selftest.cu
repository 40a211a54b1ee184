// selftest.cu - device self-tests exposed through the C ABI: the bounded
// waits of the pipelines run out on a signal that never comes and report
// CC_ETIMEOUT, leaving the context usable.
#include "cc_internal.cuh"
#include "cc_pipe.cuh"

namespace cc {

#ifdef CC_DEBUG_BOUNDS
// The debug build's record of the first failed bounds check (cc_internal.cuh).
__device__ unsigned long long cc_oob_word = 0;
#endif

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

#ifdef CC_DEBUG_BOUNDS
// The one checked access asks for element n of an n-element buffer: the
// check records it and the store is skipped.
__global__ void k_selftest_bounds(int32_t *buf, int64_t n) {
    if (threadIdx.x != 0) return;
    const int64_t i = n;
    if (CC_IN_BOUNDS(CC_SITE_SELFTEST, i, n)) buf[i] = 1;
}
#endif

}  // namespace

#ifdef CC_DEBUG_BOUNDS
cudaError_t launch_selftest_bounds(int32_t *buf, int64_t n, cudaStream_t s) {
    k_selftest_bounds<<<1, 32, 0, s>>>(buf, n);
    return cudaGetLastError();
}
#endif

cudaError_t launch_selftest_wait(int which, int64_t limit_ns, uint32_t *counter, int32_t *status,
                                 cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_selftest_wait<<<1, 32, 0, s>>>(which, (unsigned long long)limit_ns,
                                     reinterpret_cast<unsigned *>(counter), status);
    return cudaGetLastError();
}

}  // namespace cc

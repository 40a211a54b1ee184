// cc_pipe.cuh - device helpers shared by the sweeps (far-field directions
// and near-field voxels), the clustering and the ring filter: the mbarrier +
// bulk-copy and tensor-copy (TMA) pipelines with bounded waits, and the argmax
// reductions (ties: lowest index).
#pragma once

#include <cuda.h>
#include <float.h>

#include "cc_internal.cuh"

namespace cc {
namespace {

// cuTensorMapEncodeTiled from the driver, looked up once (no link to libcuda)
typedef CUresult (*TmapEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline TmapEncodeFn encode_fn() {
    static const TmapEncodeFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<TmapEncodeFn>(p);
    }();
    return fn;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void tma_bulk_load(void *dst, const void *src, unsigned bytes,
                                              unsigned long long *bar) {
    unsigned b = smem_u32(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(b)
        : "memory");
}

// A bulk copy completing on `bar` whose expected bytes were already
// announced (several copies may share one arrive.expect_tx).  Both addresses
// 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes,
                                          unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Tensor store of a shared-memory tile (bulk group; the caller commits the
// group and waits for it before the tile is reused or the CTA exits).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, const void *src) {
    asm volatile(
        "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map),
        "r"(x), "r"(y), "r"(smem_u32(src))
        : "memory");
}

// Bounded wait for an mbarrier phase: false after limit_ns.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          unsigned long long limit_ns = kWaitLimitNs) {
    unsigned b = smem_u32(bar);
    unsigned long long t0 = 0;
    for (unsigned it = 0; it < (1u << 30); ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(b), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 31) == 0) {
            unsigned long long now = globaltimer_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > limit_ns) return false;
        }
    }
    return false;
}

// Bounded spin until a counter in global memory reaches target (another CTA
// raises it): false after limit_ns.  One thread calls it; acquire ordering is
// the caller's (a fence after it returns).
__device__ __forceinline__ bool spin_until_ge(const unsigned *count, unsigned target,
                                              unsigned long long limit_ns = kWaitLimitNs) {
    const volatile unsigned *vc = count;
    unsigned long long t0 = 0;
    for (unsigned it = 0; *vc < target; ++it) {
        if ((it & 255) == 255) {
            const unsigned long long now = globaltimer_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > limit_ns) return false;
        }
    }
    return true;
}

__device__ __forceinline__ void better(float &v, int &j, float v2, int j2) {
    if (v2 > v || (v2 == v && j2 < j)) { v = v2; j = j2; }
}

// Block-wide argmax (ties: lowest index); result valid in thread 0.
__device__ __forceinline__ void block_best(float &v, int &j) {
    __shared__ float sv[32];
    __shared__ int sj[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float v2 = __shfl_xor_sync(0xffffffffu, v, o);
        int j2 = __shfl_xor_sync(0xffffffffu, j, o);
        better(v, j, v2, j2);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0) { sv[w] = v; sj[w] = j; }
    __syncthreads();
    if (w == 0) {
        v = l < nw ? sv[l] : -FLT_MAX;
        j = l < nw ? sj[l] : INT32_MAX;
        if (l >= nw) v = -__builtin_huge_valf();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float v2 = __shfl_xor_sync(0xffffffffu, v, o);
            int j2 = __shfl_xor_sync(0xffffffffu, j, o);
            better(v, j, v2, j2);
        }
    }
    __syncthreads();
}

}  // namespace
}  // namespace cc

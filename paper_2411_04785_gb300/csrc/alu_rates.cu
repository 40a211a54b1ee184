// alu_rates.cu - measures the per-SM issue rates of the units the sweep
// kernel's roofline is built from: FP32 FMA (scalar and packed FP32x2),
// MUFU ex2, MUFU sqrt / rsqrt, and FP32 min.  Standalone program (not part of
// libcompton.so); `python bench.py --alu-rates` builds and runs it.
//
// Every thread runs ILP independent dependency chains of NIT iterations;
// lane-ops per second = blocks x threads x NIT x ILP x lanes per instruction
// over the CUDA-event time of one launch (after 3 warm-up launches).  Results
// are printed as one JSON object, per SM per clock at the SM clock given on
// the command line (MHz).
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

#define NIT 4096
#define ILP 8

__device__ __forceinline__ unsigned long long pk(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0,{%1,%2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
    float a, b;
    asm("mov.b64 {%0,%1},%2;" : "=f"(a), "=f"(b) : "l"(r));
    return make_float2(a, b);
}

// The sink store is taken only for an impossible value, at o[threadIdx.x]
// (< 256 elements), so every access stays in bounds.
__global__ void k_ffma(float *o, float s) {
    float x[ILP];
    for (int i = 0; i < ILP; i++) x[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < NIT; it++)
#pragma unroll
        for (int i = 0; i < ILP; i++) x[i] = fmaf(x[i], s, 0.5f);
    float t = 0;
    for (int i = 0; i < ILP; i++) t += x[i];
    if (t == 12345.f) o[threadIdx.x] = t;
}
__global__ void k_ffma2(float *o, float s) {
    unsigned long long x[ILP];
    for (int i = 0; i < ILP; i++) x[i] = pk(threadIdx.x * 1e-3f + i, i * 0.1f);
    unsigned long long ss = pk(s, s), hh = pk(0.5f, 0.5f);
    for (int it = 0; it < NIT; it++)
#pragma unroll
        for (int i = 0; i < ILP; i++)
            asm volatile("fma.rn.f32x2 %0,%0,%1,%2;" : "+l"(x[i]) : "l"(ss), "l"(hh));
    float t = 0;
    for (int i = 0; i < ILP; i++) { float2 v = upk(x[i]); t += v.x + v.y; }
    if (t == 12345.f) o[threadIdx.x] = t;
}
#define UNARY_KERNEL(NAME, PTX, INIT)                                              \
    __global__ void NAME(float *o, float s) {                                      \
        float x[ILP];                                                              \
        for (int i = 0; i < ILP; i++) x[i] = INIT;                                 \
        for (int it = 0; it < NIT; it++)                                           \
            _Pragma("unroll") for (int i = 0; i < ILP; i++)                        \
                asm volatile(PTX " %0,%0;" : "+f"(x[i]));                          \
        float t = 0;                                                               \
        for (int i = 0; i < ILP; i++) t += x[i];                                   \
        if (t == 12345.f) o[threadIdx.x] = t;                                      \
    }
UNARY_KERNEL(k_ex2, "ex2.approx.ftz.f32", -(threadIdx.x * 1e-3f + i) * 1e-3f)
UNARY_KERNEL(k_sqrt, "sqrt.approx.ftz.f32", threadIdx.x * 1e-3f + i + 1)
UNARY_KERNEL(k_rsqrt, "rsqrt.approx.ftz.f32", threadIdx.x * 1e-3f + i + 1)
__global__ void k_min(float *o, float s) {
    float x[ILP];
    for (int i = 0; i < ILP; i++) x[i] = threadIdx.x * 1e-3f + i + 1;
    for (int it = 0; it < NIT; it++)
#pragma unroll
        for (int i = 0; i < ILP; i++) asm volatile("min.f32 %0,%0,%1;" : "+f"(x[i]) : "f"(s));
    float t = 0;
    for (int i = 0; i < ILP; i++) t += x[i];
    if (t == 12345.f) o[threadIdx.x] = t;
}

typedef void (*kern_t)(float *, float);

int main(int argc, char **argv) {
    double mhz = argc > 1 ? atof(argv[1]) : 2070.0;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, 0) != cudaSuccess) return 1;
    float *o = nullptr;
    if (cudaMalloc(&o, 256 * sizeof(float)) != cudaSuccess) return 1;
    kern_t ks[] = {k_ffma, k_ffma2, k_ex2, k_sqrt, k_rsqrt, k_min};
    const char *nm[] = {"ffma", "ffma2_lanes", "ex2", "sqrt", "rsqrt", "min"};
    const double lanes[] = {1, 2, 1, 1, 1, 1};
    const int blocks = p.multiProcessorCount * 8, threads = 256;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    printf("{\"device\": \"%s\", \"sms\": %d, \"sm_mhz_assumed\": %.0f", p.name,
           p.multiProcessorCount, mhz);
    int rc = 0;
    for (int q = 0; q < 6; q++) {
        for (int w = 0; w < 3; w++) ks[q]<<<blocks, threads>>>(o, 0.999f);
        cudaEventRecord(a);
        ks[q]<<<blocks, threads>>>(o, 0.999f);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (cudaGetLastError() != cudaSuccess) rc = 1;
        double n = (double)blocks * threads * NIT * ILP * lanes[q];
        printf(", \"%s_per_clk_sm\": %.1f", nm[q],
               n / (ms * 1e-3) / (p.multiProcessorCount * mhz * 1e6));
    }
    printf("}\n");
    cudaFree(o);
    return rc;
}

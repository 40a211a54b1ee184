// grid.cu - sky grids (the far-field counterpart of the paper's image
// universe, Sec. 3 "Spatial optimization"): Fibonacci sphere and HEALPix
// pixel centres in RING order, plus an FP64 gather of grid directions.
//
// Everything is exact integer index arithmetic plus one correctly rounded
// FP32 division and sincospif per coordinate, so each component is within a
// few ulp of the FP64 value.
#include "cc_internal.cuh"

namespace cc {
namespace {

// frac(i * (3 - sqrt 5)/2) as a 64-bit fixed-point fraction:
// round(2^64 * (3 - sqrt 5)/2).
constexpr unsigned long long kGoldenFrac = 0x61C8864680B583EAull;

__global__ void k_fibonacci(int64_t n, float *__restrict__ x, float *__restrict__ y,
                            float *__restrict__ z) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || !CC_IN_BOUNDS(CC_SITE_GRID_OUT, i, n)) return;
    // 1 - z = (2i+1)/n and 1 + z = (2n-2i-1)/n: integer numerators, so
    // rho = sqrt((1 - z)(1 + z)) keeps full precision at both poles
    float a = (float)(2 * i + 1), b = (float)(2 * (n - i) - 1), fn = (float)n;
    float rho = sqrtf(a * b) / fn;
    unsigned long long f = (unsigned long long)i * kGoldenFrac;   // mod 2^64
    float frac = (float)(f >> 40) * 5.9604644775390625e-8f;       // 2^-24
    float s, c;
    sincospif(2.0f * frac, &s, &c);
    x[i] = rho * c;
    y[i] = rho * s;
    z[i] = (float)(n - 2 * i - 1) / fn;
}

// Centre of RING pixel p (0 <= p < 12 nside^2) into out[o].
__device__ __forceinline__ void ring_pixel(int64_t nside, int64_t p, int64_t o,
                                           float *__restrict__ x, float *__restrict__ y,
                                           float *__restrict__ z) {
    const int64_t npix = 12 * nside * nside;
    const int64_t ncap = 2 * nside * (nside - 1);
    float zz, omz, num, den;   // omz = 1 - |z|; phi = pi * num / den
    if (p < ncap || p >= npix - ncap) {
        const bool north = p < ncap;
        // polar ring i holds 4i pixels; 2i(i-1) pixels precede it
        int64_t q = north ? p : npix - 1 - p;
        int64_t i = (int64_t)((1.0f + sqrtf(1.0f + 2.0f * (float)q)) * 0.5f);
        while (i > 1 && 2 * i * (i - 1) > q) i--;
        while (2 * i * (i + 1) <= q) i++;
        int64_t j = q - 2 * i * (i - 1) + 1;          // 1..4i
        if (!north) j = 4 * i + 1 - j;                 // south rings run the other way
        omz = (float)(i * i) / (float)(3 * nside * nside);
        zz = north ? 1.0f - omz : omz - 1.0f;
        num = (float)(2 * j - 1);
        den = (float)(4 * i);
    } else {
        int64_t q = p - ncap;
        int64_t i = q / (4 * nside) + nside;           // nside .. 3 nside
        int64_t j = q % (4 * nside) + 1;
        int64_t two_f = ((i + nside) & 1) ? 2 : 1;     // 2 * offset (1 or 1/2)
        zz = (float)(2 * (2 * nside - i)) / (float)(3 * nside);
        omz = 1.0f - fabsf(zz);
        num = (float)(2 * j - two_f);
        den = (float)(4 * nside);
    }
    float rho = sqrtf(fmaxf(omz * (2.0f - omz), 0.0f));
    float s, c;
    sincospif(num / den, &s, &c);
    x[o] = rho * c;
    y[o] = rho * s;
    z[o] = zz;
}

__global__ void k_healpix_ring(int64_t nside, float *__restrict__ x, float *__restrict__ y,
                               float *__restrict__ z) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < 12 * nside * nside) ring_pixel(nside, p, p, x, y, z);
}

// The even bits of v packed together (bit 2b -> bit b).
__device__ __forceinline__ int64_t even_bits(uint64_t v) {
    v &= 0x5555555555555555ull;
    v = (v | (v >> 1)) & 0x3333333333333333ull;
    v = (v | (v >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v >> 4)) & 0x00FF00FF00FF00FFull;
    v = (v | (v >> 8)) & 0x0000FFFF0000FFFFull;
    v = (v | (v >> 16)) & 0x00000000FFFFFFFFull;
    return (int64_t)v;
}

// NESTED pixel p -> RING pixel (Gorski et al. 2005): base face f, face
// coordinates (ix, iy) from the interleaved bits, then the ring counted from
// the north pole and the place in that ring.
__device__ __forceinline__ int64_t nest_to_ring(int64_t nside, int64_t p) {
    const int64_t npface = nside * nside, npix = 12 * npface, ncap = 2 * nside * (nside - 1);
    const int f = (int)(p / npface);
    const int64_t q = p - (int64_t)f * npface;
    const int64_t ix = even_bits((uint64_t)q), iy = even_bits((uint64_t)q >> 1);
    const int row = f >> 2;                                  // 0 north, 1 equator, 2 south
    const int64_t jr = (2 + row) * nside - ix - iy - 1;      // ring, 1 .. 4 nside - 1
    const int64_t jp0 = 2 * (f & 3) + (row == 1 ? 0 : 1);
    int64_t nr, start, shift = 0;
    if (jr < nside) {
        nr = jr;
        start = 2 * nr * (nr - 1);
    } else if (jr > 3 * nside) {
        nr = 4 * nside - jr;
        start = npix - 2 * nr * (nr + 1);
    } else {
        nr = nside;
        start = ncap + (jr - nside) * 4 * nside;
        shift = (jr - nside) & 1;
    }
    int64_t jp = (jp0 * nr + ix - iy + 1 + shift) / 2;
    if (jp > 4 * nside) jp -= 4 * nside;
    if (jp < 1) jp += 4 * nside;
    return start + jp - 1;
}

__global__ void k_healpix_nest(int64_t nside, float *__restrict__ x, float *__restrict__ y,
                               float *__restrict__ z) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < 12 * nside * nside) {
        const int64_t r = nest_to_ring(nside, p);
        if (CC_IN_BOUNDS(CC_SITE_GRID_OUT, r, 12 * nside * nside)) ring_pixel(nside, r, p, x, y, z);
    }
}

__global__ void k_gather(const float *__restrict__ gx, const float *__restrict__ gy,
                         const float *__restrict__ gz, int64_t M,
                         const int32_t *__restrict__ idx, int k, double *__restrict__ out) {
    int t = threadIdx.x;
    if (t >= k) return;
    int j = idx[t];
    double v[3] = {0.0, 0.0, 0.0};
    if (j >= 0 && j < M) {
        v[0] = gx[j];
        v[1] = gy[j];
        v[2] = gz[j];
        double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);   // final normalisation
        v[0] /= n;
        v[1] /= n;
        v[2] /= n;
    }
    out[3 * t] = v[0];
    out[3 * t + 1] = v[1];
    out[3 * t + 2] = v[2];
}

}  // namespace

cudaError_t launch_grid_fibonacci(int64_t n, float *x, float *y, float *z, cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    TraceScope ts(CC_STAGE_GRID, s);
    k_fibonacci<<<(unsigned)blocks, 256, 0, s>>>(n, x, y, z);
    return cudaGetLastError();
}

cudaError_t launch_grid_healpix(int32_t nside, float *x, float *y, float *z, cudaStream_t s) {
    int64_t npix = 12 * (int64_t)nside * nside;
    int64_t blocks = (npix + 255) / 256;
    TraceScope ts(CC_STAGE_GRID, s);
    k_healpix_ring<<<(unsigned)blocks, 256, 0, s>>>(nside, x, y, z);
    return cudaGetLastError();
}

cudaError_t launch_grid_healpix_nest(int32_t nside, float *x, float *y, float *z,
                                    cudaStream_t s) {
    int64_t npix = 12 * (int64_t)nside * nside;
    int64_t blocks = (npix + 255) / 256;
    TraceScope ts(CC_STAGE_GRID, s);
    k_healpix_nest<<<(unsigned)blocks, 256, 0, s>>>(nside, x, y, z);
    return cudaGetLastError();
}

cudaError_t launch_grid_gather(const cc_grid &g, const int32_t *idx, int k, double *out,
                               cudaStream_t s) {
    TraceScope ts(CC_STAGE_GATHER, s);
    k_gather<<<1, 64, 0, s>>>(g.x, g.y, g.z, g.count, idx, k, out);
    return cudaGetLastError();
}

}  // namespace cc

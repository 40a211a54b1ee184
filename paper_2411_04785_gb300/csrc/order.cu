// order.cu - a compact traversal order of the sky directions for the sweep.
//
// The sweep gives each warp a run of consecutive directions of this order.
// When a warp's directions lie close together, most rings lie wholly on one
// side of them (every angle to the ring axis below pi/2, or every one above),
// and the warp sweeps those rings without the per-pair fold and select.  The
// order is the directions sorted by their HEALPix NESTED pixel (Gorski et al.
// 2005, the hierarchical numbering: pixels close in number are close on the
// sphere) at the coarsest nside with at least as many pixels as directions,
// ties in index order.  A HEALPix RING grid comes out in its NESTED order.
//
// The sort is a stable least-significant-digit radix sort of (pixel, index)
// with 8-bit digits: per pass, every block of 1024 directions counts its
// digits, one scan orders the (digit, block) counts, and one warp per block
// scatters its directions in index order (ranks among equal digits from
// __match_any_sync).  Everything is deterministic.
//
// The near-field back projection takes its voxels in the same way by their
// Morton (Z-order) key (point_order): 10 bits per coordinate across the
// set's bounding box, so each warp's run of voxels is a compact block.
#include "cc_internal.cuh"

namespace cc {
namespace {

constexpr int kOrderTile = 1024;      // directions per block of a radix pass

__device__ __forceinline__ uint32_t spread_bits(uint32_t v) {   // bit i -> bit 2 i
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// NESTED pixel of the direction (x, y, z) at nside = 2^L (L <= 13): the base
// face and the (ix, iy) position in it, from the equal-area projection of the
// HEALPix construction; its bits interleaved (ix even, iy odd) below the face.
// A direction that is not finite sorts last.
__device__ uint32_t nest_pixel(float x, float y, float z, int L) {
    const int ns = 1 << L;
    const float r = sqrtf(fmaf(x, x, fmaf(y, y, z * z)));
    if (!(r > 0.0f) || !isfinite(r)) return 0xFFFFFFFFu;
    const float zn = fminf(fmaxf(z / r, -1.0f), 1.0f), za = fabsf(zn);
    float phi = atan2f(y, x);
    if (phi < 0.0f) phi += 2.0f * kPiF;
    float tt = phi * (2.0f / kPiF);                    // in [0, 4)
    if (!(tt < 4.0f)) tt = 0.0f;
    int face, ix, iy;
    if (za <= 2.0f / 3.0f) {                          // equatorial zone
        const float a = ns * (0.5f + tt), b = ns * zn * 0.75f;
        const int jp = (int)(a - b), jm = (int)(a + b);   // edge-line indices
        const int ifp = jp >> L, ifm = jm >> L;
        face = ifp == ifm ? (ifp | 4) : (ifp < ifm ? ifp : ifm + 8);
        ix = jm & (ns - 1);
        iy = ns - (jp & (ns - 1)) - 1;
    } else {                                          // polar caps
        int ntt = (int)tt;
        if (ntt > 3) ntt = 3;
        const float tp = tt - ntt, tmp = ns * sqrtf(3.0f * (1.0f - za));
        int jp = (int)(tp * tmp), jm = (int)((1.0f - tp) * tmp);
        jp = jp < ns - 1 ? jp : ns - 1;
        jm = jm < ns - 1 ? jm : ns - 1;
        if (zn >= 0.0f) {
            face = ntt;
            ix = ns - jm - 1;
            iy = ns - jp - 1;
        } else {
            face = ntt + 8;
            ix = jp;
            iy = jm;
        }
    }
    face = face < 0 ? 0 : (face > 11 ? 11 : face);
    ix = ix < 0 ? 0 : (ix > ns - 1 ? ns - 1 : ix);
    iy = iy < 0 ? 0 : (iy > ns - 1 ? ns - 1 : iy);
    return ((uint32_t)face << (2 * L)) | spread_bits((uint32_t)ix) | (spread_bits((uint32_t)iy) << 1);
}

__global__ void __launch_bounds__(256)
k_order_keys(const float *__restrict__ x, const float *__restrict__ y, const float *__restrict__ z,
             int64_t M, int L, uint32_t *__restrict__ keys, int32_t *__restrict__ idx) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= M) return;
    keys[j] = nest_pixel(x[j], y[j], z[j], L);
    idx[j] = (int32_t)j;
}

// Digit counts of one block of kOrderTile keys: hist[digit * nblk + block].
__global__ void __launch_bounds__(32)
k_radix_hist(const uint32_t *__restrict__ keys, int64_t M, int shift, int32_t *__restrict__ hist,
             int64_t nblk) {
    __shared__ int32_t cnt[256];
    const int lane = threadIdx.x;
    for (int d = lane; d < 256; d += 32) cnt[d] = 0;
    __syncwarp();
    const int64_t b0 = blockIdx.x * (int64_t)kOrderTile;
    for (int s = 0; s < kOrderTile; s += 32) {
        const int64_t i = b0 + s + lane;
        if (i < M) atomicAdd(&cnt[(keys[i] >> shift) & 0xFFu], 1);
    }
    __syncwarp();
    for (int d = lane; d < 256; d += 32) hist[d * nblk + blockIdx.x] = cnt[d];
}

// Stable scatter of one block: its keys in index order, each to the scanned
// offset of its (digit, block) plus its rank among the block's earlier keys
// of the same digit.
__global__ void __launch_bounds__(32)
k_radix_scatter(const uint32_t *__restrict__ kin, const int32_t *__restrict__ iin, int64_t M,
                int shift, const int32_t *__restrict__ hist, int64_t nblk,
                uint32_t *__restrict__ kout, int32_t *__restrict__ iout) {
    __shared__ int32_t base[256];
    const int lane = threadIdx.x;
    for (int d = lane; d < 256; d += 32) base[d] = hist[d * nblk + blockIdx.x];
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t b0 = blockIdx.x * (int64_t)kOrderTile;
    for (int s = 0; s < kOrderTile; s += 32) {
        const int64_t i = b0 + s + lane;
        const bool on = i < M;
        const unsigned act = __ballot_sync(0xffffffffu, on);
        if (act == 0u) break;
        uint32_t key = 0, d = 0;
        unsigned peers = 0;
        int pos = 0;
        if (on) {
            key = kin[i];
            d = (key >> shift) & 0xFFu;
            peers = __match_any_sync(act, d);
            pos = base[d] + __popc(peers & lt);
        }
        __syncwarp();
        if (on) {
            if (CC_IN_BOUNDS(CC_SITE_ORDER, pos, M)) {
                kout[pos] = key;
                iout[pos] = iin[i];
            }
            if (lane == 31 - __clz((int)peers)) base[d] += __popc(peers);   // the group's last lane
        }
        __syncwarp();
    }
}

int order_level(int64_t M) {   // coarsest L with 12 * 4^L >= M, at most 13
    int L = 0;
    while (L < 13 && 12ll << (2 * L) < M) L++;
    return L;
}

// Bounding box of a point set: one CTA, lo[3] then hi[3] into box[6]; points
// that are not finite are ignored (an empty box stays +inf / -inf).
__global__ void __launch_bounds__(1024)
k_bbox(const float *__restrict__ x, const float *__restrict__ y, const float *__restrict__ z,
       int64_t M, float *__restrict__ box) {
    __shared__ float red[6][32];
    float v[6] = {__builtin_huge_valf(), __builtin_huge_valf(), __builtin_huge_valf(),
                  -__builtin_huge_valf(), -__builtin_huge_valf(), -__builtin_huge_valf()};
    for (int64_t j = threadIdx.x; j < M; j += blockDim.x) {
        const float a = x[j], b = y[j], c = z[j];
        if (!isfinite(a) || !isfinite(b) || !isfinite(c)) continue;
        v[0] = fminf(v[0], a); v[1] = fminf(v[1], b); v[2] = fminf(v[2], c);
        v[3] = fmaxf(v[3], a); v[4] = fmaxf(v[4], b); v[5] = fmaxf(v[5], c);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 6; q++) {
            const float u = __shfl_xor_sync(0xffffffffu, v[q], o);
            v[q] = q < 3 ? fminf(v[q], u) : fmaxf(v[q], u);
        }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
        for (int q = 0; q < 6; q++) red[q][w] = v[q];
    __syncthreads();
    if (threadIdx.x < 6) {
        float a = red[threadIdx.x][0];
        for (int k = 1; k < nw; k++)
            a = threadIdx.x < 3 ? fminf(a, red[threadIdx.x][k]) : fmaxf(a, red[threadIdx.x][k]);
        box[threadIdx.x] = a;
    }
}

__device__ __forceinline__ uint32_t spread3(uint32_t v) {   // bit i -> bit 3 i (10 bits)
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Morton (Z-order) key of each point: its coordinates quantised to 10 bits
// each across the bounding box, bits interleaved (x lowest).  A point that is
// not finite sorts last.
__global__ void __launch_bounds__(256)
k_morton_keys(const float *__restrict__ x, const float *__restrict__ y,
              const float *__restrict__ z, int64_t M, const float *__restrict__ box,
              uint32_t *__restrict__ keys, int32_t *__restrict__ idx) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= M) return;
    const float p[3] = {x[j], y[j], z[j]};
    uint32_t key = 0;
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        ok = ok && isfinite(p[c]);
        const float lo = box[c], ext = box[3 + c] - box[c];
        float t = ext > 0.0f ? (p[c] - lo) * (1024.0f / ext) : 0.0f;
        t = fminf(fmaxf(t, 0.0f), 1023.0f);
        key |= spread3((uint32_t)t) << c;
    }
    keys[j] = ok ? key : 0xFFFFFFFFu;
    idx[j] = (int32_t)j;
}

// Scratch of a sort of M keys: two key buffers, one index buffer, the digit
// counts, the scan total, and a 6-float bounding box.
struct SortScratch {
    uint32_t *k0, *k1;
    int32_t *tmp, *hist;
    int64_t *total;
    float *box;
};

SortScratch carve(char *scratch, int64_t M) {
    const int64_t nblk = (M + kOrderTile - 1) / kOrderTile;
    SortScratch q;
    char *c = scratch;
    q.k0 = reinterpret_cast<uint32_t *>(c);
    c += align256((size_t)M * sizeof(uint32_t));
    q.k1 = reinterpret_cast<uint32_t *>(c);
    c += align256((size_t)M * sizeof(uint32_t));
    q.tmp = reinterpret_cast<int32_t *>(c);
    c += align256((size_t)M * sizeof(int32_t));
    q.hist = reinterpret_cast<int32_t *>(c);
    c += align256((size_t)(256 * nblk) * sizeof(int32_t));
    q.total = reinterpret_cast<int64_t *>(c);
    c += align256(sizeof(int64_t));
    q.box = reinterpret_cast<float *>(c);
    return q;
}

// Stable LSD radix sort of the (key, index) pairs in (q.k0, idx0) on the low
// `bits` bits; the sorted indices end in perm.  idx0 is q.tmp or perm, as the
// pass count requires (first_index_buffer).
cudaError_t radix_sort(const SortScratch &q, int32_t *perm, int64_t M, int bits,
                       cudaStream_t s) {
    const int64_t nblk = (M + kOrderTile - 1) / kOrderTile;
    const int passes = (bits + 7) / 8;
    int32_t *ibuf[2] = {passes % 2 ? q.tmp : perm, passes % 2 ? perm : q.tmp};
    uint32_t *kbuf[2] = {q.k0, q.k1};
    cudaError_t e;
    for (int p = 0; p < passes; p++) {
        const int a = p & 1, b = a ^ 1;
        k_radix_hist<<<(unsigned)nblk, 32, 0, s>>>(kbuf[a], M, 8 * p, q.hist, nblk);
        if ((e = launch_pack_scan(q.hist, 256 * nblk, q.total, s)) != cudaSuccess) return e;
        k_radix_scatter<<<(unsigned)nblk, 32, 0, s>>>(kbuf[a], ibuf[a], M, 8 * p, q.hist, nblk,
                                                      kbuf[b], ibuf[b]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The index buffer the keys kernel fills: the last pass must leave the
// indices in perm.
int32_t *first_index_buffer(const SortScratch &q, int32_t *perm, int bits) {
    return ((bits + 7) / 8) % 2 ? q.tmp : perm;
}

}  // namespace

size_t direction_order_bytes(int64_t M) {
    if (M < 1) return 0;
    const int64_t nblk = (M + kOrderTile - 1) / kOrderTile;
    return 2 * align256((size_t)M * sizeof(uint32_t)) + align256((size_t)M * sizeof(int32_t)) +
           align256((size_t)(256 * nblk) * sizeof(int32_t)) + align256(sizeof(int64_t)) +
           align256(6 * sizeof(float));
}

cudaError_t direction_order(const cc_grid &g, int32_t *perm, char *scratch, cudaStream_t s) {
    const int64_t M = g.count;
    if (M < 1) return cudaSuccess;
    const SortScratch q = carve(scratch, M);
    const int L = order_level(M);
    const int bits = 2 * L + 4;                       // 12 faces < 16
    k_order_keys<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(g.x, g.y, g.z, M, L, q.k0,
                                                             first_index_buffer(q, perm, bits));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return radix_sort(q, perm, M, bits, s);
}

int direction_order_kernels(int64_t M) {   // keys, then per pass: counts, scan, scatter
    return M < 1 ? 0 : 1 + 3 * ((2 * order_level(M) + 4 + 7) / 8);
}

int point_order_kernels(int64_t M) {       // box, keys, 4 passes
    return M < 1 ? 0 : 2 + 3 * 4;
}

cudaError_t point_order(const float *x, const float *y, const float *z, int64_t M, int32_t *perm,
                        char *scratch, cudaStream_t s) {
    if (M < 1) return cudaSuccess;
    const SortScratch q = carve(scratch, M);
    const int bits = 30;
    k_bbox<<<1, 1024, 0, s>>>(x, y, z, M, q.box);
    k_morton_keys<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(x, y, z, M, q.box, q.k0,
                                                              first_index_buffer(q, perm, bits));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return radix_sort(q, perm, M, bits, s);
}

}  // namespace cc

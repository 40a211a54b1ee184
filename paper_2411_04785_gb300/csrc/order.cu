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

}  // namespace

size_t direction_order_bytes(int64_t M) {
    if (M < 1) return 0;
    const int64_t nblk = (M + kOrderTile - 1) / kOrderTile;
    return 2 * align256((size_t)M * sizeof(uint32_t)) + align256((size_t)M * sizeof(int32_t)) +
           align256((size_t)(256 * nblk) * sizeof(int32_t)) + align256(sizeof(int64_t));
}

cudaError_t direction_order(const cc_grid &g, int32_t *perm, char *scratch, cudaStream_t s) {
    const int64_t M = g.count;
    if (M < 1) return cudaSuccess;
    const int64_t nblk = (M + kOrderTile - 1) / kOrderTile;
    uint32_t *k0 = reinterpret_cast<uint32_t *>(scratch);
    uint32_t *k1 = reinterpret_cast<uint32_t *>(scratch + align256((size_t)M * sizeof(uint32_t)));
    int32_t *tmp = reinterpret_cast<int32_t *>(scratch + 2 * align256((size_t)M * sizeof(uint32_t)));
    int32_t *hist = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(tmp) +
                                                align256((size_t)M * sizeof(int32_t)));
    int64_t *total = reinterpret_cast<int64_t *>(reinterpret_cast<char *>(hist) +
                                                 align256((size_t)(256 * nblk) * sizeof(int32_t)));
    const int L = order_level(M);
    const int bits = 2 * L + 4;                       // 12 faces < 16
    const int passes = (bits + 7) / 8;
    // the last pass must leave the indices in perm
    int32_t *ibuf[2] = {passes % 2 ? tmp : perm, passes % 2 ? perm : tmp};
    uint32_t *kbuf[2] = {k0, k1};
    k_order_keys<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(g.x, g.y, g.z, M, L, kbuf[0], ibuf[0]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int p = 0; p < passes; p++) {
        const int a = p & 1, b = a ^ 1;
        k_radix_hist<<<(unsigned)nblk, 32, 0, s>>>(kbuf[a], M, 8 * p, hist, nblk);
        if ((e = launch_pack_scan(hist, 256 * nblk, total, s)) != cudaSuccess) return e;
        k_radix_scatter<<<(unsigned)nblk, 32, 0, s>>>(kbuf[a], ibuf[a], M, 8 * p, hist, nblk,
                                                      kbuf[b], ibuf[b]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace cc

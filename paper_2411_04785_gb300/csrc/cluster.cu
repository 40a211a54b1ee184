// cluster.cu - event clustering of time-sorted detections by a maximum step
// between consecutive detections (Sec. 2 of the paper), one pass over HBM.
//
// Sec. 2 defines, for detections sorted by time, the step to the next
// detection, a mask "step < dt_max" on it, and the edge of a detection as the
// XOR of the masks on its two sides (no step outside the stream: false).  A
// run of detections joined by masked steps is one event; its first and last
// detection carry the edges.  The paper computes the edges with two kernels;
// here one kernel computes the edges AND builds the events: every detection
// gets its event number (-1 when isolated) and every event its first
// detection, its size and its amplitude sum.
//
// Event numbers are a prefix count of event starts (a detection whose step
// before is not masked and whose step after is), so the kernel is a
// single-pass chained scan: a CTA takes the next tile of 4096 detections from
// a ticket counter, computes the tile's aggregate, publishes it, looks back
// over the tiles before it until one has published its inclusive prefix
// (decoupled look-back; every wait is bounded), publishes its own inclusive
// prefix and writes its outputs.  t and adc are read once, coalesced; the
// outputs are written once.  The scan state of a range of detections is
// (starts in it, index of its last start, its amplitude sum, its amplitude
// sum before its last start), which composes associatively, so an event's
// amplitude sum is the difference of two prefix sums taken at its two edges
// with no per-event atomics.  All arithmetic is integer: results are exact.
//
// Layout inside a tile: the tile's t (32 KB) and adc (16 KB) arrive in
// shared memory by two TMA tensor copies (t seen as rows of 16 int64, adc as
// rows of 32 uint32; 128-byte rows in the 128B swizzle) on one mbarrier.
// Every lane owns 16 consecutive detections: it reads its own row (or half
// row) chunk by chunk - the swizzle puts the chunks of 8 neighbouring rows
// in 8 different bank groups, so the reads are conflict-free - builds its
// 16 step masks, scans its detections serially, and the lanes of a warp
// combine their aggregates in one warp scan per 16 detections.  Edges and
// event ids leave as 16-byte stores.
#include <string.h>

#include "cc_internal.cuh"
#include "cc_pipe.cuh"

namespace cc {
namespace {

constexpr int kCWarps = 8;
constexpr int kCThreads = kCWarps * 32;
constexpr int kRows = 16;
constexpr int kWarpSpan = kRows * 32;            // 512
constexpr int kTileSpan = kWarpSpan * kCWarps;   // 4096: 48 KB staged, 4 CTAs per SM
constexpr int kLook = 1;                         // predecessors per lane per look-back round

struct Carry {
    long long starts;              // event starts in the range
    long long last_start;          // index of the range's last start, -1 if none
    unsigned long long sum;        // amplitude sum over the range
    unsigned long long sum_before; // amplitude sum of the range before its last start
};

__device__ __forceinline__ Carry identity() { return Carry{0, -1, 0ull, 0ull}; }

// a covers the detections just before those of b
__device__ __forceinline__ Carry combine(const Carry &a, const Carry &b) {
    Carry c;
    c.starts = a.starts + b.starts;
    c.sum = a.sum + b.sum;
    if (b.last_start >= 0) {
        c.last_start = b.last_start;
        c.sum_before = a.sum + b.sum_before;
    } else {
        c.last_start = a.last_start;
        c.sum_before = a.sum_before;
    }
    return c;
}

struct TileState {                 // published by the CTA that owns the tile
    Carry agg;                     // its own range
    Carry incl;                    // everything up to its end
    int status;                    // 0 nothing, 1 agg ready, 2 incl ready
    int pad[3];
};

__device__ __forceinline__ void put(volatile Carry *dst, const Carry &v) {
    dst->starts = v.starts;
    dst->last_start = v.last_start;
    dst->sum = v.sum;
    dst->sum_before = v.sum_before;
}

__device__ __forceinline__ Carry get(const volatile Carry *src) {
    return Carry{src->starts, src->last_start, src->sum, src->sum_before};
}

// step from a to b in wrapping 64-bit arithmetic (meaningful for |step| < 2^63)
__device__ __forceinline__ long long step_of(long long a, long long b) {
    return (long long)((unsigned long long)b - (unsigned long long)a);
}

__device__ __forceinline__ Carry shfl_down_carry(const Carry &c, int o) {
    return Carry{__shfl_down_sync(0xffffffffu, c.starts, o),
                 __shfl_down_sync(0xffffffffu, c.last_start, o),
                 __shfl_down_sync(0xffffffffu, c.sum, o),
                 __shfl_down_sync(0xffffffffu, c.sum_before, o)};
}

// Shared memory of one CTA: the tile's time stamps (256 rows of 16) and
// amplitudes (128 rows of 32), 128-byte rows in the TMA 128B swizzle (the
// 16-byte chunk c of row r sits at chunk c ^ (r & 7)), so that a lane reading
// its own row's chunks never conflicts with the lanes beside it.
struct ClusterSmem {
    unsigned char tsw[kTileSpan * 8];     // t, swizzled
    unsigned char asw[kTileSpan * 4];     // adc, swizzled
    long long t_prev, t_next;
    unsigned long long bar;
    long long tile;
    Carry warp_agg[kCWarps];
    Carry warp_excl[kCWarps];
    Carry tile_agg, tile_excl;
    int load_failed;
};
constexpr size_t kClusterSmemBytes = sizeof(ClusterSmem) + 1024;   // + alignment of the rows

__device__ __forceinline__ int swz(int row, int chunk) { return row * 128 + ((chunk ^ (row & 7)) << 4); }

// element e of the tile: its byte offset in tsw / asw
__device__ __forceinline__ int t_off(int e) { return swz(e >> 4, (e & 15) >> 1) + ((e & 1) << 3); }
__device__ __forceinline__ int a_off(int e) { return swz(e >> 5, (e & 31) >> 2) + ((e & 3) << 2); }

__global__ void __launch_bounds__(kCThreads, 4)   // 4 CTAs per SM: 64 registers
k_cluster(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap amap,
          int use_tma, const long long *__restrict__ t, const unsigned *__restrict__ adc,
          long long N, long long dt_max, unsigned char *__restrict__ edge,
          int *__restrict__ event_id, int vec_out, long long *__restrict__ ev_first,
          int *__restrict__ ev_count, unsigned long long *__restrict__ ev_adc,
          long long *__restrict__ n_events, TileState *__restrict__ tiles,
          unsigned long long *__restrict__ ticket, int *__restrict__ status, long long ahead) {
    extern __shared__ unsigned char smem_raw[];
    ClusterSmem &S = *reinterpret_cast<ClusterSmem *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long ntiles = (N + kTileSpan - 1) / kTileSpan;
    if (threadIdx.x == 0) {
        S.tile = (long long)atomicAdd(ticket, 1ull);
        S.load_failed = 0;
        mbar_init(&S.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const long long tile = S.tile;
    const long long base = tile * kTileSpan;
    // whole tiles inside the tensor maps (rows of 32 detections) by TMA
    const bool bulk = use_tma && base + kTileSpan <= (N / 32) * 32;
    if (bulk) {
        if (threadIdx.x == 0) {
            const unsigned bytes = kTileSpan * 8u + (adc ? kTileSpan * 4u : 0u);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                             smem_u32(&S.bar)), "r"(bytes)
                         : "memory");
            tma_load_2d(S.tsw, &tmap, 0, (int)(base / 16), &S.bar);
            if (adc) tma_load_2d(S.asw, &amap, 0, (int)(base / 32), &S.bar);
        }
        if (adc == nullptr)
            for (int e = threadIdx.x; e < kTileSpan; e += kCThreads)
                *reinterpret_cast<unsigned *>(S.asw + a_off(e)) = 0u;
    } else {
        for (int e = threadIdx.x; e < kTileSpan; e += kCThreads) {
            const long long g = base + e;
            *reinterpret_cast<long long *>(S.tsw + t_off(e)) = g < N ? __ldcs(t + g) : 0;
            *reinterpret_cast<unsigned *>(S.asw + a_off(e)) =
                (adc != nullptr && g < N) ? __ldcs(adc + g) : 0u;
        }
    }
    if (use_tma && ahead > 0 && threadIdx.x >= 64 && threadIdx.x < 66) {
        // the tile that a CTA starting about one CTA lifetime from now will
        // take (tickets are handed out in order, 4 CTAs per SM are resident):
        // its time stamps and amplitudes are fetched into L2 now, so that its
        // tensor copies find them there (measured: 0.69 -> 0.67 ms on the
        // 81.7M-detection stream; twice as far ahead was slower)
        const long long pb = base + ahead * kTileSpan;
        if (pb + kTileSpan <= N && (threadIdx.x == 64 || adc != nullptr)) {
            const void *p = threadIdx.x == 64 ? (const void *)(t + pb) : (const void *)(adc + pb);
            const unsigned bytes = threadIdx.x == 64 ? kTileSpan * 8u : kTileSpan * 4u;
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
        }
    }
    if (threadIdx.x == 32) {
        S.t_prev = base > 0 ? __ldg(t + base - 1) : 0;
        S.t_next = base + kTileSpan < N ? __ldg(t + base + kTileSpan) : 0;
    }
    if (bulk && threadIdx.x == 0 && !mbar_wait(&S.bar, 0)) S.load_failed = 1;
    __syncthreads();
    if (S.load_failed) {          // a bounded wait gave up: report, publish, go on
        if (threadIdx.x == 0) atomicExch(status, (int)CC_ETIMEOUT);
        for (int i = threadIdx.x; i < kTileSpan * 12 / 16; i += kCThreads)
            reinterpret_cast<int4 *>(S.tsw)[i] = make_int4(0, 0, 0, 0);
        __syncthreads();
    }

    // ---- each lane owns 16 consecutive detections: tile elements
    // e0 .. e0 + 15, row r of the time stamps
    const int e0 = w * kWarpSpan + lane * 16;
    const long long i0 = base + e0;
    const int r = e0 >> 4;
    unsigned ma = 0, mb = 0;        // bit k: step after / before detection i0 + k is masked
    {
        long long tv[16];
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const longlong2 v = *reinterpret_cast<const longlong2 *>(S.tsw + swz(r, c));
            tv[2 * c] = v.x;
            tv[2 * c + 1] = v.y;
        }
        long long tn = __shfl_down_sync(0xffffffffu, tv[0], 1);
        long long tp = __shfl_up_sync(0xffffffffu, tv[15], 1);
        if (lane == 31) tn = e0 + 16 < kTileSpan ? *reinterpret_cast<const long long *>(S.tsw + t_off(e0 + 16)) : S.t_next;
        if (lane == 0) tp = e0 > 0 ? *reinterpret_cast<const long long *>(S.tsw + t_off(e0 - 1)) : S.t_prev;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const long long nx = k < 15 ? tv[k + 1 < 16 ? k + 1 : 15] : tn;
            const bool a_k = (i0 + k + 1 < N) && step_of(tv[k], nx) < dt_max;
            ma |= (unsigned)a_k << k;
        }
        const bool b0 = (i0 > 0) && (i0 < N) && step_of(tp, tv[0]) < dt_max;
        mb = ((ma << 1) | (unsigned)b0) & 0xFFFFu;
        if (i0 + 16 > N) {          // detections past the end have no steps
            const long long room = N - i0;
            const unsigned keep = room <= 0 ? 0u : ((1u << (unsigned)room) - 1u);
            mb &= keep;
        }
    }
    const unsigned sbits = ma & ~mb, ebits = mb & ~ma;

    // ---- the lane's aggregate and the warp's inclusive scan of them
    const int arow = e0 >> 5, ach = (lane & 1) * 4;
    auto adc_at = [&](int k) -> unsigned {
        return *reinterpret_cast<const unsigned *>(S.asw + swz(arow, ach + (k >> 2)) + ((k & 3) << 2));
    };
    Carry mine{__popc(sbits), -1, 0ull, 0ull};
    const int lastk = sbits ? 31 - __clz((int)sbits) : -1;
    if (lastk >= 0) mine.last_start = i0 + lastk;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const uint4 v = *reinterpret_cast<const uint4 *>(S.asw + swz(arow, ach + c));
        const unsigned q[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            mine.sum += q[j];
            if (4 * c + j < lastk) mine.sum_before += q[j];
        }
    }
    Carry incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Carry y{__shfl_up_sync(0xffffffffu, incl.starts, o),
                      __shfl_up_sync(0xffffffffu, incl.last_start, o),
                      __shfl_up_sync(0xffffffffu, incl.sum, o),
                      __shfl_up_sync(0xffffffffu, incl.sum_before, o)};
        if (lane >= o) incl = combine(y, incl);
    }
    Carry lane_excl{__shfl_up_sync(0xffffffffu, incl.starts, 1),
                    __shfl_up_sync(0xffffffffu, incl.last_start, 1),
                    __shfl_up_sync(0xffffffffu, incl.sum, 1),
                    __shfl_up_sync(0xffffffffu, incl.sum_before, 1)};
    if (lane == 0) lane_excl = identity();
    if (lane == 31) S.warp_agg[w] = incl;
    __syncthreads();

    // ---- tile aggregate, look-back, tile prefix.  Warp 0 looks back over
    // windows of 32 predecessors at once: it waits until each predecessor up
    // to the nearest one that has published its inclusive prefix has
    // published at least its aggregate, combines them in order, and stops
    // there.
    if (threadIdx.x == 0) {
        Carry acc = identity();
        for (int k = 0; k < kCWarps; k++) {
            S.warp_excl[k] = acc;
            acc = combine(acc, S.warp_agg[k]);
        }
        S.tile_agg = acc;
        volatile TileState *me = tiles + tile;
        if (tile == 0) put(&me->incl, acc);
        else put(&me->agg, acc);
        __threadfence();
        me->status = tile == 0 ? 2 : 1;
    }
    __syncthreads();
    if (w == 0) {
        // windows of 32 x kLook predecessors: lane l covers tiles
        // hi - kLook l - j (j = 0 nearest), all loaded in one round trip
        Carry excl = identity();
        bool timed_out = false;
        unsigned long long t0 = 0;
        for (long long hi = tile - 1; hi >= 0;) {
            int st[kLook];
            int pending = 0, incl = 0;
#pragma unroll
            for (int j = 0; j < kLook; j++) {
                const long long p = hi - kLook * lane - j;
                st[j] = p >= 0 ? ((volatile TileState *)tiles)[p].status : 2;
                pending |= st[j] == 0;
                incl |= st[j] == 2;
            }
            // only the lanes up to the nearest inclusive prefix are needed:
            // wait for those, not for older tiles beyond it
            auto waiting = [&]() {
                const unsigned im = __ballot_sync(0xffffffffu, incl);
                const int need = im ? __ffs(im) : 32;
                return __any_sync(0xffffffffu, pending && lane < need);
            };
            for (unsigned it = 0; waiting(); ++it) {
                pending = 0;
                incl = 0;
#pragma unroll
                for (int j = 0; j < kLook; j++) {
                    const long long p = hi - kLook * lane - j;
                    if (st[j] == 0) st[j] = ((volatile TileState *)tiles)[p].status;
                    pending |= st[j] == 0;
                    incl |= st[j] == 2;
                }
                if ((it & 63) == 0) {   // lane 0's clock for all: the exit stays warp-uniform
                    const unsigned long long now = __shfl_sync(0xffffffffu, globaltimer_ns(), 0);
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > kWaitLimitNs) { timed_out = true; break; }
                }
            }
            if (timed_out) break;
            __threadfence();
            // the lane's value: its tiles from the farthest in, cut at its
            // nearest inclusive prefix
            Carry v = identity();
            bool has_incl = false;
#pragma unroll
            for (int j = kLook - 1; j >= 0; j--) {
                const long long p = hi - kLook * lane - j;
                Carry x = identity();
                if (p >= 0) x = st[j] == 2 ? get(&((volatile TileState *)tiles)[p].incl)
                                           : get(&((volatile TileState *)tiles)[p].agg);
                if (st[j] == 2) { v = x; has_incl = true; }
                else v = combine(v, x);
            }
            const unsigned incl_mask = __ballot_sync(0xffffffffu, has_incl);
            const int n = incl_mask ? __ffs(incl_mask) : 32;   // lanes [0, n) take part
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {                 // ordered tree reduction
                const Carry y = shfl_down_carry(v, o);
                if (lane + o < n) v = combine(y, v);
            }
            excl = combine(v, excl);                           // lane 0's value is the window's
            if (incl_mask) break;
            hi -= 32 * kLook;
        }
        if (lane == 0) {
            if (timed_out) atomicExch(status, (int)CC_ETIMEOUT);
            if (tile > 0) {
                volatile TileState *me = tiles + tile;
                put(&me->incl, combine(excl, S.tile_agg));
                __threadfence();
                me->status = 2;
            }
            S.tile_excl = excl;
            if (tile == ntiles - 1 && n_events != nullptr)
                *n_events = combine(excl, S.tile_agg).starts;
        }
    }
    __syncthreads();

    // ---- outputs: the lane walks its 16 detections with the running prefix
    const Carry c0 = combine(S.tile_excl, combine(S.warp_excl[w], lane_excl));
    long long rank = c0.starts, last = c0.last_start;
    unsigned long long sum = c0.sum, before = c0.sum_before;
    unsigned eb[4] = {0u, 0u, 0u, 0u};
    int ids[16];
#pragma unroll
    for (int k = 0; k < 16; k++) {
        const long long i = i0 + k;
        const bool st = (sbits >> k) & 1u, en = (ebits >> k) & 1u;
        const bool in = ((ma | mb) >> k) & 1u;
        if (st) {
            last = i;
            before = sum;
        }
        sum += adc_at(k);
        rank += st;
        ids[k] = in ? (int)(rank - 1) : -1;
        eb[k >> 2] |= (unsigned)((((ma ^ mb) >> k) & 1u)) << (8 * (k & 3));
        if (en && i < N && CC_IN_BOUNDS(CC_SITE_CLUSTER_EVENT, rank - 1, N / 2)) {
            const long long id = rank - 1;
            if (ev_first) ev_first[id] = last;
            if (ev_count) ev_count[id] = (int)(i - last + 1);
            if (ev_adc) ev_adc[id] = sum - before;
        }
    }
    if (vec_out && i0 + 16 <= N && CC_IN_BOUNDS(CC_SITE_CLUSTER_OUT, i0 + 15, N)) {
        if (edge) *reinterpret_cast<uint4 *>(edge + i0) = make_uint4(eb[0], eb[1], eb[2], eb[3]);
        if (event_id) {
#pragma unroll
            for (int q = 0; q < 4; q++)
                reinterpret_cast<int4 *>(event_id + i0)[q] =
                    make_int4(ids[4 * q], ids[4 * q + 1], ids[4 * q + 2], ids[4 * q + 3]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 16; k++) {
            if (i0 + k < N && CC_IN_BOUNDS(CC_SITE_CLUSTER_OUT, i0 + k, N)) {
                if (edge) edge[i0 + k] = (unsigned char)((eb[k >> 2] >> (8 * (k & 3))) & 1u);
                if (event_id) event_id[i0 + k] = ids[k];
            }
        }
    }
}

// Histogram of event amplitudes: bin = adc / bin_width, the last bin also
// takes everything above it.  Counts in shared memory when they fit.
__global__ void __launch_bounds__(256)
k_spectrum(const unsigned long long *__restrict__ ev_adc, const long long *__restrict__ n_events,
           unsigned long long bin_width, int nbins, unsigned long long *__restrict__ hist) {
    extern __shared__ unsigned sh[];
    const bool local = nbins <= 8192;
    if (local)
        for (int b = threadIdx.x; b < nbins; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    const long long K = *n_events;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < K;
         k += (long long)gridDim.x * blockDim.x) {
        unsigned long long b = ev_adc[k] / bin_width;
        const int bi = b < (unsigned long long)nbins ? (int)b : nbins - 1;
        if (local) atomicAdd(sh + bi, 1u);
        else atomicAdd(hist + bi, 1ull);
    }
    __syncthreads();
    if (local)
        for (int b = threadIdx.x; b < nbins; b += blockDim.x)
            if (sh[b]) atomicAdd(hist + b, (unsigned long long)sh[b]);
}

}  // namespace

size_t cluster_workspace_bytes(int64_t n) {
    const int64_t tiles = n > 0 ? (n + kTileSpan - 1) / kTileSpan : 1;
    return align256(sizeof(unsigned long long)) + align256((size_t)tiles * sizeof(TileState)) +
           align256(sizeof(int));
}

cudaError_t launch_cluster(const int64_t *t, const uint32_t *adc, int64_t n, int64_t dt_max,
                           uint8_t *edge, int32_t *event_id, int64_t *ev_first, int32_t *ev_count,
                           uint64_t *ev_adc, int64_t *n_events, int32_t *status, char *ws,
                           cudaStream_t s) {
    const int64_t tiles = n > 0 ? (n + kTileSpan - 1) / kTileSpan : 1;
    auto *ticket = reinterpret_cast<unsigned long long *>(ws);
    auto *state = reinterpret_cast<TileState *>(ws + align256(sizeof(unsigned long long)));
    int32_t *st = status ? status
                         : reinterpret_cast<int32_t *>(ws + align256(sizeof(unsigned long long)) +
                                                       align256((size_t)tiles * sizeof(TileState)));
    cudaError_t e = cudaMemsetAsync(ws, 0, align256(sizeof(unsigned long long)) +
                                               (size_t)tiles * sizeof(TileState), s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(st, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    if (n == 0) {
        if (n_events) return cudaMemsetAsync(n_events, 0, sizeof(int64_t), s);
        return cudaSuccess;
    }
    // tensor maps of t as [N/16][16] int64 and adc as [N/32][32] uint32 rows,
    // 128B swizzle, boxes of one tile (256 x 16 and 128 x 32)
    CUtensorMap tmap, amap;
    memset(&tmap, 0, sizeof(tmap));
    memset(&amap, 0, sizeof(amap));
    auto al16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    int use_tma = n >= kTileSpan && al16(t) && (adc == nullptr || al16(adc)) && encode_fn() != nullptr;
    if (use_tma) {
        const cuuint64_t gst[1] = {128};
        const cuuint32_t es[2] = {1, 1};
        const cuuint64_t gdt[2] = {16, (cuuint64_t)(n / 16)};
        const cuuint32_t bt[2] = {16, (cuuint32_t)(kTileSpan / 16)};
        CUresult r = encode_fn()(&tmap, CU_TENSOR_MAP_DATA_TYPE_INT64, 2, const_cast<int64_t *>(t),
                                 gdt, gst, bt, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS && adc != nullptr) {
            const cuuint64_t gda[2] = {32, (cuuint64_t)(n / 32)};
            const cuuint32_t ba[2] = {32, (cuuint32_t)(kTileSpan / 32)};
            r = encode_fn()(&amap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t *>(adc),
                            gda, gst, ba, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        }
        if (r != CUDA_SUCCESS) use_tma = 0;          // plain loads instead
    }
    const int vec_out = (edge == nullptr || al16(edge)) && (event_id == nullptr || al16(event_id));
    // the staged tile needs more than 48 KB of shared memory (set per call:
    // the attribute belongs to the current device)
    e = cudaFuncSetAttribute((const void *)k_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kClusterSmemBytes);
    if (e != cudaSuccess) return e;
    TraceScope ts(CC_STAGE_CLUSTER, s);
    k_cluster<<<(unsigned)tiles, kCThreads, kClusterSmemBytes, s>>>(
        tmap, amap, use_tma, reinterpret_cast<const long long *>(t), adc, (long long)n,
        (long long)dt_max, edge, event_id, vec_out, reinterpret_cast<long long *>(ev_first),
        ev_count, reinterpret_cast<unsigned long long *>(ev_adc),
        reinterpret_cast<long long *>(n_events), state, ticket, st, 4LL * device_sm_count());
    return cudaGetLastError();
}

cudaError_t launch_spectrum(const uint64_t *ev_adc, const int64_t *n_events, uint64_t bin_width,
                            int32_t nbins, uint64_t *hist, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)nbins * sizeof(uint64_t), s);
    if (e != cudaSuccess) return e;
    const size_t smem = nbins <= 8192 ? (size_t)nbins * sizeof(unsigned) : 0;
    TraceScope ts(CC_STAGE_CLUSTER, s);
    k_spectrum<<<(unsigned)(device_sm_count() * 2), 256, smem, s>>>(
        reinterpret_cast<const unsigned long long *>(ev_adc),
        reinterpret_cast<const long long *>(n_events), (unsigned long long)bin_width, nbins,
        reinterpret_cast<unsigned long long *>(hist));
    return cudaGetLastError();
}

}  // namespace cc

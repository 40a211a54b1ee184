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
// Layout inside a tile: the tile's t (32 KB) and adc (16 KB) are staged in
// shared memory by two bulk copies (TMA) completing on one mbarrier, so no
// thread holds the tile in registers and four CTAs fit an SM (measured
// faster than eight 4-warp CTAs of 2048 detections and than two persistent
// double-buffered ones); warp w then reads its 512 consecutive detections as 16 rows of 32 (lane l of row r
// holds detection base + 512 w + 32 r + l), conflict-free, and the row-level
// prefix counts are ballots.
#include "cc_internal.cuh"
#include "cc_pipe.cuh"

namespace cc {
namespace {

constexpr int kCWarps = 8;
constexpr int kCThreads = kCWarps * 32;
constexpr int kRows = 16;
constexpr int kWarpSpan = kRows * 32;            // 512
constexpr int kTileSpan = kWarpSpan * kCWarps;   // 4096: 48 KB staged, 4 CTAs per SM

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

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Shared memory of one CTA: the tile's time stamps and amplitudes (staged
// by two bulk copies), the neighbours just outside it, and the scan state.
struct ClusterSmem {
    long long ts[kTileSpan];
    unsigned as[kTileSpan];
    long long t_prev, t_next;
    unsigned long long bar;
    long long tile;
};

__global__ void __launch_bounds__(kCThreads)
k_cluster(const long long *__restrict__ t, const unsigned *__restrict__ adc, long long N,
          long long dt_max, unsigned char *__restrict__ edge, int *__restrict__ event_id,
          long long *__restrict__ ev_first, int *__restrict__ ev_count,
          unsigned long long *__restrict__ ev_adc, long long *__restrict__ n_events,
          TileState *__restrict__ tiles, unsigned long long *__restrict__ ticket,
          int *__restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ClusterSmem &S = *reinterpret_cast<ClusterSmem *>(smem_raw);
    __shared__ Carry warp_agg[kCWarps];
    __shared__ Carry warp_excl[kCWarps];
    __shared__ Carry tile_excl;
    __shared__ int load_failed;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        S.tile = (long long)atomicAdd(ticket, 1ull);
        mbar_init(&S.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        load_failed = 0;
    }
    __syncthreads();
    const long long tile = S.tile;
    const long long base = tile * kTileSpan;
    const long long n_here = N - base < kTileSpan ? N - base : kTileSpan;

    // ---- stage the tile: whole aligned tiles by two bulk copies on one
    // mbarrier, the ragged last tile by plain loads
    const bool bulk = n_here == kTileSpan && ((reinterpret_cast<uintptr_t>(t) & 15u) == 0) &&
                      (adc == nullptr || (reinterpret_cast<uintptr_t>(adc) & 15u) == 0);
    if (bulk) {
        if (threadIdx.x == 0) {
            const unsigned bytes = kTileSpan * 8u + (adc ? kTileSpan * 4u : 0u);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                             smem_u32(&S.bar)), "r"(bytes)
                         : "memory");
            bulk_copy(S.ts, t + base, kTileSpan * 8u, &S.bar);
            if (adc) bulk_copy(S.as, adc + base, kTileSpan * 4u, &S.bar);
        }
        if (adc == nullptr)
            for (int i = threadIdx.x; i < kTileSpan; i += kCThreads) S.as[i] = 0u;
    } else {
        for (int i = threadIdx.x; i < kTileSpan; i += kCThreads) {
            const long long g = base + i;
            S.ts[i] = g < N ? __ldcs(t + g) : 0;
            S.as[i] = (adc != nullptr && g < N) ? __ldcs(adc + g) : 0u;
        }
    }
    if (threadIdx.x == 32) {
        S.t_prev = base > 0 ? __ldg(t + base - 1) : 0;
        S.t_next = base + kTileSpan < N ? __ldg(t + base + kTileSpan) : 0;
    }
    if (bulk && threadIdx.x == 0 && !mbar_wait(&S.bar, 0)) load_failed = 1;
    __syncthreads();
    if (load_failed) {              // a bounded wait gave up: report, publish, go on
        if (threadIdx.x == 0) atomicExch(status, (int)CC_ETIMEOUT);
        for (int i = threadIdx.x; i < kTileSpan; i += kCThreads) {
            S.ts[i] = 0;
            S.as[i] = 0u;
        }
        __syncthreads();
    }

    // ---- masks: bit r of m_after = "step from this detection to the next
    // is below dt_max", bit r of m_before = the same for the step before
    const int wl = w * kWarpSpan + lane;                // local index of row 0
    const long long seg = base + (long long)w * kWarpSpan;
    unsigned m_after = 0, m_before = 0;
#pragma unroll
    for (int r = 0; r < kRows; r++) {
        const int li = wl + 32 * r;
        const long long i = base + li;
        const long long ti = S.ts[li];
        const long long tn = li + 1 < kTileSpan ? S.ts[li + 1] : S.t_next;
        const long long tp = li > 0 ? S.ts[li - 1] : S.t_prev;
        const bool ma = (i + 1 < N) && step_of(ti, tn) < dt_max;
        const bool mb = (i > 0) && (i < N) && step_of(tp, ti) < dt_max;
        m_after |= (unsigned)ma << r;
        m_before |= (unsigned)mb << r;
    }
    // ---- pass 1: the warp's aggregate
    const unsigned starts_bits = m_after & ~m_before;
    long long cnt = 0, last = -1;
#pragma unroll
    for (int r = 0; r < kRows; r++) {
        const unsigned s = __ballot_sync(0xffffffffu, (starts_bits >> r) & 1u);
        cnt += __popc(s);
        if (s) last = seg + 32 * r + (31 - __clz((int)s));
    }
    unsigned long long own = 0, own_before = 0;
#pragma unroll
    for (int r = 0; r < kRows; r++) {
        const long long i = seg + 32 * r + lane;
        const unsigned a = S.as[wl + 32 * r];
        own += a;
        if (i < last) own_before += a;
    }
    Carry wa{cnt, last, warp_sum_u64(own), warp_sum_u64(own_before)};
    if (last < 0) wa.sum_before = 0;
    if (lane == 0) warp_agg[w] = wa;
    __syncthreads();

    // ---- tile aggregate, look-back, tile prefix.  Warp 0 looks back over
    // windows of 32 predecessors at once: it waits until each has published
    // at least its aggregate, combines (in order) back to the nearest one
    // that has published its inclusive prefix, and stops there.
    __shared__ Carry tile_agg;
    if (threadIdx.x == 0) {
        Carry acc = identity();
        for (int k = 0; k < kCWarps; k++) {
            warp_excl[k] = acc;
            acc = combine(acc, warp_agg[k]);
        }
        tile_agg = acc;
        volatile TileState *me = tiles + tile;
        if (tile == 0) {
            put(&me->incl, acc);
        } else {
            put(&me->agg, acc);
        }
        __threadfence();
        me->status = tile == 0 ? 2 : 1;
    }
    __syncthreads();
    if (w == 0) {
        Carry excl = identity();
        bool timed_out = false;
        unsigned long long t0 = 0;
        for (long long hi = tile - 1; hi >= 0;) {
            const long long p = hi - lane;              // lane 0: the nearest predecessor
            int st = p >= 0 ? ((volatile TileState *)tiles)[p].status : 2;
            for (unsigned it = 0; __any_sync(0xffffffffu, st == 0); ++it) {
                if (st == 0) st = ((volatile TileState *)tiles)[p].status;
                if ((it & 63) == 0) {   // lane 0's clock for all: the exit stays warp-uniform
                    const unsigned long long now = __shfl_sync(0xffffffffu, globaltimer_ns(), 0);
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > kWaitLimitNs) { timed_out = true; break; }
                }
            }
            if (timed_out) break;
            __threadfence();
            Carry v = identity();
            if (p >= 0) v = st == 2 ? get(&((volatile TileState *)tiles)[p].incl)
                                    : get(&((volatile TileState *)tiles)[p].agg);
            const unsigned incl_mask = __ballot_sync(0xffffffffu, st == 2);
            const int n = incl_mask ? __ffs(incl_mask) : 32;   // lanes [0, n) take part
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {                 // ordered tree reduction
                const Carry y = shfl_down_carry(v, o);
                if (lane + o < n) v = combine(y, v);
            }
            excl = combine(v, excl);                           // lane 0's value is the window's
            if (incl_mask) break;
            hi -= 32;
        }
        if (lane == 0) {
            if (timed_out) atomicExch(status, (int)CC_ETIMEOUT);
            if (tile > 0) {
                volatile TileState *me = tiles + tile;
                put(&me->incl, combine(excl, tile_agg));
                __threadfence();
                me->status = 2;
            }
            tile_excl = excl;
            if (tile == (N - 1) / kTileSpan && n_events != nullptr)
                *n_events = combine(excl, tile_agg).starts;
        }
    }
    __syncthreads();

    // ---- pass 2: outputs, row by row with the running prefix
    Carry c = combine(tile_excl, warp_excl[w]);
    const unsigned lane_le = 0xffffffffu >> (31 - lane);
#pragma unroll
    for (int r = 0; r < kRows; r++) {
        const long long i = seg + 32 * r + lane;
        const bool ma = (m_after >> r) & 1u, mb = (m_before >> r) & 1u;
        const bool st = ma && !mb, en = mb && !ma;
        const unsigned s = __ballot_sync(0xffffffffu, st);
        const unsigned a = S.as[wl + 32 * r];
        const unsigned long long incl = warp_incl_scan_u64(a, lane);
        const unsigned long long excl_here = incl - a;
        const unsigned s_le = s & lane_le;
        const int sl = s_le ? 31 - __clz((int)s_le) : 0;
        const unsigned long long before_sl = __shfl_sync(0xffffffffu, excl_here, sl);
        const long long id = c.starts + __popc(s_le) - 1;
        if (i < N) {
            if (edge) edge[i] = (unsigned char)(ma ^ mb);
            if (event_id) event_id[i] = (ma || mb) ? (int)id : -1;
            if (en) {
                const long long first = s_le ? seg + 32 * r + sl : c.last_start;
                const unsigned long long sum_before = s_le ? c.sum + before_sl : c.sum_before;
                if (ev_first) ev_first[id] = first;
                if (ev_count) ev_count[id] = (int)(i - first + 1);
                if (ev_adc) ev_adc[id] = c.sum + incl - sum_before;
            }
        }
        // advance the running prefix by this row
        const unsigned long long row_sum = __shfl_sync(0xffffffffu, incl, 31);
        const int ls = s ? 31 - __clz((int)s) : 0;
        const unsigned long long row_before = __shfl_sync(0xffffffffu, excl_here, ls);
        Carry row{__popc(s), s ? seg + 32 * r + ls : -1, row_sum, s ? row_before : 0ull};
        c = combine(c, row);
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
    // the staged tile needs more than 48 KB of shared memory (set per call:
    // the attribute belongs to the current device)
    e = cudaFuncSetAttribute((const void *)k_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(ClusterSmem));
    if (e != cudaSuccess) return e;
    TraceScope ts(CC_STAGE_CLUSTER, s);
    k_cluster<<<(unsigned)tiles, kCThreads, sizeof(ClusterSmem), s>>>(
        reinterpret_cast<const long long *>(t), adc, (long long)n, (long long)dt_max, edge,
        event_id, reinterpret_cast<long long *>(ev_first), ev_count,
        reinterpret_cast<unsigned long long *>(ev_adc), reinterpret_cast<long long *>(n_events),
        state, ticket, st);
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

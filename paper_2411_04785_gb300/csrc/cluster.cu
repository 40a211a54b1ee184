// cluster.cu - event clustering of time-sorted detections by a maximum step
// between consecutive detections (Sec. 2 of the paper).
//
// Sec. 2 defines, for detections sorted by time, the step to the next
// detection, a mask "step < dt_max" on it, and the edge of a detection as the
// XOR of the masks on its two sides (no step outside the stream: false).  A
// run of detections joined by masked steps is one event; its first and last
// detection carry the edges.  The paper computes the edges with two kernels;
// here the edges AND the events are built: every detection gets its event
// number (-1 when isolated) and every event its first detection, its size and
// its amplitude sum.
//
// Event numbers are a prefix count of event starts (a detection whose step
// before is not masked and whose step after is), so the work is a scan, done
// in three launches that never wait on one another's CTAs:
//   k_cluster_masks   per tile of 4096 detections: the step masks from t,
//                     the edges, the masks themselves (2 bits per detection,
//                     for the third launch) and the tile's aggregate, whose
//                     amplitude part needs only the detections from the
//                     tile's last event start on;
//   k_cluster_scan    the exclusive prefix of the tile aggregates within
//                     groups of 1024 tiles, and each group's total;
//   k_cluster_events  per tile: the masks and amplitudes again, the local scan
//                     from the tile's prefix, event ids and per-event outputs.
// The scan state of a range of detections is (starts in it, index of its last
// start, its tail: the amplitude sum from its last start to its end, or over
// all of it when it holds no start), which composes associatively (a
// segmented sum that restarts at every start), so an event's amplitude sum
// is the tail carried into its lane plus the lane's own prefix sum, with no
// per-event atomics.  All
// arithmetic is integer: results are exact.  A tile's time stamps and
// amplitudes arrive in shared memory by TMA tensor copies (128-byte rows in
// the 128B swizzle, so that a lane reading its own row never conflicts with
// its neighbours), and its event ids leave the same way; every lane owns 16
// consecutive detections and scans them serially, and the lanes of a warp
// combine their aggregates in one warp scan per 16 detections.
// Traffic per detection: t read, edges and masks written, then masks and adc
// read and event ids written: 8 + 1.25 + 4.25 + 4 bytes, plus the per-event
// outputs and each tile's tail amplitudes (a few dozen detections, all 4096
// for a tile inside one event), against 17 + 20 per event for the inputs and
// outputs alone.
#include <string.h>

#include "cc_internal.cuh"
#include "cc_pipe.cuh"

namespace cc {
namespace {

constexpr int kCWarps = 8;
constexpr int kCThreads = kCWarps * 32;
constexpr int kWarpSpan = 16 * 32;               // 512 detections per warp
constexpr int kTileSpan = kWarpSpan * kCWarps;   // 4096 per CTA

struct Carry {
    long long starts;              // event starts in the range
    long long last_start;          // index of the range's last start, -1 if none
    unsigned long long tail;       // amplitude sum from the last start on (all: no start)
};

__device__ __forceinline__ Carry identity() { return Carry{0, -1, 0ull}; }

// a covers the detections just before those of b
__device__ __forceinline__ Carry combine(const Carry &a, const Carry &b) {
    Carry c;
    c.starts = a.starts + b.starts;
    if (b.last_start >= 0) {
        c.last_start = b.last_start;
        c.tail = b.tail;
    } else {
        c.last_start = a.last_start;
        c.tail = a.tail + b.tail;
    }
    return c;
}

__device__ __forceinline__ Carry shfl_up_carry(const Carry &c, int o) {
    return Carry{__shfl_up_sync(0xffffffffu, c.starts, o),
                 __shfl_up_sync(0xffffffffu, c.last_start, o),
                 __shfl_up_sync(0xffffffffu, c.tail, o)};
}

// step from a to b in wrapping 64-bit arithmetic (meaningful for |step| < 2^63)
__device__ __forceinline__ long long step_of(long long a, long long b) {
    return (long long)((unsigned long long)b - (unsigned long long)a);
}

// A tile in shared memory: its time stamps (256 rows of 16 int64) and
// amplitudes (128 rows of 32 uint32) as 128-byte rows in the TMA 128B swizzle
// (16-byte chunk c of row r at chunk c ^ (r & 7)), so that a lane reading its
// own row's chunks never conflicts with the lanes beside it.
__device__ __forceinline__ int swz(int row, int chunk) { return row * 128 + ((chunk ^ (row & 7)) << 4); }
__device__ __forceinline__ int t_off(int e) { return swz(e >> 4, (e & 15) >> 1) + ((e & 1) << 3); }
__device__ __forceinline__ int a_off(int e) { return swz(e >> 5, (e & 31) >> 2) + ((e & 3) << 2); }

// Stage a tile of 4096 detections starting at `base`: by tensor copies when
// the tile is whole inside the maps (tma), else by plain loads (0 past the
// end).  `tsw` may be null (amplitudes only), `asw` null (time stamps only),
// and the amplitudes are 0 without adc.  Thread 0 waits (bounded); returns
// false on a timeout.
__device__ __forceinline__ bool stage_tile(unsigned char *tsw, unsigned char *asw,
                                           unsigned long long *bar, const CUtensorMap *tmap,
                                           const CUtensorMap *amap, bool tma,
                                           const long long *__restrict__ t,
                                           const unsigned *__restrict__ adc, long long N,
                                           long long base) {
    const bool amps = asw != nullptr, load_amps = amps && adc != nullptr;
    if (tma) {
        if (threadIdx.x == 0) {
            const unsigned bytes = (tsw ? kTileSpan * 8u : 0u) + (load_amps ? kTileSpan * 4u : 0u);
            if (bytes) {
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                 smem_u32(bar)), "r"(bytes)
                             : "memory");
                if (tsw) tma_load_2d(tsw, tmap, 0, (int)(base / 16), bar);
                if (load_amps) tma_load_2d(asw, amap, 0, (int)(base / 32), bar);
            } else {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
            }
        }
        if (amps && adc == nullptr)
            for (int e = threadIdx.x; e < kTileSpan; e += kCThreads)
                *reinterpret_cast<unsigned *>(asw + a_off(e)) = 0u;
    } else {
        for (int e = threadIdx.x; e < kTileSpan; e += kCThreads) {
            const long long g = base + e;
            if (tsw) *reinterpret_cast<long long *>(tsw + t_off(e)) = g < N ? __ldcs(t + g) : 0;
            if (amps)
                *reinterpret_cast<unsigned *>(asw + a_off(e)) =
                    (adc != nullptr && g < N) ? __ldcs(adc + g) : 0u;
        }
    }
    return !(tma && threadIdx.x == 0 && !mbar_wait(bar, 0));
}

// The 16 amplitudes of the lane's detections (tile elements e0 .. e0 + 15).
__device__ __forceinline__ void lane_adc(const unsigned char *asw, int e0, unsigned (&a)[16]) {
    const int arow = e0 >> 5, ach = ((e0 >> 4) & 1) * 4;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const uint4 v = *reinterpret_cast<const uint4 *>(asw + swz(arow, ach + c));
        a[4 * c] = v.x;
        a[4 * c + 1] = v.y;
        a[4 * c + 2] = v.z;
        a[4 * c + 3] = v.w;
    }
}

// Masks of the lane's detections (tile elements e0 .. e0 + 15, global i0 ..)
// from the staged time stamps: bit k of ma: the step after detection i0 + k
// is masked; of mb: the step before it.  t_prev / t_next: the detections just
// before and after the tile.  Every lane of the warp takes part (shuffles).
__device__ __forceinline__ void lane_masks(const unsigned char *tsw, long long t_prev,
                                           long long t_next, long long N, int e0, long long i0,
                                           long long dt_max, int lane, unsigned &ma,
                                           unsigned &mb) {
    long long tv[16];
    const int r = e0 >> 4;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const longlong2 v = *reinterpret_cast<const longlong2 *>(tsw + swz(r, c));
        tv[2 * c] = v.x;
        tv[2 * c + 1] = v.y;
    }
    long long tn = __shfl_down_sync(0xffffffffu, tv[0], 1);
    long long tp = __shfl_up_sync(0xffffffffu, tv[15], 1);
    if (lane == 31)
        tn = e0 + 16 < kTileSpan ? *reinterpret_cast<const long long *>(tsw + t_off(e0 + 16)) : t_next;
    if (lane == 0) tp = e0 > 0 ? *reinterpret_cast<const long long *>(tsw + t_off(e0 - 1)) : t_prev;
    ma = 0;
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

struct MasksSmem {
    unsigned char tsw[kTileSpan * 8];
    long long t_prev, t_next;
    unsigned long long bar;
    long long wstarts[kCWarps];
    long long wlast[kCWarps];
    unsigned long long wtail[kCWarps];
    int failed;
};

__global__ void __launch_bounds__(kCThreads, 4)
k_cluster_masks(const __grid_constant__ CUtensorMap tmap, int use_tma,
                const long long *__restrict__ t, const unsigned *__restrict__ adc, long long N,
                long long dt_max, int vec_out, unsigned char *__restrict__ edge,
                unsigned *__restrict__ masks, Carry *__restrict__ aggs, int *__restrict__ status) {
    extern __shared__ unsigned char smem_raw[];
    MasksSmem &S = *reinterpret_cast<MasksSmem *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kTileSpan;
    const bool tma = use_tma && base + kTileSpan <= (N / 32) * 32;
    if (threadIdx.x == 0) {
        S.failed = 0;
        mbar_init(&S.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 32) {
        S.t_prev = base > 0 ? __ldg(t + base - 1) : 0;
        S.t_next = base + kTileSpan < N ? __ldg(t + base + kTileSpan) : 0;
    }
    // the amplitudes of the tile's last 256 detections, loaded while the time
    // stamps arrive: the tile's tail (below) nearly always lies inside them
    const long long pref0 = base + kTileSpan - kCThreads, gp = pref0 + threadIdx.x;
    const unsigned a_pref = (adc != nullptr && gp < N) ? __ldg(adc + gp) : 0u;
    if (!stage_tile(S.tsw, nullptr, &S.bar, &tmap, nullptr, tma, t, nullptr, N, base)) S.failed = 1;
    __syncthreads();
    if (S.failed) {               // a bounded wait gave up: report, and go on with zeros
        if (threadIdx.x == 0) atomicExch(status, (int)CC_ETIMEOUT);
        for (int i = threadIdx.x; i < kTileSpan * 8 / 16; i += kCThreads)
            reinterpret_cast<int4 *>(S.tsw)[i] = make_int4(0, 0, 0, 0);
        __syncthreads();
    }
    const int e0 = w * kWarpSpan + lane * 16;
    const long long i0 = base + e0;
    unsigned ma, mb;
    lane_masks(S.tsw, S.t_prev, S.t_next, N, e0, i0, dt_max, lane, ma, mb);
    if (i0 < N && CC_IN_BOUNDS(CC_SITE_CLUSTER_OUT, i0 >> 4, (N + 15) >> 4))
        masks[i0 >> 4] = ma | (mb << 16);
    const unsigned eb = ma ^ mb;
    if (edge != nullptr) {
        if (vec_out && i0 + 16 <= N && CC_IN_BOUNDS(CC_SITE_CLUSTER_OUT, i0 + 15, N)) {
            unsigned q[4];
#pragma unroll
            for (int c = 0; c < 4; c++)
                q[c] = ((eb >> (4 * c)) & 1u) | (((eb >> (4 * c + 1)) & 1u) << 8) |
                       (((eb >> (4 * c + 2)) & 1u) << 16) | (((eb >> (4 * c + 3)) & 1u) << 24);
            *reinterpret_cast<uint4 *>(edge + i0) = make_uint4(q[0], q[1], q[2], q[3]);
        } else {
#pragma unroll
            for (int k = 0; k < 16; k++)
                if (i0 + k < N && CC_IN_BOUNDS(CC_SITE_CLUSTER_OUT, i0 + k, N))
                    edge[i0 + k] = (unsigned char)((eb >> k) & 1u);
        }
    }
    // the tile's starts and its last start
    const unsigned sbits = ma & ~mb;
    long long st = __popc(sbits);
    long long last = sbits ? i0 + (31 - __clz((int)sbits)) : -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        st += __shfl_xor_sync(0xffffffffu, st, o);
        last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
    }
    if (lane == 0) {
        S.wstarts[w] = st;
        S.wlast[w] = last;
    }
    __syncthreads();
    long long tile_starts = 0, tile_last = -1;
#pragma unroll
    for (int k = 0; k < kCWarps; k++) {
        tile_starts += S.wstarts[k];
        tile_last = max(tile_last, S.wlast[k]);
    }
    // its tail: the amplitudes from the last start to the tile's end (the
    // whole tile when it holds no start)
    unsigned long long tail = 0;
    if (adc != nullptr) {
        const long long end = base + kTileSpan < N ? base + kTileSpan : N;
        const long long from = tile_last >= 0 ? tile_last : base;
        if (gp >= from && gp < end) tail = a_pref;
        const long long stop = end < pref0 ? end : pref0;   // the rest: a long last event
        for (long long g = from + threadIdx.x; g < stop; g += kCThreads) tail += __ldg(adc + g);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tail += __shfl_xor_sync(0xffffffffu, tail, o);
        if (lane == 0) S.wtail[w] = tail;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int k = 1; k < kCWarps; k++) tail += S.wtail[k];
    }
    if (threadIdx.x == 0) aggs[blockIdx.x] = Carry{tile_starts, tile_last, tail};
}
constexpr size_t kMasksSmemBytes = sizeof(MasksSmem) + 1024;

// Exclusive prefix of the tile aggregates within groups of 1024 tiles: one
// CTA per group, one tile per thread, an ordered warp scan and a scan of the
// warps' totals; the group's total goes to gtot[group].
constexpr int kScanThreads = 1024;
__device__ __forceinline__ Carry warp_incl_scan(Carry v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Carry y = shfl_up_carry(v, o);
        if (lane >= o) v = combine(y, v);
    }
    return v;
}

__global__ void __launch_bounds__(kScanThreads)
k_cluster_scan(const Carry *__restrict__ aggs, long long ntiles, Carry *__restrict__ excl,
               Carry *__restrict__ gtot) {
    __shared__ Carry wtot[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const long long tile = (long long)blockIdx.x * kScanThreads + tid;
    const Carry v = tile < ntiles ? aggs[tile] : identity();
    const Carry incl = warp_incl_scan(v, lane);
    if (lane == 31) wtot[w] = incl;
    __syncthreads();
    if (w == 0) {
        const Carry s = warp_incl_scan(wtot[lane], lane);
        Carry before = shfl_up_carry(s, 1);
        if (lane == 0) before = identity();
        wtot[lane] = before;
        if (lane == 31) gtot[blockIdx.x] = s;
    }
    __syncthreads();
    Carry ex = shfl_up_carry(incl, 1);
    if (lane == 0) ex = identity();
    if (tile < ntiles) excl[tile] = combine(wtot[w], ex);
}

// The prefix of groups [0, g) by one warp (every lane returns it).
__device__ __forceinline__ Carry groups_before(const Carry *__restrict__ gtot, long long g,
                                               int lane) {
    Carry run = identity();
    for (long long b = 0; b < g; b += 32) {
        const Carry v = b + lane < g ? gtot[b + lane] : identity();
        const Carry s = warp_incl_scan(v, lane);
        const Carry chunk = Carry{__shfl_sync(0xffffffffu, s.starts, 31),
                                  __shfl_sync(0xffffffffu, s.last_start, 31),
                                  __shfl_sync(0xffffffffu, s.tail, 31)};
        run = combine(run, chunk);
    }
    return run;
}

// n_events alone (when no per-detection or per-event output is asked for)
__global__ void k_cluster_total(const Carry *__restrict__ gtot, long long ngroups,
                                long long *__restrict__ n_events) {
    const Carry all = groups_before(gtot, ngroups, threadIdx.x & 31);
    if (threadIdx.x == 0 && n_events != nullptr) *n_events = all.starts;
}

struct EventsSmem {
    unsigned char asw[kTileSpan * 4];     // amplitudes, swizzled; then the event ids (tensor store)
    unsigned long long psum[16][kCThreads];   // per lane: its amplitudes' prefix sums
    unsigned long long bar;
    Carry wagg[kCWarps];
    Carry tile_pre;
    int failed;
};
constexpr size_t kEventsSmemBytes = sizeof(EventsSmem) + 1024;

__global__ void __launch_bounds__(kCThreads, 4)
k_cluster_events(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap imap,
                 int use_tma, int id_tma, const unsigned *__restrict__ masks,
                 const unsigned *__restrict__ adc, long long N, int vec_out,
                 const Carry *__restrict__ excl, const Carry *__restrict__ gtot, long long ngroups,
                 long long *__restrict__ n_events, int *__restrict__ event_id,
                 long long *__restrict__ ev_first, int *__restrict__ ev_count,
                 unsigned long long *__restrict__ ev_adc, long long ev_cap,
                 int *__restrict__ status) {
    extern __shared__ unsigned char smem_raw[];
    EventsSmem &S = *reinterpret_cast<EventsSmem *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kTileSpan;
    const bool whole = base + kTileSpan <= (N / 32) * 32;
    if (threadIdx.x == 0) {
        S.failed = 0;
        mbar_init(&S.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int e0 = w * kWarpSpan + lane * 16;
    const long long i0 = base + e0;
    const unsigned m = i0 < N ? __ldcs(masks + (i0 >> 4)) : 0u;
    // the amplitudes' tensor copy first, then (warp 0, while it is in flight)
    // the tile's prefix: its group's, then its own in the group
    const bool tma = use_tma && whole;
    if (tma && threadIdx.x == 0 && adc != nullptr) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         smem_u32(&S.bar)), "r"(kTileSpan * 4u)
                     : "memory");
        tma_load_2d(S.asw, &amap, 0, (int)(base / 32), &S.bar);
    }
    if (w == 0) {
        const Carry own = excl[blockIdx.x];           // issued before the group walk
        const long long g = blockIdx.x / kScanThreads;
        const Carry pre = combine(groups_before(gtot, g, lane), own);
        if (lane == 0) S.tile_pre = pre;
        if (blockIdx.x == gridDim.x - 1 && n_events != nullptr) {
            const Carry all = groups_before(gtot, ngroups, lane);
            if (lane == 0) *n_events = all.starts;
        }
    }
    if (tma) {
        if (adc == nullptr)
            for (int e = threadIdx.x; e < kTileSpan; e += kCThreads)
                *reinterpret_cast<unsigned *>(S.asw + a_off(e)) = 0u;
        else if (threadIdx.x == 0 && !mbar_wait(&S.bar, 0))
            S.failed = 1;
    } else if (!stage_tile(nullptr, S.asw, &S.bar, nullptr, &amap, false, nullptr, adc, N, base)) {
        S.failed = 1;
    }
    const unsigned ma = m & 0xFFFFu, mb = m >> 16;
    const unsigned sbits = ma & ~mb, ebits = mb & ~ma, inb = ma | mb;
    __syncthreads();
    if (S.failed) {
        if (threadIdx.x == 0) atomicExch(status, (int)CC_ETIMEOUT);
        for (int i = threadIdx.x; i < kTileSpan / 4; i += kCThreads)
            reinterpret_cast<int4 *>(S.asw)[i] = make_int4(0, 0, 0, 0);
        __syncthreads();
    }
    Carry mine{__popc(sbits), -1, 0ull};
    {
        unsigned a[16];
        lane_adc(S.asw, e0, a);
        unsigned long long run = 0;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            run += a[k];
            S.psum[k][threadIdx.x] = run;
        }
        const int lastk = sbits ? 31 - __clz((int)sbits) : -1;
        mine.tail = run;
        if (lastk >= 0) {
            mine.last_start = i0 + lastk;
            mine.tail = run - (lastk > 0 ? S.psum[lastk - 1][threadIdx.x] : 0ull);
        }
    }
    const Carry incl = warp_incl_scan(mine, lane);
    Carry lane_ex = shfl_up_carry(incl, 1);
    if (lane == 0) lane_ex = identity();
    if (lane == 31) S.wagg[w] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {       // the warps' exclusive prefixes, from the tile's
        Carry acc = S.tile_pre;
        for (int k = 0; k < kCWarps; k++) {
            const Carry next = combine(acc, S.wagg[k]);
            S.wagg[k] = acc;
            acc = next;
        }
    }
    __syncthreads();
    const Carry c0 = combine(S.wagg[w], lane_ex);

    // per-event outputs at the lane's ends: the event's id is the count of
    // starts up to it, its first detection the last start before it (in the
    // lane, or carried in), its sum a difference of the lane's prefix sums
    // (start in the lane) or the carried tail plus the lane's prefix sum
    const unsigned valid = i0 + 16 <= N ? 0xFFFFu : (i0 >= N ? 0u : (1u << (unsigned)(N - i0)) - 1u);
    for (unsigned e = ebits & valid; e; e &= e - 1) {
        const int k = __ffs(e) - 1;
        const unsigned upto = sbits & ((2u << k) - 1u);
        const long long id = c0.starts + __popc(upto) - 1;
        const int lk = upto ? 31 - __clz((int)upto) : -1;
        const long long first = lk >= 0 ? i0 + lk : c0.last_start;
        const unsigned long long upto_k = S.psum[k][threadIdx.x];
        const unsigned long long sum =
            lk >= 0 ? upto_k - (lk > 0 ? S.psum[lk - 1][threadIdx.x] : 0ull) : c0.tail + upto_k;
        if (CC_IN_BOUNDS(CC_SITE_CLUSTER_EVENT, id, ev_cap)) {
            if (ev_first) ev_first[id] = first;
            if (ev_count) ev_count[id] = (int)(i0 + k - first + 1);
            if (ev_adc) ev_adc[id] = sum;
        }
    }
    // event ids (fewer than 2^31 detections: they fit in 32 bits)
    int ids[16];
    {
        int rank = (int)c0.starts;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            rank += (sbits >> k) & 1u;
            ids[k] = ((inb >> k) & 1u) ? rank - 1 : -1;
        }
    }
    if (event_id == nullptr) return;
    if (id_tma && whole) {        // through shared memory, one tensor store per tile
        const int arow = e0 >> 5, ach = ((e0 >> 4) & 1) * 4;   // the amplitudes are all read
#pragma unroll
        for (int c = 0; c < 4; c++)
            *reinterpret_cast<int4 *>(S.asw + swz(arow, ach + c)) =
                make_int4(ids[4 * c], ids[4 * c + 1], ids[4 * c + 2], ids[4 * c + 3]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0 && CC_IN_BOUNDS(CC_SITE_CLUSTER_OUT, base + kTileSpan - 1, N)) {
            tma_store_2d(&imap, 0, (int)(base / 32), S.asw);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // the tile is read
        }
        return;
    }
    if (vec_out && i0 + 16 <= N && CC_IN_BOUNDS(CC_SITE_CLUSTER_OUT, i0 + 15, N)) {
#pragma unroll
        for (int q = 0; q < 4; q++)
            reinterpret_cast<int4 *>(event_id + i0)[q] =
                make_int4(ids[4 * q], ids[4 * q + 1], ids[4 * q + 2], ids[4 * q + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < 16; k++)
            if (i0 + k < N && CC_IN_BOUNDS(CC_SITE_CLUSTER_OUT, i0 + k, N)) event_id[i0 + k] = ids[k];
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
    const int64_t rows = n > 0 ? (n + 15) / 16 : 1;
    const int64_t groups = (tiles + kScanThreads - 1) / kScanThreads;
    return 2 * align256((size_t)tiles * sizeof(Carry)) + align256((size_t)rows * sizeof(unsigned)) +
           align256((size_t)groups * sizeof(Carry)) + align256(sizeof(int));
}

// [rows][cols] elements of `bytes` each as a TMA map, 128B swizzle, boxes of
// `box_rows` rows
static bool row_map(CUtensorMap *m, CUtensorMapDataType type, const void *p, int cols,
                    int64_t rows, int box_rows) {
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {128};
    const cuuint32_t box[2] = {(cuuint32_t)cols, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return encode_fn()(m, type, 2, const_cast<void *>(p), dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_cluster(const int64_t *t, const uint32_t *adc, int64_t n, int64_t dt_max,
                           uint8_t *edge, int32_t *event_id, int64_t *ev_first, int32_t *ev_count,
                           uint64_t *ev_adc, int64_t *n_events, int32_t *status, char *ws,
                           cudaStream_t s) {
    const int64_t tiles = n > 0 ? (n + kTileSpan - 1) / kTileSpan : 1;
    const int64_t rows = n > 0 ? (n + 15) / 16 : 1;
    const int64_t groups = (tiles + kScanThreads - 1) / kScanThreads;
    Carry *aggs = reinterpret_cast<Carry *>(ws);
    Carry *excl = reinterpret_cast<Carry *>(ws + align256((size_t)tiles * sizeof(Carry)));
    unsigned *masks = reinterpret_cast<unsigned *>(ws + 2 * align256((size_t)tiles * sizeof(Carry)));
    Carry *gtot = reinterpret_cast<Carry *>(ws + 2 * align256((size_t)tiles * sizeof(Carry)) +
                                            align256((size_t)rows * sizeof(unsigned)));
    int32_t *st = status ? status
                         : reinterpret_cast<int32_t *>(reinterpret_cast<char *>(gtot) +
                                                       align256((size_t)groups * sizeof(Carry)));
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    if (n == 0) {
        if (n_events) return cudaMemsetAsync(n_events, 0, sizeof(int64_t), s);
        return cudaSuccess;
    }
    // tensor maps of t as [N/16][16] int64, adc and event_id as [N/32][32]
    // 32-bit rows, 128B swizzle, boxes of one tile (256 x 16, 128 x 32)
    auto al16 = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    CUtensorMap tmap, amap, imap;
    memset(&tmap, 0, sizeof(tmap));
    memset(&amap, 0, sizeof(amap));
    memset(&imap, 0, sizeof(imap));
    int use_tma = n >= kTileSpan && al16(t) && (adc == nullptr || al16(adc)) && encode_fn() != nullptr;
    if (use_tma)
        use_tma = row_map(&tmap, CU_TENSOR_MAP_DATA_TYPE_INT64, t, 16, n / 16, kTileSpan / 16) &&
                  (adc == nullptr ||
                   row_map(&amap, CU_TENSOR_MAP_DATA_TYPE_UINT32, adc, 32, n / 32, kTileSpan / 32));
    int id_tma = use_tma && event_id != nullptr && al16(event_id) &&
                 row_map(&imap, CU_TENSOR_MAP_DATA_TYPE_INT32, event_id, 32, n / 32, kTileSpan / 32);
    const int vec_out = (edge == nullptr || al16(edge)) && (event_id == nullptr || al16(event_id));
    const auto *tl = reinterpret_cast<const long long *>(t);
    if ((e = cudaFuncSetAttribute((const void *)k_cluster_masks,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kMasksSmemBytes)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute((const void *)k_cluster_events,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kEventsSmemBytes)) != cudaSuccess)
        return e;
    TraceScope ts(CC_STAGE_CLUSTER, s, 3);   // masks, scan, events (or the total alone)
    k_cluster_masks<<<(unsigned)tiles, kCThreads, kMasksSmemBytes, s>>>(
        tmap, use_tma, tl, adc, (long long)n, (long long)dt_max, vec_out, edge, masks, aggs, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_cluster_scan<<<(unsigned)groups, kScanThreads, 0, s>>>(aggs, (long long)tiles, excl, gtot);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    auto *ne = reinterpret_cast<long long *>(n_events);
    if (event_id == nullptr && ev_first == nullptr && ev_count == nullptr && ev_adc == nullptr) {
        k_cluster_total<<<1, 32, 0, s>>>(gtot, (long long)groups, ne);
        return cudaGetLastError();
    }
    k_cluster_events<<<(unsigned)tiles, kCThreads, kEventsSmemBytes, s>>>(
        amap, imap, use_tma, id_tma, masks, adc, (long long)n, vec_out, excl, gtot,
        (long long)groups, ne, event_id, reinterpret_cast<long long *>(ev_first), ev_count,
        reinterpret_cast<unsigned long long *>(ev_adc), (long long)n / 2, st);
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

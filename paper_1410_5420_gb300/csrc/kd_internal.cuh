// kd_internal.cuh -- device helpers and launch declarations shared by the
// kernel files and the host orchestration of the GB300 k-d tree builder.
#pragma once

#include <cstdint>
#include <utility>

#include <cuda_runtime.h>

namespace kd {

// ------------------------------------------------------------------ limits
constexpr int MAXK = 8;
constexpr int RADIX = 256;
constexpr int MAXPAY = 10;          // payload planes carried by one sort pass
constexpr int LEVEL_THREADS = 256;
constexpr int LEVEL_WARPS = LEVEL_THREADS / 32;
constexpr int LEVEL_NSMAX = 4;      // level-L segments one level-pass tile may touch
constexpr int FIN_THREADS = 256;

// device error word bits
constexpr int ERR_NAN = 1;
constexpr int ERR_TIMEOUT = 2;
constexpr int ERR_INTERNAL = 4;

// Poll limit of every wait (look-back flags, mbarriers).  The awaited block
// or copy was already running when the wait began, so a wait normally ends
// within microseconds; the bound only keeps a fault from hanging the GPU.
constexpr uint32_t SPIN_LIMIT = 1u << 24;

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}
__device__ __forceinline__ void st_volatile(uint32_t* p, uint32_t v) {
    *reinterpret_cast<volatile uint32_t*>(p) = v;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ----------------------------------------- bulk async copies (TMA engine)
// cp.async.bulk moves a contiguous global range into shared memory and
// signals an mbarrier with the bytes it wrote.  Both addresses must be
// 16-byte aligned and the size a multiple of 16 bytes.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t arrivals) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(arrivals) : "memory");
}
// Make barrier initialisation visible to the async proxy (before first use).
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes to the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    // suspend for up to 1 us per poll while the phase is incomplete
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Programmatic dependent launch.  A kernel launched by launch_dependent()
// may start while the previous kernel on its stream is still running; it
// calls pdl_wait() before its first global-memory access, which returns once
// that kernel has completed and its writes are visible (at once when the
// kernel was launched without the attribute).  pdl_trigger() lets the
// dependent grid launch as soon as every block of this grid has issued it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... P, typename... A>
inline cudaError_t launch_dependent(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                    A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// Named barrier 1 over the first NT threads of the block (the consumer
// warps of a kernel whose last warp is a producer that never joins it).
template <int NT>
__device__ __forceinline__ void consumer_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}
template <int NT>
__device__ __forceinline__ bool consumer_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.cta.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(NT)
        : "memory");
    return r != 0;
}
// Wait for phase `parity` of an mbarrier to complete; false after
// SPIN_LIMIT polls (each poll suspends for at most 1 us: about 17 s in all).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t spins = 0; spins < SPIN_LIMIT; ++spins)
        if (mbar_test(bar, parity)) return true;
    return false;
}

// Exclusive scan of one value per thread over a 256-thread block; *total
// (if not null) receives the block sum.  s_warp holds 8 words.
__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t v, uint32_t* s_warp, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < 8 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < 8) s_warp[lane] = w;
    }
    __syncthreads();
    uint32_t excl = x - v + (warp > 0 ? s_warp[warp - 1] : 0u);
    if (total) *total = s_warp[7];
    __syncthreads();
    return excl;
}

// Exclusive scan of one value per thread over an NT-thread block.
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) s_warp[lane] = w;
    }
    __syncthreads();
    uint32_t excl = x - v + (warp > 0 ? s_warp[warp - 1] : 0u);
    if (total) *total = s_warp[NW - 1];
    __syncthreads();
    return excl;
}

__host__ __device__ __forceinline__ int64_t pad4(int64_t x) { return (x + 3) & ~(int64_t)3; }

// ---------------------------------------------- tile-major look-back
// Each tile publishes a flag word (0 nothing, 1 aggregate, 2 inclusive) and
// two count records: its own counts (aggregate) and, once known, the counts
// of every tile up to and including itself (inclusive).  A record is written
// before its flag (fence in between); a reader loads the flag, fences, then
// the record.  Walking back, warp 0 reads 32 predecessor flags per round
// trip; the nearest inclusive record plus the aggregates above it give the
// exclusive prefix.  Records are rows of `nslot` words, so every slot's
// read is coalesced across the block.
constexpr uint32_t FLAG_AGG = 1u;
constexpr uint32_t FLAG_INC = 2u;

__device__ __forceinline__ void publish_flag(uint32_t* flags, int64_t tile, uint32_t f) {
    __threadfence();
    st_volatile(flags + tile, f);
}

// Called by the whole block (uniform control flow).  Thread `tid < nslot`
// receives the exclusive prefix of slot tid in *excl.  AggT is the word type
// of aggregate records.  s_ctl: one shared word.  Bounded wait: after
// `spin_limit` polls that find a predecessor without a record, the block
// sets ERR_TIMEOUT, *timed_out (if given) becomes true for every thread and
// the returned prefix is meaningless.
template <typename AggT>
__device__ __forceinline__ uint32_t block_lookback(const uint32_t* flags, const AggT* aggrec, const uint32_t* increc,
                                                   int nslot, int64_t tile, uint32_t* s_ctl, int* err,
                                                   int stride = 0, uint32_t spin_limit = SPIN_LIMIT,
                                                   bool* timed_out = nullptr) {
    if (stride == 0) stride = nslot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t excl = 0;
    int64_t hi = tile - 1;
    uint32_t spins = 0;
    while (hi >= 0) {
        if (warp == 0) {
            const int64_t u = hi - lane;
            const uint32_t f = u >= 0 ? ld_volatile(flags + u) : FLAG_INC;
            const uint32_t binc = __ballot_sync(0xffffffffu, f == FLAG_INC && u >= 0);
            const uint32_t bnr = __ballot_sync(0xffffffffu, f == 0u);
            const int L = binc ? __ffs(binc) - 1 : 32;
            const uint32_t upto = L >= 31 ? 0xffffffffu : ((2u << L) - 1u);
            if (lane == 0) *s_ctl = (bnr & upto) ? 0xffffffffu : (uint32_t)L;
        }
        __syncthreads();
        const uint32_t L = *s_ctl;
        __syncthreads();
        if (L == 0xffffffffu) {
            if (++spins > spin_limit) {
                if (tid == 0) atomicOr(err, ERR_TIMEOUT);
                if (timed_out) *timed_out = true;
                break;
            }
            __nanosleep(32);
            continue;
        }
        __threadfence();
        if (tid < nslot) {
            const int nagg = (int)(L < 32 ? L : 32);
            for (int i = 0; i < nagg; ++i) {
                const int64_t u = hi - i;
                if (u >= 0) excl += (uint32_t)(*reinterpret_cast<const volatile AggT*>(aggrec + u * stride + tid));
            }
            if (L < 32) excl += *reinterpret_cast<const volatile uint32_t*>(increc + (hi - (int64_t)L) * stride + tid);
        }
        if (L < 32) break;
        hi -= 32;
    }
    return excl;
}

// ------------------------------------------------- order-preserving keys
// Unsigned words whose unsigned order equals the numeric order of the
// coordinates (the super key parts of Section 2.1 compare numerically).
__device__ __forceinline__ uint32_t key_of(float f, int* nan_flag) {
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7fffffffu) > 0x7f800000u) *nan_flag = 1;
    if (u == 0x80000000u) u = 0;  // -0.0 compares equal to +0.0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ uint32_t key_of(int32_t v, int*) { return (uint32_t)v ^ 0x80000000u; }
__device__ __forceinline__ uint64_t key_of(int64_t v, int*) {
    return (uint64_t)v ^ 0x8000000000000000ull;
}

// ------------------------------------------------------------ tree shape
// The segments of level L of a tree over m addresses: level 0 is [0, m-1];
// a segment [lo, hi] has median mid = lo + (hi - lo) / 2 and children
// [lo, mid-1] and [mid+1, hi].  Segment index s at level L counts segments
// left to right (children of s are 2s and 2s+1).
struct Seg {
    int32_t lo, hi, idx;  // idx < 0: the address is a node of a shallower level
};

__device__ __forceinline__ Seg segment_of(int32_t i, int32_t m, int L) {
    int32_t lo = 0, hi = m - 1, s = 0;
    for (int l = 0; l < L; ++l) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if (i < mid) {
            hi = mid - 1;
            s = 2 * s;
        } else if (i > mid) {
            lo = mid + 1;
            s = 2 * s + 1;
        } else {
            return Seg{lo, hi, -1};
        }
    }
    return Seg{lo, hi, s};
}

// Bounds of segment index s at level L (may be empty: hi < lo).
__device__ __forceinline__ void segment_bounds(int32_t m, int L, int32_t s, int32_t& lo, int32_t& hi) {
    lo = 0;
    hi = m - 1;
    for (int l = L - 1; l >= 0; --l) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if ((s >> l) & 1)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
}

__host__ __device__ __forceinline__ int32_t child_mid(int32_t lo, int32_t hi) {
    return hi < lo ? -1 : lo + ((hi - lo) >> 1);
}

// Level-L segments touching the tile [pos0, pos0 + npos): at most
// LEVEL_NSMAX (the host sizes tiles so that this holds).  Thread 0 only.
__device__ __forceinline__ int tile_segments(int32_t pos0, int32_t npos, int32_t m, int L, int32_t* lo, int32_t* hi,
                                             int32_t* idx, int* err) {
    int ns = 0;
    int32_t i = pos0;
    const int32_t pend = pos0 + npos - 1;
    while (i <= pend) {
        const Seg sg = segment_of(i, m, L);
        if (sg.idx < 0) {
            ++i;
            continue;
        }
        if (ns == LEVEL_NSMAX) {
            atomicOr(err, ERR_INTERNAL);
            break;
        }
        lo[ns] = sg.lo;
        hi[ns] = sg.hi;
        idx[ns] = sg.idx;
        ++ns;
        i = sg.hi + 1;
    }
    return ns;
}

// Segment slot of cloud-local position pos among the tile's ns segments
// [lo[x], hi[x]]; -1 for an address that is a node of a shallower level
// (no element there).
__device__ __forceinline__ int tile_slot(const int32_t (&lo)[LEVEL_NSMAX], const int32_t (&hi)[LEVEL_NSMAX], int ns,
                                         int32_t pos) {
    int sj = 0;
    int32_t a = lo[0], z = hi[0];
#pragma unroll
    for (int x = 1; x < LEVEL_NSMAX; ++x)
        if (x < ns && pos >= lo[x]) {
            sj = x;
            a = lo[x];
            z = hi[x];
        }
    return (ns > 0 && pos >= a && pos <= z) ? sj : -1;
}

// ------------------------------------------------------ launch plumbing
struct PayloadArgs {
    const uint32_t* src[MAXPAY];  // nullptr: the source position (iota)
    uint32_t* dst[MAXPAY];
    int n;
};

enum KeyMode { KEY_DIRECT = 0, KEY_GATHER = 1, KEY_BUF = 2 };

// One device cloud's coordinates to be packed into a batch's buffer.
struct PackDesc {
    const void* src;
    int64_t words;     // 32-bit words
    int64_t dst_word;  // first destination word
};

// Per-cloud facts the build kernels need (one entry per cloud of a batch).
struct CloudDev {
    int64_t off;        // first position of the cloud in the batched arrays
    int64_t in_off;     // first input tuple of the cloud (tuple ids are global)
    int32_t m;          // tuples after dedup
    int32_t lam;        // level at which the on-chip finisher takes over
    int64_t medr_off;   // medr table base: level L starts at medr_off + 2^L - 1
    int32_t* node;      // outputs (cloud-local addresses and tuple indices)
    int32_t* left;
    int32_t* right;
    uint8_t* dim;
    uint8_t buf[MAXK];  // finisher: buffer set holding array q (0 initial, 1, 2)
};

// One tile of a level pass.
struct LevelTile {
    int32_t cloud;
    int32_t lev_in;   // level of the input view (after the free split)
    int32_t lev_out;  // level after the pass
    int32_t src_buf, dst_buf;
    int32_t write_med;  // LEVEL_MED: lev_out is this array's primary level and < lam; | LEVEL_FINAL
    int64_t pos0;       // first cloud-local position of the tile
    int32_t npos;       // positions in the tile
    int32_t first;      // 1: first tile of this cloud in this launch (no look-back past it)
};

struct FinUnit {
    int32_t cloud;
    int32_t seg;  // segment index at level lam of the cloud
};

// Flags of a level job: the pass writes the medians of lev_out
// (LEVEL_MED); it is the array's last move before the finisher, which reads
// rank 0 alone, so the other planes are not written (LEVEL_FINAL).
constexpr int32_t LEVEL_MED = 1;
constexpr int32_t LEVEL_FINAL = 2;

// One cloud's share of a level step: its tiles are tile_begin ..
// tile_begin + ceil(m / tile) - 1 of the launch.
struct LevelJob {
    int32_t cloud;
    int32_t lev_in, lev_out;
    int32_t src_buf, dst_buf;
    int32_t write_med;
    int64_t tile_begin;
};

// Index of the last entry of a non-decreasing prefix array <= x.
__device__ __forceinline__ int last_le(const int64_t* __restrict__ a, int n, int64_t x) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// Tile t of a level step, from the step's jobs (tile_begin ascending).
__device__ __forceinline__ LevelTile job_tile(const LevelJob* __restrict__ jobs, int njobs, int t, int tile,
                                              const CloudDev* __restrict__ clouds) {
    int lo = 0, hi = njobs;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (jobs[mid].tile_begin <= t) lo = mid; else hi = mid;
    }
    const LevelJob J = jobs[lo];
    LevelTile T;
    T.cloud = J.cloud;
    T.lev_in = J.lev_in;
    T.lev_out = J.lev_out;
    T.src_buf = J.src_buf;
    T.dst_buf = J.dst_buf;
    T.write_med = J.write_med;
    T.pos0 = (int64_t)(t - J.tile_begin) * tile;
    const int64_t rem = clouds[J.cloud].m - T.pos0;
    T.npos = (int32_t)(rem < tile ? rem : tile);
    T.first = T.pos0 == 0;
    return T;
}

// Stable warp ranking of digits below `marker` (the marker: no element):
// the lanes holding an equal digit come from one match instruction; the
// lowest of them advances the warp's counter of the digit.
template <int IPT>
__device__ __forceinline__ void warp_rank(const uint32_t (&dig)[IPT], uint32_t marker, uint32_t* __restrict__ wc,
                                          uint32_t (&rank)[IPT]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const uint32_t d = dig[j];
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader && d < marker) old = atomicAdd(&wc[d], (uint32_t)__popc(peers));
        old = __shfl_sync(0xffffffffu, old, leader);
        rank[j] = old + __popc(peers & lanemask_lt());
    }
}

// Stable warp ranking that picks its method per call: the first key is
// ranked with a match instruction, and the number of distinct digits among
// the warp's 32 first keys decides the rest.  Few distinct digits (long
// runs, as in the top bytes of clustered coordinates) stay with the match
// instruction; many go through shared-memory match words: each lane ORs its
// bit into its digit's word, reads back the lanes sharing its digit, and
// the highest of them advances the warp's counter of the digit and clears
// the word, so `match` is all zero between calls.  Both leave the same
// per-warp counts in wc.  Digits below `marker` (the marker: no element).
constexpr int RANK_DISTINCT_MAX = 16;  // at most this many distinct first digits: match instruction
template <int IPT>
__device__ __forceinline__ void warp_rank_adaptive(const uint32_t (&dig)[IPT], uint32_t marker,
                                                   uint32_t* __restrict__ wc, uint32_t* __restrict__ match,
                                                   uint32_t (&rank)[IPT]) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    uint32_t peers = __match_any_sync(0xffffffffu, dig[0]);
    int leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if (lane == leader && dig[0] < marker) old = atomicAdd(&wc[dig[0]], (uint32_t)__popc(peers));
    rank[0] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
    const int distinct = __popc(__ballot_sync(0xffffffffu, lane == leader));
    if (distinct <= RANK_DISTINCT_MAX) {
#pragma unroll
        for (int j = 1; j < IPT; ++j) {
            const uint32_t d = dig[j];
            peers = __match_any_sync(0xffffffffu, d);
            leader = __ffs(peers) - 1;
            old = 0;
            if (lane == leader && d < marker) old = atomicAdd(&wc[d], (uint32_t)__popc(peers));
            rank[j] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
        }
    } else {
        __syncwarp();
#pragma unroll
        for (int j = 1; j < IPT; ++j) {
            const uint32_t d = dig[j];
            if (d < marker) atomicOr(&match[d], 1u << lane);
            __syncwarp();
            const uint32_t pw = d < marker ? match[d] : (1u << lane);
            __syncwarp();
            const int ld = 31 - __clz(pw);
            uint32_t o = 0;
            if (lane == ld && d < marker) {
                o = wc[d];
                wc[d] = o + (uint32_t)__popc(pw);
                match[d] = 0;
            }
            __syncwarp();
            o = __shfl_sync(0xffffffffu, o, ld);
            rank[j] = o + __popc(pw & lt);
        }
    }
}

// rec[d][p]: plane p (ranks in super-key-p order) of index array d.
struct AllPlanes {
    uint32_t* p[MAXK][MAXK];
};

// Build buffers: [array d][buffer set: 0 initial records, 1, 2][plane p].
struct AllBufs {
    uint32_t* p[MAXK][3][MAXK];
};

// Buffer set holding an array after `moves` level passes.
__host__ __device__ __forceinline__ int buf_after(int moves) { return moves == 0 ? 0 : ((moves & 1) ? 1 : 2); }

}  // namespace kd

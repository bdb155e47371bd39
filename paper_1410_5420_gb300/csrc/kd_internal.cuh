// kd_internal.cuh -- device helpers and launch declarations shared by the
// kernel files and the host orchestration of the GB300 k-d tree builder.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace kd {

// ------------------------------------------------------------------ limits
constexpr int MAXK = 8;
constexpr int RADIX = 256;
constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int MAXPAY = 10;          // payload planes carried by one sort pass
constexpr int LEVEL_THREADS = 256;
constexpr int LEVEL_WARPS = LEVEL_THREADS / 32;
constexpr int LEVEL_NSMAX = 4;      // level-L segments one level-pass tile may touch
constexpr int FIN_THREADS = 256;

// device error word bits
constexpr int ERR_NAN = 1;
constexpr int ERR_TIMEOUT = 2;
constexpr int ERR_INTERNAL = 4;

// Decoupled look-back status word: 2 flag bits above a 30-bit count.
constexpr uint32_t ST_AGG = 1u << 30;
constexpr uint32_t ST_INC = 2u << 30;
constexpr uint32_t ST_FLAGS = 3u << 30;
constexpr uint32_t ST_COUNT = (1u << 30) - 1;

// Spin limit of a look-back wait.  A predecessor tile took its tile id (and
// so was already running) before the waiter did, so the wait normally ends
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

// Walk back from tile `tile - 1` over the status words (stride `stride`
// words per tile, word `slot` of each) until an inclusive prefix is found;
// returns the sum of everything before `tile`.  Sets ERR_TIMEOUT and
// returns what it has if a wait exceeds SPIN_LIMIT.
__device__ __forceinline__ uint32_t lookback(const uint32_t* status, int64_t tile, int stride,
                                             int slot, int* err) {
    uint32_t excl = 0;
    int64_t t = tile - 1;
    uint32_t spins = 0;
    while (t >= 0) {
        uint32_t s = ld_volatile(status + t * stride + slot);
        if ((s & ST_FLAGS) == 0) {
            if (++spins > SPIN_LIMIT) {
                atomicOr(err, ERR_TIMEOUT);
                break;
            }
            __nanosleep(64);
            continue;
        }
        excl += s & ST_COUNT;
        if ((s & ST_FLAGS) == ST_INC) break;
        --t;
    }
    return excl;
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

// ------------------------------------------------------ launch plumbing
struct PayloadArgs {
    const uint32_t* src[MAXPAY];  // nullptr: the source position (iota)
    uint32_t* dst[MAXPAY];
    int n;
};

enum KeyMode { KEY_DIRECT = 0, KEY_GATHER = 1, KEY_BUF = 2 };

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
    int32_t write_med;  // lev_out is this array's primary level and < lam
    int64_t pos0;       // first cloud-local position of the tile
    int32_t npos;       // positions in the tile
    int32_t first;      // 1: first tile of this cloud in this launch (no look-back past it)
};

struct FinUnit {
    int32_t cloud;
    int32_t seg;  // segment index at level lam of the cloud
};

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

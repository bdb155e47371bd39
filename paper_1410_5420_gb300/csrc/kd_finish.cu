// kd_finish.cu -- on-chip finisher of the GB300 k-d tree builder, in the
// paper's own form (Section 2.1, partition and recursion paragraphs).
//
// Once the level passes have split a cloud into subtrees of at most 1024
// tuples, one CTA finishes each subtree ("unit") in shared memory.  Every
// tuple is packed into one word holding its local rank in each super-key
// order (10 bits per dimension: k <= 3 fit a 32-bit word, k <= 6 a 64-bit
// word), so a compare of super keys is a compare of two bit fields and no
// lookup is needed.  The k index arrays are kept as word arrays, array q
// sorted by its super key within every current segment.  Per level with
// primary array p:
//   - the median of each segment is the word at its middle address of
//     array p: it becomes the node;
//   - each other array that a later level still reads is stably partitioned
//     around the median (less -> [lo, mid-1], greater -> [mid+1, hi], the
//     median itself dropped), every array and segment of the unit in one
//     block-wide scan of packed (less, greater) counters;
//   - array p itself is already split: its halves are in place.
// When every segment holds at most 3 tuples, the primary array gives every
// remaining node directly (the paper's termination at 1, 2 and 3 elements).
// The tree outputs of the unit are then written with coalesced stores.
#include <cstdint>
#include <type_traits>

#include "kd_internal.cuh"

namespace kd {

constexpr int FP_THREADS = 256;
constexpr int FP_SMAX = 1024;                    // tuples per unit
constexpr int FP_PPT = FP_SMAX / FP_THREADS;     // consecutive positions per thread
constexpr int FP_B = 10;                          // bits per local rank
constexpr int FP_WARPS = FP_THREADS / 32;
constexpr uint32_t FP_DONE = 0x80000000u;         // segment word: the position is a node

template <int K>
using fp_word_t = typename std::conditional<(K * FP_B <= 32), uint32_t, uint64_t>::type;

// Segment word of a position: lo (bits 0-11), hi (12-23), level at which it
// became a node (24-30), FP_DONE.
__device__ __forceinline__ uint32_t fp_seg(int lo, int hi) { return (uint32_t)lo | ((uint32_t)hi << 12); }
__device__ __forceinline__ int fp_lo(uint32_t w) { return (int)(w & 0xfffu); }
__device__ __forceinline__ int fp_hi(uint32_t w) { return (int)((w >> 12) & 0xfffu); }
__device__ __forceinline__ int fp_lvl(uint32_t w) { return (int)((w >> 24) & 0x7fu); }

template <typename W>
__device__ __forceinline__ uint32_t fp_rank(W w, int p) {
    return (uint32_t)(w >> (FP_B * p)) & ((1u << FP_B) - 1u);
}

// Four consecutive words at a 16-byte-aligned (32-bit words) or 32-byte-
// aligned (64-bit words) shared-memory address, as vector accesses.
__device__ __forceinline__ void fp_ld4(const uint32_t* a, uint32_t (&v)[4]) {
    const uint4 x = *reinterpret_cast<const uint4*>(a);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void fp_ld4(const uint64_t* a, uint64_t (&v)[4]) {
    const ulonglong2 x = reinterpret_cast<const ulonglong2*>(a)[0];
    const ulonglong2 y = reinterpret_cast<const ulonglong2*>(a)[1];
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}
__device__ __forceinline__ void fp_st4(uint32_t* a, const uint32_t (&v)[4]) {
    *reinterpret_cast<uint4*>(a) = make_uint4(v[0], v[1], v[2], v[3]);
}

// Shared memory of a unit (dynamic): the word arrays A[2][K][SMAX] (two
// buffers per array), the segment word of every position, the exclusive
// prefix of the packed counters of every non-primary array at every
// position, and the local rank 0 (lid) of the node at every position.
template <int K>
struct FpSmem {
    fp_word_t<K> A[2][K][FP_SMAX];
    uint32_t seg[FP_SMAX];
    uint32_t pre[K - 1][FP_SMAX];
    uint16_t node_lid[FP_SMAX];
};

template <int K>
constexpr size_t fp_smem_bytes() {
    return sizeof(FpSmem<K>);
}

// Largest unit size at level l of a unit of S tuples (segments at most halve).
__device__ __forceinline__ int fp_max_seg(int S, int l) { return S >> l; }

template <int K>
__global__ void __launch_bounds__(FP_THREADS, K <= 3 ? 5 : 2)
    k_finish_packed(const __grid_constant__ AllBufs bufs, const int64_t* __restrict__ unit_prefix, int ncloud,
                    int64_t unit_base, const CloudDev* __restrict__ clouds, const uint32_t* __restrict__ perm0,
                    int* __restrict__ err) {
    using W = fp_word_t<K>;
    constexpr int NQ = K - 1;
    extern __shared__ __align__(16) unsigned char fp_raw[];
    FpSmem<K>& sm = *reinterpret_cast<FpSmem<K>*>(fp_raw);
    __shared__ uint32_t s_wtot[NQ][FP_WARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t unit = unit_base + blockIdx.x;
    const int ci = last_le(unit_prefix, ncloud + 1, unit);
    const CloudDev& C = clouds[ci];
    int32_t ulo, uhi;
    segment_bounds(C.m, C.lam, (int32_t)(unit - unit_prefix[ci]), ulo, uhi);
    const int S = uhi - ulo + 1;
    if (S <= 0) return;
    if (S > FP_SMAX) {
        if (tid == 0) atomicOr(err, ERR_INTERNAL);
        return;
    }
    const int64_t g = C.off + ulo;
    bool bad = false;
    const int i0 = tid * FP_PPT;  // this thread's positions i0 .. i0 + FP_PPT - 1

    // ---- load: local ranks of every tuple --------------------------------
    // Array 0 is sorted by rank 0: the position of a tuple in it is its
    // local rank 0 (lid).  Array d >= 1 carries each element's rank 0; the
    // element's lid is found by binary search in array 0's rank-0 plane, and
    // its position in array d is the tuple's local rank d.
    uint32_t* r0 = reinterpret_cast<uint32_t*>(&sm.A[1][0][0]);     // array 0's rank-0 plane
    uint16_t* rho = reinterpret_cast<uint16_t*>(&sm.pre[0][0]);      // rho[(d-1)*SMAX + lid]
    uint16_t* lids = reinterpret_cast<uint16_t*>(&sm.A[1][1][0]);    // lids[(d-1)*SMAX + j]
    static_assert(sizeof(sm.pre) >= (size_t)NQ * FP_SMAX * 2, "rho fits the prefix area");
    static_assert(sizeof(W) * FP_SMAX * (K - 1) >= (size_t)NQ * FP_SMAX * 2, "lids fit the second buffer");
    {
        const uint32_t* a0 = bufs.p[0][C.buf[0]][0] + g;
        uint32_t rv[NQ][FP_PPT];
#pragma unroll
        for (int d = 1; d < K; ++d) {
            const uint32_t* ad = bufs.p[d][C.buf[d]][0] + g;
#pragma unroll
            for (int e = 0; e < FP_PPT; ++e) rv[d - 1][e] = i0 + e < S ? ad[i0 + e] : 0u;
        }
#pragma unroll
        for (int e = 0; e < FP_PPT; ++e)
            if (i0 + e < S) r0[i0 + e] = a0[i0 + e];
        __syncthreads();
#pragma unroll
        for (int d = 1; d < K; ++d) {
#pragma unroll
            for (int e = 0; e < FP_PPT; ++e) {
                const int j = i0 + e;
                if (j < S) {
                    int pos = 0;
#pragma unroll
                    for (int step = FP_SMAX / 2; step >= 1; step >>= 1)
                        if (pos + step <= S && r0[pos + step - 1] < rv[d - 1][e]) pos += step;
                    if (pos >= S || r0[pos] != rv[d - 1][e]) {
                        bad = true;
                        pos = 0;
                    }
                    lids[(d - 1) * FP_SMAX + j] = (uint16_t)pos;
                    rho[(d - 1) * FP_SMAX + pos] = (uint16_t)j;
                }
            }
        }
        __syncthreads();
        // array 0 in lid order: the packed word of tuple lid
#pragma unroll
        for (int e = 0; e < FP_PPT; ++e) {
            const int i = i0 + e;
            if (i < S) {
                W w = (W)i;
#pragma unroll
                for (int d = 1; d < K; ++d) w |= (W)rho[(d - 1) * FP_SMAX + i] << (FP_B * d);
                sm.A[0][0][i] = w;
            }
            sm.seg[i] = i < S ? fp_seg(0, S - 1) : FP_DONE;
        }
        __syncthreads();
#pragma unroll
        for (int d = 1; d < K; ++d)
#pragma unroll
            for (int e = 0; e < FP_PPT; ++e) {
                const int j = i0 + e;
                if (j < S) sm.A[0][d][j] = sm.A[0][0][lids[(d - 1) * FP_SMAX + j]];
            }
        __syncthreads();
    }

    // ---- levels -------------------------------------------------------------
    uint32_t cur = 0;  // bit q: the buffer holding array q
    int l = 0;
    for (; fp_max_seg(S, l) > 3; ++l) {
        const int p = (C.lam + l) % K;
        // last level with a partition: lf - 1, where lf is the final step's level
        int lf = l;
        while (fp_max_seg(S, lf) > 3) ++lf;
        // the non-primary arrays, in a fixed order, and whether a later
        // level reads them
        int qs[NQ];
        bool need[NQ];
#pragma unroll
        for (int x = 0; x < NQ; ++x) {
            const int q = (p + 1 + x) % K;
            qs[x] = q;
            // q is primary at level lq = l + 1 + x (the first later level where it is)
            need[x] = l + 1 + x <= lf;
        }
        static_assert(FP_PPT == 4, "four positions per thread");
        uint32_t sw[FP_PPT];
        int mid[FP_PPT];
        uint32_t mp[FP_PPT];
        uint32_t cnt[NQ][FP_PPT];
        W v[NQ][FP_PPT];
        const W* Ap = sm.A[(cur >> p) & 1u][p];
        fp_ld4(&sm.seg[i0], sw);
#pragma unroll
        for (int x = 0; x < NQ; ++x) {
            if (need[x]) fp_ld4(&sm.A[(cur >> qs[x]) & 1u][qs[x]][i0], v[x]);
            else
#pragma unroll
                for (int e = 0; e < FP_PPT; ++e) v[x][e] = 0;
        }
#pragma unroll
        for (int e = 0; e < FP_PPT; ++e) {
            const int i = i0 + e;
            const bool live = !(sw[e] & FP_DONE);
            const int lo = fp_lo(sw[e]), hi = fp_hi(sw[e]);
            mid[e] = lo + ((hi - lo) >> 1);
            const W M = live ? Ap[mid[e]] : (W)0;
            mp[e] = fp_rank(M, p);
            if (live && i == mid[e]) sm.node_lid[i] = (uint16_t)fp_rank(M, 0);
#pragma unroll
            for (int x = 0; x < NQ; ++x) {
                const uint32_t r = fp_rank(v[x][e], p);
                cnt[x][e] = (live && need[x]) ? ((r < mp[e] ? 1u : 0u) | (r > mp[e] ? 0x10000u : 0u)) : 0u;
            }
        }
        // exclusive prefix of the packed counters over positions: in the
        // thread, over the warp, over the block
        uint32_t tot[NQ];
#pragma unroll
        for (int x = 0; x < NQ; ++x) {
            uint32_t run = 0;
#pragma unroll
            for (int e = 0; e < FP_PPT; ++e) {
                const uint32_t c = cnt[x][e];
                cnt[x][e] = run;  // exclusive within the thread
                run += c;
            }
            uint32_t incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) s_wtot[x][warp] = incl;
            tot[x] = incl - run;  // exclusive within the warp
        }
        __syncthreads();
#pragma unroll
        for (int x = 0; x < NQ; ++x) {
            uint32_t wp = 0;
#pragma unroll
            for (int w2 = 0; w2 < FP_WARPS; ++w2) wp += w2 < warp ? s_wtot[x][w2] : 0u;
            tot[x] += wp;
#pragma unroll
            for (int e = 0; e < FP_PPT; ++e) cnt[x][e] += tot[x];
            fp_st4(&sm.pre[x][i0], cnt[x]);
        }
        __syncthreads();
        // destinations: less -> lo + (less before i in the segment), greater
        // -> mid + 1 + (greater before i in the segment); the median is dropped
        uint32_t nsw[FP_PPT];
#pragma unroll
        for (int e = 0; e < FP_PPT; ++e) {
            const int i = i0 + e;
            nsw[e] = sw[e];
            if (sw[e] & FP_DONE) continue;
            const int lo = fp_lo(sw[e]), hi = fp_hi(sw[e]);
#pragma unroll
            for (int x = 0; x < NQ; ++x) {
                if (!need[x]) continue;
                const uint32_t r = fp_rank(v[x][e], p);
                if (r == mp[e]) continue;
                const uint32_t base = sm.pre[x][lo];
                const uint32_t before = cnt[x][e] - base;
                const int dst = r < mp[e] ? lo + (int)(before & 0xffffu) : mid[e] + 1 + (int)(before >> 16);
                const bool ok = r < mp[e] ? dst < mid[e] : (dst > mid[e] && dst <= hi);
                if (ok) sm.A[((cur >> qs[x]) & 1u) ^ 1u][qs[x]][dst] = v[x][e]; else bad = true;
            }
            if (i == mid[e]) nsw[e] = sw[e] | FP_DONE | ((uint32_t)l << 24);
            else if (i < mid[e]) nsw[e] = fp_seg(lo, mid[e] - 1);
            else nsw[e] = fp_seg(mid[e] + 1, hi);
        }
        fp_st4(&sm.seg[i0], nsw);
#pragma unroll
        for (int x = 0; x < NQ; ++x)
            if (need[x]) cur ^= 1u << qs[x];
        __syncthreads();
    }
    // ---- final step: every segment holds at most 3 tuples ----------------
    // Array p (primary at level l) is sorted within each segment, so the
    // tuple at position i of array p is the node at address i: the median at
    // level l, its children at level l + 1.
    {
        const int p = (C.lam + l) % K;
        const W* Ap = sm.A[(cur >> p) & 1u][p];
#pragma unroll
        for (int e = 0; e < FP_PPT; ++e) {
            const int i = i0 + e;
            const uint32_t sw = sm.seg[i];
            if (i >= S || (sw & FP_DONE)) continue;
            const int lo = fp_lo(sw), hi = fp_hi(sw);
            const int md = lo + ((hi - lo) >> 1);
            sm.node_lid[i] = (uint16_t)fp_rank(Ap[i], 0);
            sm.seg[i] = (i == md) ? (sw | FP_DONE | ((uint32_t)l << 24))
                                  : (fp_seg(i, i) | FP_DONE | ((uint32_t)(l + 1) << 24));
        }
    }
    __syncthreads();
    // ---- outputs, coalesced: node tuple, children, split dimension --------
    const uint32_t* a0 = bufs.p[0][C.buf[0]][0] + g;
    for (int i = tid; i < S; i += FP_THREADS) {
        const uint32_t sw = sm.seg[i];
        if (!(sw & FP_DONE)) {
            bad = true;
            continue;
        }
        const int lo = fp_lo(sw), hi = fp_hi(sw), lv = fp_lvl(sw);
        const int32_t addr = ulo + i;
        const uint32_t rr = a0[sm.node_lid[i]];
        if (rr >= C.off && rr < C.off + C.m)
            C.node[addr] = (int32_t)((int64_t)perm0[rr] - C.in_off);
        else
            bad = true;
        if (C.left) C.left[addr] = lo <= i - 1 ? ulo + child_mid(lo, i - 1) : -1;
        if (C.right) C.right[addr] = i + 1 <= hi ? ulo + child_mid(i + 1, hi) : -1;
        if (C.dim) C.dim[addr] = (uint8_t)((C.lam + lv) % K);
    }
    if (bad) atomicOr(err, ERR_INTERNAL);
}

// Largest k the packed finisher serves (six 10-bit ranks in a 64-bit word).
constexpr int FP_KMAX = 6;

int finish_packed_kmax() { return FP_KMAX; }
int finish_packed_smax() { return FP_SMAX; }

template <int K>
static cudaError_t fp_init() {
    return cudaFuncSetAttribute((const void*)k_finish_packed<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fp_smem_bytes<K>());
}

cudaError_t init_finish_packed() {
    cudaError_t e = fp_init<2>();
    if (e == cudaSuccess) e = fp_init<3>();
    if (e == cudaSuccess) e = fp_init<4>();
    if (e == cudaSuccess) e = fp_init<5>();
    if (e == cudaSuccess) e = fp_init<6>();
    return e;
}

// Finisher over units [unit_base, unit_base + nunits) of subtrees of at most
// 1024 tuples, 2 <= k <= 6.
cudaError_t launch_finish_packed(const AllBufs& bufs, int k, const int64_t* unit_prefix, int ncloud,
                                 int64_t unit_base, int nunits, const CloudDev* clouds, const uint32_t* perm0,
                                 int* err, cudaStream_t s) {
    if (nunits == 0) return cudaSuccess;
    switch (k) {
#define KD_FP_CASE(KK)                                                                                      \
    case KK:                                                                                              \
        k_finish_packed<KK><<<nunits, FP_THREADS, fp_smem_bytes<KK>(), s>>>(bufs, unit_prefix, ncloud,   \
                                                                            unit_base, clouds, perm0, err); \
        break;
        KD_FP_CASE(2)
        KD_FP_CASE(3)
        KD_FP_CASE(4)
        KD_FP_CASE(5)
        KD_FP_CASE(6)
#undef KD_FP_CASE
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace kd

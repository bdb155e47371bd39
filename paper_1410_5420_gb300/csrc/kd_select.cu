// kd_select.cu -- the O(n log n) k-d tree build of the paper's "Comparative
// Performance" section ("The O(n log n) Algorithm"), on the GPU.
//
// The paper's comparison algorithm sorts one index array by one super key,
// removes duplicate tuples, and then, at every level of the recursion, finds
// the median of each sub-array in the level's super key with a linear-time
// selection and partitions the sub-array around it.  It builds the same
// tree as the presorting method (every median is unique under the total
// super-key order), but without the other k-1 presorts.
//
// Here the index array is the presorting build's array 0 (super key 0,
// duplicates removed) and it carries its tuples' key words as planes (the
// tuple index plus k key planes, moved together).  Every segment of a level
// is processed by the same launches:
//   k_sel_hist / k_sel_choose  most-significant-digit radix selection.  Per
//       round, a 256-bin histogram of the next byte of the level's super key
//       over each segment's candidates (elements whose earlier bytes equal
//       the prefix chosen so far); the bin that holds the median's rank
//       becomes the next prefix byte.  A segment is resolved once its bin
//       holds a single element.  Each round reads every element once, so a
//       level is O(n) work, as with the paper's median of medians.
//   k_sel_move  partition around the medians: less -> the lower half,
//       greater -> the upper half, the median becomes the node.  Since the
//       next level selects afresh, the halves need not keep an order: slots
//       are claimed with atomics.
//   k_sel_finish  a segment of at most SEL_T tuples is finished by one CTA in
//       shared memory (4-bit selection rounds while sub-segments exceed 32
//       tuples), then one warp per sub-segment of at most 32 tuples (each
//       lane's rank in every super key from pairwise compares).
#include <cstdint>

#include "kd_internal.cuh"

namespace kd {

constexpr int SEL_THREADS = 256;
constexpr int SEL_TILE = 2048;   // largest tile of the level kernels (positions)
constexpr int SEL_IPT = SEL_TILE / SEL_THREADS;
constexpr int SEL_FIN_SUBMAX = 64;  // sub-segments of a finisher unit while they exceed 32 tuples

// Planes of the index array: tuple index and key words of each coordinate,
// two buffers.
template <typename KW>
struct SelBufs {
    uint32_t* id[2];
    KW* key[2][MAXK];
};

// Selection state of one segment of the current level.
template <typename KW>
struct SelSeg {
    int32_t lo, hi;
    int32_t pos;      // array position of the median; -1 unresolved, -2 empty segment
    uint32_t target;  // rank of the median among the current candidates
    uint32_t cnt[2];  // partition: elements placed in the lower / upper half
    int32_t start;    // first byte of the super key the candidates do not all share
    uint32_t pad;
    KW span_and, span_or;  // AND and OR of the segment's leading key words
    KW prefix[MAXK];  // super-key words; the bytes chosen so far (high bytes first)
};

// Byte r of a super key of k words of B bytes: word r / B, counted from the
// most significant byte.
template <typename KW>
__device__ __forceinline__ int sel_shift(int r) {
    constexpr int B = sizeof(KW);
    return 8 * (B - 1 - r % B);
}

template <typename KW>
__global__ void k_sel_init(int32_t m, int L, int nseg, SelSeg<KW>* __restrict__ segs, uint32_t* __restrict__ ghist) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
        SelSeg<KW> S;
        segment_bounds(m, L, s, S.lo, S.hi);
        S.pos = S.hi < S.lo ? -2 : -1;
        S.target = S.hi < S.lo ? 0u : (uint32_t)((S.hi - S.lo) >> 1);
        S.cnt[0] = S.cnt[1] = 0;
        S.start = 0;
        S.pad = 0;
        S.span_and = ~(KW)0;
        S.span_or = 0;
        for (int j = 0; j < MAXK; ++j) S.prefix[j] = 0;
        segs[s] = S;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)nseg * RADIX;
         i += (int64_t)gridDim.x * blockDim.x)
        ghist[i] = 0;
}

// The tile's segments (at most LEVEL_NSMAX) and their selection state.
template <typename KW>
struct SelTile {
    int ns;
    int32_t lo[LEVEL_NSMAX], hi[LEVEL_NSMAX], idx[LEVEL_NSMAX];
    int32_t pos[LEVEL_NSMAX];
    int32_t start[LEVEL_NSMAX];
    KW prefix[LEVEL_NSMAX][MAXK];
};

template <typename KW>
__device__ __forceinline__ void sel_load_tile(SelTile<KW>& T, int32_t pos0, int32_t npos, int32_t m, int L,
                                              const SelSeg<KW>* __restrict__ segs, int* err) {
    if (threadIdx.x == 0) {
        T.ns = tile_segments(pos0, npos, m, L, T.lo, T.hi, T.idx, err);
        for (int x = 0; x < T.ns; ++x) {
            const SelSeg<KW>& S = segs[T.idx[x]];
            T.pos[x] = S.pos;
            T.start[x] = S.start;
            for (int j = 0; j < MAXK; ++j) T.prefix[x][j] = S.prefix[j];
        }
    }
    __syncthreads();
}

// One selection round: histogram of super-key byte r over the candidates.
template <typename KW>
__global__ void __launch_bounds__(SEL_THREADS) k_sel_hist(const __grid_constant__ SelBufs<KW> bufs, int cur, int k,
                                                          int32_t m, int L, int r, int tile,
                                                          const SelSeg<KW>* __restrict__ segs,
                                                          uint32_t* __restrict__ ghist, int32_t* __restrict__ gany,
                                                          int* __restrict__ err) {
    __shared__ SelTile<KW> T;
    __shared__ uint32_t h[LEVEL_NSMAX][RADIX];
    __shared__ int32_t any[LEVEL_NSMAX][RADIX];
    const int tid = threadIdx.x;
    const int32_t pos0 = blockIdx.x * tile;
    const int32_t npos = min(tile, m - pos0);
    sel_load_tile(T, pos0, npos, m, L, segs, err);
    bool open = false;
    for (int x = 0; x < T.ns; ++x) open |= T.pos[x] == -1 && r >= T.start[x];
    if (!open) return;  // uniform: every segment of the tile is resolved, or shares byte r
    for (int i = tid; i < LEVEL_NSMAX * RADIX; i += SEL_THREADS) (&h[0][0])[i] = 0;
    __syncthreads();
    constexpr int B = sizeof(KW);
    const int j = r / B, sh = sel_shift<KW>(r);
    const int p = L % k;
    for (int e = 0; e < SEL_IPT; ++e) {
        const int o = e * SEL_THREADS + tid;
        const int32_t pos = pos0 + o;
        int sj = o < npos ? tile_slot(T.lo, T.hi, T.ns, pos) : -1;
        bool cand = sj >= 0 && T.pos[sj] == -1 && r >= T.start[sj];
        uint32_t dig = 0;
        if (cand) {
            // the words of the super key up to word j, compared with the prefix
            KW wj = 0;
#pragma unroll
            for (int jj = 0; jj < MAXK; ++jj) {
                if (jj > j) break;
                int d = p + jj;
                if (d >= k) d -= k;
                const KW x = bufs.key[cur][d][pos];
                if (jj < j) cand = cand && x == T.prefix[sj][jj];
                else wj = x;
            }
            if (cand && sh + 8 < 8 * B) cand = (wj >> (sh + 8)) == (T.prefix[sj][j] >> (sh + 8));
            dig = (uint32_t)(wj >> sh) & 255u;
        }
        // candidates of one segment and digit in this warp add once (long runs of
        // equal top bytes would otherwise serialise on one counter)
        const uint32_t key = cand ? ((uint32_t)sj << 8 | dig) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        if (cand && (threadIdx.x & 31) == __ffs(peers) - 1) {
            atomicAdd(&h[sj][dig], (uint32_t)__popc(peers));
            any[sj][dig] = pos;
        }
    }
    __syncthreads();
    for (int x = 0; x < T.ns; ++x) {
        if (T.pos[x] != -1) continue;
        const uint32_t c = h[x][tid];
        if (c) {
            atomicAdd(&ghist[(int64_t)T.idx[x] * RADIX + tid], c);
            gany[(int64_t)T.idx[x] * RADIX + tid] = any[x][tid];
        }
    }
}

// AND and OR of a 64- or 32-bit word over the lanes of `mask` (all calling).
__device__ __forceinline__ void sel_warp_and_or(uint32_t mask, uint32_t w, uint32_t& a, uint32_t& o) {
    a = __reduce_and_sync(mask, w);
    o = __reduce_or_sync(mask, w);
}
__device__ __forceinline__ void sel_warp_and_or(uint32_t mask, uint64_t w, uint64_t& a, uint64_t& o) {
    const uint32_t ah = __reduce_and_sync(mask, (uint32_t)(w >> 32)), al = __reduce_and_sync(mask, (uint32_t)w);
    const uint32_t oh = __reduce_or_sync(mask, (uint32_t)(w >> 32)), ol = __reduce_or_sync(mask, (uint32_t)w);
    a = ((uint64_t)ah << 32) | al;
    o = ((uint64_t)oh << 32) | ol;
}

__device__ __forceinline__ void sel_atomic_and_or(uint32_t* a, uint32_t* o, uint32_t va, uint32_t vo) {
    atomicAnd(a, va);
    atomicOr(o, vo);
}
__device__ __forceinline__ void sel_atomic_and_or(uint64_t* a, uint64_t* o, uint64_t va, uint64_t vo) {
    atomicAnd(reinterpret_cast<unsigned long long*>(a), (unsigned long long)va);
    atomicOr(reinterpret_cast<unsigned long long*>(o), (unsigned long long)vo);
}

// Span of every segment's leading key words (x_p of super key p): the
// bits on which AND and OR agree are shared by all of its elements.
template <typename KW>
__global__ void __launch_bounds__(SEL_THREADS) k_sel_span(const __grid_constant__ SelBufs<KW> bufs, int cur, int k,
                                                          int32_t m, int L, int tile, SelSeg<KW>* __restrict__ segs,
                                                          int* __restrict__ err) {
    __shared__ SelTile<KW> T;
    __shared__ KW s_and[LEVEL_NSMAX], s_or[LEVEL_NSMAX];
    const int tid = threadIdx.x;
    const int32_t pos0 = blockIdx.x * tile;
    const int32_t npos = min(tile, m - pos0);
    if (tid < LEVEL_NSMAX) {
        s_and[tid] = ~(KW)0;
        s_or[tid] = 0;
    }
    sel_load_tile(T, pos0, npos, m, L, segs, err);  // (synchronises the block)
    const int p = L % k;
    // warp, then block, then one global update per segment of the tile
    for (int e = 0; e < SEL_IPT; ++e) {
        const int o = e * SEL_THREADS + tid;
        const int sj = o < npos ? tile_slot(T.lo, T.hi, T.ns, pos0 + o) : -1;
        const KW w = sj >= 0 ? bufs.key[cur][p][pos0 + o] : (KW)0;
        const uint32_t peers = __match_any_sync(0xffffffffu, (uint32_t)sj);  // lanes of one segment
        KW a, b;
        sel_warp_and_or(peers, w, a, b);
        if (sj >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) sel_atomic_and_or(&s_and[sj], &s_or[sj], a, b);
    }
    __syncthreads();
    if (tid < T.ns) sel_atomic_and_or(&segs[T.idx[tid]].span_and, &segs[T.idx[tid]].span_or, s_and[tid], s_or[tid]);
}

// The leading bytes every element of a segment shares become its prefix;
// selection starts at the first byte where they differ.  *first receives
// the smallest such byte over the level's open segments.
template <typename KW>
__global__ void k_sel_skip(int nseg, SelSeg<KW>* __restrict__ segs, int32_t* __restrict__ first) {
    constexpr int B = sizeof(KW);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
        SelSeg<KW>& S = segs[s];
        if (S.pos != -1) continue;
        const KW diff = S.span_and ^ S.span_or;
        const int lead = diff == 0 ? 8 * B : (B == 8 ? __clzll((long long)diff) : __clz((int)(uint32_t)diff));
        const int cb = lead / 8 < B ? lead / 8 : B - 1;  // keep at least the last byte of the word to select
        const KW mask = cb == 0 ? (KW)0 : ~(KW)0 << (8 * (B - cb));
        S.prefix[0] = S.span_and & mask;
        S.start = cb;
        atomicMin(first, cb);
    }
}

// One warp per segment: the bin holding the median's rank becomes the next
// prefix byte; a bin of one element resolves the segment.
template <typename KW>
__global__ void k_sel_choose(int nseg, int r, int nbytes, SelSeg<KW>* __restrict__ segs,
                             uint32_t* __restrict__ ghist, const int32_t* __restrict__ gany,
                             uint32_t* __restrict__ unresolved, int* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nseg) return;
    SelSeg<KW>& S = segs[s];
    if (S.pos != -1 || r < S.start) return;  // uniform per warp (byte r is shared: already in the prefix)
    uint32_t* hs = ghist + (int64_t)s * RADIX;
    uint32_t v[8], sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        v[i] = hs[lane * 8 + i];
        sum += v[i];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t target = S.target;
    const uint32_t excl = incl - sum;
    const bool mine = target >= excl && target < incl;
    const uint32_t who = __ballot_sync(0xffffffffu, mine);
    if (who == 0) {  // the candidates do not cover the rank: inconsistent state
        if (lane == 0) {
            atomicOr(err, ERR_INTERNAL);
            S.pos = -2;
        }
        return;
    }
    if (mine) {
        uint32_t c = excl;  // elements of the bins before b
        int b = 0;
        uint32_t cnt = 0;
        bool found = false;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (!found) {
                if (target < c + v[i]) {
                    b = lane * 8 + i;
                    cnt = v[i];
                    found = true;
                } else {
                    c += v[i];
                }
            }
        }
        S.target = target - c;
        const int j = r / (int)sizeof(KW);
        S.prefix[j] |= (KW)b << sel_shift<KW>(r);
        if (cnt == 1) {
            S.pos = gany[(int64_t)s * RADIX + b];
        } else if (r + 1 >= nbytes) {
            atomicOr(err, ERR_INTERNAL);  // two elements with equal super keys after deduplication
            S.pos = -2;
        } else {
            atomicAdd(unresolved, 1u);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) hs[lane * 8 + i] = 0;
}

// Partition around the resolved medians; the median of each segment becomes
// the node at the segment's middle address.
template <typename KW>
__global__ void __launch_bounds__(SEL_THREADS) k_sel_move(const __grid_constant__ SelBufs<KW> bufs, int cur, int k,
                                                          int32_t m, int L, int tile, SelSeg<KW>* __restrict__ segs,
                                                          int32_t* __restrict__ node, int64_t in_off,
                                                          int* __restrict__ err) {
    __shared__ SelTile<KW> T;
    __shared__ KW med[LEVEL_NSMAX][MAXK];
    __shared__ uint32_t scnt[LEVEL_NSMAX][2], sbase[LEVEL_NSMAX][2];
    const int tid = threadIdx.x;
    const int32_t pos0 = blockIdx.x * tile;
    const int32_t npos = min(tile, m - pos0);
    sel_load_tile(T, pos0, npos, m, L, segs, err);
    const int p = L % k;
    if (tid < T.ns * MAXK) {
        const int x = tid / MAXK, j = tid % MAXK;
        int d = p + j;
        while (d >= k) d -= k;
        const int32_t mp = T.pos[x];
        med[x][j] = (j < k && mp >= T.lo[x] && mp <= T.hi[x]) ? bufs.key[cur][d][mp] : (KW)0;
    }
    if (tid < LEVEL_NSMAX * 2) (&scnt[0][0])[tid] = 0;
    __syncthreads();
    int flag[SEL_IPT];
    uint32_t local[SEL_IPT];
    int slot[SEL_IPT];
#pragma unroll
    for (int e = 0; e < SEL_IPT; ++e) {
        const int o = e * SEL_THREADS + tid;
        flag[e] = -1;
        slot[e] = -1;
        local[e] = 0;
        if (o >= npos) continue;
        const int32_t pos = pos0 + o;
        const int sj = tile_slot(T.lo, T.hi, T.ns, pos);
        if (sj < 0) continue;
        if (T.pos[sj] < T.lo[sj] || T.pos[sj] > T.hi[sj]) {
            atomicOr(err, ERR_INTERNAL);
            continue;
        }
        int c = 0;
#pragma unroll
        for (int j = 0; j < MAXK; ++j) {
            if (j >= k || c != 0) break;
            int d = p + j;
            if (d >= k) d -= k;
            const KW x = bufs.key[cur][d][pos], y = med[sj][j];
            if (x != y) c = x < y ? -1 : 1;
        }
        slot[e] = sj;
        if (c == 0) {
            if (pos != T.pos[sj]) atomicOr(err, ERR_INTERNAL);
            const int32_t mid = T.lo[sj] + ((T.hi[sj] - T.lo[sj]) >> 1);
            node[mid] = (int32_t)((int64_t)bufs.id[cur][pos] - in_off);
            continue;
        }
        flag[e] = c > 0 ? 1 : 0;
        local[e] = atomicAdd(&scnt[sj][flag[e]], 1u);
    }
    __syncthreads();
    if (tid < T.ns * 2) {
        const int x = tid >> 1, f = tid & 1;
        sbase[x][f] = atomicAdd(&segs[T.idx[x]].cnt[f], scnt[x][f]);
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < SEL_IPT; ++e) {
        if (flag[e] < 0) continue;
        const int sj = slot[e];
        const int32_t lo = T.lo[sj], hi = T.hi[sj], mid = lo + ((hi - lo) >> 1);
        const int32_t dst = (flag[e] ? mid + 1 : lo) + (int32_t)(sbase[sj][flag[e]] + local[e]);
        if (flag[e] ? (dst <= mid || dst > hi) : (dst >= mid)) {
            atomicOr(err, ERR_INTERNAL);
            continue;
        }
        const int32_t pos = pos0 + e * SEL_THREADS + tid;  // < pos0 + npos: flag[e] >= 0
        bufs.id[cur ^ 1][dst] = bufs.id[cur][pos];
        for (int d = 0; d < k; ++d) bufs.key[cur ^ 1][d][dst] = bufs.key[cur][d][pos];
    }
}

// ------------------------------------------------------------- finisher
// One CTA per segment of at most SEL_T tuples at level lam.  Shared memory
// (dynamic): two buffers of (index, k key planes) for up to T elements,
// then the segment word of every position (lo | hi << 12 | level << 24 |
// done), the sub-segment index of every position, and the selection state of
// the sub-segments.
constexpr uint32_t SF_DONE = 0x80000000u;

template <typename KW>
struct SelSub {
    int32_t lo, hi, pos;
    uint32_t target;
    uint32_t cnt[2];
    int32_t start;  // first nibble of the super key the sub-segment's elements do not all share
    uint32_t pad;
    KW sand, sor;   // AND and OR of its leading key words
    uint32_t hist[16];
    int32_t any[16];
    KW prefix[MAXK];
};

template <typename KW>
size_t sel_finish_smem(int k, int T) {
    return (size_t)2 * T * (4 + (size_t)k * sizeof(KW)) + (size_t)T * 4 + (size_t)T + 16 +
           sizeof(SelSub<KW>) * SEL_FIN_SUBMAX + 64;
}

template <typename KW>
__device__ __forceinline__ void sf_emit(int32_t* node, int32_t* left, int32_t* right, uint8_t* dim, int32_t ulo,
                                        int32_t a, int32_t b, int32_t c, uint32_t id, int64_t in_off, int d) {
    const int32_t addr = ulo + c;
    node[addr] = (int32_t)((int64_t)id - in_off);
    if (left) left[addr] = a <= c - 1 ? ulo + child_mid(a, c - 1) : -1;
    if (right) right[addr] = c + 1 <= b ? ulo + child_mid(c + 1, b) : -1;
    if (dim) dim[addr] = (uint8_t)d;
}

template <typename KW>
__global__ void __launch_bounds__(SEL_THREADS) k_sel_finish(const __grid_constant__ SelBufs<KW> bufs, int cur, int k,
                                                            int32_t m, int lam, int T, int32_t* __restrict__ node,
                                                            int32_t* __restrict__ left, int32_t* __restrict__ right,
                                                            uint8_t* __restrict__ dim, int64_t in_off,
                                                            int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char sf_raw[];
    __shared__ int s_first;  // smallest first nibble to select over the sub-segments of a level
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int32_t ulo, uhi;
    segment_bounds(m, lam, blockIdx.x, ulo, uhi);
    const int S = uhi - ulo + 1;
    if (S <= 0) return;
    if (S > T) {
        if (tid == 0) atomicOr(err, ERR_INTERNAL);
        return;
    }
    // shared memory layout (see sel_finish_smem)
    unsigned char* q = sf_raw;
    KW* const keys0 = reinterpret_cast<KW*>(q);
    q += (size_t)T * k * sizeof(KW);
    uint32_t* const ids0 = reinterpret_cast<uint32_t*>(q);
    q += (size_t)T * 4;
    KW* const keys1 = reinterpret_cast<KW*>(q);
    q += (size_t)T * k * sizeof(KW);
    uint32_t* const ids1 = reinterpret_cast<uint32_t*>(q);
    q += (size_t)T * 4;
    // buffer bb of the element planes (selected, not indexed, to stay in registers)
    auto KB = [&](int bb) { return bb ? keys1 : keys0; };
    auto IB = [&](int bb) { return bb ? ids1 : ids0; };
    uint32_t* segw = reinterpret_cast<uint32_t*>(q);
    q += (size_t)T * 4;
    uint8_t* subid = q;
    q += ((size_t)T + 15) & ~(size_t)15;
    SelSub<KW>* sub = reinterpret_cast<SelSub<KW>*>(q);
    for (int i = tid; i < S; i += SEL_THREADS) {
        ids0[i] = bufs.id[cur][ulo + i];
        for (int d = 0; d < k; ++d) keys0[d * T + i] = bufs.key[cur][d][ulo + i];
        segw[i] = (uint32_t)(S - 1) << 12;  // lo 0, hi S-1
        subid[i] = 0;
    }
    __syncthreads();
    int b = 0;  // buffer holding the elements
    int l = 0;
    bool bad = false;
    constexpr int B = sizeof(KW);
    const int nnib = 2 * k * B;
    // ---- block levels: sub-segments of more than 32 tuples ----------------
    for (; (S >> l) > 32; ++l) {
        const int p = (lam + l) % k;
        const int nsub = 1 << l;  // at most S / 32 <= SEL_FIN_SUBMAX
        for (int s = tid; s < nsub; s += SEL_THREADS) {
            int32_t lo = 0, hi = S - 1;
            for (int f = l - 1; f >= 0; --f) {
                const int32_t c = lo + ((hi - lo) >> 1);
                if ((s >> f) & 1) lo = c + 1; else hi = c - 1;
            }
            SelSub<KW>& U = sub[s];
            U.lo = lo;
            U.hi = hi;
            U.pos = hi < lo ? -2 : -1;
            U.target = hi < lo ? 0u : (uint32_t)((hi - lo) >> 1);
            U.cnt[0] = U.cnt[1] = 0;
            U.start = 0;
            U.sand = ~(KW)0;
            U.sor = 0;
            for (int x = 0; x < 16; ++x) U.hist[x] = 0;
            for (int j = 0; j < MAXK; ++j) U.prefix[j] = 0;
        }
        if (tid == 0) s_first = 2 * B - 1;
        __syncthreads();
        // the leading nibbles every element of a sub-segment shares become
        // its prefix; its selection starts at the first nibble where they differ
        for (int i0 = 0; i0 < S; i0 += SEL_THREADS) {
            const int i = i0 + tid;
            const bool v = i < S && !(segw[i] & SF_DONE);
            const uint32_t su = v ? subid[i] : 0xffffffffu;
            const KW w = v ? KB(b)[p * T + i] : (KW)0;
            const uint32_t peers = __match_any_sync(0xffffffffu, su);
            KW a, o;
            sel_warp_and_or(peers, w, a, o);
            if (v && lane == __ffs(peers) - 1) sel_atomic_and_or(&sub[su].sand, &sub[su].sor, a, o);
        }
        __syncthreads();
        for (int s = tid; s < nsub; s += SEL_THREADS) {
            SelSub<KW>& U = sub[s];
            if (U.pos != -1) continue;
            const KW diff = U.sand ^ U.sor;
            const int lead = diff == 0 ? 8 * B : (B == 8 ? __clzll((long long)diff) : __clz((int)(uint32_t)diff));
            const int cn = lead / 4 < 2 * B ? lead / 4 : 2 * B - 1;
            U.prefix[0] = cn == 0 ? (KW)0 : (U.sand & (~(KW)0 << (4 * (2 * B - cn))));
            U.start = cn;
            atomicMin(&s_first, cn);
        }
        __syncthreads();
        // selection: 4-bit rounds, most significant nibble first
        for (int r4 = s_first; r4 < nnib; ++r4) {
            const int r = r4 >> 1;
            const int j = r / B;
            const int sh = 8 * (B - 1 - r % B) + ((r4 & 1) ? 0 : 4);
            int dj = p + j;
            if (dj >= k) dj -= k;
            for (int i0 = 0; i0 < S; i0 += SEL_THREADS) {  // whole warps, for the aggregation below
                const int i = i0 + tid;
                bool cand = i < S && !(segw[i] & SF_DONE);
                const int su = cand ? subid[i] : 0;
                cand = cand && sub[su].pos == -1 && r4 >= sub[su].start;
                uint32_t nib = 0;
                if (cand) {
                    const SelSub<KW>& U = sub[su];
                    for (int jj = 0; jj < j && cand; ++jj) {
                        int d = p + jj;
                        if (d >= k) d -= k;
                        cand = KB(b)[d * T + i] == U.prefix[jj];
                    }
                    const KW wj = KB(b)[dj * T + i];
                    if (cand && sh + 4 < 8 * B) cand = (wj >> (sh + 4)) == (U.prefix[j] >> (sh + 4));
                    nib = (uint32_t)(wj >> sh) & 15u;
                }
                const uint32_t key = cand ? ((uint32_t)su << 4 | nib) : 0xffffffffu;
                const uint32_t peers = __match_any_sync(0xffffffffu, key);
                if (cand && lane == __ffs(peers) - 1) {
                    atomicAdd(&sub[su].hist[nib], (uint32_t)__popc(peers));
                    sub[su].any[nib] = i;
                }
            }
            __syncthreads();
            bool open = false;
            for (int s = tid; s < nsub; s += SEL_THREADS) {
                SelSub<KW>& U = sub[s];
                if (U.pos != -1) continue;
                if (r4 < U.start) {  // this nibble is shared: already in the prefix
                    open = true;
                    continue;
                }
                uint32_t c = 0, hb = 0;
                int bb = -1;
                for (int x = 0; x < 16; ++x) {
                    const uint32_t h = U.hist[x];
                    if (bb < 0) {
                        if (U.target < c + h) {
                            bb = x;
                            hb = h;
                        } else {
                            c += h;
                        }
                    }
                    U.hist[x] = 0;
                }
                if (bb < 0) {
                    bad = true;
                    U.pos = -2;
                    continue;
                }
                U.target -= c;
                U.prefix[j] |= (KW)bb << sh;
                if (hb == 1) {
                    U.pos = U.any[bb];
                } else if (r4 + 1 >= nnib) {
                    bad = true;  // equal super keys after deduplication
                    U.pos = -2;
                } else {
                    open = true;
                }
            }
            if (!__syncthreads_or(open)) break;
        }
        // partition around the medians (the median becomes the node)
        for (int i = tid; i < S; i += SEL_THREADS) {
            if (segw[i] & SF_DONE) continue;
            SelSub<KW>& U = sub[subid[i]];
            if (U.pos < U.lo || U.pos > U.hi) {
                bad = true;
                continue;
            }
            const int32_t mid = U.lo + ((U.hi - U.lo) >> 1);
            int c = 0;
            for (int jj = 0; jj < k && c == 0; ++jj) {
                int d = p + jj;
                if (d >= k) d -= k;
                const KW x = KB(b)[d * T + i], y = KB(b)[d * T + U.pos];
                if (x != y) c = x < y ? -1 : 1;
            }
            if (c == 0) {
                if (i != U.pos) bad = true;
                sf_emit<KW>(node, left, right, dim, ulo, U.lo, U.hi, mid, IB(b)[i], in_off, p);
                continue;
            }
            const int f = c > 0 ? 1 : 0;
            const int32_t dst = (f ? mid + 1 : U.lo) + (int32_t)atomicAdd(&U.cnt[f], 1u);
            if (f ? (dst <= mid || dst > U.hi) : (dst >= mid)) {
                bad = true;
                continue;
            }
            IB(b ^ 1)[dst] = IB(b)[i];
            for (int d = 0; d < k; ++d) KB(b ^ 1)[d * T + dst] = KB(b)[d * T + i];
        }
        __syncthreads();
        // the segment of every position at the next level
        for (int i = tid; i < S; i += SEL_THREADS) {
            if (segw[i] & SF_DONE) continue;
            const int s = subid[i];
            const int32_t lo = sub[s].lo, hi = sub[s].hi, mid = lo + ((hi - lo) >> 1);
            if (i == mid) {
                segw[i] |= SF_DONE;
            } else if (i < mid) {
                subid[i] = (uint8_t)(2 * s);
                segw[i] = (uint32_t)lo | ((uint32_t)(mid - 1) << 12);
            } else {
                subid[i] = (uint8_t)(2 * s + 1);
                segw[i] = (uint32_t)(mid + 1) | ((uint32_t)hi << 12);
            }
        }
        b ^= 1;
        __syncthreads();
    }
    // ---- warp levels: one warp per sub-segment of at most 32 tuples --------
    // Each lane holds one tuple.  LESS_q (the lanes whose super key q is
    // smaller) comes from pairwise compares; a lane's rank in its current
    // sub-segment at a level with primary p is popc(LESS_p & SUB).
    const int nsub = 1 << l;
    const uint32_t lt = lanemask_lt();
    for (int s = warp; s < nsub; s += SEL_THREADS / 32) {
        int32_t lo = 0, hi = S - 1;
        for (int f = l - 1; f >= 0; --f) {
            const int32_t c = lo + ((hi - lo) >> 1);
            if ((s >> f) & 1) lo = c + 1; else hi = c - 1;
        }
        const int n = hi - lo + 1;
        if (n <= 0) continue;  // uniform per warp
        if (n > 32) {
            bad = true;
            continue;
        }
        const bool in = lane < n;
        KW w[MAXK];
        uint32_t id = in ? IB(b)[lo + lane] : 0u;
#pragma unroll
        for (int d = 0; d < MAXK; ++d) w[d] = (in && d < k) ? KB(b)[d * T + lo + lane] : (KW)0;
        uint32_t less[MAXK];
#pragma unroll
        for (int qd = 0; qd < MAXK; ++qd) less[qd] = 0;
        // per source lane: which of its coordinate words are below / equal to
        // this lane's (bit d); super key q then reads them rotated by q
        const uint32_t full = (1u << k) - 1u;
        for (int src = 0; src < n; ++src) {
            uint32_t ltm = 0, eqm = 0;
#pragma unroll
            for (int d = 0; d < MAXK; ++d) {
                if (d < k) {
                    const KW o = __shfl_sync(0xffffffffu, w[d], src);
                    ltm |= (o < w[d] ? 1u : 0u) << d;
                    eqm |= (o == w[d] ? 1u : 0u) << d;
                }
            }
#pragma unroll
            for (int qd = 0; qd < MAXK; ++qd) {
                if (qd < k) {
                    const uint32_t ne = ~((eqm >> qd) | (eqm << (k - qd))) & full;
                    const uint32_t lt = ((ltm >> qd) | (ltm << (k - qd))) & full;
                    if (ne && ((lt >> (__ffs(ne) - 1)) & 1u)) less[qd] |= 1u << src;
                }
            }
        }
        uint32_t subm = __ballot_sync(0xffffffffu, in);
        bool active = in;
        int32_t mlo = lo, mhi = hi;
        for (int lv = l; __any_sync(0xffffffffu, active); ++lv) {
            if (active && (mhi < mlo || lv >= l + 32)) {  // inconsistent ranks: report, never spin
                bad = true;
                active = false;
            }
            const int p = (lam + lv) % k;
            uint32_t lp = 0;
#pragma unroll
            for (int qd = 0; qd < MAXK; ++qd)
                if (qd == p) lp = less[qd];
            const int rank = __popc(lp & subm);
            const int32_t c = mlo + ((mhi - mlo) >> 1);
            const bool goL = active && rank < c - mlo;
            const bool goR = active && rank > c - mlo;
            if (active && rank == c - mlo) {
                sf_emit<KW>(node, left, right, dim, ulo, mlo, mhi, c, id, in_off, p);
                active = false;
            }
            const uint32_t Lm = __ballot_sync(0xffffffffu, goL);
            const uint32_t Rm = __ballot_sync(0xffffffffu, goR);
            if (goL) {
                mhi = c - 1;
                subm &= Lm;
            } else if (goR) {
                mlo = c + 1;
                subm &= Rm;
            }
        }
        (void)lt;
    }
    if (bad) atomicOr(err, ERR_INTERNAL);
}

// ------------------------------------------------------------ launchers
template <typename KW>
static SelBufs<KW> sel_bufs(void* const* id, void* const* key, int k) {
    SelBufs<KW> B{};
    for (int b = 0; b < 2; ++b) {
        B.id[b] = static_cast<uint32_t*>(id[b]);
        for (int d = 0; d < k; ++d) B.key[b][d] = static_cast<KW*>(key[b * MAXK + d]);
    }
    return B;
}

size_t sel_seg_bytes(int key64) { return key64 ? sizeof(SelSeg<uint64_t>) : sizeof(SelSeg<uint32_t>); }

// Largest finisher unit (2048, 1024 or 512 tuples) whose shared memory fits.
int sel_finish_tile(int key64, int k) {
    for (int T = 2048; T >= 512; T /= 2) {
        const size_t b = key64 ? sel_finish_smem<uint64_t>(k, T) : sel_finish_smem<uint32_t>(k, T);
        if (b <= 160 * 1024) return T;
    }
    return 512;
}

template <typename KW>
static cudaError_t sel_level(const SelBufs<KW>& B, int cur, int k, int32_t m, int L, int tile, void* segs,
                             uint32_t* ghist, int32_t* gany, uint32_t* unresolved, int32_t* node, int64_t in_off,
                             int* err, cudaStream_t s, int round_begin, int round_end, int phase) {
    const int nseg = 1 << L;
    const int ntiles = (m + tile - 1) / tile;
    SelSeg<KW>* sg = static_cast<SelSeg<KW>*>(segs);
    if (phase == 0) {
        const int g = std::min(152 * 16, (int)(((int64_t)nseg * RADIX + 255) / 256));
        k_sel_init<KW><<<g, 256, 0, s>>>(m, L, nseg, sg, ghist);
        return cudaGetLastError();
    }
    if (phase == 3) {
        k_sel_span<KW><<<ntiles, SEL_THREADS, 0, s>>>(B, cur, k, m, L, tile, sg, err);
        k_sel_skip<KW><<<std::min(152 * 8, (nseg + 255) / 256), 256, 0, s>>>(nseg, sg,
                                                                            reinterpret_cast<int32_t*>(unresolved));
        return cudaGetLastError();
    }
    if (phase == 1) {
        for (int r = round_begin; r < round_end; ++r) {
            k_sel_hist<KW><<<ntiles, SEL_THREADS, 0, s>>>(B, cur, k, m, L, r, tile, sg, ghist, gany, err);
            k_sel_choose<KW><<<(nseg * 32 + 255) / 256, 256, 0, s>>>(nseg, r, k * (int)sizeof(KW), sg, ghist, gany,
                                                                     unresolved, err);
        }
        return cudaGetLastError();
    }
    k_sel_move<KW><<<ntiles, SEL_THREADS, 0, s>>>(B, cur, k, m, L, tile, sg, node, in_off, err);
    return cudaGetLastError();
}

// One level of the selection build over every segment of level L, in tiles
// of `tile` positions (a tile must touch at most LEVEL_NSMAX segments: with
// segments of at least T tuples, 2048 for T >= 1024 and 1024 for T = 512).
// phase 0: reset the segments' state; 3: the shared leading bytes of every
// segment (*unresolved, as an int32, receives the smallest first byte to
// select; it must hold the byte count before); 1: selection rounds
// [round_begin, round_end) (each adds the segments still unresolved to
// *unresolved); 2: partition around the medians.
cudaError_t launch_sel_level(int key64, void* const* id, void* const* key, int cur, int k, int32_t m, int L, int tile,
                             void* segs, uint32_t* ghist, int32_t* gany, uint32_t* unresolved, int32_t* node,
                             int64_t in_off, int* err, cudaStream_t s, int round_begin, int round_end, int phase) {
    if (m <= 0) return cudaSuccess;
    if (tile != SEL_TILE && tile != SEL_TILE / 2) return cudaErrorInvalidValue;
    if (key64)
        return sel_level<uint64_t>(sel_bufs<uint64_t>(id, key, k), cur, k, m, L, tile, segs, ghist, gany, unresolved,
                                   node, in_off, err, s, round_begin, round_end, phase);
    return sel_level<uint32_t>(sel_bufs<uint32_t>(id, key, k), cur, k, m, L, tile, segs, ghist, gany, unresolved,
                               node, in_off, err, s, round_begin, round_end, phase);
}

cudaError_t init_select_kernels() {
    cudaError_t e = cudaFuncSetAttribute((const void*)k_sel_finish<uint32_t>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)k_sel_finish<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
    return e;
}

// Finisher over the 2^lam units of level lam (each at most T tuples).
cudaError_t launch_sel_finish(int key64, void* const* id, void* const* key, int cur, int k, int32_t m, int lam, int T,
                              int32_t* node, int32_t* left, int32_t* right, uint8_t* dim, int64_t in_off, int* err,
                              cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const unsigned units = 1u << lam;
    if (key64) {
        const size_t smem = sel_finish_smem<uint64_t>(k, T);
        k_sel_finish<uint64_t><<<units, SEL_THREADS, smem, s>>>(sel_bufs<uint64_t>(id, key, k), cur, k, m, lam, T,
                                                                node, left, right, dim, in_off, err);
    } else {
        const size_t smem = sel_finish_smem<uint32_t>(k, T);
        k_sel_finish<uint32_t><<<units, SEL_THREADS, smem, s>>>(sel_bufs<uint32_t>(id, key, k), cur, k, m, lam, T,
                                                                node, left, right, dim, in_off, err);
    }
    return cudaGetLastError();
}

}  // namespace kd

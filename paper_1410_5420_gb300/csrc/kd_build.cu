// kd_build.cu -- tree-level kernels of the GB300 k-d tree builder.
//
// Section 2.1 builds the tree recursively: the median of the primary index
// array's segment becomes a node; the other k-1 arrays are partitioned in
// address order around the median's super key, each half keeping its
// sorted order, and the primary dimension cycles.  Here every tree level of
// every segment (and every cloud of a batch) is processed by one launch:
//
//   k_level_pass  moves one index array through up to k-1 tree levels at
//                 once.  Array q sorted within the segments of level L
//                 (where q is primary) is already split at level L for free
//                 (its halves are in place); the pass then applies the
//                 splits of levels L+1..L+k-1, whose medians come from the
//                 arrays that were primary there, as a stable 2^(k-1)-way
//                 segmented multisplit (warp match ranking, smem-staged
//                 coalesced scatter).  The counts of a segment's elements in
//                 earlier tiles come from a count pass (k_level_count, which
//                 reads only the decision planes) and a segmented scan over
//                 tiles (k_level_scan).  With this schedule each tree level
//                 costs one pass over one array.  Elements carry their rank
//                 in every super-key order, so each compare is one integer
//                 compare (super keys are unique after deduplication).
//   k_finish      once segments hold at most a few thousand tuples, one CTA
//                 finishes a whole subtree in shared memory.  Every tuple
//                 carries a segment label; while segments exceed 32 tuples,
//                 each level is one pass over the primary array ranking
//                 tuples within their labels (the median offset becomes the
//                 node, the others take their half's label).  A stable
//                 multisplit by label then orders every array within the
//                 remaining segments, and one warp finishes each segment of
//                 at most 32 tuples with per-dimension precedence masks,
//                 down to single elements (same result as the paper's
//                 1/2/3 element termination).
//   k_top_nodes   children and split dimension of the nodes above the
//                 finisher level (pure functions of m and the address).
#include <algorithm>

#include "kd_internal.cuh"

namespace kd {

constexpr uint32_t INV = 0xffffffffu;

// ------------------------------------------------------------ level step
// A level step is four launches:
//   k_level_tiles  one warp per tile: the tile's level-lev_in segments and
//                  the medians of the F decision levels below each of them,
//                  written as one tile record;
//   k_level_count  per tile, the bucket counts of its last segment;
//   k_level_scan   segmented scan of those counts over tiles;
//   k_level_pass   the move: route, stable warp ranking, scatter.
// The count and move passes are persistent: a producer warp takes tile ids
// from a counter and streams each tile's record and plane slices into a
// shared-memory stage with bulk async copies (full/empty mbarriers), while
// eight consumer warps work on the previous stage.
//
// Tile record (u32 words): [0] ns, [1..4] segment lo, [5..8] hi, [9..12]
// segment index, [13] pos0, [14] npos, [15] job; then at TR_HEAD +
// x * NBMAX + h the median rank of heap node h (1 = the segment itself,
// children 2h, 2h+1) of segment x.
constexpr int TR_HEAD = 16;
constexpr int LEVEL_STAGES = 2;
constexpr int PLANE_SLACK = 8;  // staged slice = tile rounded out to 16-byte boundaries
constexpr int LEVEL_BLOCK = LEVEL_THREADS + 32;  // eight consumer warps + one producer warp

// Elements per thread of a level-step tile: 8 (tiles of 2048 positions) or 4
// (1024), chosen per step by the host; k > 4 uses 4 (its planes fill the
// registers).  The default is the larger tile where it exists.
__host__ __device__ constexpr int level_ipt_of(int K) { return K <= 4 ? 8 : 4; }
__host__ __device__ constexpr int level_tile_of(int K) { return LEVEL_THREADS * level_ipt_of(K); }
__host__ __device__ constexpr bool level_ipt_ok(int K, int IPT) { return IPT == 4 || (IPT == 8 && K <= 4); }
__host__ __device__ constexpr int level_nbp(int K) { return (1 << (K - 1)) < 4 ? 4 : (1 << (K - 1)); }
__host__ __device__ constexpr int trec_words(int K) { return TR_HEAD + LEVEL_NSMAX * (1 << (K - 1)); }

struct StageMeta {
    int32_t t;  // tile, or -1: no more tiles
    int32_t cloud, lev_in, F, src_buf, dst_buf, write_med;
    int32_t shift;  // offset of the tile's first element in the staged slices
    int32_t pos0, npos, m, has_incl;
    int64_t goff;
};

template <int K, int IPT>
__global__ void __launch_bounds__(256) k_level_tiles(const LevelJob* __restrict__ jobs, int njobs, int ntiles,
                                                     const CloudDev* __restrict__ clouds,
                                                     const uint32_t* __restrict__ medr, uint32_t* __restrict__ trec,
                                                     uint32_t* __restrict__ ctrs, uint32_t* __restrict__ scan_flags,
                                                     int nflags, int* __restrict__ err) {
    constexpr int NBMAX = 1 << (K - 1);
    constexpr int TW = trec_words(K);
    constexpr int TILE = LEVEL_THREADS * IPT;
    pdl_wait();  // the previous step's counters and medians
    pdl_trigger();
    if (blockIdx.x == 0) {
        if (threadIdx.x < 3) ctrs[threadIdx.x] = 0;  // tile counters of the two passes, scan ticket
        for (int i = threadIdx.x; i < nflags; i += blockDim.x) scan_flags[i] = 0;
    }
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= ntiles) return;
    int lo = 0, hi = njobs;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (jobs[mid].tile_begin <= t) lo = mid; else hi = mid;
    }
    const LevelJob J = jobs[lo];
    const int32_t m = clouds[J.cloud].m;
    const int64_t medr_off = clouds[J.cloud].medr_off;
    const int32_t pos0 = (int32_t)((int64_t)(t - J.tile_begin) * TILE);
    const int32_t npos = (m - pos0) < TILE ? (m - pos0) : TILE;
    uint32_t* rec = trec + (int64_t)t * TW;
    int32_t slo[LEVEL_NSMAX], shi[LEVEL_NSMAX], sidx[LEVEL_NSMAX];
    int ns = 0;
    if (lane == 0) {
        ns = tile_segments(pos0, npos, m, J.lev_in, slo, shi, sidx, err);
        rec[0] = (uint32_t)ns;
        for (int x = 0; x < LEVEL_NSMAX; ++x) {
            rec[1 + x] = (uint32_t)(x < ns ? slo[x] : 0);
            rec[5 + x] = (uint32_t)(x < ns ? shi[x] : -1);
            rec[9 + x] = (uint32_t)(x < ns ? sidx[x] : 0);
        }
        rec[13] = (uint32_t)pos0;
        rec[14] = (uint32_t)npos;
        rec[15] = (uint32_t)lo;
    }
    ns = __shfl_sync(0xffffffffu, ns, 0);
    int32_t seg[LEVEL_NSMAX];
#pragma unroll
    for (int x = 0; x < LEVEL_NSMAX; ++x) seg[x] = __shfl_sync(0xffffffffu, lane == 0 && x < ns ? sidx[x] : 0, 0);
    const int F = J.lev_out - J.lev_in;
    const int per = (1 << F) - 1;
    for (int e = lane; e < ns * per; e += 32) {
        const int j = e / per;
        const int h = e - j * per + 1;
        const int f = 31 - __clz(h);
        int32_t sj = seg[0];
#pragma unroll
        for (int x = 1; x < LEVEL_NSMAX; ++x)
            if (j == x) sj = seg[x];
        const int64_t gseg = ((int64_t)sj << f) + (h - (1 << f));
        rec[TR_HEAD + j * NBMAX + h] = medr[medr_off + ((int64_t)1 << (J.lev_in + f)) - 1 + gseg];
    }
}

// Producer of the persistent level kernels (lane 0 of the last warp): for
// each tile it takes, waits until the stage is free, records the tile's
// facts in the stage's meta entry and starts the bulk copies of the tile
// record, `nplanes` plane slices and (move pass) the scanned counts of the
// previous tile.  Ends by publishing t = -1.
template <int K, int IPT, bool MOVE>
__device__ __forceinline__ void level_producer(const AllBufs& bufs, int q, const LevelJob* __restrict__ jobs,
                                               int njobs, int ntiles, const CloudDev* __restrict__ clouds,
                                               const uint32_t* __restrict__ trec, const uint32_t* __restrict__ incl,
                                               uint32_t* ctr, uint32_t* smem, StageMeta* meta, uint64_t* full,
                                               uint64_t* empty, int* err) {
    constexpr int TW = trec_words(K);
    constexpr int TILE = LEVEL_THREADS * IPT;
    constexpr int PST = TILE + PLANE_SLACK;
    constexpr int NP = MOVE ? K : K - 1;
    constexpr int NBP = level_nbp(K);
    constexpr int SW = TW + NBP + NP * PST;
    for (int it = 0;; ++it) {
        const int s = it % LEVEL_STAGES;
        const uint32_t ph = (uint32_t)(it / LEVEL_STAGES) & 1u;
        if (it >= LEVEL_STAGES && !mbar_wait(&empty[s], ph ^ 1u)) {
            atomicOr(err, ERR_TIMEOUT);
            meta[s].t = -1;
            mbar_arrive(&full[s]);
            return;
        }
        const int t = (int)atomicAdd(ctr, 1u);
        StageMeta M;
        M.t = t < ntiles ? t : -1;
        if (M.t < 0) {
            meta[s] = M;
            mbar_arrive(&full[s]);
            return;
        }
        const LevelTile T = job_tile(jobs, njobs, t, TILE, clouds);
        M.cloud = T.cloud;
        M.lev_in = T.lev_in;
        M.F = T.lev_out - T.lev_in;
        M.src_buf = T.src_buf;
        M.dst_buf = T.dst_buf;
        M.write_med = T.write_med;
        M.pos0 = (int32_t)T.pos0;
        M.npos = T.npos;
        M.m = clouds[T.cloud].m;
        M.goff = clouds[T.cloud].off;
        M.has_incl = MOVE && T.pos0 > 0;
        const int64_t g0 = M.goff + T.pos0;
        const int64_t a0 = g0 & ~(int64_t)3;
        const int64_t e1 = (g0 + T.npos + 3) & ~(int64_t)3;
        M.shift = (int32_t)(g0 - a0);
        const uint32_t pb = (uint32_t)((e1 - a0) * 4);
        // the move stages every plane but the array's own (its rank in
        // super key q, which only array 0 carries); the count the F
        // decision planes
        const int npl = MOVE ? K : M.F;
        const int skip = (MOVE && q != 0) ? (q - T.lev_in % K + K) % K : -1;
        meta[s] = M;
        uint32_t* st = smem + (size_t)s * SW;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&full[s], TW * 4 + (M.has_incl ? NBP * 4 : 0) + (uint32_t)(npl - (skip >= 0)) * pb);
        bulk_g2s(st, trec + (int64_t)t * TW, TW * 4, &full[s]);
        if (M.has_incl) bulk_g2s(st + TW, incl + (int64_t)(t - 1) * NBP, NBP * 4, &full[s]);
        for (int f = 0; f < npl; ++f)
            if (f != skip)
                bulk_g2s(st + TW + NBP + f * PST, bufs.p[q][T.src_buf][(T.lev_in + f) % K] + a0, pb, &full[s]);
    }
}

template <int K, int IPT>
constexpr size_t level_smem_bytes(bool move) {
    return (size_t)LEVEL_STAGES *
           (trec_words(K) + level_nbp(K) + (move ? K : K - 1) * (LEVEL_THREADS * IPT + PLANE_SLACK)) * 4;
}

// Segment bounds of a tile record, in registers.
__device__ __forceinline__ void tile_bounds(const uint32_t* rec, int32_t (&lo)[LEVEL_NSMAX],
                                            int32_t (&hi)[LEVEL_NSMAX]) {
#pragma unroll
    for (int x = 0; x < LEVEL_NSMAX; ++x) {
        lo[x] = (int32_t)rec[1 + x];
        hi[x] = (int32_t)rec[5 + x];
    }
}

// Single-segment tiles with every decision level: the medians of the
// segment's K-1 decision levels held in registers (heap order, mh[1..]),
// and an element's bucket found by K-1 compares.  Returns false for an
// element equal to a median.
template <int K>
__device__ __forceinline__ bool route_fast(const uint32_t (&mh)[1 << (K - 1)], const uint32_t* r, uint32_t& bucket) {
    uint32_t h = 1;
    bool eq = false;
#pragma unroll
    for (int f = 0; f < K - 1; ++f) {
        uint32_t mv = mh[1 << f];
#pragma unroll
        for (int c = (1 << f) + 1; c < (2 << f); ++c)
            if (h == (uint32_t)c) mv = mh[c];
        eq |= r[f] == mv;
        h = 2 * h + (r[f] > mv ? 1u : 0u);
    }
    bucket = h - (1u << (K - 1));
    return !eq;
}

// Bucket of an element of segment slot sj after F decision levels: r[f] is
// its rank in super key (lev_in + f) mod K, compared with the medians of
// the tile record; INV for an element equal to a median (the node itself).
template <int K>
__device__ __forceinline__ uint32_t route_rec(const uint32_t (&r)[K], int F, int sj, const uint32_t* rec) {
    constexpr int NBMAX = 1 << (K - 1);
    const uint32_t* med = rec + TR_HEAD + sj * NBMAX;
    uint32_t h = 1;
#pragma unroll
    for (int f = 0; f < K - 1; ++f) {
        if (f < F) {
            const uint32_t mv = med[h];
            if (r[f] == mv) return INV;
            h = 2 * h + (r[f] > mv ? 1u : 0u);
        }
    }
    return ((uint32_t)sj << F) + (h - (1u << F));
}

// Count pass: per tile, the bucket counts of its last segment (cnt[t][b],
// row stride level_nbp(K)) and whether that segment starts inside the tile
// (head[t]).  Reads the F decision planes only.
template <int K, int IPT>
__global__ void __launch_bounds__(LEVEL_BLOCK)
    k_level_count(const __grid_constant__ AllBufs bufs, int q, const LevelJob* __restrict__ jobs, int njobs,
                  int ntiles, const CloudDev* __restrict__ clouds, const uint32_t* __restrict__ trec,
                  uint32_t* __restrict__ cnt, uint32_t* __restrict__ head, uint32_t* __restrict__ ctr,
                  int* __restrict__ err) {
    constexpr int TILE = LEVEL_THREADS * IPT;
    constexpr int PST = TILE + PLANE_SLACK;
    constexpr int NBMAX = 1 << (K - 1);
    constexpr int NDMAX = LEVEL_NSMAX * NBMAX;
    constexpr int NBP = level_nbp(K);
    constexpr int TW = trec_words(K);
    constexpr int SW = TW + NBP + (K - 1) * PST;
    extern __shared__ __align__(128) uint32_t lsm[];
    __shared__ __align__(8) uint64_t full[LEVEL_STAGES], empty[LEVEL_STAGES];
    __shared__ StageMeta meta[LEVEL_STAGES];
    __shared__ uint32_t s_cnt[LEVEL_STAGES][NDMAX];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < LEVEL_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], LEVEL_WARPS);
        }
        fence_mbar_init();
    }
    for (int i = tid; i < LEVEL_STAGES * NDMAX; i += LEVEL_BLOCK) (&s_cnt[0][0])[i] = 0;
    __syncthreads();
    pdl_wait();  // the tile records and counters
    pdl_trigger();
    if (warp == LEVEL_WARPS) {
        if (lane == 0)
            level_producer<K, IPT, false>(bufs, q, jobs, njobs, ntiles, clouds, trec, nullptr, ctr, lsm, meta, full, empty,
                                     err);
        return;
    }
    const int wbase = warp * 32 * IPT;
    for (int it = 0;; ++it) {
        const int s = it % LEVEL_STAGES;
        const bool ok = mbar_wait(&full[s], (uint32_t)(it / LEVEL_STAGES) & 1u);
        if (consumer_or<LEVEL_THREADS>(!ok)) {
            if (tid == 0) atomicOr(err, ERR_TIMEOUT);
            break;
        }
        const StageMeta M = meta[s];
        if (M.t < 0) break;
        const uint32_t* st = lsm + (size_t)s * SW;
        const uint32_t* rec = st;
        const int ns = (int)rec[0];
        int32_t tlo[LEVEL_NSMAX], thi[LEVEL_NSMAX];
        tile_bounds(rec, tlo, thi);
        const int32_t lo0 = tlo[0];
        const int F = M.F;
        if (ns == 1 && F == K - 1) {  // one segment, every decision level
            uint32_t mh[K <= 4 ? NBMAX : 1];
            if constexpr (K <= 4) {
#pragma unroll
                for (int h = 0; h < NBMAX; ++h) mh[h] = rec[TR_HEAD + h];
            }
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const int o = wbase + j * 32 + lane;
                const int32_t pos = M.pos0 + o;
                if (o < M.npos && pos >= tlo[0] && pos <= thi[0]) {
                    uint32_t r[K];
#pragma unroll
                    for (int f = 0; f < K - 1; ++f) r[f] = st[TW + NBP + f * PST + M.shift + o];
                    uint32_t b;
                    bool keep;
                    if constexpr (K <= 4) {
                        keep = route_fast<K>(mh, r, b);
                    } else {
                        const uint32_t d = route_rec<K>(r, F, 0, rec);
                        keep = d != INV;
                        b = d;
                    }
                    if (keep) atomicAdd(&s_cnt[s][b], 1u);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const int o = wbase + j * 32 + lane;
                if (o < M.npos) {
                    const int32_t pos = M.pos0 + o;
                    const int sj = tile_slot(tlo, thi, ns, pos);
                    if (sj >= 0) {
                        uint32_t r[K];
#pragma unroll
                        for (int f = 0; f < K; ++f) r[f] = (f < F) ? st[TW + NBP + f * PST + M.shift + o] : 0u;
                        const uint32_t d = route_rec<K>(r, F, sj, rec);
                        if (d != INV) atomicAdd(&s_cnt[s][d], 1u);
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        consumer_sync<LEVEL_THREADS>();
        const int NB = 1 << F;
        if (tid < NBP) cnt[(int64_t)M.t * NBP + tid] = (ns > 0 && tid < NB) ? s_cnt[s][(ns - 1) * NB + tid] : 0u;
        if (tid == 0) head[M.t] = (ns == 1 && lo0 < M.pos0) ? 0u : 1u;
        // the next stage's counters were last read before this iteration's first barrier
        for (int i = tid; i < NDMAX; i += LEVEL_THREADS) s_cnt[(s + 1) % LEVEL_STAGES][i] = 0;
    }
}

// Segmented inclusive scan over the tiles of a level step:
// incl[t][b] = cnt[t][b] + (head[t] ? 0 : incl[t-1][b]) (row stride
// `stride`), one block per (chunk of LS_CHUNK tiles, bucket b), ids taken
// in launch order from a ticket.  Each thread loads LS_V consecutive tiles
// at once and scans them in registers; the threads' (flag, value) pairs are
// scanned across the block; a chunk then publishes what it carries out
// (inclusive at once when it holds a head) and takes what comes in by a
// decoupled look-back over the earlier chunks of its bucket.
constexpr int LS_V = 4;
constexpr int LS_CHUNK = 1024 * LS_V;
__host__ __device__ __forceinline__ int level_scan_chunks(int ntiles) { return (ntiles + LS_CHUNK - 1) / LS_CHUNK; }

__global__ void __launch_bounds__(1024) k_level_scan(int ntiles, int ncol, int stride, const uint32_t* __restrict__ cnt,
                                                     const uint32_t* __restrict__ head, uint32_t* __restrict__ incl,
                                                     uint32_t* __restrict__ lb, uint32_t* __restrict__ ticket,
                                                     int* __restrict__ err) {
    __shared__ uint32_t s_f[32], s_v[32];
    __shared__ uint32_t s_ctl, s_id, s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    pdl_wait();
    pdl_trigger();
    if (tid == 0) s_id = atomicAdd(ticket, 1u);
    __syncthreads();
    const int nch = level_scan_chunks(ntiles);
    const int id = (int)s_id;
    const int c = id / ncol, b = id - (id / ncol) * ncol;
    if (c >= nch) return;
    uint32_t* flags = lb + (size_t)b * nch;  // [ncol][nch] flags, aggregates, inclusive values
    uint32_t* agg = lb + (size_t)(ncol + b) * nch;
    uint32_t* inc = lb + (size_t)(2 * ncol + b) * nch;
    const int tb = c * LS_CHUNK + tid * LS_V;
    uint32_t lv[LS_V];
    uint32_t hf = 0;  // bit e: tile tb + e starts a segment (tiles past the end count as heads)
    if (tb + LS_V <= ntiles) {
        const uint4 h = *reinterpret_cast<const uint4*>(head + tb);  // tb is a multiple of LS_V
        hf = (h.x != 0u ? 1u : 0u) | (h.y != 0u ? 2u : 0u) | (h.z != 0u ? 4u : 0u) | (h.w != 0u ? 8u : 0u);
    } else {
#pragma unroll
        for (int e = 0; e < LS_V; ++e) {
            const int t = tb + e;
            hf |= ((t >= ntiles || head[t] != 0u) ? 1u : 0u) << e;
        }
    }
#pragma unroll
    for (int e = 0; e < LS_V; ++e) {
        const int t = tb + e;
        lv[e] = t < ntiles ? cnt[(int64_t)t * stride + b] : 0u;
    }
    // inclusive within the thread: a head starts a new segment
#pragma unroll
    for (int e = 1; e < LS_V; ++e)
        if (!((hf >> e) & 1u)) lv[e] += lv[e - 1];
    // (flag, value) pairs of the threads: inclusive scan within the warp
    uint32_t xf = hf != 0u ? 1u : 0u, xv = lv[LS_V - 1];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t yf = __shfl_up_sync(0xffffffffu, xf, o);
        const uint32_t yv = __shfl_up_sync(0xffffffffu, xv, o);
        if (lane >= o) {
            if (!xf) xv += yv;
            xf |= yf;
        }
    }
    uint32_t ef = __shfl_up_sync(0xffffffffu, xf, 1), ev = __shfl_up_sync(0xffffffffu, xv, 1);
    if (lane == 0) {
        ef = 0;
        ev = 0;
    }
    if (lane == 31) {
        s_f[warp] = xf;
        s_v[warp] = xv;
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t wf = s_f[lane], wv = s_v[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t yf = __shfl_up_sync(0xffffffffu, wf, o);
            const uint32_t yv = __shfl_up_sync(0xffffffffu, wv, o);
            if (lane >= o) {
                if (!wf) wv += yv;
                wf |= yf;
            }
        }
        s_f[lane] = wf;
        s_v[lane] = wv;
    }
    __syncthreads();
    // what the chunk carries out, ignoring what comes in: inclusive when the
    // chunk holds a head (or is the first)
    const bool blk_head = s_f[31] != 0u;
    if (tid == 0) {
        if (c == 0 || blk_head) {
            inc[c] = s_v[31];
            publish_flag(flags, c, FLAG_INC);
        } else {
            agg[c] = s_v[31];
            publish_flag(flags, c, FLAG_AGG);
        }
    }
    uint32_t carry = 0;
    if (c > 0) {
        const uint32_t ex = block_lookback<uint32_t>(flags, agg, inc, 1, c, &s_ctl, err, 1);
        if (tid == 0) {
            s_carry = ex;
            if (!blk_head) {
                inc[c] = ex + s_v[31];
                publish_flag(flags, c, FLAG_INC);
            }
        }
        __syncthreads();
        carry = s_carry;
    }
    // everything before this thread: earlier chunks, earlier warps, earlier lanes
    uint32_t pv = carry;
    if (warp > 0) pv = s_f[warp - 1] ? s_v[warp - 1] : carry + s_v[warp - 1];
    const uint32_t xv0 = ef ? ev : pv + ev;
#pragma unroll
    for (int e = 0; e < LS_V; ++e) {
        const int t = tb + e;
        // a head at or before e inside this thread cuts the carried prefix
        const bool cut = (hf << (31 - e)) != 0u;
        if (t < ntiles) incl[(int64_t)t * stride + b] = cut ? lv[e] : xv0 + lv[e];
    }
}

// Value of the rotated plane holding super key p: v[f] is plane (lev_in + f) mod K.
template <int K, int IPT>
__device__ __forceinline__ uint32_t plane_value(const uint32_t (&v)[K][IPT], int j, int f_sel) {
    uint32_t x = 0;
#pragma unroll
    for (int f = 0; f < K; ++f)
        if (f == f_sel) x = v[f][j];
    return x;
}

// Move pass: each element of array q goes to its bucket of the tile's
// segments after F decision levels, keeping its order (stable warp
// ranking), with all K planes.  The element landing on the middle of a
// final segment of level lev_out (its primary level) is that segment's
// median: its rank in super key q goes to medr and its tuple to the node.
template <int K, int IPT>
__global__ void __launch_bounds__(LEVEL_BLOCK, K <= 3 ? 3 : 2)
    k_level_pass(const __grid_constant__ AllBufs bufs, int q, const LevelJob* __restrict__ jobs, int njobs,
                 int ntiles, const CloudDev* __restrict__ clouds, uint32_t* __restrict__ medr,
                 const uint32_t* __restrict__ perm0, const uint32_t* __restrict__ trec,
                 const uint32_t* __restrict__ incl, uint32_t* __restrict__ ctr, int* __restrict__ err) {
    constexpr int TILE = LEVEL_THREADS * IPT;
    constexpr int PST = TILE + PLANE_SLACK;
    constexpr int NBMAX = 1 << (K - 1);
    constexpr int NDMAX = LEVEL_NSMAX * NBMAX;
    constexpr int NBP = level_nbp(K);
    constexpr int TW = trec_words(K);
    constexpr int SW = TW + NBP + K * PST;
    extern __shared__ __align__(128) uint32_t lsm[];
    __shared__ __align__(8) uint64_t full[LEVEL_STAGES], empty[LEVEL_STAGES];
    __shared__ StageMeta meta[LEVEL_STAGES];
    __shared__ uint32_t s_wc[LEVEL_WARPS][NDMAX];
    __shared__ int2 s_dlh[NDMAX];   // final segment [lo, hi] of each digit
    __shared__ int32_t s_dmid[NDMAX];
    __shared__ int32_t s_segidx[LEVEL_NSMAX];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < LEVEL_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], LEVEL_WARPS);
        }
        fence_mbar_init();
    }
    for (int i = tid; i < LEVEL_WARPS * NDMAX; i += LEVEL_BLOCK) (&s_wc[0][0])[i] = 0;
    __syncthreads();
    pdl_wait();  // the scanned counts
    pdl_trigger();
    if (warp == LEVEL_WARPS) {
        if (lane == 0)
            level_producer<K, IPT, true>(bufs, q, jobs, njobs, ntiles, clouds, trec, incl, ctr, lsm, meta, full, empty, err);
        return;
    }
    const int wbase = warp * 32 * IPT;
    for (int it = 0;; ++it) {
        const int s = it % LEVEL_STAGES;
        const bool ok = mbar_wait(&full[s], (uint32_t)(it / LEVEL_STAGES) & 1u);
        if (consumer_or<LEVEL_THREADS>(!ok)) {
            if (tid == 0) atomicOr(err, ERR_TIMEOUT);
            break;
        }
        const StageMeta M = meta[s];
        if (M.t < 0) break;
        const uint32_t* st = lsm + (size_t)s * SW;
        const uint32_t* rec = st;
        const int ns = (int)rec[0];
        int32_t tlo[LEVEL_NSMAX], thi[LEVEL_NSMAX];
        tile_bounds(rec, tlo, thi);
        const int F = M.F;
        const int NB = 1 << F;
        const uint32_t marker = (uint32_t)(ns * NB);
        const int own = q != 0 ? (q - M.lev_in % K + K) % K : -1;  // slot of the array's own plane: not carried
        uint32_t v[K][IPT];
        uint32_t dig[IPT];
        uint32_t rank[IPT];
        if (ns == 1 && F == K - 1) {
            // one segment and every decision level: compile-time routing and
            // (buckets 0 .. NB-1, marker NB)
            uint32_t mh[K <= 4 ? NBMAX : 1];
            if constexpr (K <= 4) {
#pragma unroll
                for (int h = 0; h < NBMAX; ++h) mh[h] = rec[TR_HEAD + h];
            }
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const int o = wbase + j * 32 + lane;
                const int32_t pos = M.pos0 + o;
                dig[j] = marker;
#pragma unroll
                for (int f = 0; f < K; ++f) v[f][j] = 0;
                if (o < M.npos) {
#pragma unroll
                    for (int f = 0; f < K; ++f) v[f][j] = st[TW + NBP + f * PST + M.shift + o];  // slot `own` is unused
                    if (pos >= tlo[0] && pos <= thi[0]) {
                        uint32_t r[K];
#pragma unroll
                        for (int f = 0; f < K; ++f) r[f] = v[f][j];
                        if constexpr (K <= 4) {
                            uint32_t b;
                            if (route_fast<K>(mh, r, b)) dig[j] = b;
                        } else {
                            const uint32_t d = route_rec<K>(r, F, 0, rec);
                            if (d != INV) dig[j] = d;
                        }
                    }
                }
            }
            warp_rank<IPT>(dig, marker, s_wc[warp], rank);
        } else {
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const int o = wbase + j * 32 + lane;
                dig[j] = marker;
#pragma unroll
                for (int f = 0; f < K; ++f) v[f][j] = 0;
                if (o < M.npos) {
#pragma unroll
                    for (int f = 0; f < K; ++f) v[f][j] = st[TW + NBP + f * PST + M.shift + o];  // slot `own` is unused
                    const int sj = tile_slot(tlo, thi, ns, M.pos0 + o);
                    if (sj >= 0) {
                        uint32_t r[K];
#pragma unroll
                        for (int f = 0; f < K; ++f) r[f] = v[f][j];
                        const uint32_t d = route_rec<K>(r, F, sj, rec);
                        if (d != INV) dig[j] = d;
                    }
                }
            }
            warp_rank<IPT>(dig, marker, s_wc[warp], rank);
        }
        consumer_sync<LEVEL_THREADS>();
        // per digit: prefix over warps; base, bounds and middle of its final
        // segment; the first segment continues the scanned counts of earlier tiles
        const bool first_cont = ns > 0 && tlo[0] < M.pos0;
        for (int d = tid; d < ns * NB; d += LEVEL_THREADS) {
            const int sj = d >> F;
            const int b = d - (sj << F);
            int32_t a = (int32_t)rec[1 + sj], z = (int32_t)rec[5 + sj];
            for (int f = F - 1; f >= 0; --f) {
                const int32_t mid = a + ((z - a) >> 1);
                if ((b >> f) & 1) a = mid + 1; else z = mid - 1;
            }
            // each warp's row: the destination of its first element of digit d
            uint32_t c = (uint32_t)(a + ((sj == 0 && first_cont && M.has_incl) ? (int32_t)st[TW + b] : 0));
#pragma unroll
            for (int w = 0; w < LEVEL_WARPS; ++w) {
                const uint32_t x = s_wc[w][d];
                s_wc[w][d] = c;
                c += x;
            }
            s_dlh[d] = make_int2(a, z);
            s_dmid[d] = (M.write_med & LEVEL_MED) ? a + ((z - a) >> 1) : -1;
        }
        if (tid < LEVEL_NSMAX) s_segidx[tid] = (int32_t)rec[9 + tid];
        consumer_sync<LEVEL_THREADS>();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage
        const CloudDev& C = clouds[M.cloud];
        int32_t dest[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            dest[j] = -1;
            const uint32_t d = dig[j];
            if (d < marker) {
                const int32_t dd = (int32_t)(s_wc[warp][d] + rank[j]);
                // the destination must lie in the element's final segment; any
                // other value means inconsistent inputs and is never written
                const int2 lh = s_dlh[d];
                if (dd >= lh.x && dd <= lh.y) {
                    dest[j] = dd;
                    if ((M.write_med & LEVEL_MED) && dd == s_dmid[d]) {
                        const int sj = (int)(d >> F);
                        const int32_t si = (s_segidx[sj] << F) + (int32_t)(d - ((uint32_t)sj << F));
                        // rank 0 of the median (its position in array 0) gives
                        // its tuple and, through array 0's initial record,
                        // its rank in super key q
                        const int f0 = (K - M.lev_in % K) % K;
                        const uint32_t r0 = plane_value<K, IPT>(v, j, f0);
                        const int64_t lev_out = M.lev_in + F;
                        if (r0 >= M.goff && r0 < M.goff + M.m) {
                            const uint32_t rq = q == 0 ? r0 : bufs.p[0][0][q][r0];
                            medr[C.medr_off + ((int64_t)1 << lev_out) - 1 + si] = rq;
                            C.node[dd] = (int32_t)((int64_t)perm0[r0] - C.in_off);
                        } else {
                            atomicOr(err, ERR_INTERNAL);
                        }
                    }
                } else {
                    atomicOr(err, ERR_INTERNAL);
                }
            }
        }
        // each run of equal digits goes to consecutive addresses: stores from
        // registers, coalesced per run
        const bool final_move = (M.write_med & LEVEL_FINAL) != 0;  // only rank 0 is read after it
#pragma unroll
        for (int f = 0; f < K; ++f) {
            if (f == own || (final_move && (M.lev_in + f) % K != 0)) continue;
            uint32_t* dp = bufs.p[q][M.dst_buf][(M.lev_in + f) % K] + M.goff;
#pragma unroll
            for (int j = 0; j < IPT; ++j)
                if (dest[j] >= 0) dp[dest[j]] = v[f][j];
        }
        // this warp's counters start the next tile at zero (only this warp
        // reads its row after the digit loop above)
        __syncwarp();
        for (int d = lane; d < NDMAX; d += 32) s_wc[warp][d] = 0;
        __syncwarp();
    }
}

// ------------------------------------------------------------- finisher

__device__ __forceinline__ uint32_t seg_pack(int32_t a, int32_t b) { return (uint32_t)a | ((uint32_t)b << 16); }

constexpr int FIN_WARPS = FIN_THREADS / 32;
constexpr uint8_t LAB_DONE = 0xff;  // the tuple is a node already

// Labels of the last block level: segments at relative level l number 2^l.
__host__ __device__ constexpr int fin_labels(int smax) { return smax / 32; }

// Unit-relative address range [a, b] of segment X at relative level l.
__device__ __forceinline__ void label_range(int S, int l, int X, int32_t& a, int32_t& b) {
    a = 0;
    b = S - 1;
    for (int f = l - 1; f >= 0; --f) {
        const int32_t c = a + ((b - a) >> 1);
        if ((X >> f) & 1) a = c + 1; else b = c - 1;
    }
}

// One pass over array A (lids in key order): each live tuple's rank among
// the tuples of its segment label, in A's order (stable warp ranking, then
// the counts of earlier warps).  On return s_wc[w][X] holds the count of
// label X in warps before w, s_lab[X] = (a, b) of segment X, and a label
// whose count differs from its segment's size is reported.
template <int SMAX>
__device__ __forceinline__ void fin_label_rank(const uint16_t* __restrict__ A, int S, int l,
                                               const uint8_t* __restrict__ lab, uint32_t (*s_wc)[fin_labels(SMAX)],
                                               int2* s_lab,
                                               uint32_t (&lid)[SMAX / FIN_THREADS],
                                               uint32_t (&dig)[SMAX / FIN_THREADS],
                                               uint32_t (&rank)[SMAX / FIN_THREADS], int* bad) {
    constexpr int IPT = SMAX / FIN_THREADS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t marker = 1u << l;
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int i = warp * 32 * IPT + j * 32 + lane;
        lid[j] = i < S ? A[i] : 0u;
        const uint32_t x = i < S ? lab[lid[j]] : LAB_DONE;
        dig[j] = x == LAB_DONE ? marker : x;
    }
    warp_rank<IPT>(dig, marker, s_wc[warp], rank);
    __syncthreads();
    for (int X = tid; X < (int)marker; X += FIN_THREADS) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < FIN_WARPS; ++w) {
            const uint32_t x = s_wc[w][X];
            s_wc[w][X] = c;
            c += x;
        }
        int32_t a, b;
        label_range(S, l, X, a, b);
        s_lab[X] = make_int2(a, b);
        if ((int32_t)c != (b >= a ? b - a + 1 : 0)) *bad = 1;
    }
    __syncthreads();
}

// The warp's own counter row back to zero for the next pass.
template <int SMAX>
__device__ __forceinline__ void fin_clear_row(uint32_t (*s_wc)[fin_labels(SMAX)]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncwarp();
    for (int X = lane; X < fin_labels(SMAX); X += 32) s_wc[warp][X] = 0;
    __syncwarp();
}

// The node at unit position c (median of unit-relative [a, b]) is tuple
// lid: its children and dimension are written now; its tuple index is
// resolved for all nodes of the unit at the end (nodelid[c] = lid), so that
// the random perm0 reads are issued together rather than on every level's
// critical path.
__device__ __forceinline__ void fin_emit(const CloudDev& C, uint16_t* nodelid, int32_t lo, int32_t a, int32_t b,
                                         int32_t c, uint16_t lid, int p) {
    const int32_t addr = lo + c;
    nodelid[c] = lid;
    if (C.left) C.left[addr] = a <= c - 1 ? lo + child_mid(a, c - 1) : -1;
    if (C.right) C.right[addr] = c + 1 <= b ? lo + child_mid(c + 1, b) : -1;
    if (C.dim) C.dim[addr] = (uint8_t)p;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Phase tracing (optional): thread 0 adds the time since the previous
// barrier-aligned stamp to phase_ns[ph]; block-time sums over all units.
#define FIN_STAMP(ph)                                                              \
    do {                                                                           \
        if (phase_ns && tid == 0) {                                                \
            const unsigned long long now_ = global_ns();                           \
            atomicAdd(&phase_ns[ph], now_ - t_prev);                               \
            t_prev = now_;                                                         \
        }                                                                          \
    } while (0)

// Slot of entry i of the unit's rank table: within each run of 32 entries
// the low five index bits are XORed with the entry's block of SMAX / 32,
// so that the lanes of a warp searching different blocks at the same
// offset read different banks.
template <int SMAX>
__device__ __forceinline__ int rk_slot(int i) {
    constexpr int SH = SMAX == 1024 ? 5 : (SMAX == 2048 ? 6 : 7);
    static_assert((SMAX >> SH) == 32, "32 blocks per unit");
    return i ^ ((i >> SH) & 31);
}

// A finisher unit's input: rk[i] = rank 0 of array 0's element i (array 0
// is sorted by rank 0), and for arrays d >= 1 the lid of each element (its
// position in array 0).  All K loads per position are in flight before the
// first is used.  (Array 0's other rank planes are not needed here: the
// unit's levels compare positions in the arrays.)
template <int K, int SMAX>
__device__ __forceinline__ void fin_load_unit(const AllBufs& bufs, const CloudDev& C, int64_t g, int S,
                                              uint32_t* rk, uint16_t* arr, int* bad) {
    constexpr int PPT = SMAX / FIN_THREADS;
    const int tid = threadIdx.x;
    uint32_t v[K][PPT];
#pragma unroll
    for (int p = 0; p < K; ++p) {
        const uint32_t* src = bufs.p[p][C.buf[p]][0];  // rank 0 of array p
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const int i = tid + j * FIN_THREADS;
            v[p][j] = i < S ? src[g + i] : 0u;
        }
    }
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        const int i = tid + j * FIN_THREADS;
        if (i < S) rk[rk_slot<SMAX>(i)] = v[0][j];
    }
    __syncthreads();
    // The K-1 arrays' searches advance together: (K-1) x PPT independent
    // chains.  The first five halvings pick one of 32 blocks of SMAX / 32
    // positions by the last rank 0 of each block, held one per lane and
    // read by shuffles (no shared-memory bank conflicts); the rest search
    // the block in shared memory.
    constexpr int BK = SMAX / 32;
    const int lane = tid & 31;
    const bool svalid = lane * BK + BK - 1 < S;  // block `lane` is full
    const uint32_t sample = svalid ? rk[rk_slot<SMAX>(lane * BK + BK - 1)] : 0u;
    int pos[K - 1][PPT];
#pragma unroll
    for (int d = 0; d < K - 1; ++d)
#pragma unroll
        for (int j = 0; j < PPT; ++j) pos[d][j] = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
#pragma unroll
        for (int d = 0; d < K - 1; ++d)
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                const int c = pos[d][j] + step - 1;  // block index
                const uint32_t sc = __shfl_sync(0xffffffffu, sample, c);
                if (c * BK + BK - 1 < S && sc < v[d + 1][j]) pos[d][j] += step;
            }
    }
#pragma unroll
    for (int d = 0; d < K - 1; ++d)
#pragma unroll
        for (int j = 0; j < PPT; ++j) pos[d][j] *= BK;
#pragma unroll
    for (int step = BK / 2; step >= 1; step >>= 1) {
#pragma unroll
        for (int d = 0; d < K - 1; ++d)
#pragma unroll
            for (int j = 0; j < PPT; ++j)
                if (pos[d][j] + step <= S && rk[rk_slot<SMAX>(pos[d][j] + step - 1)] < v[d + 1][j])
                    pos[d][j] += step;
    }
#pragma unroll
    for (int d = 1; d < K; ++d)
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const int i = tid + j * FIN_THREADS;
            if (i < S) {
                if (pos[d - 1][j] >= S || rk[rk_slot<SMAX>(pos[d - 1][j])] != v[d][j]) *bad = 1;
                arr[d * SMAX + i] = (uint16_t)min(pos[d - 1][j], S - 1);
            }
        }
}

// Largest k each on-chip subtree size serves (the host clamps accordingly),
// so that one kernel's registers are not sized for every k.
__host__ __device__ constexpr int fin_kmax(int smax) { return smax >= 4096 ? 3 : (smax >= 2048 ? 4 : 8); }

// Blocks per SM the finisher is compiled for: at 1024 tuples and k <= 4
// six blocks fit the shared memory, and trading registers for them (a few
// spills) hides more of the shared-memory latency (3.20 ms per 2^26 step at
// k = 3, against 3.33 at five blocks and 3.58 at seven); wider tuples fit
// fewer.  At 2048 tuples five blocks (3.77 ms) beat four (3.88).
__host__ __device__ constexpr int fin_min_blocks(int smax, int k) {
    return smax >= 4096 ? 2 : (smax >= 2048 ? 5 : (k <= 4 ? 6 : (k <= 6 ? 5 : 4)));
}

// K: the number of dimensions, so that the unit's per-dimension arrays and
// loops are sized exactly.
template <int SMAX, int K>
__global__ void __launch_bounds__(FIN_THREADS, fin_min_blocks(SMAX, K))
    k_finish(const __grid_constant__ AllBufs bufs, const int64_t* __restrict__ unit_prefix, int ncloud,
             int64_t unit_base, const CloudDev* __restrict__ clouds, const uint32_t* __restrict__ perm0,
             int* __restrict__ err, unsigned long long* __restrict__ phase_ns) {
    constexpr int GMAX = SMAX / FIN_THREADS;
    constexpr int smax = SMAX;
    constexpr int k = K;
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ uint32_t s_wc[FIN_WARPS][fin_labels(SMAX)];
    __shared__ int2 s_lab[fin_labels(SMAX)];
    __shared__ int s_cur[MAXK + 1];
    __shared__ int s_nseg;
    uint32_t* rk = sm;                                          // rk[rk_slot(lid)]: rank 0
    uint32_t* seg = rk + smax;                                  // packed segment per position
    uint16_t* arr = reinterpret_cast<uint16_t*>(seg + smax);   // (k+1) storages of lids
    uint16_t* nodelid = arr + (size_t)(k + 1) * smax;           // tuple chosen at each position
    uint8_t* lab = reinterpret_cast<uint8_t*>(nodelid + smax);   // per lid: segment label at the current level
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    FinUnit U;
    const int64_t unit = unit_base + blockIdx.x;
    U.cloud = last_le(unit_prefix, ncloud + 1, unit);
    U.seg = (int32_t)(unit - unit_prefix[U.cloud]);
    const CloudDev& C = clouds[U.cloud];
    int32_t lo, hi;
    segment_bounds(C.m, C.lam, U.seg, lo, hi);
    const int S = hi - lo + 1;
    if (S <= 0) return;
    if (S > smax) {
        if (tid == 0) atomicOr(err, ERR_INTERNAL);
        return;
    }
    const int64_t g = C.off + lo;
    unsigned long long t_prev = phase_ns && tid == 0 ? global_ns() : 0ull;
    if (tid <= k) s_cur[tid] = tid;
    if (tid == 0) s_nseg = 0;
    int bad = 0;
    // Load the unit at once: array 0's k rank planes (the rank table, rows
    // sorted by rank 0) and the rank-0 plane of arrays 1..k-1; every load is
    // issued before any is used.  Then each element of array d finds its lid
    // (its position in array 0) by a branch-free binary search of its rank 0.
    fin_load_unit<K, SMAX>(bufs, C, g, S, rk, arr, &bad);
    for (int i = tid; i < S; i += FIN_THREADS) {
        arr[i] = (uint16_t)i;  // array 0 is the rank table's own order
        lab[i] = 0;
        nodelid[i] = 0xffffu;  // every address gets its node below; checked at the end
    }
    for (int i = tid; i < FIN_WARPS * fin_labels(SMAX); i += FIN_THREADS) (&s_wc[0][0])[i] = 0;
    __syncthreads();
    FIN_STAMP(0);  // rank table and lids of the unit
    // Block levels, while a segment may hold more than 32 tuples.  The k
    // arrays keep their unit-level order (array d sorted by super key d) and
    // every tuple carries its segment label at the current level (lab[lid],
    // LAB_DONE once it is a node).  At level l a pass over the primary array
    // p ranks each tuple among its label's tuples in key-p order: the one at
    // the segment's median offset becomes the node, the others take the
    // label of their half.
    int dl = 0;
    int ordered = -1;  // the array the last block level leaves in final segment order
    for (; (S >> dl) > 32; ++dl) {
        const int p = (C.lam + dl) % k;
        const bool last_block_level = (S >> (dl + 1)) <= 32;
        if (last_block_level) ordered = p;
        if (dl == 0) {
            // the unit is one segment: a tuple's rank is its position in array p
            const uint16_t* A = arr + p * smax;
            const int32_t off = (S - 1) >> 1;
            for (int i = tid; i < S; i += FIN_THREADS) {
                const uint16_t lid = A[i];
                if (i == off) {
                    fin_emit(C, nodelid, lo, 0, S - 1, off, lid, p);
                    lab[lid] = LAB_DONE;
                } else {
                    lab[lid] = (uint8_t)(i > off ? 1 : 0);
                }
            }
            __syncthreads();
            continue;
        }
        uint32_t lid[GMAX], dig[GMAX], rank[GMAX];
        fin_label_rank<SMAX>(arr + p * smax, S, dl, lab, s_wc, s_lab, lid, dig, rank, &bad);
        const uint32_t marker = 1u << dl;
#pragma unroll
        for (int j = 0; j < GMAX; ++j) {
            if (dig[j] < marker) {
                const int X = (int)dig[j];
                const int2 ab = s_lab[X];
                const int32_t off = (ab.y - ab.x) >> 1;
                const int32_t r = (int32_t)(s_wc[warp][X] + rank[j]);
                if (r == off) {
                    fin_emit(C, nodelid, lo, ab.x, ab.y, ab.x + off, (uint16_t)lid[j], p);
                    lab[lid[j]] = LAB_DONE;
                } else {
                    lab[lid[j]] = (uint8_t)(2 * X + (r > off ? 1 : 0));
                    // the halves of segment X are [a, c-1] and [c+1, b]:
                    // rank r in key-p order puts the tuple at a + r in both
                    // (every read of the array preceded the ranking's barrier)
                    if (last_block_level) arr[p * smax + ab.x + r] = (uint16_t)lid[j];
                }
            }
        }
        fin_clear_row<SMAX>(s_wc);
        __syncthreads();
    }
    FIN_STAMP(1);  // block levels
    // every array in key order within each remaining segment: a stable
    // multisplit by label, in place (all reads precede the first barrier);
    // the last block level's primary array is in that order already (at
    // dl = 0 each half keeps its place, deeper levels wrote it above)
    for (int q = 0; q < k; ++q) {
        if (q == ordered) continue;
        uint16_t* A = arr + q * smax;
        uint32_t lid[GMAX], dig[GMAX], rank[GMAX];
        fin_label_rank<SMAX>(A, S, dl, lab, s_wc, s_lab, lid, dig, rank, &bad);
        const uint32_t marker = 1u << dl;
#pragma unroll
        for (int j = 0; j < GMAX; ++j) {
            if (dig[j] < marker) {
                const int2 ab = s_lab[dig[j]];
                const int32_t o = ab.x + (int32_t)(s_wc[warp][dig[j]] + rank[j]);
                if (o <= ab.y) A[o] = (uint16_t)lid[j]; else bad = 1;
            }
        }
        fin_clear_row<SMAX>(s_wc);
        __syncthreads();
    }
    if (tid <= k) s_cur[tid] = tid;
    __syncthreads();
    FIN_STAMP(4);  // final splits by segment
    // warp levels: every remaining segment has at most 32 tuples; one warp
    // finishes a segment with one tuple per lane, in the order of the
    // current primary array.  For every dimension q the lane holds LESS_q,
    // the set of lanes whose tuples precede its own in super key q (from
    // the segment's sorted array q); a lane's rank in its sub-segment SUB is
    // then popc(LESS_p & SUB): equal to the median offset -> node, below ->
    // left child, above -> right child.
    uint32_t* list = reinterpret_cast<uint32_t*>(arr + s_cur[k] * smax);  // spare storage, first smax bytes
    for (int X = tid; X < (1 << dl); X += FIN_THREADS) {
        int32_t a, b;
        label_range(S, dl, X, a, b);
        if (b >= a) {
            const int e = atomicAdd(&s_nseg, 1);
            if (e < smax / 4) list[e] = seg_pack(a, b); else bad = 1;  // below lane_of (byte smax)
        }
    }
    __syncthreads();
    const int nseg = min(s_nseg, smax / 4);
    const int p0 = (C.lam + dl) % k;
    const uint16_t* prim0 = arr + s_cur[p0] * smax;
    // lane_of[lid]: lane holding tuple lid in its warp (each tuple is in
    // exactly one segment); it lives in the free upper half of the spare
    // storage, above the segment list (at most S/16 words).  Per-segment
    // scratch words come from `seg`, whose entries are no longer read.
    uint8_t* lane_of = reinterpret_cast<uint8_t*>(arr + s_cur[k] * smax) + smax;
    const uint32_t lt = lanemask_lt();
    for (int e = warp; e < nseg; e += FIN_THREADS / 32) {
        const uint32_t sg = list[e];
        const int32_t a0 = sg & 0xffff, b0 = sg >> 16;
        const int n = b0 - a0 + 1;
        const bool in = lane < n;
        const uint16_t lid = in ? prim0[a0 + lane] : 0;
        uint32_t* scr = seg + a0;  // n words, owned by this warp for this segment
        if (in) lane_of[lid] = (uint8_t)lane;
        __syncwarp();
        uint32_t less[K];
#pragma unroll
        for (int q = 0; q < K; ++q) {
            less[q] = 0;
            if (q < k) {
                if (q == p0) {
                    less[q] = lt;
                } else {
                    // lane i reads the tuple at sorted position i of array q
                    // and the lane x that holds it
                    const uint16_t* aq = arr + s_cur[q] * smax;
                    const uint32_t x = in ? lane_of[aq[a0 + lane]] : 0u;
                    // prefix-OR over sorted order gives, at position i, the lanes of
                    // positions < i; push it to lane x
                    uint32_t bit = in ? (1u << x) : 0u;
                    uint32_t incl = bit;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl |= y;
                    }
                    __syncwarp();
                    if (in) scr[x] = incl & ~bit;
                    __syncwarp();
                    less[q] = in ? scr[lane] : 0u;
                }
            }
        }
        __syncwarp();
        uint32_t sub = __ballot_sync(0xffffffffu, in);
        bool active = in;
        int32_t mlo = a0, mhi = b0;
        int p = p0;  // the dimension of level l
        for (int l = dl; __any_sync(0xffffffffu, active); ++l, p = p + 1 == K ? 0 : p + 1) {
            uint32_t lp = 0;
#pragma unroll
            for (int q = 0; q < K; ++q)
                if (q == p) lp = less[q];
            const int rank = __popc(lp & sub);
            const int32_t c = mlo + ((mhi - mlo) >> 1);
            const bool goL = active && rank < c - mlo;
            const bool goR = active && rank > c - mlo;
            if (active && rank == c - mlo) {
                fin_emit(C, nodelid, lo, mlo, mhi, c, lid, p);
                active = false;
            }
            const uint32_t Lm = __ballot_sync(0xffffffffu, goL);
            const uint32_t Rm = __ballot_sync(0xffffffffu, goR);
            if (goL) {
                mhi = c - 1;
                sub &= Lm;
            } else if (goR) {
                mlo = c + 1;
                sub &= Rm;
            }
        }
    }
    // tuple of every node of the unit: rank 0 -> input index, all reads in flight together
    __syncthreads();
    FIN_STAMP(2);  // warp levels
#pragma unroll 4
    for (int i = tid; i < S; i += FIN_THREADS) {
        const uint32_t nl = nodelid[i];
        if (nl >= (uint32_t)S) {
            bad = 1;
            continue;
        }
        const uint32_t r0 = rk[rk_slot<SMAX>((int)nl)];
        if (r0 >= C.off && r0 < C.off + C.m)
            C.node[lo + i] = (int32_t)((int64_t)perm0[r0] - C.in_off);
        else
            bad = 1;
    }
    if (bad) atomicOr(err, ERR_INTERNAL);
    __syncthreads();
    FIN_STAMP(3);  // node tuples
}

// ------------------------------------------------------------ top nodes
// Entries j of cloud c (j < 2^lam - 1, breadth-first: level L = floor(log2
// (j+1)), index s = j + 1 - 2^L) are the nodes above the finisher level.
// all_nodes (k = 1): also the tuple of every node, the a-th sorted tuple.
__global__ void k_top_nodes(const CloudDev* __restrict__ clouds, const int64_t* __restrict__ prefix,
                            int ncloud, int k, const uint32_t* __restrict__ perm0, uint32_t* __restrict__ medr,
                            int all_nodes) {
    const int64_t total = prefix[ncloud];
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int lo_c = 0, hi_c = ncloud;
        while (hi_c - lo_c > 1) {
            const int mid = (lo_c + hi_c) >> 1;
            if (prefix[mid] <= idx) lo_c = mid; else hi_c = mid;
        }
        const CloudDev C = clouds[lo_c];
        const int64_t j = idx - prefix[lo_c];
        const int L = 63 - __clzll(j + 1);
        const int32_t s = (int32_t)(j + 1 - ((int64_t)1 << L));
        int32_t lo, hi;
        segment_bounds(C.m, L, s, lo, hi);
        if (hi < lo) continue;
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (C.left) C.left[mid] = child_mid(lo, mid - 1);
        if (C.right) C.right[mid] = child_mid(mid + 1, hi);
        if (C.dim) C.dim[mid] = (uint8_t)(L % k);
        if (L == 0 || all_nodes) C.node[mid] = (int32_t)((int64_t)perm0[C.off + mid] - C.in_off);
        if (L == 0 && medr && !all_nodes) medr[C.medr_off] = (uint32_t)(C.off + mid);
    }
}

// --------------------------------------------------------------- shape
// Children and split dimension of every address of one tree over m
// addresses: pure functions of m (the walk from the root to the segment
// whose median is the address).  Used when the tree goes to host memory, so
// that these outputs are copied back while the level passes run.
__global__ void k_shape(int32_t m, int k, int32_t* __restrict__ left, int32_t* __restrict__ right,
                        uint8_t* __restrict__ dim) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = (int32_t)i;
        int32_t lo = 0, hi = m - 1;
        int depth = 0;
        for (; depth < 32; ++depth) {  // at most ceil(log2(m + 1)) steps
            const int32_t mid = lo + ((hi - lo) >> 1);
            if (a == mid) break;
            if (a < mid) hi = mid - 1; else lo = mid + 1;
        }
        if (left) left[a] = child_mid(lo, a - 1);
        if (right) right[a] = child_mid(a + 1, hi);
        if (dim) dim[a] = (uint8_t)(depth % k);
    }
}

cudaError_t launch_shape(int32_t m, int k, int32_t* left, int32_t* right, uint8_t* dim, cudaStream_t s) {
    if (m <= 0 || (!left && !right && !dim)) return cudaSuccess;
    int64_t g = ((int64_t)m + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    k_shape<<<(unsigned)g, 256, 0, s>>>(m, k, left, right, dim);
    return cudaGetLastError();
}

// ------------------------------------------------------------ launchers
int level_tile(int k) { return level_tile_of(k); }
bool level_tile_supported(int k, int tile) {
    return tile == LEVEL_THREADS * 4 || (tile == LEVEL_THREADS * 8 && level_ipt_ok(k, 8));
}

// Resident blocks per SM of the persistent level kernels ([0] count,
// [1] move; by K and tile variant: [0] 4, [1] 8 elements per thread) and
// the SM count, set by init_build_kernels.
static int g_level_occ[2][MAXK + 1][2];
static int g_num_sms = 0;

// Status area of one level step (u32 words, every region 16-byte aligned):
// counts [t][nbp], scanned counts [t][nbp], head flags [t], tile records
// [t][trec_words], two tile counters.
struct LevelStatus {
    uint32_t *cnt, *incl, *head, *trec, *lb, *ctrs;
};
static size_t level_lb_words(int k, int ntiles) {
    return ((size_t)3 * level_nbp(k) * level_scan_chunks(ntiles) + 3) & ~(size_t)3;
}
static LevelStatus level_status_layout(int k, int ntiles, uint32_t* status) {
    const size_t t4 = ((size_t)ntiles + 3) & ~(size_t)3;
    const size_t nbp = (size_t)level_nbp(k);
    LevelStatus L;
    L.cnt = status;
    L.incl = L.cnt + t4 * nbp;
    L.head = L.incl + t4 * nbp;
    L.trec = L.head + t4;
    L.lb = L.trec + t4 * (size_t)trec_words(k);
    L.ctrs = L.lb + level_lb_words(k, ntiles);
    return L;
}

size_t level_status_words(int k, int ntiles) {
    const size_t t4 = ((size_t)ntiles + 3) & ~(size_t)3;
    return t4 * (2 * (size_t)level_nbp(k) + 1 + (size_t)trec_words(k)) + level_lb_words(k, ntiles) + 4;
}

template <int K, int IPT>
static cudaError_t level_step(const AllBufs& bufs, int q, const LevelJob* jobs, int njobs, int ntiles,
                              const CloudDev* clouds, uint32_t* medr, const uint32_t* perm0, const LevelStatus& L,
                              int* err, cudaStream_t s) {
    const int v = IPT == 8 ? 1 : 0;
    const int nbmax = 1 << (K - 1);
    const int nch = level_scan_chunks(ntiles);
    const int nflags = nbmax * nch;  // look-back flags of the scan, [bucket][chunk]
    const int gc = std::min(ntiles, g_num_sms * g_level_occ[0][K][v]);
    const int gm = std::min(ntiles, g_num_sms * g_level_occ[1][K][v]);
    cudaError_t e = launch_dependent(k_level_tiles<K, IPT>, dim3((ntiles + 7) / 8), dim3(256), 0, s, jobs, njobs,
                                     ntiles, clouds, (const uint32_t*)medr, L.trec, L.ctrs, L.lb, nflags, err);
    if (e == cudaSuccess)
        e = launch_dependent(k_level_count<K, IPT>, dim3(gc), dim3(LEVEL_BLOCK), level_smem_bytes<K, IPT>(false), s,
                             bufs, q, jobs, njobs, ntiles, clouds, (const uint32_t*)L.trec, L.cnt, L.head, L.ctrs, err);
    if (e == cudaSuccess)
        e = launch_dependent(k_level_scan, dim3(nbmax * nch), dim3(1024), 0, s, ntiles, nbmax, level_nbp(K),
                             (const uint32_t*)L.cnt, (const uint32_t*)L.head, L.incl, L.lb, L.ctrs + 2, err);
    if (e == cudaSuccess)
        e = launch_dependent(k_level_pass<K, IPT>, dim3(gm), dim3(LEVEL_BLOCK), level_smem_bytes<K, IPT>(true), s, bufs,
                             q, jobs, njobs, ntiles, clouds, medr, perm0, (const uint32_t*)L.trec,
                             (const uint32_t*)L.incl, L.ctrs + 1, err);
    return e;
}

// One level step of array q over the jobs' tiles of `tile` positions
// (1024, or 2048 for k <= 4).
cudaError_t launch_level_pass(int k, int tile, const AllBufs& bufs, int q, const LevelJob* jobs, int njobs,
                              int ntiles, const CloudDev* clouds, uint32_t* medr, const uint32_t* perm0,
                              uint32_t* status, int* err, cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    if (k < 2 || k > MAXK || g_num_sms == 0 || !level_tile_supported(k, tile)) return cudaErrorInvalidValue;
    const LevelStatus L = level_status_layout(k, ntiles, status);
    const bool big = tile == LEVEL_THREADS * 8;
    cudaError_t e = cudaSuccess;
    switch (k) {
        case 2: e = big ? level_step<2, 8>(bufs, q, jobs, njobs, ntiles, clouds, medr, perm0, L, err, s)
                        : level_step<2, 4>(bufs, q, jobs, njobs, ntiles, clouds, medr, perm0, L, err, s); break;
        case 3: e = big ? level_step<3, 8>(bufs, q, jobs, njobs, ntiles, clouds, medr, perm0, L, err, s)
                        : level_step<3, 4>(bufs, q, jobs, njobs, ntiles, clouds, medr, perm0, L, err, s); break;
        case 4: e = big ? level_step<4, 8>(bufs, q, jobs, njobs, ntiles, clouds, medr, perm0, L, err, s)
                        : level_step<4, 4>(bufs, q, jobs, njobs, ntiles, clouds, medr, perm0, L, err, s); break;
        case 5: e = level_step<5, 4>(bufs, q, jobs, njobs, ntiles, clouds, medr, perm0, L, err, s); break;
        case 6: e = level_step<6, 4>(bufs, q, jobs, njobs, ntiles, clouds, medr, perm0, L, err, s); break;
        case 7: e = level_step<7, 4>(bufs, q, jobs, njobs, ntiles, clouds, medr, perm0, L, err, s); break;
        case 8: e = level_step<8, 4>(bufs, q, jobs, njobs, ntiles, clouds, medr, perm0, L, err, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int K, int IPT>
static cudaError_t init_level_kernels() {
    const int v = IPT == 8 ? 1 : 0;
    const size_t sc = level_smem_bytes<K, IPT>(false), sm = level_smem_bytes<K, IPT>(true);
    cudaError_t e = cudaFuncSetAttribute((const void*)k_level_count<K, IPT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)k_level_pass<K, IPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
    int oc = 0, om = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, k_level_count<K, IPT>, LEVEL_BLOCK, sc);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&om, k_level_pass<K, IPT>, LEVEL_BLOCK, sm);
    g_level_occ[0][K][v] = oc > 0 ? oc : 1;
    g_level_occ[1][K][v] = om > 0 ? om : 1;
    return e;
}

int finish_kmax(int smax) { return fin_kmax(smax); }
size_t finish_smem(int k, int smax) {
    return (size_t)smax * 4 + (size_t)smax * 4 + (size_t)(k + 2) * smax * 2 + (size_t)smax;
}

cudaError_t init_build_kernels() {
    cudaError_t e = cudaSuccess;
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = init_level_kernels<2, 8>();
    if (e == cudaSuccess) e = init_level_kernels<2, 4>();
    if (e == cudaSuccess) e = init_level_kernels<3, 8>();
    if (e == cudaSuccess) e = init_level_kernels<3, 4>();
    if (e == cudaSuccess) e = init_level_kernels<4, 8>();
    if (e == cudaSuccess) e = init_level_kernels<4, 4>();
    if (e == cudaSuccess) e = init_level_kernels<5, 4>();
    if (e == cudaSuccess) e = init_level_kernels<6, 4>();
    if (e == cudaSuccess) e = init_level_kernels<7, 4>();
    if (e == cudaSuccess) e = init_level_kernels<8, 4>();
    auto set = [&](const void* f, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set((const void*)k_finish<1024, 2>, finish_smem(2, 1024));
    set((const void*)k_finish<1024, 3>, finish_smem(3, 1024));
    set((const void*)k_finish<1024, 4>, finish_smem(4, 1024));
    set((const void*)k_finish<1024, 5>, finish_smem(5, 1024));
    set((const void*)k_finish<1024, 6>, finish_smem(6, 1024));
    set((const void*)k_finish<1024, 7>, finish_smem(7, 1024));
    set((const void*)k_finish<1024, 8>, finish_smem(8, 1024));
    set((const void*)k_finish<2048, 2>, finish_smem(2, 2048));
    set((const void*)k_finish<2048, 3>, finish_smem(3, 2048));
    set((const void*)k_finish<2048, 4>, finish_smem(4, 2048));
    set((const void*)k_finish<4096, 2>, finish_smem(2, 4096));
    set((const void*)k_finish<4096, 3>, finish_smem(3, 4096));
    return e;
}

// Finisher over units [unit_base, unit_base + nunits).
template <int SMAX, int K>
static void finish_as(const AllBufs& bufs, const int64_t* unit_prefix, int ncloud, int64_t unit_base, int nunits,
                      const CloudDev* clouds, const uint32_t* perm0, size_t smem, int* err,
                      unsigned long long* phase_ns, cudaStream_t s) {
    if constexpr (K <= fin_kmax(SMAX))
        k_finish<SMAX, K><<<nunits, FIN_THREADS, smem, s>>>(bufs, unit_prefix, ncloud, unit_base, clouds, perm0, err,
                                                           phase_ns);
}

template <int SMAX>
static cudaError_t finish_for(int k, const AllBufs& bufs, const int64_t* unit_prefix, int ncloud, int64_t unit_base,
                              int nunits, const CloudDev* clouds, const uint32_t* perm0, size_t smem, int* err,
                              unsigned long long* phase_ns, cudaStream_t s) {
#define KD_FIN(K)                                                                                              \
    case K:                                                                                                    \
        finish_as<SMAX, K>(bufs, unit_prefix, ncloud, unit_base, nunits, clouds, perm0, smem, err, phase_ns, s); \
        break;
    switch (k) {
        KD_FIN(2) KD_FIN(3) KD_FIN(4) KD_FIN(5) KD_FIN(6) KD_FIN(7) KD_FIN(8)
        default: return cudaErrorInvalidValue;
    }
#undef KD_FIN
    return cudaGetLastError();
}

cudaError_t launch_finish(const AllBufs& bufs, int k, const int64_t* unit_prefix, int ncloud, int64_t unit_base,
                          int nunits, const CloudDev* clouds, const uint32_t* perm0, int smax, int* err,
                          unsigned long long* phase_ns, cudaStream_t s) {
    if (nunits == 0) return cudaSuccess;
    if (k > fin_kmax(smax)) return cudaErrorInvalidValue;
    const size_t smem = finish_smem(k, smax);
    if (smax == 2048)
        return finish_for<2048>(k, bufs, unit_prefix, ncloud, unit_base, nunits, clouds, perm0, smem, err, phase_ns, s);
    if (smax == 1024)
        return finish_for<1024>(k, bufs, unit_prefix, ncloud, unit_base, nunits, clouds, perm0, smem, err, phase_ns, s);
    if (smax == 4096)
        return finish_for<4096>(k, bufs, unit_prefix, ncloud, unit_base, nunits, clouds, perm0, smem, err, phase_ns, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_top_nodes(const CloudDev* clouds, const int64_t* prefix, int ncloud, int64_t total, int k,
                             const uint32_t* perm0, uint32_t* medr, int all_nodes, cudaStream_t s) {
    if (total == 0) return cudaSuccess;
    int64_t g = (total + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    k_top_nodes<<<(unsigned)g, 256, 0, s>>>(clouds, prefix, ncloud, k, perm0, medr, all_nodes);
    return cudaGetLastError();
}

}  // namespace kd

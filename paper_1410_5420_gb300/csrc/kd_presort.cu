// kd_presort.cu -- presort kernels of the GB300 k-d tree builder.
//
// The presort of Section 2.1 (k index arrays sorted by the cyclic super keys
// x_d : x_{d+1} : ... : x_{d-1}, then one pass removing duplicate tuples) is
// computed here as:
//   k_transform   coordinates -> order-preserving unsigned key planes (SoA)
//                 plus 256-bin histograms of every key byte;
//   k_rs_count / k_rs_scan / k_rs_move
//                 one stable 8-bit LSD pass as reduce (per-tile digit
//                 histograms), scan (per-digit tile offsets) and a persistent
//                 move kernel fed by bulk async copies (stable warp ranking,
//                 tile ordered by digit in shared memory, coalesced runs).
//                 Sorting least-significant part first over x_{k-1}, ...,
//                 x_0 leaves the index array in x:y:... order; each further
//                 array d is a stable sort of array d+1 by x_d alone (ties
//                 keep the order of super key d+1, which equals super key
//                 d's order on them);
//   k_gather      the keys of the next coordinate in the current order;
//   k_dedup       adjacent-compare of the sorted array 0 and stream
//                 compaction (Section 2.1, duplicates paragraph);
//   k_records     rank vectors: rec[d][p][i] = position, in super-key-p
//                 order, of the tuple at position i of array d.  After
//                 deduplication super keys are unique, so comparing super
//                 keys equals comparing these ranks.
#include <algorithm>

#include "kd_internal.cuh"

namespace kd {

// -------------------------------------------------------------- helpers
// ------------------------------------------------------------ transform
// hist layout: row (d * D + b) for coordinate d, key byte b; then rows
// (k * D + b) for the cloud-id plane of a batch.  Dynamic smem: the block's
// histogram rows followed by a 256-point staging tile of coordinates.
template <typename T, typename KW>
__global__ void __launch_bounds__(256) k_transform(const T* __restrict__ coords, int64_t n, int k,
                                                   KW* __restrict__ keys, int64_t stride, KW* __restrict__ tail,
                                                   const int64_t* __restrict__ cloud_start, int ncloud,
                                                   uint32_t* __restrict__ cloud_plane,
                                                   int cloud_digits, uint32_t* __restrict__ hist,
                                                   int* __restrict__ err) {
    constexpr int D = sizeof(KW);
    extern __shared__ uint32_t smem[];
    const int nrows = k * D + cloud_digits;
    uint32_t* sh = smem;
    T* sc = reinterpret_cast<T*>(smem + nrows * RADIX);
    const int tid = threadIdx.x;
    for (int i = tid; i < nrows * RADIX; i += 256) sh[i] = 0;
    int nan = 0;
    __syncthreads();
    for (int64_t base = (int64_t)blockIdx.x * 256; base < n; base += (int64_t)gridDim.x * 256) {
        const int cnt = (int)(n - base < 256 ? n - base : 256);
        for (int i = tid; i < cnt * k; i += 256) sc[i] = coords[base * k + i];
        __syncthreads();
        if (tid < cnt) {
            const int64_t p = base + tid;
            for (int d = 0; d < k; ++d) {
                KW key = key_of(sc[tid * k + d], &nan);
                keys[d * stride + p] = key;
                if (tail && d > 0) tail[p * (k - 1) + d - 1] = key;
#pragma unroll
                for (int b = 0; b < D; ++b)
                    atomicAdd(&sh[(d * D + b) * RADIX + (uint32_t)((key >> (8 * b)) & 255u)], 1u);
            }
            if (ncloud > 1) {
                int lo = 0, hi = ncloud;  // largest c with cloud_start[c] <= p
                while (hi - lo > 1) {
                    int mid = (lo + hi) >> 1;
                    if (cloud_start[mid] <= p) lo = mid; else hi = mid;
                }
                cloud_plane[p] = (uint32_t)lo;
                for (int b = 0; b < cloud_digits; ++b)
                    atomicAdd(&sh[(k * D + b) * RADIX + ((lo >> (8 * b)) & 255)], 1u);
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < nrows * RADIX; i += 256)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
    if (nan) atomicOr(err, ERR_NAN);
}

// ---------------------------------------------------------- sort passes
// One stable LSD digit pass is three launches (reduce, scan, move):
//   k_rs_count  per tile, the 256-bin histogram of the pass digit;
//   k_rs_scan   per digit, the exclusive prefix over tiles plus the digit's
//               global base: chunks of RS_CHUNK tiles, chained by a
//               decoupled look-back over chunk totals;
//   k_rs_move   persistent: a producer warp streams each tile's offsets row,
//               keys and up to SP payload planes into a shared-memory stage
//               with bulk async copies (full/empty mbarriers); eight consumer
//               warps rank the keys stably (match instruction or match
//               words, chosen per warp and tile by how many distinct digits
//               the first 32 keys hold; per-warp counters), order the tile
//               by digit in shared memory and
//               write every plane with runs of equal digits to consecutive
//               addresses.
// Stability: within a tile, elements are ranked in position order (warp by
// warp, lane by lane); across tiles, the scan orders tiles by index.
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_BLOCK = RS_THREADS + 32;  // + producer warp
constexpr int RS_CHUNK = 64;               // tiles per scan chunk
constexpr int RS_TILE_MIN = 1024;          // smallest tile of any variant (sizes the status area)

struct SortMeta {
    int32_t t;  // tile, or -1: no more tiles
    int32_t n;  // elements in the tile
    int64_t base;
};

template <typename KW>
__device__ __forceinline__ uint32_t digit_of(KW key, int shift) {
    return (uint32_t)(key >> shift) & 255u;
}

constexpr int RS_CT = 2;  // tiles counted per block (their loads in flight together)

template <typename KW, int TILE>
__global__ void __launch_bounds__(256) k_rs_count(const int64_t* __restrict__ count_ptr, const KW* __restrict__ key_src,
                                                  int shift, uint32_t* __restrict__ cnt,
                                                  uint32_t* __restrict__ scan_flags, int nflags,
                                                  uint32_t* __restrict__ scan_ctr) {
    constexpr int V = 16 / sizeof(KW);            // keys per 16-byte load
    constexpr int NV = TILE / V / 256;            // loads per thread and tile
    __shared__ uint32_t s_h[RS_CT][8][RADIX];
    const int tid = threadIdx.x, warp = tid >> 5;
    pdl_wait();  // the previous pass's keys
    pdl_trigger();
    if (blockIdx.x == 0) {  // the scan of this pass starts from cleared flags
        for (int i = tid; i < nflags; i += 256) scan_flags[i] = 0;
        if (tid == 0) *scan_ctr = 0;
    }
    for (int i = tid; i < RS_CT * 8 * RADIX; i += 256) (&s_h[0][0][0])[i] = 0;
    __syncthreads();
    const int64_t count = *count_ptr;
    const int64_t ntiles = (count + TILE - 1) / TILE;
    uint4 x[RS_CT][NV];
#pragma unroll
    for (int c = 0; c < RS_CT; ++c) {
        const int64_t base = ((int64_t)blockIdx.x * RS_CT + c) * TILE;
        const int n = base >= count ? 0 : (int)(count - base < TILE ? count - base : (int64_t)TILE);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int o = (v * 256 + tid) * V;
            x[c][v] = o + V <= n ? *reinterpret_cast<const uint4*>(key_src + base + o) : make_uint4(0, 0, 0, 0);
        }
    }
#pragma unroll
    for (int c = 0; c < RS_CT; ++c) {
        const int64_t base = ((int64_t)blockIdx.x * RS_CT + c) * TILE;
        const int n = base >= count ? 0 : (int)(count - base < TILE ? count - base : (int64_t)TILE);
        const KW* src = key_src + base;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int o = (v * 256 + tid) * V;
            if (o + V <= n) {
                const KW* kv = reinterpret_cast<const KW*>(&x[c][v]);
#pragma unroll
                for (int e = 0; e < V; ++e) atomicAdd(&s_h[c][warp][digit_of(kv[e], shift)], 1u);
            } else {
                for (int e = 0; e < V; ++e)
                    if (o + e < n) atomicAdd(&s_h[c][warp][digit_of(src[o + e], shift)], 1u);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < RS_CT; ++c) {
        const int64_t t = (int64_t)blockIdx.x * RS_CT + c;
        if (t >= ntiles) break;
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) sum += s_h[c][w][tid];
        cnt[t * RADIX + tid] = sum;
    }
}

// offs[t][d] = digit_base[d] + (elements of digit d in tiles before t).
// spin_limit bounds the look-back's polls; a chunk whose wait runs out
// stores nothing and reports ERR_TIMEOUT.  withhold (failure-detection
// tests only): chunk 0 never publishes its flag, so every later chunk's
// wait runs out.
__global__ void __launch_bounds__(256) k_rs_scan(const int64_t* __restrict__ count_ptr, int tile,
                                                 const uint32_t* __restrict__ cnt,
                                                 const uint32_t* __restrict__ digit_base, uint32_t* __restrict__ offs,
                                                 uint32_t* __restrict__ flags, uint32_t* __restrict__ agg,
                                                 uint32_t* __restrict__ inc, uint32_t* __restrict__ scan_ctr,
                                                 uint32_t* __restrict__ move_ctr, int* __restrict__ err,
                                                 uint32_t spin_limit, int withhold) {
    __shared__ uint32_t s_chunk, s_ctl;
    const int tid = threadIdx.x;
    pdl_wait();
    pdl_trigger();
    if (tid == 0) s_chunk = atomicAdd(scan_ctr, 1u);
    if (blockIdx.x == 0 && tid == 0) *move_ctr = 0;  // the move pass starts after this kernel
    __syncthreads();
    const int64_t count = *count_ptr;
    const int64_t ntiles = (count + tile - 1) / tile;
    const int64_t nchunks = (ntiles + RS_CHUNK - 1) / RS_CHUNK;
    const int64_t c = s_chunk;
    if (c >= nchunks) return;
    const int64_t t0 = c * RS_CHUNK;
    const int64_t t1 = t0 + RS_CHUNK < ntiles ? t0 + RS_CHUNK : ntiles;
    // the chunk's counts of digit tid, all loads in flight together
    uint32_t v[RS_CHUNK];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < RS_CHUNK; ++j) v[j] = t0 + j < t1 ? cnt[(t0 + j) * RADIX + tid] : 0u;
#pragma unroll
    for (int j = 0; j < RS_CHUNK; ++j) sum += v[j];
    if (c == 0) inc[tid] = sum;
    else agg[c * RADIX + tid] = sum;
    __syncthreads();
    if (tid == 0 && !(withhold && c == 0)) publish_flag(flags, c, c == 0 ? FLAG_INC : FLAG_AGG);
    uint32_t excl = 0;
    if (c > 0) {
        __shared__ bool s_late;
        if (tid == 0) s_late = false;
        __syncthreads();
        excl = block_lookback<uint32_t>(flags, agg, inc, RADIX, c, &s_ctl, err, 0, spin_limit, &s_late);
        if (s_late) return;  // uniform: set by the look-back for the whole block
        inc[c * RADIX + tid] = excl + sum;
        __syncthreads();
        if (tid == 0) publish_flag(flags, c, FLAG_INC);
    }
    uint32_t run = digit_base[tid] + excl;
#pragma unroll
    for (int j = 0; j < RS_CHUNK; ++j) {
        if (t0 + j < t1) offs[(t0 + j) * RADIX + tid] = run;
        run += v[j];
    }
}

// The tile is ordered by digit in shared memory before it is written out.
// 32-bit keys: in place, over the key and payload words of the stage the
// tile came in (every value is in registers by then).  64-bit keys: in a
// separate buffer of TILE key words.
template <typename KW>
constexpr bool rs_inplace() { return sizeof(KW) == 4; }

template <typename KW, int TILE, int SP>
constexpr size_t rs_move_smem() {
    return ((size_t)2 * (RADIX + TILE * (sizeof(KW) / 4) + SP * TILE) + (rs_inplace<KW>() ? 0 : (size_t)TILE * 2)) *
           4;
}

// Resident blocks the move kernel is compiled for: as many as its shared
// memory allows (32-bit keys: 4 with one staged payload, 3 with two, 2
// with three).
template <typename KW, int TILE, int SP>
constexpr int rs_min_blocks() {
    return rs_inplace<KW>() ? (SP == 1 ? 4 : (SP == 2 ? 3 : 2)) : 2;
}

template <typename KW, int TILE, int SP>
__global__ void __launch_bounds__(RS_BLOCK, (rs_min_blocks<KW, TILE, SP>()))
    k_rs_move(const int64_t* __restrict__ count_ptr, const KW* __restrict__ key_src, KW* __restrict__ key_dst,
              const __grid_constant__ PayloadArgs pay, const uint32_t* __restrict__ offs, int shift,
              uint32_t* __restrict__ ctr, int* __restrict__ err) {
    constexpr int IPT = TILE / RS_THREADS;
    constexpr int KWW = sizeof(KW) / 4;
    constexpr int SW = RADIX + TILE * KWW + SP * TILE;  // stage words: offsets row | keys | payloads
    constexpr bool INPLACE = rs_inplace<KW>();
    constexpr bool PAIR = sizeof(KW) == 4 && SP == 1;    // key and payload sorted together
    constexpr bool TRIPLE = sizeof(KW) == 4 && SP == 2;  // key and two payloads: an 8-byte and a 4-byte word
    constexpr bool QUAD = sizeof(KW) == 4 && SP == 3;    // key and three payloads: two 8-byte words
    extern __shared__ __align__(128) uint32_t rsm[];     // [2][SW] stages (then the sorted tile for 64-bit keys)
    __shared__ __align__(8) uint64_t full[2], empty[2];
    __shared__ SortMeta meta[2];
    __shared__ uint32_t s_wc[RS_WARPS][RADIX];
    __shared__ uint32_t s_match[RS_WARPS][RADIX];  // lane masks of the ranking; all zero between uses
    __shared__ uint32_t s_goff[RADIX], s_tstart[RADIX];
    __shared__ uint32_t s_wsum[RS_WARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], RS_WARPS);
        }
        fence_mbar_init();
    }
    for (int i = tid; i < RS_WARPS * RADIX; i += RS_BLOCK) {
        (&s_wc[0][0])[i] = 0;
        (&s_match[0][0])[i] = 0;
    }
    __syncthreads();
    pdl_wait();  // the scan's offsets and tile counter
    pdl_trigger();
    const int64_t count = *count_ptr;
    const int64_t ntiles = (count + TILE - 1) / TILE;
    if (warp == RS_WARPS) {  // producer
        if (lane != 0) return;
        for (int it = 0;; ++it) {
            const int s = it & 1;
            const uint32_t ph = (uint32_t)(it >> 1) & 1u;
            if (it >= 2 && !mbar_wait(&empty[s], ph ^ 1u)) {
                atomicOr(err, ERR_TIMEOUT);
                meta[s].t = -1;
                mbar_arrive(&full[s]);
                return;
            }
            const int64_t t = atomicAdd(ctr, 1u);
            SortMeta M;
            M.t = t < ntiles ? (int32_t)t : -1;
            if (M.t < 0) {
                meta[s] = M;
                mbar_arrive(&full[s]);
                return;
            }
            M.base = t * TILE;
            M.n = (int32_t)(count - M.base < TILE ? count - M.base : (int64_t)TILE);
            const uint32_t kb = ((uint32_t)M.n * sizeof(KW) + 15u) & ~15u;
            const uint32_t pb = ((uint32_t)M.n * 4u + 15u) & ~15u;
            int nst = 0;
            for (int p = 0; p < pay.n && p < SP; ++p) nst += pay.src[p] != nullptr;
            meta[s] = M;
            uint32_t* st = rsm + (size_t)s * SW;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&full[s], RADIX * 4 + kb + (uint32_t)nst * pb);
            bulk_g2s(st, offs + t * RADIX, RADIX * 4, &full[s]);
            bulk_g2s(st + RADIX, key_src + M.base, kb, &full[s]);
            for (int p = 0; p < pay.n && p < SP; ++p)
                if (pay.src[p]) bulk_g2s(st + RADIX + TILE * KWW + p * TILE, pay.src[p] + M.base, pb, &full[s]);
        }
    }
    const int wbase = warp * 32 * IPT;
    for (int it = 0;; ++it) {
        const int s = it & 1;
        const bool ok = mbar_wait(&full[s], (uint32_t)(it >> 1) & 1u);
        if (consumer_or<RS_THREADS>(!ok)) {
            if (tid == 0) atomicOr(err, ERR_TIMEOUT);
            break;
        }
        const SortMeta M = meta[s];
        if (M.t < 0) break;
        uint32_t* st = rsm + (size_t)s * SW;
        // the tile's keys and staged payloads into registers
        KW kreg[IPT];
        uint32_t preg[SP][IPT];
        {
            const KW* skeys = reinterpret_cast<const KW*>(st + RADIX);
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const int o = wbase + j * 32 + lane;
                const bool v = o < M.n;
                kreg[j] = v ? skeys[o] : (KW)0;
#pragma unroll
                for (int p = 0; p < SP; ++p) {
                    const uint32_t* sp = st + RADIX + TILE * KWW + p * TILE;
                    preg[p][j] = (p < pay.n && pay.src[p]) ? (v ? sp[o] : 0u) : (uint32_t)(M.base + o);
                }
            }
        }
        // stable warp ranking (match instruction or match words)
        uint32_t dig[IPT], slot[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j)
            dig[j] = wbase + j * 32 + lane < M.n ? digit_of(kreg[j], shift) : (uint32_t)RADIX;
        warp_rank_adaptive<IPT>(dig, RADIX, s_wc[warp], s_match[warp], slot);
        consumer_sync<RS_THREADS>();  // every warp has ranked, and has read the stage into registers
        // digit tid: prefix over warps in place, tile count, tile start
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t x = s_wc[w][tid];
            s_wc[w][tid] = c;
            c += x;
        }
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[warp] = x;
        consumer_sync<RS_THREADS>();
        uint32_t wpre = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) wpre += w < warp ? s_wsum[w] : 0u;
        const uint32_t tstart = wpre + x - c;
        s_tstart[tid] = tstart;
        s_goff[tid] = st[tid] - tstart;  // destination of sorted slot i with digit d: s_goff[d] + i
        consumer_sync<RS_THREADS>();
#pragma unroll
        for (int j = 0; j < IPT; ++j)
            if (dig[j] < RADIX) slot[j] += s_tstart[dig[j]] + s_wc[warp][dig[j]];
        __syncwarp();
        for (int d = lane; d < RADIX; d += 32) s_wc[warp][d] = 0;  // own row, read above only by this warp
        // the sorted tile: over this stage's keys and payloads, or a separate buffer
        uint32_t* sb32 = INPLACE ? st + RADIX : rsm + (size_t)2 * SW;
        KW* sbuf = reinterpret_cast<KW*>(sb32);
        if constexpr (PAIR) {
            if (pay.n == 1) {
                // 32-bit keys with one payload: both go through the sorted
                // tile as one 8-byte word
                uint2* sb2 = reinterpret_cast<uint2*>(sb32);
#pragma unroll
                for (int j = 0; j < IPT; ++j)
                    if (dig[j] < RADIX) sb2[slot[j]] = make_uint2((uint32_t)kreg[j], preg[0][j]);
                consumer_sync<RS_THREADS>();
                uint32_t* dst = pay.dst[0];
#pragma unroll
                for (int r = 0; r < IPT; ++r) {
                    const int i = r * RS_THREADS + tid;
                    if (i < M.n) {
                        const uint2 kv = sb2[i];
                        const uint32_t dd = s_goff[digit_of((KW)kv.x, shift)] + (uint32_t)i;
                        if ((int64_t)dd < count) {
                            if (key_dst) key_dst[dd] = (KW)kv.x;
                            dst[dd] = kv.y;
                        } else {
                            atomicOr(err, ERR_INTERNAL);
                        }
                    }
                }
                if (INPLACE) fence_proxy_async_smem();  // our writes to the stage before the next bulk copy into it
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);  // this warp's reads of the stage are done
                continue;
            }
        }
        if constexpr (TRIPLE) {
            if (pay.n == 2) {
                uint2* sb2 = reinterpret_cast<uint2*>(sb32);
                uint32_t* sb1 = sb32 + 2 * TILE;
#pragma unroll
                for (int j = 0; j < IPT; ++j) {
                    if (dig[j] < RADIX) {
                        sb2[slot[j]] = make_uint2((uint32_t)kreg[j], preg[0][j]);
                        sb1[slot[j]] = preg[1][j];
                    }
                }
                consumer_sync<RS_THREADS>();
                uint32_t* dst0 = pay.dst[0];
                uint32_t* dst1 = pay.dst[1];
#pragma unroll
                for (int r = 0; r < IPT; ++r) {
                    const int i = r * RS_THREADS + tid;
                    if (i < M.n) {
                        const uint2 kv = sb2[i];
                        const uint32_t dd = s_goff[digit_of((KW)kv.x, shift)] + (uint32_t)i;
                        if ((int64_t)dd < count) {
                            if (key_dst) key_dst[dd] = (KW)kv.x;
                            dst0[dd] = kv.y;
                            dst1[dd] = sb1[i];
                        } else {
                            atomicOr(err, ERR_INTERNAL);
                        }
                    }
                }
                if (INPLACE) fence_proxy_async_smem();  // our writes to the stage before the next bulk copy into it
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);  // this warp's reads of the stage are done
                continue;
            }
        }
        if constexpr (QUAD) {
            if (pay.n == 3) {
                uint2* sa = reinterpret_cast<uint2*>(sb32);             // (key, payload 0)
                uint2* sq = reinterpret_cast<uint2*>(sb32 + 2 * TILE);  // (payload 1, payload 2)
#pragma unroll
                for (int j = 0; j < IPT; ++j) {
                    if (dig[j] < RADIX) {
                        sa[slot[j]] = make_uint2((uint32_t)kreg[j], preg[0][j]);
                        sq[slot[j]] = make_uint2(preg[1][j], preg[2][j]);
                    }
                }
                consumer_sync<RS_THREADS>();
                uint32_t* dst0 = pay.dst[0];
                uint32_t* dst1 = pay.dst[1];
                uint32_t* dst2 = pay.dst[2];
#pragma unroll
                for (int r = 0; r < IPT; ++r) {
                    const int i = r * RS_THREADS + tid;
                    if (i < M.n) {
                        const uint2 kv = sa[i];
                        const uint2 pq = sq[i];
                        const uint32_t dd = s_goff[digit_of((KW)kv.x, shift)] + (uint32_t)i;
                        if ((int64_t)dd < count) {
                            if (key_dst) key_dst[dd] = (KW)kv.x;
                            dst0[dd] = kv.y;
                            dst1[dd] = pq.x;
                            dst2[dd] = pq.y;
                        } else {
                            atomicOr(err, ERR_INTERNAL);
                        }
                    }
                }
                if (INPLACE) fence_proxy_async_smem();  // our writes to the stage before the next bulk copy into it
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);  // this warp's reads of the stage are done
                continue;
            }
        }
#pragma unroll
        for (int j = 0; j < IPT; ++j)
            if (dig[j] < RADIX) sbuf[slot[j]] = kreg[j];
        consumer_sync<RS_THREADS>();
        // A destination outside [0, count) can only come from inconsistent
        // counts; it is reported and never written.
        uint32_t dest[IPT];
#pragma unroll
        for (int r = 0; r < IPT; ++r) {
            const int i = r * RS_THREADS + tid;
            dest[r] = 0xffffffffu;
            if (i < M.n) {
                const KW kk = sbuf[i];
                const uint32_t dd = s_goff[digit_of(kk, shift)] + (uint32_t)i;
                if ((int64_t)dd < count) {
                    dest[r] = dd;
                    if (key_dst) key_dst[dd] = kk;
                } else {
                    atomicOr(err, ERR_INTERNAL);
                }
            }
        }
        if constexpr (sizeof(KW) == 8) {
            // payload planes two at a time through the sorted tile (8-byte
            // words); staged planes come from registers, the others from global
            // memory in source order
            uint2* sbp = reinterpret_cast<uint2*>(sb32);
            for (int p = 0; p < pay.n; p += 2) {
                const bool two = p + 1 < pay.n;
                consumer_sync<RS_THREADS>();  // earlier readers of the sorted tile are done
#pragma unroll
                for (int j = 0; j < IPT; ++j) {
                    const int o = wbase + j * 32 + lane;
                    if (dig[j] < RADIX) {
                        uint32_t a = 0, b = 0;
                        if (p < SP) {
#pragma unroll
                            for (int q = 0; q < SP; ++q)
                                if (q == p) a = preg[q][j];
                        } else {
                            a = pay.src[p] ? pay.src[p][M.base + o] : (uint32_t)(M.base + o);
                        }
                        if (two) {
                            if (p + 1 < SP) {
#pragma unroll
                                for (int q = 0; q < SP; ++q)
                                    if (q == p + 1) b = preg[q][j];
                            } else {
                                b = pay.src[p + 1] ? pay.src[p + 1][M.base + o] : (uint32_t)(M.base + o);
                            }
                        }
                        sbp[slot[j]] = make_uint2(a, b);
                    }
                }
                consumer_sync<RS_THREADS>();
                uint32_t* dst0 = pay.dst[p];
                uint32_t* dst1 = two ? pay.dst[p + 1] : nullptr;
#pragma unroll
                for (int r = 0; r < IPT; ++r) {
                    if (dest[r] != 0xffffffffu) {
                        const uint2 v = sbp[r * RS_THREADS + tid];
                        dst0[dest[r]] = v.x;
                        if (two) dst1[dest[r]] = v.y;
                    }
                }
            }
        } else {
            // one plane at a time (these kernels also hold the one- and
            // two-payload forms above, whose registers this keeps)
            for (int p = 0; p < pay.n; ++p) {
                consumer_sync<RS_THREADS>();  // earlier readers of the sorted tile are done
                const uint32_t* src = pay.src[p];
#pragma unroll
                for (int j = 0; j < IPT; ++j) {
                    const int o = wbase + j * 32 + lane;
                    if (dig[j] < RADIX) {
                        uint32_t val = 0;
                        if (p < SP) {  // staged: already in registers
#pragma unroll
                            for (int q = 0; q < SP; ++q)
                                if (q == p) val = preg[q][j];
                        } else {
                            val = src ? src[M.base + o] : (uint32_t)(M.base + o);
                        }
                        sb32[slot[j]] = val;
                    }
                }
                consumer_sync<RS_THREADS>();
                uint32_t* dst = pay.dst[p];
#pragma unroll
                for (int r = 0; r < IPT; ++r)
                    if (dest[r] != 0xffffffffu) dst[dest[r]] = sb32[r * RS_THREADS + tid];
            }
        }
        // every read of this stage (and of the sorted tile over it) is behind the barriers above
        if (INPLACE) fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

// Gather of key words by tuple id: out[pos] = plane[ids[pos]], positions in
// [0, *count_ptr).  Each thread issues GI independent gathers, so a random
// read of the key plane keeps many requests in flight.
template <typename KW, int GI>
__global__ void __launch_bounds__(256) k_gather(const int64_t* __restrict__ count_ptr, const KW* __restrict__ plane,
                                                const uint32_t* __restrict__ ids, int64_t gather_limit,
                                                KW* __restrict__ out, int* __restrict__ err) {
    const int64_t count = *count_ptr;
    const int64_t base = (int64_t)blockIdx.x * 256 * GI + threadIdx.x;
    uint32_t id[GI];
#pragma unroll
    for (int j = 0; j < GI; ++j) {
        const int64_t p = base + (int64_t)j * 256;
        id[j] = p < count ? ids[p] : 0u;
    }
    KW v[GI];
#pragma unroll
    for (int j = 0; j < GI; ++j) {
        const int64_t p = base + (int64_t)j * 256;
        v[j] = 0;
        if (p < count) {
            if ((int64_t)id[j] < gather_limit) v[j] = plane[id[j]]; else atomicOr(err, ERR_INTERNAL);
        }
    }
#pragma unroll
    for (int j = 0; j < GI; ++j) {
        const int64_t p = base + (int64_t)j * 256;
        if (p < count) out[p] = v[j];
    }
}

// Exclusive prefix of each 256-bin histogram row: bases[r][d].
__global__ void k_digit_bases(const uint32_t* __restrict__ hist, uint32_t* __restrict__ bases) {
    __shared__ uint32_t s_warp[8];
    const int r = blockIdx.x;
    bases[r * RADIX + threadIdx.x] = block_excl_scan256(hist[r * RADIX + threadIdx.x], s_warp, nullptr);
}

// ---------------------------------------------------------------- dedup
// keep[i] = i is the first of its run of identical tuples (same cloud) in
// the array sorted by super key 0.  Three steps, no inter-tile waiting:
// k_dedup_flags writes keep bits and per-tile keep counts (and subtracts
// each dropped tuple's key bytes from the histograms, so that they describe
// the kept tuples for the sorts that follow); k_tile_scan turns the counts
// into tile offsets (and m); k_dedup_compact writes the kept ids in order.
constexpr int DEDUP_TILE = 4096;

// Duplicate flags over array 0 (sorted by super key 0, equal tuples in index
// order): a tuple equal to its predecessor goes.  The keys x_1..x_{k-1} of
// position i are T[d * tstride + i], in array-0 order (the predecessor's
// are the neighbour lane's).  The kept tuples' counts leave the digit
// histograms.  TM: the most tail planes the kernel compares (k - 1 at
// most), so that k <= 3 keeps two of them in registers, not MAXK - 1.
template <typename KW, int TM>
__global__ void __launch_bounds__(256) k_dedup_flags(int64_t n, const KW* __restrict__ key0,
                                                     const uint32_t* __restrict__ ids, const KW* __restrict__ T,
                                                     int64_t tstride, int k, const uint32_t* __restrict__ cloud_plane,
                                                     int cloud_digits,
                                                     uint32_t* __restrict__ keepbits, uint32_t* __restrict__ tile_cnt,
                                                     uint32_t* __restrict__ hist, int32_t* __restrict__ mcloud,
                                                     int* __restrict__ err) {
    constexpr int IPT = DEDUP_TILE / 256;
    constexpr int D = sizeof(KW);
    __shared__ uint32_t s_wsum[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tk = k - 1;
    const int64_t base = (int64_t)blockIdx.x * DEDUP_TILE;
    const int wbase = warp * 32 * IPT;
    // the predecessor of this warp's first element
    KW last[TM];
    KW lastk0 = 0;
    uint32_t lastid = 0;
#pragma unroll
    for (int d = 0; d < TM; ++d) last[d] = 0;
    {
        const int64_t p0 = base + wbase;
        if (p0 > 0 && p0 - 1 < n) {
            if (cloud_plane) {
                lastid = ids[p0 - 1];
                if ((int64_t)lastid >= n) {
                    atomicOr(err, ERR_INTERNAL);
                    lastid = 0;
                }
            }
            lastk0 = key0[p0 - 1];
#pragma unroll
            for (int d = 0; d < TM; ++d)
                if (d < tk) last[d] = T[d * tstride + p0 - 1];
        }
    }
    uint32_t wcount = 0;
    // rows are taken U at a time, all their loads issued before the first
    // is used (ids matter only for the cloud test of a batch)
    constexpr int U = D == 4 ? 4 : 2;
    static_assert(IPT % U == 0, "rows per warp must be a multiple of the batch");
#pragma unroll 1
    for (int j0 = 0; j0 < IPT; j0 += U) {
        uint32_t idb[U];
        KW k0b[U], rb[U][TM];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t pos = base + wbase + (j0 + u) * 32 + lane;
            const bool valid = pos < n;
            idb[u] = (valid && cloud_plane) ? ids[pos] : 0u;
            k0b[u] = valid ? key0[pos] : (KW)0;
#pragma unroll
            for (int d = 0; d < TM; ++d) rb[u][d] = (valid && d < tk) ? T[d * tstride + pos] : (KW)0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + u;
            const int64_t pos = base + wbase + j * 32 + lane;
            const bool valid = pos < n;
            uint32_t id = idb[u];
            if ((int64_t)id >= n) {
                atomicOr(err, ERR_INTERNAL);
                id = 0;
            }
            const KW k0 = k0b[u];
            KW r[TM];
#pragma unroll
            for (int d = 0; d < TM; ++d) r[d] = rb[u][d];
            KW pk0 = __shfl_up_sync(0xffffffffu, k0, 1);
            uint32_t pid = __shfl_up_sync(0xffffffffu, id, 1);
            bool same = true;
#pragma unroll
            for (int d = 0; d < TM; ++d) {
                KW q = __shfl_up_sync(0xffffffffu, r[d], 1);
                if (lane == 0) q = last[d];
                same = same && (d >= tk || q == r[d]);
                last[d] = __shfl_sync(0xffffffffu, r[d], 31);
            }
            if (lane == 0) {
                pk0 = lastk0;
                pid = lastid;
            }
            lastk0 = __shfl_sync(0xffffffffu, k0, 31);
            lastid = __shfl_sync(0xffffffffu, id, 31);
            bool dup = valid && pos > 0 && pk0 == k0 && same;
            if (dup && cloud_plane && cloud_plane[id] != cloud_plane[pid]) dup = false;
            if (dup) {
                for (int b = 0; b < D; ++b) atomicSub(&hist[b * RADIX + (uint32_t)((k0 >> (8 * b)) & 255u)], 1u);
#pragma unroll
                for (int d = 0; d < TM; ++d)
                    if (d < tk)
                        for (int b = 0; b < D; ++b)
                            atomicSub(&hist[((d + 1) * D + b) * RADIX + (uint32_t)((r[d] >> (8 * b)) & 255u)], 1u);
                if (cloud_plane) {
                    const uint32_t c = cloud_plane[id];
                    for (int b = 0; b < cloud_digits; ++b)
                        atomicSub(&hist[(k * D + b) * RADIX + ((c >> (8 * b)) & 255u)], 1u);
                    atomicSub(&mcloud[c], 1);
                } else if (mcloud) {
                    atomicSub(&mcloud[0], 1);
                }
            }
            const uint32_t ball = __ballot_sync(0xffffffffu, valid && !dup);
            if (lane == 0 && base + wbase + j * 32 < n) keepbits[(base + wbase + j * 32) >> 5] = ball;
            wcount += __popc(ball);
        }
    }
    if (lane == 0) s_wsum[warp] = wcount;
    __syncthreads();
    if (tid == 0) {
        uint32_t acc = 0;
        for (int w = 0; w < 8; ++w) acc += s_wsum[w];
        tile_cnt[blockIdx.x] = acc;
    }
}

// Exclusive scan of per-tile counts in one block; *total_out = sum.
__global__ void __launch_bounds__(1024) k_tile_scan(int64_t ntiles, const uint32_t* __restrict__ cnt,
                                                    uint32_t* __restrict__ offs, int64_t* __restrict__ total_out) {
    __shared__ uint32_t s_warp[32];
    uint32_t carry = 0;
    for (int64_t t0 = 0; t0 < ntiles; t0 += 1024) {
        const int64_t t = t0 + threadIdx.x;
        const uint32_t v = t < ntiles ? cnt[t] : 0u;
        uint32_t tot;
        const uint32_t ex = block_excl_scan<1024>(v, s_warp, &tot);
        if (t < ntiles) offs[t] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

template <typename KW>
__global__ void __launch_bounds__(256) k_dedup_compact(int64_t n, const uint32_t* __restrict__ ids,
                                                       const uint32_t* __restrict__ keepbits,
                                                       const uint32_t* __restrict__ offs,
                                                       uint32_t* __restrict__ ids_out, const KW* __restrict__ y1,
                                                       const KW* __restrict__ y2, KW* __restrict__ y1_out,
                                                       KW* __restrict__ y2_out) {
    // y1 / y2: planes of x_{k-1} and x_{k-2} in array-0 order (NULL: not
    // wanted); the kept tuples' values go to y1_out / y2_out
    constexpr int IPT = DEDUP_TILE / 256;
    __shared__ uint32_t s_wsum[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * DEDUP_TILE;
    const int wbase = warp * 32 * IPT;
    uint32_t ball[IPT];
    uint32_t wcount = 0;
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int64_t row = base + wbase + j * 32;
        ball[j] = row < n ? keepbits[row >> 5] : 0u;
        wcount += __popc(ball[j]);
    }
    if (lane == 0) s_wsum[warp] = wcount;
    __syncthreads();
    uint32_t out = offs[blockIdx.x];
    for (int w = 0; w < warp; ++w) out += s_wsum[w];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int64_t pos = base + wbase + j * 32 + lane;
        if ((ball[j] >> lane) & 1u) {
            const uint32_t o = out + __popc(ball[j] & lanemask_lt());
            ids_out[o] = ids[pos];
            if (y1 && y1_out) y1_out[o] = y1[pos];
            if (y2 && y2_out) y2_out[o] = y2[pos];
        }
        out += __popc(ball[j]);
    }
}

// ------------------------------------------------------------- tie runs
// Array 0 in super-key-0 order from a sort by x_0 alone.  A stable sort of
// the ids (index order) by x_0 leaves every run of equal x_0 in index
// order; super key 0 orders such a run by x_1, ..., x_{k-1}, and equal
// tuples keep index order (Section 2.1: the super key definition, and the
// duplicates paragraph, which keeps one of the equal tuples).
//   k_run_stats    one warp per tile of RT_TILE positions: the runs'
//                  lengths L (whether one exceeds rmax, and the sum of L^2
//                  over runs of L > RT_WARP, the work of ordering them by
//                  compares: the caller sorts array 0 by the whole super key
//                  instead when either is too large), and the tile's range
//                  of whole runs for k_run_tiles: from its first run start
//                  to the next tile's, less a run of more than RT_EXT
//                  positions at its end, which is listed instead;
//   k_tail_gather  T[d][i] = x_{d+1} of the tuple at position i (its tail
//                  record, read once per position), so that everything
//                  after it streams;
//   k_run_tiles    one block per tile range (at most RT_CAP positions),
//                  staged in shared memory: each position of a run goes to
//                  run start + the number of run members whose (x_1, ...,
//                  x_{k-1}, index) is smaller (no two are equal);
//   k_run_cross    one block per listed run, the same ranking over up to
//                  rmax positions.
constexpr int RT_TILE = 2048;
constexpr int RT_EXT = 512;
constexpr int RT_CAP = RT_TILE + RT_EXT;  // positions a tile range holds at most
constexpr int RT_WARP = 32;
constexpr int RUN_BLOCK = 4096;
constexpr int RS_ROWS = 8;  // rows of 32 positions whose loads k_run_stats issues together
static_assert((RT_TILE / 32) % RS_ROWS == 0, "a tile's rows must be a multiple of the batch");

// Shared memory of k_run_tiles (x_0, tk tail words or a packed 64-bit key,
// and the id per staged position) and of k_run_cross (tk tail words and
// the id).
static size_t run_tile_smem(int key64, int tk) {
    const size_t w = key64 ? 8 : 4;
    return (size_t)RT_CAP * (w + std::max<size_t>((size_t)tk * w, 8) + 4);
}
static size_t run_cross_smem(int key64, int tk, int rmax) { return (size_t)rmax * ((size_t)tk * (key64 ? 8 : 4) + 4); }
// Longest run k_run_cross orders: RUN_BLOCK, halved while its stage would
// exceed 160 KB (64-bit keys with many dimensions).
int run_block_max(int key64, int tk) {
    int r = RUN_BLOCK;
    while (r > RT_TILE && run_cross_smem(key64, tk, r) > (size_t)160 * 1024) r >>= 1;
    return r;
}

// Last position of the run of key0[i] = v holding position i, searched up
// to i + limit (key0 is sorted): galloping, then bisection.
template <typename KW>
__device__ __forceinline__ int64_t run_last(const KW* __restrict__ key0, int64_t n, int64_t i, KW v, int64_t limit) {
    const int64_t cap = n - 1 < i + limit ? n - 1 : i + limit;
    int64_t lo = i, step = 1;
    while (lo + step <= cap && key0[lo + step] == v) {
        lo += step;
        step <<= 1;
    }
    int64_t hi = lo + step - 1 < cap ? lo + step - 1 : cap;  // key0[lo] == v; key0[hi + 1] != v or hi == cap
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (key0[mid] == v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// run_meta: [0..1] sum of L^2 over runs of more than RT_WARP positions
// (64-bit), [2] a run exceeds rmax positions, [3] runs listed for
// k_run_cross.  range[t] = (first, end) positions of tile t's whole runs.
// A run's length is the distance from its first position to the next
// run's, both in the tile, or found by galloping for the run open at the
// tile's end (the tile holding a run's first position accounts for it).
template <typename KW>
__global__ void __launch_bounds__(256) k_run_stats(const int64_t* __restrict__ count_ptr, const KW* __restrict__ key0,
                                                   int rmax, uint2* __restrict__ range, uint2* __restrict__ cross_runs,
                                                   uint32_t* __restrict__ run_meta) {
    __shared__ unsigned long long s_cost[8];
    const int64_t n = *count_ptr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    unsigned long long cost = 0;
    bool lng = false;
#define RUN_ACCOUNT(L_)                                                 \
    do {                                                                \
        const int64_t l_ = (L_);                                        \
        if (l_ > rmax) lng = true;                                      \
        else if (l_ > RT_WARP) cost += (unsigned long long)(l_ * l_);   \
    } while (0)
    const int64_t ntiles = (n + RT_TILE - 1) / RT_TILE;
    for (int64_t t = (int64_t)blockIdx.x * 8 + warp; t < ntiles; t += (int64_t)gridDim.x * 8) {
        const int64_t c0 = t * RT_TILE;
        // positions relative to c0 while scanning the tile
        int open_r = -1;   // first position of the run still open, if it began in this tile
        int first_r = -1;  // the tile's first run start
        const int valid_r = n - c0 < RT_TILE ? (int)(n - c0) : RT_TILE;  // positions of the tile
        // x_0 at the position before each row (the tile's predecessor first)
        KW carry = c0 > 0 ? key0[c0 - 1] : (KW)0;
        const KW* tile = key0 + c0;
#pragma unroll 1
        for (int r0 = 0; r0 < RT_TILE / 32; r0 += RS_ROWS) {
            KW vb[RS_ROWS];  // all rows' loads in flight before the first is used
#pragma unroll
            for (int u = 0; u < RS_ROWS; ++u) {
                const int i = (r0 + u) * 32 + lane;
                vb[u] = i < valid_r ? tile[i] : (KW)0;
            }
#pragma unroll
            for (int u = 0; u < RS_ROWS; ++u) {
                const int rb = (r0 + u) * 32;
                const int i = rb + lane;
                const KW v = vb[u];
                KW pv = __shfl_up_sync(0xffffffffu, v, 1);
                if (lane == 0) pv = carry;
                carry = __shfl_sync(0xffffffffu, v, 31);
                const bool head = i < valid_r && ((c0 == 0 && i == 0) || pv != v);
                const uint32_t hb = __ballot_sync(0xffffffffu, head);
                const uint32_t below = hb & lt;
                const int prev = below ? rb + 31 - __clz(below) : open_r;
                if (head && prev >= 0) RUN_ACCOUNT(i - prev);
                if (hb) {
                    if (first_r < 0) first_r = rb + __ffs(hb) - 1;
                    open_r = rb + 31 - __clz(hb);
                }
            }
        }
        const int64_t open = open_r >= 0 ? c0 + open_r : -1;
        int64_t first = first_r >= 0 ? c0 + first_r : -1;
        if (lane == 0) {
            // the run holding the tile's last position ends at `last`
            const int64_t tl = c0 + RT_TILE - 1 < n - 1 ? c0 + RT_TILE - 1 : n - 1;
            const int64_t last = run_last<KW>(key0, n, tl, key0[tl], rmax);
            const int64_t next = last + 1;  // the next tile's first run start (or n)
            int64_t end = next;
            if (open >= 0) {
                const int64_t L = last - open + 1;
                RUN_ACCOUNT(L);
                if (last > tl && L > RT_EXT) {  // a long run leaving the tile: listed
                    end = open;
                    if (L <= rmax) {
                        const uint32_t slot = atomicAdd(&run_meta[3], 1u);
                        cross_runs[slot] = make_uint2((uint32_t)open, (uint32_t)L);
                    }
                }
            }
            if (first < 0) first = next;  // the tile lies inside one run
            range[t] = make_uint2((uint32_t)first, (uint32_t)(end > first ? end : first));
        }
    }
#undef RUN_ACCOUNT
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) cost += __shfl_xor_sync(0xffffffffu, cost, o);
    if (lane == 0) s_cost[warp] = cost;
    lng = __syncthreads_or(lng);
    if (tid == 0) {
        unsigned long long c = 0;
        for (int w = 0; w < 8; ++w) c += s_cost[w];
        if (c) atomicAdd(reinterpret_cast<unsigned long long*>(run_meta), c);
        if (lng) atomicOr(&run_meta[2], 1u);
    }
}

constexpr int TG_ITEMS = 8;  // positions per thread of k_tail_gather
template <typename KW>
__global__ void __launch_bounds__(256) k_tail_gather(const int64_t* __restrict__ count_ptr,
                                                     const uint32_t* __restrict__ ids, const KW* __restrict__ tail,
                                                     int tk, int64_t id_limit, KW* __restrict__ T, int64_t tstride,
                                                     int* __restrict__ err) {
    constexpr int TM = MAXK - 1;
    const int64_t n = *count_ptr;
    const int64_t base = (int64_t)blockIdx.x * 256 * TG_ITEMS + threadIdx.x;
    if (base >= n) return;
    uint32_t id[TG_ITEMS];
#pragma unroll
    for (int e = 0; e < TG_ITEMS; ++e) {
        const int64_t i = base + (int64_t)e * 256;
        id[e] = i < n ? ids[i] : 0u;
        if (i < n && (int64_t)id[e] >= id_limit) {
            atomicOr(err, ERR_INTERNAL);
            id[e] = 0;
        }
    }
    if (tk * sizeof(KW) == 8) {  // one 8-byte record (two 32-bit words or one 64-bit word)
        uint2 v[TG_ITEMS];
        const uint2* rec = reinterpret_cast<const uint2*>(tail);
#pragma unroll
        for (int e = 0; e < TG_ITEMS; ++e) v[e] = base + (int64_t)e * 256 < n ? rec[id[e]] : make_uint2(0u, 0u);
#pragma unroll
        for (int e = 0; e < TG_ITEMS; ++e) {
            const int64_t i = base + (int64_t)e * 256;
            if (i < n) {
                if (sizeof(KW) == 8) {
                    T[i] = (KW)(((uint64_t)v[e].y << 32) | v[e].x);
                } else {
                    T[i] = (KW)v[e].x;
                    T[tstride + i] = (KW)v[e].y;
                }
            }
        }
        return;
    }
#pragma unroll
    for (int d = 0; d < TM; ++d) {
        if (d >= tk) break;
        KW v[TG_ITEMS];
#pragma unroll
        for (int e = 0; e < TG_ITEMS; ++e) v[e] = base + (int64_t)e * 256 < n ? tail[(int64_t)id[e] * tk + d] : (KW)0;
#pragma unroll
        for (int e = 0; e < TG_ITEMS; ++e) {
            const int64_t i = base + (int64_t)e * 256;
            if (i < n) T[d * tstride + i] = v[e];
        }
    }
}

// Number of positions j in [s, f] of a staged run whose (tail words, id)
// precede those of position i (tail word d of j at st[d * stride + j]).
// TK > 0: that many tail words, known at compile time; 0: tk of them.
template <typename KW, int TK>
__device__ __forceinline__ uint32_t run_rank(const KW* __restrict__ st, int stride, const uint32_t* __restrict__ sid,
                                             int tk, int s, int f, int i) {
    constexpr int TM = TK > 0 ? TK : MAXK - 1;
    const int nk = TK > 0 ? TK : tk;
    KW a[TM];
#pragma unroll
    for (int d = 0; d < TM; ++d) a[d] = d < nk ? st[d * stride + i] : (KW)0;
    const uint32_t ia = sid[i];
    uint32_t r = 0;
    for (int j = s; j <= f; ++j) {
        bool less = false, eq = true;
#pragma unroll
        for (int d = 0; d < TM; ++d) {
            if (d < nk) {
                const KW b = st[d * stride + j];
                less = less || (eq && b < a[d]);
                eq = eq && b == a[d];
            }
        }
        r += (less || (eq && sid[j] < ia)) ? 1u : 0u;
    }
    return r;
}

// First / last position of the staged run holding position e (sk sorted
// over [0, cnt)).
template <typename KW>
__device__ __forceinline__ int staged_first(const KW* __restrict__ sk, int e) {
    const KW v = sk[e];
    int lo = 0, hi = e;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sk[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}
template <typename KW>
__device__ __forceinline__ int staged_last(const KW* __restrict__ sk, int cnt, int e) {
    const KW v = sk[e];
    int lo = e, hi = cnt - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sk[mid] > v) hi = mid - 1; else lo = mid;
    }
    return lo;
}

// Packed rank keys, one 64-bit word per staged position, for the common
// widths: 1 = x_1 << 32 | id (32-bit keys, k = 2: the id completes the
// key), 2 = x_1 << 32 | x_2 (32-bit keys, k = 3), 3 = x_1 (64-bit keys,
// k = 2); ties of forms 2 and 3 go to the id.  0: tail words as staged.
template <typename KW, int TK>
__host__ __device__ constexpr int packed_form() {
    return (sizeof(KW) == 4 && TK == 1) ? 1 : (sizeof(KW) == 4 && TK == 2) ? 2 : (sizeof(KW) == 8 && TK == 1) ? 3 : 0;
}

// A tile range holds whole runs.  Bounds: warp w takes staged positions
// [w * RT_CAP / 8, ...) as rows of 32; a run's first and last positions
// come from ballots of the "differs from the previous / next position"
// flags, carried from row to row (and found by bisection once per warp for
// a run entering or leaving its span).  Ranking: row R goes to warp R mod
// 8, so that a long run is shared by all warps.
template <typename KW, int TK>
__global__ void __launch_bounds__(256) k_run_tiles(const int64_t* __restrict__ count_ptr, const KW* __restrict__ key0,
                                                   const uint2* __restrict__ range, uint32_t* __restrict__ ids,
                                                   KW* __restrict__ T, int64_t tstride, int tk,
                                                   int* __restrict__ err) {
    constexpr int ROWS = RT_CAP / 256;  // rows per warp
    constexpr int SPAN = ROWS * 32;     // positions per warp for the bounds
    constexpr int PF = packed_form<KW, TK>();
    extern __shared__ __align__(16) unsigned char rt_smem[];
    KW* sk = reinterpret_cast<KW*>(rt_smem);                                // [RT_CAP] x_0, then packed bounds
    uint64_t* pk = reinterpret_cast<uint64_t*>(sk + RT_CAP);                // [RT_CAP] packed keys (PF > 0)
    KW* st = sk + RT_CAP;                                                   // [tk][RT_CAP] tail words (PF == 0)
    uint32_t* sid = PF ? reinterpret_cast<uint32_t*>(pk + RT_CAP)          // [RT_CAP]
                       : reinterpret_cast<uint32_t*>(st + (size_t)tk * RT_CAP);
    uint32_t* sb = reinterpret_cast<uint32_t*>(sk);                         // [RT_CAP] first | last << 16
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t le = lt | (1u << lane), ge = ~lt;
    const int wb = warp * SPAN;
    const int64_t n = *count_ptr;
    const int64_t ntiles = (n + RT_TILE - 1) / RT_TILE;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint2 R = range[t];
        const int64_t base = R.x;
        const int64_t span = (int64_t)R.y - (int64_t)R.x;
        int cnt = (int)span;
        if (span < 0 || span > RT_CAP || (int64_t)R.y > n) {
            if (tid == 0) atomicOr(err, ERR_INTERNAL);
            cnt = 0;
        }
        if (cnt <= 1) continue;  // (uniform over the block)
        for (int e = tid; e < cnt; e += 256) {
            const int64_t g = base + e;
            sk[e] = key0[g];
            const uint32_t id = ids[g];
            if constexpr (PF == 1) {
                pk[e] = ((uint64_t)(uint32_t)T[g] << 32) | id;
            } else if constexpr (PF == 2) {
                pk[e] = ((uint64_t)(uint32_t)T[g] << 32) | (uint32_t)T[tstride + g];
                sid[e] = id;
            } else if constexpr (PF == 3) {
                pk[e] = (uint64_t)T[g];
                sid[e] = id;
            } else {
                sid[e] = id;
                for (int d = 0; d < tk; ++d) st[d * RT_CAP + e] = T[d * tstride + g];
            }
        }
        __syncthreads();
        int fs[ROWS], ls[ROWS];
        {
            int carry = wb;  // first position of the run holding the warp's first position
            if (wb > 0 && wb < cnt && sk[wb - 1] == sk[wb]) carry = staged_first<KW>(sk, wb);
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const int e = wb + r * 32 + lane;
                const bool head = e >= cnt || e == 0 || sk[e - 1] != sk[e];
                const uint32_t hb = __ballot_sync(0xffffffffu, head);
                const uint32_t m = hb & le;
                fs[r] = m ? wb + r * 32 + 31 - __clz(m) : carry;
                if (hb) carry = wb + r * 32 + 31 - __clz(hb);
            }
        }
        {
            const int wl = wb + SPAN - 1 < cnt - 1 ? wb + SPAN - 1 : cnt - 1;  // the warp's last position
            int carry = wl;  // last position of the run holding it
            if (wl >= wb && wl + 1 < cnt && sk[wl + 1] == sk[wl]) carry = staged_last<KW>(sk, cnt, wl);
#pragma unroll
            for (int r = ROWS - 1; r >= 0; --r) {
                const int e = wb + r * 32 + lane;
                const bool tail = e >= cnt - 1 || sk[e + 1] != sk[e];
                const uint32_t tb = __ballot_sync(0xffffffffu, tail);
                const uint32_t m = tb & ge;
                ls[r] = m ? wb + r * 32 + __ffs(m) - 1 : carry;
                if (tb) carry = wb + r * 32 + __ffs(tb) - 1;
            }
        }
        __syncthreads();  // every read of x_0 is done: the bounds replace it
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int e = wb + r * 32 + lane;
            if (e < cnt) sb[e] = (uint32_t)fs[r] | ((uint32_t)ls[r] << 16);
        }
        __syncthreads();
        // every global read of the staged positions precedes the barriers
        // above, so each position is written as soon as it is ranked
#pragma unroll 1
        for (int q = 0; q < ROWS; ++q) {
            const int e = (q * 8 + warp) * 32 + lane;
            if (e >= cnt) continue;
            const uint32_t bnd = sb[e];
            const int f0 = (int)(bnd & 0xffffu), f1 = (int)(bnd >> 16);
            if (f1 == f0) continue;
            if constexpr (PF == 1) {
                const uint64_t a = pk[e];
                uint32_t r = 0;
#pragma unroll 4
                for (int j = f0; j <= f1; ++j) r += pk[j] < a ? 1u : 0u;
                const int64_t o = base + f0 + r;
                if (o != base + e) {
                    ids[o] = (uint32_t)a;
                    T[o] = (KW)(uint32_t)(a >> 32);
                }
            } else if constexpr (PF == 2 || PF == 3) {
                const uint64_t a = pk[e];
                const uint32_t ia = sid[e];
                uint32_t r = 0, eq = 0;
#pragma unroll 4
                for (int j = f0; j <= f1; ++j) {
                    const uint64_t b = pk[j];
                    r += b < a ? 1u : 0u;
                    eq += b == a ? 1u : 0u;
                }
                if (eq > 1) {  // equal tuples (besides itself): index order among them
                    for (int j = f0; j <= f1; ++j) r += (pk[j] == a && sid[j] < ia) ? 1u : 0u;
                }
                const int64_t o = base + f0 + r;
                if (o != base + e) {
                    ids[o] = ia;
                    if constexpr (PF == 2) {
                        T[o] = (KW)(uint32_t)(a >> 32);
                        T[tstride + o] = (KW)(uint32_t)a;
                    } else {
                        T[o] = (KW)a;
                    }
                }
            } else {
                const int o = f0 + (int)run_rank<KW, TK>(st, RT_CAP, sid, tk, f0, f1, e);
                if (o != e) {
                    ids[base + o] = sid[e];
                    for (int d = 0; d < tk; ++d) T[d * tstride + base + o] = st[d * RT_CAP + e];
                }
            }
        }
        __syncthreads();  // the stage is reused by the next tile
    }
}

template <typename KW>
__global__ void __launch_bounds__(256) k_run_cross(const uint32_t* __restrict__ run_meta,
                                                   const uint2* __restrict__ runs, int64_t max_count,
                                                   uint32_t* __restrict__ ids, KW* __restrict__ T, int64_t tstride,
                                                   int tk, int rmax) {
    extern __shared__ __align__(16) unsigned char rc_smem[];
    KW* st = reinterpret_cast<KW*>(rc_smem);                              // [tk][rmax]
    uint32_t* sid = reinterpret_cast<uint32_t*>(st + (size_t)tk * rmax);  // [rmax]
    const int tid = threadIdx.x;
    const uint32_t nr = run_meta[3];
    for (uint32_t r = blockIdx.x; r < nr; r += gridDim.x) {
        const uint2 R = runs[r];
        const int L = R.y <= (uint32_t)rmax && (int64_t)R.x + R.y <= max_count ? (int)R.y : 0;
        for (int i = tid; i < L; i += 256) {
            sid[i] = ids[R.x + i];
            for (int d = 0; d < tk; ++d) st[d * rmax + i] = T[d * tstride + R.x + i];
        }
        __syncthreads();
        // every read of the run precedes the barrier: positions are written as ranked
        for (int i = tid; i < L; i += 256) {
            const uint32_t o = run_rank<KW, 0>(st, rmax, sid, tk, 0, L - 1, i);
            ids[R.x + o] = sid[i];
            for (int d = 0; d < tk; ++d) T[d * tstride + R.x + o] = st[d * rmax + i];
        }
        __syncthreads();  // the stage is reused by the next run
    }
}

// -------------------------------------------------------------- records
// rec[d][p][i]: rank in super-key-p order of the tuple at position i of index
// array d.  After deduplication super keys are unique, so comparing super
// keys equals comparing these ranks.  The chain sorts write most planes,
// the permutation below the rest; an array's own plane is its position.
// Array 0's own rank plane: rec[0][0][i] = i.  (The other arrays' own
// planes are never read: a level pass moves array d >= 1 without its rank
// in super key d.)
__global__ void __launch_bounds__(256) k_own_ranks(const int64_t* __restrict__ m_ptr, int k, AllPlanes rec) {
    const int64_t m = *m_ptr;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        rec.p[0][0][i] = (uint32_t)i;
}

// Permutation by destination index, in two streaming steps: a sort pass on
// the top bits of the destination (digit bases below) groups the elements
// into destination ranges small enough to stay in L2, then k_perm_scatter
// writes each element to its destination.  Destinations are a permutation
// of [0, m), so range d holds min(2^shift, m - d * 2^shift) elements.
__global__ void k_perm_bases(const int64_t* __restrict__ m_ptr, int shift, uint32_t* __restrict__ bases) {
    __shared__ uint32_t s_warp[8];
    const int64_t m = *m_ptr;
    const int64_t lo = (int64_t)threadIdx.x << shift;
    const int64_t c = m - lo < 0 ? 0 : (m - lo > ((int64_t)1 << shift) ? ((int64_t)1 << shift) : m - lo);
    bases[threadIdx.x] = block_excl_scan256((uint32_t)c, s_warp, nullptr);
}

// Scatter of nval planes by destination: dst[j][dest[i]] = src[j][i].  Each
// thread moves PS_ITEMS elements with all their loads in flight at once.
constexpr int PS_ITEMS = 4;  // 4: 1.88 ms for the records per 2^26 step, 8: 1.93, 16: 1.96
__global__ void __launch_bounds__(256) k_perm_scatter(const int64_t* __restrict__ m_ptr,
                                                      const uint32_t* __restrict__ dest, int nval,
                                                      const __grid_constant__ PayloadArgs pa) {
    const int64_t m = *m_ptr;
    const int64_t base = (int64_t)blockIdx.x * 256 * PS_ITEMS + threadIdx.x;
    if (base >= m) return;
    uint32_t d[PS_ITEMS];
#pragma unroll
    for (int e = 0; e < PS_ITEMS; ++e) {
        const int64_t i = base + (int64_t)e * 256;
        d[e] = i < m ? dest[i] : 0xffffffffu;
    }
    for (int j = 0; j < nval; ++j) {
        uint32_t v[PS_ITEMS];
#pragma unroll
        for (int e = 0; e < PS_ITEMS; ++e) {
            const int64_t i = base + (int64_t)e * 256;
            v[e] = i < m ? pa.src[j][i] : 0u;
        }
#pragma unroll
        for (int e = 0; e < PS_ITEMS; ++e)
            if ((int64_t)d[e] < m) pa.dst[j][d[e]] = v[e];  // an inconsistent destination is never written
    }
}

// Tuple ids of array d (for checking the presort): out[d*m + i] =
// perm0[rec[d][0][off + i]] - in_off, per cloud (single cloud here).
__global__ void k_arrays_out(const int64_t* __restrict__ m_ptr, int k, AllPlanes rec,
                             const uint32_t* __restrict__ perm0, int32_t* __restrict__ out) {
    const int64_t m = *m_ptr;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m * k;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(i / m);
        const int64_t j = i - (int64_t)d * m;
        const uint32_t r0 = rec.p[d][0][j];
        out[i] = (int64_t)r0 < m ? (int32_t)perm0[r0] : -1;
    }
}

// ------------------------------------------------------------ launchers
static int grid_for(int64_t work, int per_block, int cap) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// Largest dynamic shared memory of k_transform: histogram rows for k = 8
// 64-bit keys plus 2 cloud-id digit rows, and the 256-point coordinate tile.
constexpr size_t TRANSFORM_SMEM_MAX = (size_t)(MAXK * 8 + 4) * RADIX * 4 + 256 * MAXK * 8;

// Concatenation of device clouds: block b copies the 32-bit words of the
// clouds whose descriptors it strides over (src, words, destination word).
__global__ void __launch_bounds__(256) k_pack_clouds(const PackDesc* __restrict__ d, int count,
                                                     uint32_t* __restrict__ dst) {
    for (int c = blockIdx.x; c < count; c += gridDim.x) {
        const PackDesc e = d[c];
        const uint32_t* src = static_cast<const uint32_t*>(e.src);
        for (int64_t i = threadIdx.x; i < e.words; i += 256) dst[e.dst_word + i] = src[i];
    }
}

cudaError_t launch_pack_clouds(const PackDesc* d, int count, void* dst, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    k_pack_clouds<<<std::min(count, 152 * 16), 256, 0, s>>>(d, count, static_cast<uint32_t*>(dst));
    return cudaGetLastError();
}

cudaError_t launch_transform(int dtype, const void* coords, int64_t n, int k, void* keys, int64_t stride, void* tail,
                             const int64_t* cloud_start, int ncloud, uint32_t* cloud_plane,
                             int cloud_digits, uint32_t* hist, int* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int D = dtype == 1 ? 8 : 4;
    const size_t tsz = dtype == 1 ? 8 : 4;
    const size_t smem = (size_t)(k * D + cloud_digits) * RADIX * 4 + 256 * k * tsz;
    if (smem > TRANSFORM_SMEM_MAX) return cudaErrorInvalidValue;
    const int grid = grid_for(n, 256, 152 * 8);
    if (dtype == 0)
        k_transform<int32_t, uint32_t><<<grid, 256, smem, s>>>((const int32_t*)coords, n, k, (uint32_t*)keys, stride,
                                                              (uint32_t*)tail, cloud_start, ncloud, cloud_plane, cloud_digits, hist, err);
    else if (dtype == 1)
        k_transform<int64_t, uint64_t><<<grid, 256, smem, s>>>((const int64_t*)coords, n, k, (uint64_t*)keys, stride,
                                                              (uint64_t*)tail, cloud_start, ncloud, cloud_plane, cloud_digits, hist, err);
    else
        k_transform<float, uint32_t><<<grid, 256, smem, s>>>((const float*)coords, n, k, (uint32_t*)keys, stride,
                                                            (uint32_t*)tail, cloud_start, ncloud, cloud_plane, cloud_digits, hist, err);
    return cudaGetLastError();
}

// Status area of the sort passes, reused by every pass (u32 words, regions
// 16-byte aligned): tile counts [tiles][256] | tile offsets [tiles][256] |
// chunk flags [chunks] | chunk aggregates [chunks][256] | chunk inclusive
// prefixes [chunks][256] | scan and move tile counters.  Sized for the
// smallest tile.
struct SortStatusArea {
    uint32_t *cnt, *offs, *flags, *agg, *inc, *ctrs;
    int64_t nchunks;
};
static SortStatusArea sort_status_layout(int64_t max_count, uint32_t* status) {
    const int64_t tiles = pad4((max_count + RS_TILE_MIN - 1) / RS_TILE_MIN);
    const int64_t chunks = pad4((tiles + RS_CHUNK - 1) / RS_CHUNK);
    SortStatusArea A;
    A.cnt = status;
    A.offs = A.cnt + tiles * RADIX;
    A.flags = A.offs + tiles * RADIX;
    A.agg = A.flags + chunks;
    A.inc = A.agg + chunks * RADIX;
    A.ctrs = A.inc + chunks * RADIX;
    A.nchunks = chunks;
    return A;
}
size_t sort_status_words(int64_t max_count) {
    const int64_t tiles = pad4((max_count + RS_TILE_MIN - 1) / RS_TILE_MIN);
    const int64_t chunks = pad4((tiles + RS_CHUNK - 1) / RS_CHUNK);
    return (size_t)(2 * tiles * RADIX + chunks + 2 * chunks * RADIX + 4);
}

// Resident blocks per SM of the move kernels (by variant) and the SM count.
static int g_rs_occ[5];
static int g_rs_sms = 0;

template <typename KW, int TILE, int SP>
static cudaError_t rs_pass(const int64_t* count_ptr, int64_t max_count, const void* key_src, void* key_dst,
                           const PayloadArgs& pay, const uint32_t* digit_base, int shift, const SortStatusArea& A,
                           int occ, int* err, uint32_t spin_limit, int withhold, cudaStream_t s) {
    const int64_t tiles = (max_count + TILE - 1) / TILE;
    const int64_t chunks = (tiles + RS_CHUNK - 1) / RS_CHUNK;
    cudaError_t e = launch_dependent(k_rs_count<KW, TILE>, dim3((unsigned)((tiles + RS_CT - 1) / RS_CT)), dim3(256), 0,
                                     s, count_ptr, (const KW*)key_src, shift, A.cnt, A.flags, (int)A.nchunks, A.ctrs);
    if (e != cudaSuccess) return e;
    e = launch_dependent(k_rs_scan, dim3((unsigned)chunks), dim3(256), 0, s, count_ptr, TILE,
                                     (const uint32_t*)A.cnt, digit_base, A.offs, A.flags, A.agg, A.inc, A.ctrs,
                                     A.ctrs + 1, err, spin_limit, withhold);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)g_rs_sms * occ);
    e = launch_dependent(k_rs_move<KW, TILE, SP>, dim3((unsigned)grid), dim3(RS_BLOCK), rs_move_smem<KW, TILE, SP>(),
                         s, count_ptr, (const KW*)key_src, (KW*)key_dst, pay, (const uint32_t*)A.offs, shift,
                         A.ctrs + 1, err);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// One stable LSD pass over *count_ptr (<= max_count) elements on digit
// (key >> shift) & 255: keys from key_src (written to key_dst when not
// NULL), payload planes moved along (a NULL source means the position).
// Key, payload and plane buffers must be 16-byte aligned and readable up to
// the count rounded up to a multiple of 4 elements.  spin_limit bounds the
// scan's look-back polls; withhold is the failure-detection tests' switch
// (k_rs_scan).
cudaError_t launch_sort_pass(int key64, const int64_t* count_ptr, int64_t max_count, const void* key_src,
                             void* key_dst, const PayloadArgs& pay, const uint32_t* digit_base, int shift,
                             uint32_t* status, int* err, cudaStream_t s, uint32_t spin_limit, int withhold) {
    if (max_count == 0) return cudaSuccess;
    if (g_rs_sms == 0) return cudaErrorInvalidValue;
    const SortStatusArea A = sort_status_layout(max_count, status);
    const bool many = pay.n > 1;
    if (!key64 && pay.n >= 3)
        return rs_pass<uint32_t, 2048, 3>(count_ptr, max_count, key_src, key_dst, pay, digit_base, shift, A,
                                          g_rs_occ[4], err, spin_limit, withhold, s);
    if (key64)
        return many ? rs_pass<uint64_t, 1024, 4>(count_ptr, max_count, key_src, key_dst, pay, digit_base, shift, A,
                                                 g_rs_occ[3], err, spin_limit, withhold, s)
                    : rs_pass<uint64_t, 2048, 1>(count_ptr, max_count, key_src, key_dst, pay, digit_base, shift, A,
                                                 g_rs_occ[2], err, spin_limit, withhold, s);
    return many ? rs_pass<uint32_t, 2048, 2>(count_ptr, max_count, key_src, key_dst, pay, digit_base, shift, A,
                                             g_rs_occ[1], err, spin_limit, withhold, s)
                : rs_pass<uint32_t, 2048, 1>(count_ptr, max_count, key_src, key_dst, pay, digit_base, shift, A,
                                             g_rs_occ[0], err, spin_limit, withhold, s);
}

template <typename KW, int TILE, int SP>
static cudaError_t init_rs_move(int* occ) {
    const size_t smem = rs_move_smem<KW, TILE, SP>();
    cudaError_t e = cudaFuncSetAttribute((const void*)k_rs_move<KW, TILE, SP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int o = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_rs_move<KW, TILE, SP>, RS_BLOCK, smem);
    *occ = o > 0 ? o : 1;
    return e;
}

cudaError_t init_presort_kernels() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set((const void*)k_transform<int32_t, uint32_t>, TRANSFORM_SMEM_MAX);
    set((const void*)k_transform<int64_t, uint64_t>, TRANSFORM_SMEM_MAX);
    set((const void*)k_transform<float, uint32_t>, TRANSFORM_SMEM_MAX);
    set((const void*)k_run_tiles<uint32_t, 0>, run_tile_smem(0, MAXK - 1));
    set((const void*)k_run_tiles<uint32_t, 1>, run_tile_smem(0, 1));
    set((const void*)k_run_tiles<uint32_t, 2>, run_tile_smem(0, 2));
    set((const void*)k_run_tiles<uint32_t, 3>, run_tile_smem(0, 3));
    set((const void*)k_run_tiles<uint64_t, 0>, run_tile_smem(1, MAXK - 1));
    set((const void*)k_run_tiles<uint64_t, 1>, run_tile_smem(1, 1));
    set((const void*)k_run_tiles<uint64_t, 2>, run_tile_smem(1, 2));
    for (int key64 = 0; key64 < 2; ++key64) {
        size_t most = 0;  // the largest stage over every tuple width
        for (int tk = 1; tk < MAXK; ++tk) most = std::max(most, run_cross_smem(key64, tk, run_block_max(key64, tk)));
        set(key64 ? (const void*)k_run_cross<uint64_t> : (const void*)k_run_cross<uint32_t>, most);
    }
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_rs_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = init_rs_move<uint32_t, 2048, 1>(&g_rs_occ[0]);
    if (e == cudaSuccess) e = init_rs_move<uint32_t, 2048, 2>(&g_rs_occ[1]);
    if (e == cudaSuccess) e = init_rs_move<uint64_t, 2048, 1>(&g_rs_occ[2]);
    if (e == cudaSuccess) e = init_rs_move<uint64_t, 1024, 4>(&g_rs_occ[3]);
    if (e == cudaSuccess) e = init_rs_move<uint32_t, 2048, 3>(&g_rs_occ[4]);
    return e;
}

cudaError_t launch_gather(int key64, const int64_t* count_ptr, int64_t max_count, const void* plane,
                          const uint32_t* ids, void* out, int* err, cudaStream_t s) {
    constexpr int GI = 8;
    const int64_t blocks = (max_count + 256 * GI - 1) / (256 * GI);
    if (blocks == 0) return cudaSuccess;
    if (key64)
        k_gather<uint64_t, GI><<<(unsigned)blocks, 256, 0, s>>>(count_ptr, (const uint64_t*)plane, ids, max_count,
                                                               (uint64_t*)out, err);
    else
        k_gather<uint32_t, GI><<<(unsigned)blocks, 256, 0, s>>>(count_ptr, (const uint32_t*)plane, ids, max_count,
                                                               (uint32_t*)out, err);
    return cudaGetLastError();
}

cudaError_t launch_digit_bases(const uint32_t* hist, int nrows, uint32_t* bases, cudaStream_t s) {
    if (nrows == 0) return cudaSuccess;
    k_digit_bases<<<nrows, RADIX, 0, s>>>(hist, bases);
    return cudaGetLastError();
}

// Scratch words dedup needs: keep bits, tile counts, tile offsets.
size_t dedup_scratch_words(int64_t n) {
    const int64_t tiles = (n + DEDUP_TILE - 1) / DEDUP_TILE;
    return (size_t)((n + 31) / 32) + 2 * (size_t)tiles + 4;
}

cudaError_t launch_dedup(int key64, int64_t n, const void* key0, const uint32_t* ids, const void* T, int64_t tstride,
                         int k, const uint32_t* cloud_plane, int cloud_digits, uint32_t* ids_out, void* y1_out,
                         void* y2_out, uint32_t* scratch, int64_t* m_out, uint32_t* hist,
                         int32_t* mcloud, int* err, cudaStream_t s) {
    const int64_t tiles = (n + DEDUP_TILE - 1) / DEDUP_TILE;
    if (tiles == 0) return cudaSuccess;
    uint32_t* keepbits = scratch;
    uint32_t* tcnt = keepbits + (n + 31) / 32;
    uint32_t* toff = tcnt + tiles;
#define KD_DEDUP(KW)                                                                                          \
    if (k <= 3)                                                                                               \
        k_dedup_flags<KW, 2><<<(unsigned)tiles, 256, 0, s>>>(n, (const KW*)key0, ids, (const KW*)T, tstride, k, \
                                                             cloud_plane, cloud_digits, keepbits, tcnt, hist,   \
                                                             mcloud, err);                                      \
    else                                                                                                      \
        k_dedup_flags<KW, MAXK - 1><<<(unsigned)tiles, 256, 0, s>>>(n, (const KW*)key0, ids, (const KW*)T,      \
                                                                    tstride, k, cloud_plane, cloud_digits,      \
                                                                    keepbits, tcnt, hist, mcloud, err);         \
    k_tile_scan<<<1, 1024, 0, s>>>(tiles, tcnt, toff, m_out);                                                 \
    k_dedup_compact<KW><<<(unsigned)tiles, 256, 0, s>>>(                                                      \
        n, ids, keepbits, toff, ids_out, (y1_out && k >= 2) ? (const KW*)T + (int64_t)(k - 2) * tstride : nullptr, \
        (y2_out && k >= 3) ? (const KW*)T + (int64_t)(k - 3) * tstride : nullptr, (KW*)y1_out, (KW*)y2_out);
    if (key64) {
        KD_DEDUP(uint64_t)
    } else {
        KD_DEDUP(uint32_t)
    }
#undef KD_DEDUP
    return cudaGetLastError();
}

// Run statistics of array 0 after its sort by x_0 alone, and the tile
// ranges and long crossing runs for launch_tie_runs (run_meta 4 words,
// cleared here; range ntiles entries, cross_runs ntiles entries, ntiles =
// ceil(max_count / RT_TILE); see k_run_stats).
cudaError_t launch_run_stats(int key64, const int64_t* count_ptr, int64_t max_count, const void* key0, int tk,
                             uint2* range, uint2* cross_runs, uint32_t* run_meta, cudaStream_t s) {
    const int rmax = run_block_max(key64, tk);
    cudaError_t e = cudaMemsetAsync(run_meta, 0, 4 * sizeof(uint32_t), s);
    if (e != cudaSuccess || max_count < 2) return e;
    const int grid = grid_for((max_count + RT_TILE - 1) / RT_TILE, 8, 152 * 8);
    if (key64)
        k_run_stats<uint64_t><<<grid, 256, 0, s>>>(count_ptr, (const uint64_t*)key0, rmax, range, cross_runs,
                                                   run_meta);
    else
        k_run_stats<uint32_t><<<grid, 256, 0, s>>>(count_ptr, (const uint32_t*)key0, rmax, range, cross_runs,
                                                   run_meta);
    return cudaGetLastError();
}

size_t run_tile_count(int64_t max_count) { return (size_t)((max_count + RT_TILE - 1) / RT_TILE); }

// T[d][i] (plane stride tstride words) = tail word d of the tuple ids[i].
cudaError_t launch_tail_gather(int key64, const int64_t* count_ptr, int64_t max_count, const uint32_t* ids,
                               const void* tail, int tk, void* T, int64_t tstride, int* err, cudaStream_t s) {
    if (max_count == 0 || tk < 1) return cudaSuccess;
    const int64_t blocks = (max_count + 256 * TG_ITEMS - 1) / (256 * TG_ITEMS);
    if (key64)
        k_tail_gather<uint64_t><<<(unsigned)blocks, 256, 0, s>>>(count_ptr, ids, (const uint64_t*)tail, tk, max_count,
                                                                 (uint64_t*)T, tstride, err);
    else
        k_tail_gather<uint32_t><<<(unsigned)blocks, 256, 0, s>>>(count_ptr, ids, (const uint32_t*)tail, tk, max_count,
                                                                 (uint32_t*)T, tstride, err);
    return cudaGetLastError();
}

template <typename KW, int TK>
static void run_tiles_as(int grid, size_t smem, const int64_t* count_ptr, const void* key0, const uint2* range,
                         uint32_t* ids, void* T, int64_t tstride, int tk, int* err, cudaStream_t s) {
    k_run_tiles<KW, TK><<<grid, 256, smem, s>>>(count_ptr, (const KW*)key0, range, ids, (KW*)T, tstride, tk, err);
}

// Orders every run of equal x_0 (ids and the T planes, in place) by the
// tail words and then the id: the tile ranges and listed runs of
// launch_run_stats, which must have found no run above run_block_max
// positions.
cudaError_t launch_tie_runs(int key64, const int64_t* count_ptr, int64_t max_count, const void* key0, uint32_t* ids,
                            void* T, int64_t tstride, int tk, const uint2* range, const uint2* cross_runs,
                            const uint32_t* run_meta, int* err, cudaStream_t s) {
    if (max_count < 2 || tk < 1) return cudaSuccess;
    const int rmax = run_block_max(key64, tk);
    const int tgrid = grid_for((max_count + RT_TILE - 1) / RT_TILE, 1, 152 * 8);
    const int cgrid = grid_for(max_count / RT_TILE + 1, 1, 152 * 4);
    const size_t tsm = run_tile_smem(key64, tk);
    if (key64) {
        if (tk == 1) run_tiles_as<uint64_t, 1>(tgrid, tsm, count_ptr, key0, range, ids, T, tstride, tk, err, s);
        else if (tk == 2) run_tiles_as<uint64_t, 2>(tgrid, tsm, count_ptr, key0, range, ids, T, tstride, tk, err, s);
        else run_tiles_as<uint64_t, 0>(tgrid, tsm, count_ptr, key0, range, ids, T, tstride, tk, err, s);
        k_run_cross<uint64_t><<<cgrid, 256, run_cross_smem(1, tk, rmax), s>>>(run_meta, cross_runs, max_count, ids,
                                                                              (uint64_t*)T, tstride, tk, rmax);
    } else {
        if (tk == 1) run_tiles_as<uint32_t, 1>(tgrid, tsm, count_ptr, key0, range, ids, T, tstride, tk, err, s);
        else if (tk == 2) run_tiles_as<uint32_t, 2>(tgrid, tsm, count_ptr, key0, range, ids, T, tstride, tk, err, s);
        else if (tk == 3) run_tiles_as<uint32_t, 3>(tgrid, tsm, count_ptr, key0, range, ids, T, tstride, tk, err, s);
        else run_tiles_as<uint32_t, 0>(tgrid, tsm, count_ptr, key0, range, ids, T, tstride, tk, err, s);
        k_run_cross<uint32_t><<<cgrid, 256, run_cross_smem(0, tk, rmax), s>>>(run_meta, cross_runs, max_count, ids,
                                                                              (uint32_t*)T, tstride, tk, rmax);
    }
    return cudaGetLastError();
}

cudaError_t launch_own_ranks(const int64_t* m_ptr, int64_t max_m, int k, const AllPlanes& rec, cudaStream_t s) {
    if (max_m == 0) return cudaSuccess;
    k_own_ranks<<<grid_for(max_m, 256, 152 * 16), 256, 0, s>>>(m_ptr, k, rec);
    return cudaGetLastError();
}

cudaError_t launch_perm_bases(const int64_t* m_ptr, int shift, uint32_t* bases, cudaStream_t s) {
    k_perm_bases<<<1, 256, 0, s>>>(m_ptr, shift, bases);
    return cudaGetLastError();
}

cudaError_t launch_perm_scatter(const int64_t* m_ptr, int64_t max_m, const uint32_t* dest, const PayloadArgs& pa,
                                cudaStream_t s) {
    if (max_m == 0) return cudaSuccess;
    const int64_t blocks = (max_m + 256 * PS_ITEMS - 1) / (256 * PS_ITEMS);
    k_perm_scatter<<<(unsigned)blocks, 256, 0, s>>>(m_ptr, dest, pa.n, pa);
    return cudaGetLastError();
}

cudaError_t launch_arrays_out(const int64_t* m_ptr, int64_t max_m, int k, const AllPlanes& rec,
                              const uint32_t* perm0, int32_t* out, cudaStream_t s) {
    if (max_m == 0) return cudaSuccess;
    k_arrays_out<<<grid_for(max_m * k, 256, 152 * 16), 256, 0, s>>>(m_ptr, k, rec, perm0, out);
    return cudaGetLastError();
}

}  // namespace kd

// kd_presort.cu -- presort kernels of the GB300 k-d tree builder.
//
// The presort of Section 2.1 (k index arrays sorted by the cyclic super keys
// x_d : x_{d+1} : ... : x_{d-1}, then one pass removing duplicate tuples) is
// computed here as:
//   k_transform   coordinates -> order-preserving unsigned key planes (SoA)
//                 plus 256-bin histograms of every key byte;
//   k_sort_pass   one stable 8-bit LSD pass (onesweep: warp match/popc
//                 ranking, decoupled look-back over tiles, smem-staged
//                 coalesced scatter).  Sorting least-significant part first
//                 over x_{k-1}, ..., x_0 leaves the index array in x:y:...
//                 order; each further array d is a stable sort of array d+1
//                 by x_d alone (ties keep the order of super key d+1, which
//                 equals super key d's order on them);
//   k_dedup       adjacent-compare of the sorted array 0 and stream
//                 compaction (Section 2.1, duplicates paragraph);
//   k_records     rank vectors: rec[d][p][i] = position, in super-key-p
//                 order, of the tuple at position i of array d.  After
//                 deduplication super keys are unique, so comparing super
//                 keys equals comparing these ranks.
#include "kd_internal.cuh"

namespace kd {

// -------------------------------------------------------------- helpers
// ------------------------------------------------------------ transform
// hist layout: row (d * D + b) for coordinate d, key byte b; then rows
// (k * D + b) for the cloud-id plane of a batch.  Dynamic smem: the block's
// histogram rows followed by a 256-point staging tile of coordinates.
template <typename T, typename KW>
__global__ void __launch_bounds__(256) k_transform(const T* __restrict__ coords, int64_t n, int k,
                                                   KW* __restrict__ keys, int64_t stride,
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

// ------------------------------------------------------------ sort pass
// One stable LSD pass over `*count_ptr` elements on digit (key >> shift) & 255.
//   MODE KEY_BUF:    key = key_src[pos]           (keys of the previous pass)
//   MODE KEY_DIRECT: key = key_src[pos]           (a key plane, identity order)
//   MODE KEY_GATHER: key = key_src[gidx[pos]]     (a key plane, by tuple id)
// Payload planes move with the key; a null source emits the source position.
// digit_base holds, per digit, the number of elements of this sort with a
// smaller digit (exclusive prefix of the digit histogram).
// Tile pipeline (8192 keys, 512 threads): load; warp multisplit ranking
// (equal-digit lane masks from 9 ballots, per-warp digit counters advanced
// by one shared-memory atomic per group); publish the tile's digit counts;
// tile-local prefix and staging of keys in digit order; look-back over
// tile-major count records; then every digit's run is written with
// consecutive addresses, keys first, then each payload plane.
struct SortStatus {
    uint32_t* flags;     // [tiles]
    uint16_t* aggrec;    // [tiles][256]
    uint32_t* increc;    // [tiles][256]
};

template <typename KW, int MODE>
__global__ void __launch_bounds__(SORT_THREADS, 2)
    k_sort_pass(const int64_t* __restrict__ count_ptr, const KW* __restrict__ key_src,
                const uint32_t* __restrict__ gidx, KW* __restrict__ key_dst, const __grid_constant__ PayloadArgs pay,
                const uint32_t* __restrict__ digit_base, int shift, SortStatus st,
                uint32_t* __restrict__ tile_ctr, int* __restrict__ err, int64_t gather_limit) {
    constexpr int IPT = sizeof(KW) == 8 ? SORT_IPT / 2 : SORT_IPT;  // 64-bit keys: half tiles
    constexpr int TILE = SORT_THREADS * IPT;
    __shared__ uint32_t s_wc[SORT_WARPS][RADIX];
    __shared__ uint32_t s_goff[RADIX];
    __shared__ uint32_t s_tstart[RADIX];
    __shared__ uint32_t s_warp[SORT_WARPS];
    __shared__ uint32_t s_tile, s_ctl;
    // s_dyn: [TILE * 8 bytes] keys, later dest | values;  then s_slot [TILE] u16
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint16_t* s_slot = reinterpret_cast<uint16_t*>(s_dyn + (size_t)TILE * 8);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
    for (int i = tid; i < SORT_WARPS * RADIX; i += SORT_THREADS) (&s_wc[0][0])[i] = 0;
    __syncthreads();
    const int64_t count = *count_ptr;
    const int64_t tile = s_tile;
    const int64_t base = tile * TILE;
    if (base >= count) return;
    const int tile_n = (int)(count - base < TILE ? count - base : (int64_t)TILE);
    const int wbase = warp * 32 * IPT;

    KW key[IPT];
    uint32_t rank[IPT];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int o = wbase + j * 32 + lane;
        key[j] = 0;
        if (o < tile_n) {
            const int64_t pos = base + o;
            if (MODE == KEY_GATHER) {
                const uint32_t id = gidx[pos];
                if ((int64_t)id < gather_limit) key[j] = key_src[id]; else atomicOr(err, ERR_INTERNAL);
            } else {
                key[j] = key_src[pos];
            }
        }
    }
    // warp multisplit: lanes with equal digits (9 bits: 8 digit bits and the
    // out-of-range marker) found by ballots; ranks follow item order
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int o = wbase + j * 32 + lane;
        const uint32_t d = (o < tile_n) ? (uint32_t)((key[j] >> shift) & 255u) : (uint32_t)RADIX;
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int bit = 0; bit < 9; ++bit) {
            const uint32_t bb = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
            peers &= ((d >> bit) & 1u) ? bb : ~bb;
        }
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader && d < RADIX) old = atomicAdd(&s_wc[warp][d], (uint32_t)__popc(peers));
        old = __shfl_sync(0xffffffffu, old, leader);
        rank[j] = old + __popc(peers & lanemask_lt());
    }
    __syncthreads();
    // threads < 256 own digit tid: tile count, published at once
    uint32_t cnt = 0;
    if (tid < RADIX) {
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) {
            const uint32_t c = s_wc[w][tid];
            s_wc[w][tid] = cnt;
            cnt += c;
        }
        if (tile == 0) st.increc[tid] = cnt;
        else st.aggrec[tile * RADIX + tid] = (uint16_t)cnt;
    }
    __syncthreads();
    if (tid == 0) publish_flag(st.flags, tile, tile == 0 ? FLAG_INC : FLAG_AGG);
    const uint32_t tstart = block_excl_scan<SORT_THREADS>(cnt, s_warp, nullptr);
    if (tid < RADIX) s_tstart[tid] = tstart;
    __syncthreads();
    // stage keys in tile order (sorted by digit); remember each item's slot
    KW* s_key = reinterpret_cast<KW*>(s_dyn);
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int o = wbase + j * 32 + lane;
        if (o < tile_n) {
            const uint32_t d = (uint32_t)((key[j] >> shift) & 255u);
            const uint32_t slot = s_tstart[d] + s_wc[warp][d] + rank[j];
            s_key[slot] = key[j];
            s_slot[o] = (uint16_t)slot;
        }
    }
    uint32_t excl = 0;
    if (tile > 0) {
        excl = block_lookback<uint16_t>(st.flags, st.aggrec, st.increc, RADIX, tile, &s_ctl, err);
        if (tid < RADIX) st.increc[tile * RADIX + tid] = excl + cnt;
        __syncthreads();
        if (tid == 0) publish_flag(st.flags, tile, FLAG_INC);
    }
    if (tid < RADIX) s_goff[tid] = digit_base[tid] + excl - tstart;  // dest = s_goff[digit] + slot (mod 2^32)
    __syncthreads();
    // A destination outside [0, count) can only come from an inconsistent
    // histogram; it is reported and never written.
    uint32_t dest[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int s = i * SORT_THREADS + tid;
        dest[i] = 0xffffffffu;
        if (s < tile_n) {
            const KW kk = s_key[s];
            const uint32_t dd = s_goff[(uint32_t)((kk >> shift) & 255u)] + (uint32_t)s;
            if ((int64_t)dd < count) {
                dest[i] = dd;
                if (key_dst) key_dst[dd] = kk;
            } else {
                atomicOr(err, ERR_INTERNAL);
            }
        }
    }
    if (pay.n == 0) return;
    __syncthreads();
    uint32_t* s_dest = reinterpret_cast<uint32_t*>(s_dyn);
    uint32_t* s_val = reinterpret_cast<uint32_t*>(s_dyn + (size_t)TILE * 4);
#pragma unroll
    for (int i = 0; i < IPT; ++i) s_dest[i * SORT_THREADS + tid] = dest[i];
    for (int p = 0; p < pay.n; ++p) {
        const uint32_t* src = pay.src[p];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const int o = wbase + j * 32 + lane;
            if (o < tile_n) {
                const int64_t pos = base + o;
                s_val[s_slot[o]] = src ? src[pos] : (uint32_t)pos;
            }
        }
        __syncthreads();
        uint32_t* dst = pay.dst[p];
        for (int s = tid; s < tile_n; s += SORT_THREADS) {
            const uint32_t dd = s_dest[s];
            if (dd != 0xffffffffu) dst[dd] = s_val[s];
        }
        __syncthreads();
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

template <typename KW>
__global__ void __launch_bounds__(256) k_dedup_flags(int64_t n, const KW* __restrict__ key0,
                                                     const uint32_t* __restrict__ ids, const KW* __restrict__ keys,
                                                     int64_t stride, int k, const uint32_t* __restrict__ cloud_plane,
                                                     int cloud_digits, uint32_t* __restrict__ keepbits,
                                                     uint32_t* __restrict__ tile_cnt, uint32_t* __restrict__ hist,
                                                     int32_t* __restrict__ mcloud, int* __restrict__ err) {
    constexpr int IPT = DEDUP_TILE / 256;
    constexpr int D = sizeof(KW);
    __shared__ uint32_t s_wsum[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * DEDUP_TILE;
    const int wbase = warp * 32 * IPT;
    uint32_t wcount = 0;
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int64_t pos = base + wbase + j * 32 + lane;
        bool keep = false;
        if (pos < n) {
            uint32_t id = ids[pos];
            if ((int64_t)id >= n) {
                atomicOr(err, ERR_INTERNAL);
                id = 0;
            }
            const KW k0 = key0[pos];
            bool dup = false;
            if (pos > 0 && key0[pos - 1] == k0 && (int64_t)ids[pos - 1] < n) {
                const uint32_t pid = ids[pos - 1];
                dup = true;
                for (int d = 1; d < k && dup; ++d)
                    if (keys[d * stride + id] != keys[d * stride + pid]) dup = false;
                if (dup && cloud_plane && cloud_plane[id] != cloud_plane[pid]) dup = false;
            }
            keep = !dup;
            if (dup) {
                for (int d = 0; d < k; ++d) {
                    const KW kd = keys[d * stride + id];
                    for (int b = 0; b < D; ++b)
                        atomicSub(&hist[(d * D + b) * RADIX + (uint32_t)((kd >> (8 * b)) & 255u)], 1u);
                }
                if (cloud_plane) {
                    const uint32_t c = cloud_plane[id];
                    for (int b = 0; b < cloud_digits; ++b)
                        atomicSub(&hist[(k * D + b) * RADIX + ((c >> (8 * b)) & 255u)], 1u);
                    atomicSub(&mcloud[c], 1);
                } else if (mcloud) {
                    atomicSub(&mcloud[0], 1);
                }
            }
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, keep);
        if (lane == 0 && base + wbase + j * 32 < n) keepbits[(base + wbase + j * 32) >> 5] = ball;
        wcount += __popc(ball);
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

__global__ void __launch_bounds__(256) k_dedup_compact(int64_t n, const uint32_t* __restrict__ ids,
                                                       const uint32_t* __restrict__ keepbits,
                                                       const uint32_t* __restrict__ offs,
                                                       uint32_t* __restrict__ ids_out) {
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
        if ((ball[j] >> lane) & 1u) ids_out[out + __popc(ball[j] & lanemask_lt())] = ids[pos];
        out += __popc(ball[j]);
    }
}

// -------------------------------------------------------------- records
// rec[d][p][i]: rank in super-key-p order of the tuple at position i of index
// array d.  After deduplication super keys are unique, so comparing super
// keys equals comparing these ranks.  The chain sorts write most planes,
// the permutation below the rest; an array's own plane is its position.
__global__ void __launch_bounds__(256) k_own_ranks(const int64_t* __restrict__ m_ptr, int k, AllPlanes rec) {
    const int64_t m = *m_ptr;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        for (int d = 0; d < k; ++d) rec.p[d][d][i] = (uint32_t)i;
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

__global__ void __launch_bounds__(256) k_perm_scatter(const int64_t* __restrict__ m_ptr,
                                                      const uint32_t* __restrict__ dest, int nval,
                                                      const __grid_constant__ PayloadArgs pa) {
    const int64_t m = *m_ptr;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t d = dest[i];
        if ((int64_t)d >= m) continue;  // inconsistent input: never written out of range
        for (int j = 0; j < nval; ++j) pa.dst[j][d] = pa.src[j][i];
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

cudaError_t launch_transform(int dtype, const void* coords, int64_t n, int k, void* keys, int64_t stride,
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
                                                              cloud_start, ncloud, cloud_plane, cloud_digits, hist, err);
    else if (dtype == 1)
        k_transform<int64_t, uint64_t><<<grid, 256, smem, s>>>((const int64_t*)coords, n, k, (uint64_t*)keys, stride,
                                                              cloud_start, ncloud, cloud_plane, cloud_digits, hist, err);
    else
        k_transform<float, uint32_t><<<grid, 256, smem, s>>>((const float*)coords, n, k, (uint32_t*)keys, stride,
                                                            cloud_start, ncloud, cloud_plane, cloud_digits, hist, err);
    return cudaGetLastError();
}

int sort_tile(int key64) { return key64 ? SORT_TILE / 2 : SORT_TILE; }
// Status words of one pass: flags [tiles] | aggregate records [tiles][256]
// u16 | inclusive records [tiles][256] u32.  Only the flags need zeroing.
// Sized for the smaller (64-bit key) tiles, which covers both key widths.
static int64_t sort_tiles_max(int64_t max_count) { return (max_count + SORT_TILE / 2 - 1) / (SORT_TILE / 2); }
size_t sort_status_words(int64_t max_count) {
    const int64_t tiles = sort_tiles_max(max_count);
    return (size_t)pad4(tiles) + (size_t)tiles * RADIX / 2 + (size_t)tiles * RADIX;
}
size_t sort_flag_words(int64_t max_count) { return (size_t)pad4(sort_tiles_max(max_count)); }

cudaError_t launch_sort_pass(int key64, int mode, const int64_t* count_ptr, int64_t max_count,
                             const void* key_src, const uint32_t* gidx, void* key_dst,
                             const PayloadArgs& pay, const uint32_t* digit_base, int shift,
                             uint32_t* status, uint32_t* tile_ctr, int* err, cudaStream_t s) {
    const int64_t gather_limit = max_count;  // tuple ids index planes of max_count entries
    const int tile = sort_tile(key64);
    const int64_t tiles = (max_count + tile - 1) / tile;
    if (tiles == 0) return cudaSuccess;
    const int64_t tmax = sort_tiles_max(max_count);
    SortStatus st;
    st.flags = status;
    st.aggrec = reinterpret_cast<uint16_t*>(status + pad4(tmax));
    st.increc = status + pad4(tmax) + tmax * RADIX / 2;
    const size_t smem = (size_t)tile * 8 + (size_t)tile * 2;
#define KD_SORT_LAUNCH(KW, MODE)                                                                          \
    do {                                                                                                  \
        auto kf = k_sort_pass<KW, MODE>;                                                                  \
        kf<<<(unsigned)tiles, SORT_THREADS, smem, s>>>(count_ptr, (const KW*)key_src, gidx, (KW*)key_dst, \
                                                       pay, digit_base, shift, st, tile_ctr, err,         \
                                                       gather_limit);                                     \
    } while (0)
    if (key64) {
        if (mode == KEY_DIRECT) KD_SORT_LAUNCH(uint64_t, KEY_DIRECT);
        else if (mode == KEY_GATHER) KD_SORT_LAUNCH(uint64_t, KEY_GATHER);
        else KD_SORT_LAUNCH(uint64_t, KEY_BUF);
    } else {
        if (mode == KEY_DIRECT) KD_SORT_LAUNCH(uint32_t, KEY_DIRECT);
        else if (mode == KEY_GATHER) KD_SORT_LAUNCH(uint32_t, KEY_GATHER);
        else KD_SORT_LAUNCH(uint32_t, KEY_BUF);
    }
#undef KD_SORT_LAUNCH
    return cudaGetLastError();
}

// Dynamic shared memory limits, set once per process at their maxima (a
// per-launch setting would race between threads launching on the same
// kernels with different sizes).
cudaError_t init_presort_kernels() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set((const void*)k_transform<int32_t, uint32_t>, TRANSFORM_SMEM_MAX);
    set((const void*)k_transform<int64_t, uint64_t>, TRANSFORM_SMEM_MAX);
    set((const void*)k_transform<float, uint32_t>, TRANSFORM_SMEM_MAX);
    const size_t s32 = (size_t)SORT_TILE * 10, s64 = (size_t)(SORT_TILE / 2) * 10;
    set((const void*)k_sort_pass<uint32_t, KEY_DIRECT>, s32);
    set((const void*)k_sort_pass<uint32_t, KEY_GATHER>, s32);
    set((const void*)k_sort_pass<uint32_t, KEY_BUF>, s32);
    set((const void*)k_sort_pass<uint64_t, KEY_DIRECT>, s64);
    set((const void*)k_sort_pass<uint64_t, KEY_GATHER>, s64);
    set((const void*)k_sort_pass<uint64_t, KEY_BUF>, s64);
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

cudaError_t launch_dedup(int key64, int64_t n, const void* key0, const uint32_t* ids, const void* keys,
                         int64_t stride, int k, const uint32_t* cloud_plane, int cloud_digits, uint32_t* ids_out,
                         uint32_t* scratch, int64_t* m_out, uint32_t* hist, int32_t* mcloud, int* err,
                         cudaStream_t s) {
    const int64_t tiles = (n + DEDUP_TILE - 1) / DEDUP_TILE;
    if (tiles == 0) return cudaSuccess;
    uint32_t* keepbits = scratch;
    uint32_t* tcnt = keepbits + (n + 31) / 32;
    uint32_t* toff = tcnt + tiles;
    if (key64)
        k_dedup_flags<uint64_t><<<(unsigned)tiles, 256, 0, s>>>(n, (const uint64_t*)key0, ids, (const uint64_t*)keys,
                                                               stride, k, cloud_plane, cloud_digits, keepbits, tcnt,
                                                               hist, mcloud, err);
    else
        k_dedup_flags<uint32_t><<<(unsigned)tiles, 256, 0, s>>>(n, (const uint32_t*)key0, ids, (const uint32_t*)keys,
                                                               stride, k, cloud_plane, cloud_digits, keepbits, tcnt,
                                                               hist, mcloud, err);
    k_tile_scan<<<1, 1024, 0, s>>>(tiles, tcnt, toff, m_out);
    k_dedup_compact<<<(unsigned)tiles, 256, 0, s>>>(n, ids, keepbits, toff, ids_out);
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
    k_perm_scatter<<<grid_for(max_m, 256, 152 * 8), 256, 0, s>>>(m_ptr, dest, pa.n, pa);
    return cudaGetLastError();
}

cudaError_t launch_arrays_out(const int64_t* m_ptr, int64_t max_m, int k, const AllPlanes& rec,
                              const uint32_t* perm0, int32_t* out, cudaStream_t s) {
    if (max_m == 0) return cudaSuccess;
    k_arrays_out<<<grid_for(max_m * k, 256, 152 * 16), 256, 0, s>>>(m_ptr, k, rec, perm0, out);
    return cudaGetLastError();
}

}  // namespace kd

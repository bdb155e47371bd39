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
// hist_row holds the 256 digit counts over all elements of this sort.
template <typename KW, int MODE, int IPT>
__global__ void __launch_bounds__(SORT_THREADS) k_sort_pass(const int64_t* __restrict__ count_ptr,
                                                            const KW* __restrict__ key_src,
                                                            const uint32_t* __restrict__ gidx,
                                                            KW* __restrict__ key_dst, PayloadArgs pay,
                                                            const uint32_t* __restrict__ hist_row, int shift,
                                                            uint32_t* __restrict__ status,
                                                            uint32_t* __restrict__ tile_ctr,
                                                            int* __restrict__ err, int64_t gather_limit) {
    constexpr int TILE = SORT_THREADS * IPT;
    __shared__ uint32_t s_wc[SORT_WARPS][RADIX];
    __shared__ uint32_t s_goff[RADIX];
    __shared__ uint32_t s_tstart[RADIX];
    __shared__ uint32_t s_warp[SORT_WARPS];
    __shared__ uint32_t s_tile;
    extern __shared__ __align__(16) unsigned char s_dyn[];

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
    // warp-level multisplit: rank among equal digits of this warp, in order
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int o = wbase + j * 32 + lane;
        const uint32_t d = (o < tile_n) ? (uint32_t)((key[j] >> shift) & 255u) : (uint32_t)RADIX;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = 0;
        if (d < RADIX) before = s_wc[warp][d];
        rank[j] = before + __popc(peers & lanemask_lt());
        __syncwarp();
        if (d < RADIX && lane == __ffs(peers) - 1) s_wc[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread tid owns digit tid: exclusive prefix over warps, tile count
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < SORT_WARPS; ++w) {
        const uint32_t c = s_wc[w][tid];
        s_wc[w][tid] = cnt;
        cnt += c;
    }
    uint32_t* st = status + tile * RADIX;
    st_volatile(st + tid, (tile == 0 ? ST_INC : ST_AGG) | cnt);
    const uint32_t hbase = block_excl_scan256(hist_row[tid], s_warp, nullptr);
    const uint32_t tstart = block_excl_scan256(cnt, s_warp, nullptr);
    uint32_t excl = 0;
    if (tile > 0) {
        excl = lookback(status, tile, RADIX, tid, err);
        st_volatile(st + tid, ST_INC | ((excl + cnt) & ST_COUNT));
    }
    s_tstart[tid] = tstart;
    s_goff[tid] = hbase + excl - tstart;  // dest = s_goff[digit] + slot (mod 2^32)
    __syncthreads();

    // stage keys in tile order (sorted by digit), then write runs out
    KW* s_key = reinterpret_cast<KW*>(s_dyn);
    uint32_t slot[IPT];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int o = wbase + j * 32 + lane;
        if (o < tile_n) {
            const uint32_t d = (uint32_t)((key[j] >> shift) & 255u);
            slot[j] = s_tstart[d] + s_wc[warp][d] + rank[j];
            s_key[slot[j]] = key[j];
        }
    }
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
    uint32_t* s_val = reinterpret_cast<uint32_t*>(s_dyn);
    for (int p = 0; p < pay.n; ++p) {
        __syncthreads();
        const uint32_t* src = pay.src[p];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const int o = wbase + j * 32 + lane;
            if (o < tile_n) {
                const int64_t pos = base + o;
                s_val[slot[j]] = src ? src[pos] : (uint32_t)pos;
            }
        }
        __syncthreads();
        uint32_t* dst = pay.dst[p];
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int s = i * SORT_THREADS + tid;
            if (s < tile_n && dest[i] != 0xffffffffu) dst[dest[i]] = s_val[s];
        }
    }
}

// ---------------------------------------------------------------- dedup
// keep[i] = i is the first of its run of identical tuples (same cloud) in
// the array sorted by super key 0; kept ids are compacted in order.  Each
// dropped tuple's key bytes are subtracted from the histograms so that they
// describe the kept tuples for the sorts that follow.
template <typename KW>
__global__ void __launch_bounds__(256) k_dedup(int64_t n, const KW* __restrict__ key0,
                                               const uint32_t* __restrict__ ids, const KW* __restrict__ keys,
                                               int64_t stride, int k,
                                               const uint32_t* __restrict__ cloud_plane, int cloud_digits,
                                               uint32_t* __restrict__ ids_out, uint32_t* __restrict__ status,
                                               uint32_t* __restrict__ tile_ctr, int64_t* __restrict__ m_out,
                                               uint32_t* __restrict__ hist, int32_t* __restrict__ mcloud,
                                               int* __restrict__ err) {
    constexpr int IPT = 16;
    constexpr int TILE = 256 * IPT;
    constexpr int D = sizeof(KW);
    __shared__ uint32_t s_tile, s_excl, s_wsum[8], s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * TILE;
    if (base >= n) return;
    const int tile_n = (int)(n - base < TILE ? n - base : (int64_t)TILE);
    const int wbase = warp * 32 * IPT;
    uint32_t ball[IPT];
    uint32_t id[IPT];
    uint32_t wcount = 0;
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int o = wbase + j * 32 + lane;
        bool keep = false;
        id[j] = 0;
        if (o < tile_n) {
            const int64_t pos = base + o;
            id[j] = ids[pos];
            if ((int64_t)id[j] >= n) {
                atomicOr(err, ERR_INTERNAL);
                id[j] = 0;
            }
            const KW k0 = key0[pos];
            bool dup = false;
            if (pos > 0 && key0[pos - 1] == k0 && (int64_t)ids[pos - 1] < n) {
                const uint32_t pid = ids[pos - 1];
                dup = true;
                for (int d = 1; d < k && dup; ++d)
                    if (keys[d * stride + id[j]] != keys[d * stride + pid]) dup = false;
                if (dup && cloud_plane && cloud_plane[id[j]] != cloud_plane[pid]) dup = false;
            }
            keep = !dup;
            if (dup) {
                for (int d = 0; d < k; ++d) {
                    const KW kd = keys[d * stride + id[j]];
                    for (int b = 0; b < D; ++b)
                        atomicSub(&hist[(d * D + b) * RADIX + (uint32_t)((kd >> (8 * b)) & 255u)], 1u);
                }
                if (cloud_plane) {
                    const uint32_t c = cloud_plane[id[j]];
                    for (int b = 0; b < cloud_digits; ++b)
                        atomicSub(&hist[(k * D + b) * RADIX + ((c >> (8 * b)) & 255u)], 1u);
                    atomicSub(&mcloud[c], 1);
                } else if (mcloud) {
                    atomicSub(&mcloud[0], 1);
                }
            }
        }
        ball[j] = __ballot_sync(0xffffffffu, keep);
        wcount += __popc(ball[j]);
    }
    if (lane == 0) s_wsum[warp] = wcount;
    __syncthreads();
    if (tid == 0) {
        uint32_t acc = 0;
        for (int w = 0; w < 8; ++w) {
            const uint32_t c = s_wsum[w];
            s_wsum[w] = acc;
            acc += c;
        }
        s_total = acc;
        st_volatile(status + tile, (tile == 0 ? ST_INC : ST_AGG) | acc);
        uint32_t excl = 0;
        if (tile > 0) {
            excl = lookback(status, tile, 1, 0, err);
            st_volatile(status + tile, ST_INC | ((excl + acc) & ST_COUNT));
        }
        s_excl = excl;
        if (base + tile_n == n) *m_out = (int64_t)excl + acc;
    }
    __syncthreads();
    uint32_t out = s_excl + s_wsum[warp];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        if ((ball[j] >> lane) & 1u) ids_out[out + __popc(ball[j] & lanemask_lt())] = id[j];
        out += __popc(ball[j]);
    }
}

// -------------------------------------------------------------- records
// From array 1's complete rank vectors (rec[1][p] for p != 1; its own rank
// is the position), fill every plane of every array that the chain sorts
// did not write: rec[d][d][i] = i, and rec[d][p][rank_d] = rank_p by scatter.
// Bits 8d..8d+7 of present_bits: the planes already written for array d.
__global__ void __launch_bounds__(256) k_records(const int64_t* __restrict__ m_ptr, int k,
                                                 AllPlanes rec, uint64_t present_bits) {
    const int64_t m = *m_ptr;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v[MAXK];
        for (int p = 0; p < k; ++p) v[p] = (p == 1) ? (uint32_t)i : rec.p[1][p][i];
        for (int d = 0; d < k; ++d) {
            const uint32_t present = (uint32_t)(present_bits >> (d * MAXK)) & 0xffu;
            if (!((present >> d) & 1u)) rec.p[d][d][i] = (uint32_t)i;
            if (d == 1) continue;
            const uint32_t r = v[d];
            if ((int64_t)r >= m) continue;  // inconsistent ranks: never written out of range
            for (int p = 0; p < k; ++p)
                if (p != d && !((present >> p) & 1u)) rec.p[d][p][r] = v[p];
        }
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

cudaError_t launch_transform(int dtype, const void* coords, int64_t n, int k, void* keys, int64_t stride,
                             const int64_t* cloud_start, int ncloud, uint32_t* cloud_plane,
                             int cloud_digits, uint32_t* hist, int* err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int D = dtype == 1 ? 8 : 4;
    const size_t tsz = dtype == 1 ? 8 : 4;
    const size_t smem = (size_t)(k * D + cloud_digits) * RADIX * 4 + 256 * k * tsz;
    const int grid = grid_for(n, 256, 152 * 8);
    cudaError_t e = cudaSuccess;
    if (dtype == 0) {
        auto kf = k_transform<int32_t, uint32_t>;
        e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            kf<<<grid, 256, smem, s>>>((const int32_t*)coords, n, k, (uint32_t*)keys, stride, cloud_start,
                                       ncloud, cloud_plane, cloud_digits, hist, err);
    } else if (dtype == 1) {
        auto kf = k_transform<int64_t, uint64_t>;
        e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            kf<<<grid, 256, smem, s>>>((const int64_t*)coords, n, k, (uint64_t*)keys, stride, cloud_start,
                                       ncloud, cloud_plane, cloud_digits, hist, err);
    } else {
        auto kf = k_transform<float, uint32_t>;
        e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            kf<<<grid, 256, smem, s>>>((const float*)coords, n, k, (uint32_t*)keys, stride, cloud_start,
                                       ncloud, cloud_plane, cloud_digits, hist, err);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

constexpr int SORT_IPT = 16;
int sort_tile() { return SORT_THREADS * SORT_IPT; }

cudaError_t launch_sort_pass(int key64, int mode, const int64_t* count_ptr, int64_t max_count,
                             const void* key_src, const uint32_t* gidx, void* key_dst,
                             const PayloadArgs& pay, const uint32_t* hist_row, int shift,
                             uint32_t* status, uint32_t* tile_ctr, int* err, cudaStream_t s) {
    const int64_t gather_limit = max_count;  // tuple ids index planes of max_count entries
    const int tile = SORT_THREADS * SORT_IPT;
    const int64_t tiles = (max_count + tile - 1) / tile;
    if (tiles == 0) return cudaSuccess;
    const size_t smem = (size_t)tile * (key64 ? 8 : 4);
#define KD_SORT_LAUNCH(KW, MODE)                                                                      \
    k_sort_pass<KW, MODE, SORT_IPT><<<(unsigned)tiles, SORT_THREADS, smem, s>>>(                    \
        count_ptr, (const KW*)key_src, gidx, (KW*)key_dst, pay, hist_row, shift, status, tile_ctr, err,  \
        gather_limit)
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

cudaError_t launch_dedup(int key64, int64_t n, const void* key0, const uint32_t* ids, const void* keys,
                         int64_t stride, int k, const uint32_t* cloud_plane, int cloud_digits,
                         uint32_t* ids_out, uint32_t* status, uint32_t* tile_ctr, int64_t* m_out,
                         uint32_t* hist, int32_t* mcloud, int* err, cudaStream_t s) {
    const int64_t tiles = (n + 4095) / 4096;
    if (tiles == 0) return cudaSuccess;
    if (key64)
        k_dedup<uint64_t><<<(unsigned)tiles, 256, 0, s>>>(n, (const uint64_t*)key0, ids, (const uint64_t*)keys,
                                                         stride, k, cloud_plane, cloud_digits, ids_out,
                                                         status, tile_ctr, m_out, hist, mcloud, err);
    else
        k_dedup<uint32_t><<<(unsigned)tiles, 256, 0, s>>>(n, (const uint32_t*)key0, ids, (const uint32_t*)keys,
                                                         stride, k, cloud_plane, cloud_digits, ids_out,
                                                         status, tile_ctr, m_out, hist, mcloud, err);
    return cudaGetLastError();
}

cudaError_t launch_records(const int64_t* m_ptr, int64_t max_m, int k, const AllPlanes& rec,
                           uint64_t present_bits, cudaStream_t s) {
    if (max_m == 0) return cudaSuccess;
    k_records<<<grid_for(max_m, 256, 152 * 16), 256, 0, s>>>(m_ptr, k, rec, present_bits);
    return cudaGetLastError();
}

cudaError_t launch_arrays_out(const int64_t* m_ptr, int64_t max_m, int k, const AllPlanes& rec,
                              const uint32_t* perm0, int32_t* out, cudaStream_t s) {
    if (max_m == 0) return cudaSuccess;
    k_arrays_out<<<grid_for(max_m * k, 256, 152 * 16), 256, 0, s>>>(m_ptr, k, rec, perm0, out);
    return cudaGetLastError();
}

}  // namespace kd

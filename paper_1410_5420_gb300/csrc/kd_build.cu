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
//                 segmented multisplit (warp match/popc ranking, decoupled
//                 look-back across tiles of one segment, smem-staged
//                 coalesced scatter).  With this schedule each tree level
//                 costs one pass over one array.  Elements carry their rank
//                 in every super-key order, so each compare is one integer
//                 compare (super keys are unique after deduplication).
//   k_finish      once segments hold at most a few thousand tuples, one CTA
//                 finishes a whole subtree in shared memory: per level the
//                 primary array's medians become nodes and the other arrays
//                 are stably partitioned with a segmented block scan, down
//                 to single elements (same result as the paper's 1/2/3
//                 element termination).
//   k_top_nodes   children and split dimension of the nodes above the
//                 finisher level (pure functions of m and the address).
#include "kd_internal.cuh"

namespace kd {

constexpr uint32_t INV = 0xffffffffu;

template <int K, int IPT>
__global__ void __launch_bounds__(LEVEL_THREADS)
    k_level_pass(const __grid_constant__ AllBufs bufs, int q, const LevelTile* __restrict__ tiles, int ntiles,
                 const CloudDev* __restrict__ clouds, uint32_t* __restrict__ medr,
                 const uint32_t* __restrict__ perm0, uint32_t* __restrict__ status,
                 uint32_t* __restrict__ tile_ctr, int* __restrict__ err) {
    constexpr int TILE = LEVEL_THREADS * IPT;
    constexpr int NBMAX = 1 << (K - 1);
    constexpr int NDMAX = LEVEL_NSMAX * NBMAX;
    __shared__ uint32_t s_wc[LEVEL_WARPS][NDMAX];
    __shared__ uint32_t s_cnt[NDMAX];
    __shared__ uint32_t s_tstart[NDMAX];
    __shared__ int32_t s_dbase[NDMAX];
    __shared__ uint32_t s_excl[NBMAX];
    __shared__ int32_t s_seglo[LEVEL_NSMAX], s_seghi[LEVEL_NSMAX], s_segidx[LEVEL_NSMAX];
    __shared__ int s_ns;
    __shared__ uint32_t s_tile, s_total;
    __shared__ uint32_t s_warp[LEVEL_WARPS];
    extern __shared__ __align__(16) uint32_t s_dyn[];  // s_dest[TILE] | s_val[TILE]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const int t = (int)s_tile;
    if (t >= ntiles) return;
    const LevelTile T = tiles[t];
    const CloudDev C = clouds[T.cloud];
    const int F = T.lev_out - T.lev_in;
    const int NB = 1 << F;
    const int ND = LEVEL_NSMAX * NB;
    const int32_t m = C.m;
    const int32_t pos0 = (int32_t)T.pos0;
    const int32_t pend = pos0 + T.npos - 1;
    if (tid == 0) {
        int ns = 0;
        int32_t i = pos0;
        while (i <= pend) {
            const Seg sg = segment_of(i, m, T.lev_in);
            if (sg.idx < 0) {
                ++i;
                continue;
            }
            if (ns == LEVEL_NSMAX) {
                atomicOr(err, ERR_INTERNAL);
                break;
            }
            s_seglo[ns] = sg.lo;
            s_seghi[ns] = sg.hi;
            s_segidx[ns] = sg.idx;
            ++ns;
            i = sg.hi + 1;
        }
        s_ns = ns;
    }
    for (int i = tid; i < LEVEL_WARPS * NDMAX; i += LEVEL_THREADS) (&s_wc[0][0])[i] = 0;
    __syncthreads();
    const int ns = s_ns;

    const int wbase = warp * 32 * IPT;
    const int64_t goff = C.off;
    uint32_t v[K][IPT];
    uint32_t dig[IPT];
    int32_t flo[IPT], fhi[IPT], fmid[IPT], fsi[IPT];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int o = wbase + j * 32 + lane;
        dig[j] = INV;
        flo[j] = 0;
        fhi[j] = -1;
        fmid[j] = -1;
        fsi[j] = 0;
#pragma unroll
        for (int p = 0; p < K; ++p) v[p][j] = 0;
        if (o < T.npos) {
            const int32_t pos = pos0 + o;
            // plane order rotated so that level lev_in + f reads v[f] (compile-time index)
#pragma unroll
            for (int f = 0; f < K; ++f) v[f][j] = bufs.p[q][T.src_buf][(T.lev_in + f) % K][goff + pos];
            int sj = -1;
#pragma unroll
            for (int x = 0; x < LEVEL_NSMAX; ++x)
                if (x < ns && pos >= s_seglo[x] && pos <= s_seghi[x]) sj = x;
            if (sj >= 0) {
                int32_t a = s_seglo[sj], z = s_seghi[sj], si = s_segidx[sj];
                uint32_t b = 0;
                bool drop = false;
#pragma unroll
                for (int f = 0; f < K - 1; ++f) {
                    if (f < F && !drop) {
                        const int L = T.lev_in + f;
                        const int32_t mid = a + ((z - a) >> 1);
                        const uint32_t mv = medr[C.medr_off + ((int64_t)1 << L) - 1 + si];
                        const uint32_t r = v[f][j];  // rank in super key L mod K
                        if (r < mv) {
                            z = mid - 1;
                            si = 2 * si;
                            b = 2 * b;
                        } else if (r > mv) {
                            a = mid + 1;
                            si = 2 * si + 1;
                            b = 2 * b + 1;
                        } else {
                            drop = true;  // the median of level L: a node, not copied
                        }
                    }
                }
                if (!drop) {
                    dig[j] = (uint32_t)(sj * NB) + b;
                    flo[j] = a;
                    fhi[j] = z;
                    fmid[j] = a + ((z - a) >> 1);
                    fsi[j] = si;
                }
            }
        }
    }
    // warp multisplit ranking on (segment, bucket)
    uint32_t rank[IPT];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const uint32_t d = dig[j];
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = 0;
        if (d != INV) before = s_wc[warp][d];
        rank[j] = before + __popc(peers & lanemask_lt());
        __syncwarp();
        if (d != INV && lane == __ffs(peers) - 1) s_wc[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = tid; d < ND; d += LEVEL_THREADS) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < LEVEL_WARPS; ++w) {
            const uint32_t x = s_wc[w][d];
            s_wc[w][d] = c;
            c += x;
        }
        s_cnt[d] = c;
    }
    __syncthreads();
    // look-back: only the first segment can have begun in an earlier tile;
    // each tile publishes the bucket counts of its last segment.
    const bool first_cont = ns > 0 && s_seglo[0] < pos0;
    if (tid < NB) {
        uint32_t* st = status + (int64_t)t * NBMAX;
        const uint32_t c = ns > 0 ? s_cnt[(ns - 1) * NB + tid] : 0u;
        const bool last_is_cont = (ns == 1) && first_cont;
        st_volatile(st + tid, (last_is_cont ? ST_AGG : ST_INC) | c);
        uint32_t e = 0;
        if (first_cont) {
            e = lookback(status, t, NBMAX, tid, err);
            if (last_is_cont) st_volatile(st + tid, ST_INC | ((e + c) & ST_COUNT));
        }
        s_excl[tid] = e;
    }
    {
        const int per = (ND + LEVEL_THREADS - 1) / LEVEL_THREADS;
        uint32_t loc = 0;
        for (int x = 0; x < per; ++x) {
            const int d = tid * per + x;
            if (d < ND) loc += s_cnt[d];
        }
        uint32_t tot = 0;
        uint32_t ex = block_excl_scan256(loc, s_warp, &tot);
        for (int x = 0; x < per; ++x) {
            const int d = tid * per + x;
            if (d < ND) {
                s_tstart[d] = ex;
                ex += s_cnt[d];
            }
        }
        if (tid == 0) s_total = tot;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < IPT; ++j)
        if (dig[j] != INV) {
            const uint32_t d = dig[j];
            const int sj = (int)d / NB;
            const int b = (int)d - sj * NB;
            s_dbase[d] = flo[j] + (sj == 0 ? (int32_t)s_excl[b] : 0);
        }
    __syncthreads();
    uint32_t* s_dest = s_dyn;
    uint32_t* s_val = s_dyn + TILE;
    uint32_t slot[IPT];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        slot[j] = INV;
        if (dig[j] != INV) {
            const uint32_t d = dig[j];
            const uint32_t within = s_wc[warp][d] + rank[j];
            slot[j] = s_tstart[d] + within;
            const int32_t dest = s_dbase[d] + (int32_t)within;
            // the destination must lie in the element's final segment; any
            // other value means inconsistent inputs and is never written
            const bool ok = dest >= flo[j] && dest <= fhi[j];
            if (!ok) atomicOr(err, ERR_INTERNAL);
            s_dest[slot[j]] = ok ? (uint32_t)(goff + dest) : INV;
            if (ok && T.write_med && dest == fmid[j]) {
                // the new median of level lev_out (rare: re-read its planes q and 0)
                const int64_t gsrc = goff + pos0 + wbase + j * 32 + lane;
                const uint32_t rq = bufs.p[q][T.src_buf][q][gsrc];
                const uint32_t r0 = bufs.p[q][T.src_buf][0][gsrc];
                medr[C.medr_off + ((int64_t)1 << T.lev_out) - 1 + fsi[j]] = rq;
                if (r0 >= goff && r0 < goff + m)
                    C.node[dest] = (int32_t)((int64_t)perm0[r0] - C.in_off);
                else
                    atomicOr(err, ERR_INTERNAL);
            }
        }
    }
    const int nvalid = (int)s_total;
#pragma unroll
    for (int f = 0; f < K; ++f) {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < IPT; ++j)
            if (slot[j] != INV) s_val[slot[j]] = v[f][j];
        __syncthreads();
        uint32_t* dp = bufs.p[q][T.dst_buf][(T.lev_in + f) % K];
        for (int s = tid; s < nvalid; s += LEVEL_THREADS)
            if (s_dest[s] != INV) dp[s_dest[s]] = s_val[s];
    }
}

// ------------------------------------------------------------- finisher
constexpr uint32_t HOLE = 0xffffffffu;

__device__ __forceinline__ uint32_t seg_pack(int32_t a, int32_t b) { return (uint32_t)a | ((uint32_t)b << 16); }

// Stable partition of one array (lids in src) around the medians of the
// current level, into dst.  Segmented block scan of packed (less, greater)
// counts; positions are blocked per thread.
__device__ __forceinline__ void fin_partition(const uint16_t* __restrict__ src, uint16_t* __restrict__ dst,
                                              const uint16_t* __restrict__ prim, const uint32_t* __restrict__ rkp,
                                              const uint32_t* __restrict__ seg, int S, int32_t* s_fl,
                                              uint32_t* s_fv, int* bad) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (S + FIN_THREADS - 1) / FIN_THREADS;
    const int i0 = tid * per;
    int tf = 0;
    uint32_t tv = 0;
    for (int x = 0; x < per; ++x) {
        const int i = i0 + x;
        if (i >= S) break;
        const uint32_t sg = seg[i];
        if (sg == HOLE) continue;
        const int32_t a = sg & 0xffff, b = sg >> 16, c = a + ((b - a) >> 1);
        if (i == a) {
            tf = 1;
            tv = 0;
        }
        const uint32_t r = rkp[src[i]], mv = rkp[prim[c]];
        tv += r < mv ? 1u : (r > mv ? 0x10000u : 0u);
    }
    int f = tf;
    uint32_t v = tv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int f2 = __shfl_up_sync(0xffffffffu, f, o);
        const uint32_t v2 = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) {
            if (!f) v += v2;
            f |= f2;
        }
    }
    int ef = __shfl_up_sync(0xffffffffu, f, 1);
    uint32_t ev = __shfl_up_sync(0xffffffffu, v, 1);
    if (lane == 0) {
        ef = 0;
        ev = 0;
    }
    if (lane == 31) {
        s_fl[warp] = f;
        s_fv[warp] = v;
    }
    __syncthreads();
    int wf = 0;
    uint32_t wv = 0;
    for (int w = 0; w < warp; ++w) {
        wv = s_fl[w] ? s_fv[w] : wv + s_fv[w];
        wf |= s_fl[w];
    }
    uint32_t acc = ef ? ev : wv + ev;
    for (int x = 0; x < per; ++x) {
        const int i = i0 + x;
        if (i >= S) break;
        const uint32_t sg = seg[i];
        if (sg == HOLE) continue;
        const int32_t a = sg & 0xffff, b = sg >> 16, c = a + ((b - a) >> 1);
        if (i == a) acc = 0;
        const uint16_t lid = src[i];
        const uint32_t r = rkp[lid], mv = rkp[prim[c]];
        if (r < mv) {
            const int32_t o = a + (int32_t)(acc & 0xffffu);
            if (o < c) dst[o] = lid; else *bad = 1;
            acc += 1u;
        } else if (r > mv) {
            const int32_t o = c + 1 + (int32_t)(acc >> 16);
            if (o <= b) dst[o] = lid; else *bad = 1;
            acc += 0x10000u;
        }
    }
}

__global__ void __launch_bounds__(FIN_THREADS)
    k_finish(const __grid_constant__ AllBufs bufs, int k, const FinUnit* __restrict__ units,
             const CloudDev* __restrict__ clouds, const uint32_t* __restrict__ perm0, int smax,
             int* __restrict__ err) {
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ int32_t s_fl[FIN_THREADS / 32];
    __shared__ uint32_t s_fv[FIN_THREADS / 32];
    __shared__ int s_cur[MAXK + 1];
    uint32_t* rk = sm;                                          // rk[p * smax + lid]
    uint32_t* seg = rk + (size_t)k * smax;                      // packed segment per position
    uint16_t* arr = reinterpret_cast<uint16_t*>(seg + smax);   // (k+1) storages of lids
    const int tid = threadIdx.x;
    const FinUnit U = units[blockIdx.x];
    const CloudDev C = clouds[U.cloud];
    int32_t lo, hi;
    segment_bounds(C.m, C.lam, U.seg, lo, hi);
    const int S = hi - lo + 1;
    if (S <= 0) return;
    if (S > smax) {
        if (tid == 0) atomicOr(err, ERR_INTERNAL);
        return;
    }
    const int64_t g = C.off + lo;
    for (int p = 0; p < k; ++p) {
        const uint32_t* src = bufs.p[0][C.buf[0]][p];
        for (int i = tid; i < S; i += FIN_THREADS) rk[p * smax + i] = src[g + i];
    }
    if (tid <= k) s_cur[tid] = tid;
    __syncthreads();
    for (int i = tid; i < S; i += FIN_THREADS) {
        arr[i] = (uint16_t)i;
        seg[i] = seg_pack(0, S - 1);
    }
    for (int d = 1; d < k; ++d) {
        const uint32_t* src0 = bufs.p[d][C.buf[d]][0];
        for (int i = tid; i < S; i += FIN_THREADS) {
            const uint32_t r0 = src0[g + i];
            int a = 0, b = S;  // array 0 is sorted by rank 0 within the segment
            while (a < b) {
                const int mid = (a + b) >> 1;
                if (rk[mid] < r0) a = mid + 1; else b = mid;
            }
            if (a >= S || rk[a] != r0) atomicOr(err, ERR_INTERNAL);
            arr[d * smax + i] = (uint16_t)min(a, S - 1);
        }
    }
    __syncthreads();
    int nlev = 0;
    while ((1 << nlev) <= S) ++nlev;  // ceil(log2(S + 1))
    int bad = 0;
    for (int dl = 0; dl < nlev; ++dl) {
        const int L = C.lam + dl;
        const int p = L % k;
        const uint16_t* prim = arr + s_cur[p] * smax;
        const uint32_t* rkp = rk + p * smax;
        for (int i = tid; i < S; i += FIN_THREADS) {
            const uint32_t sg = seg[i];
            if (sg == HOLE) continue;
            const int32_t a = sg & 0xffff, b = sg >> 16, c = a + ((b - a) >> 1);
            if (i != c) continue;
            const int32_t addr = lo + c;
            const uint32_t r0 = rk[prim[c]];
            if (r0 >= C.off && r0 < C.off + C.m)
                C.node[addr] = (int32_t)((int64_t)perm0[r0] - C.in_off);
            else
                bad = 1;
            if (C.left) C.left[addr] = a <= c - 1 ? lo + child_mid(a, c - 1) : -1;
            if (C.right) C.right[addr] = c + 1 <= b ? lo + child_mid(c + 1, b) : -1;
            if (C.dim) C.dim[addr] = (uint8_t)p;
        }
        for (int j = 1; j < k; ++j) {
            const int d = (p + j) % k;
            fin_partition(arr + s_cur[d] * smax, arr + s_cur[k] * smax, prim, rkp, seg, S, s_fl, s_fv, &bad);
            __syncthreads();
            if (tid == 0) {
                const int x = s_cur[d];
                s_cur[d] = s_cur[k];
                s_cur[k] = x;
            }
            __syncthreads();
        }
        for (int i = tid; i < S; i += FIN_THREADS) {
            const uint32_t sg = seg[i];
            if (sg == HOLE) continue;
            const int32_t a = sg & 0xffff, b = sg >> 16, c = a + ((b - a) >> 1);
            seg[i] = (i == c) ? HOLE : (i < c ? seg_pack(a, c - 1) : seg_pack(c + 1, b));
        }
        __syncthreads();
    }
    if (bad) atomicOr(err, ERR_INTERNAL);
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

// ------------------------------------------------------------ launchers
int level_ipt(int k) { return 8; }
int level_tile(int k) { return LEVEL_THREADS * level_ipt(k); }
int level_status_stride(int k) { return 1 << (k - 1); }

cudaError_t launch_level_pass(int k, const AllBufs& bufs, int q, const LevelTile* tiles, int ntiles,
                              const CloudDev* clouds, uint32_t* medr, const uint32_t* perm0, uint32_t* status,
                              uint32_t* tile_ctr, int* err, cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    const size_t smem = (size_t)2 * level_tile(k) * sizeof(uint32_t);
#define KD_LEVEL_CASE(KK)                                                                                  \
    case KK:                                                                                             \
        k_level_pass<KK, 8><<<ntiles, LEVEL_THREADS, smem, s>>>(bufs, q, tiles, ntiles, clouds, medr, perm0, \
                                                              status, tile_ctr, err);                     \
        break;
    switch (k) {
        KD_LEVEL_CASE(2)
        KD_LEVEL_CASE(3)
        KD_LEVEL_CASE(4)
        KD_LEVEL_CASE(5)
        KD_LEVEL_CASE(6)
        KD_LEVEL_CASE(7)
        KD_LEVEL_CASE(8)
        default:
            return cudaErrorInvalidValue;
    }
#undef KD_LEVEL_CASE
    return cudaGetLastError();
}

size_t finish_smem(int k, int smax) { return (size_t)k * smax * 4 + (size_t)smax * 4 + (size_t)(k + 1) * smax * 2; }

cudaError_t launch_finish(const AllBufs& bufs, int k, const FinUnit* units, int nunits, const CloudDev* clouds,
                          const uint32_t* perm0, int smax, int* err, cudaStream_t s) {
    if (nunits == 0) return cudaSuccess;
    const size_t smem = finish_smem(k, smax);
    cudaError_t e = cudaFuncSetAttribute(k_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_finish<<<nunits, FIN_THREADS, smem, s>>>(bufs, k, units, clouds, perm0, smax, err);
    return cudaGetLastError();
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

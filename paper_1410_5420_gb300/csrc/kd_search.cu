// kd_search.cu -- searches over a built tree: m nearest neighbours and
// region search (the "Nearest Neighbors" subsection and the region search
// of the source-code subsection of the paper).
//
// A search index holds the tree's tuples in address order (node a's k
// coordinates side by side, AoS) and the tuple index of every node, so that
// a walk reads one contiguous record per visited node.  The tree is the
// in-order layout the builder writes: the subtree of a node covers a
// contiguous address range [lo, hi], its node is the median lo + (hi-lo)/2,
// its children cover [lo, mid-1] and [mid+1, hi], and the split dimension
// of depth t is t mod k.  A subtree on the "less" side holds only tuples
// with x_d <= the node's x_d, the "greater" side only x_d >= (super keys
// order ties by the next coordinates), which is what both searches prune on.
//
//   k_index_gather  node_coords[a] = coords[node_tuple[a]]
//   k_knn           one thread per query: depth-first walk, near side first,
//                   the far side only while its splitting-plane distance
//                   does not exceed the current m-th best; the m best kept
//                   sorted by (distance, tuple index)
//   k_region        one thread per box: depth-first walk visiting a side
//                   only if the box reaches it; counts, then (second launch
//                   after a scan of the counts) the indices
//
// Distances are defined exactly (no fused multiply-add): per dimension the
// absolute difference (integers: |a - b| as an unsigned 64-bit value,
// rounded to double; floats: the double difference of the two values),
// squared and summed in double in dimension order.
#include <algorithm>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "kd_internal.cuh"
#include "kdtree.h"

namespace kd {
int ctx_device(const kd_ctx* ctx);
cudaStream_t ctx_stream(const kd_ctx* ctx);
void ctx_set_error(kd_ctx* ctx, const std::string& msg);
void ctx_add_launches(kd_ctx* ctx, int n);
kd_status ctx_alloc(kd_ctx* ctx, void** p, size_t bytes);
void ctx_free(kd_ctx* ctx, void* p);
std::recursive_mutex& ctx_mutex(kd_ctx* ctx);
}  // namespace kd

struct kd_index_s {
    kd_ctx* ctx = nullptr;
    int64_t m = 0;
    int k = 0;
    int dtype = 0;
    void* node_coords = nullptr;  // m x k, address order, input dtype
    int32_t* node_tuple = nullptr;
};

namespace {

using kd::ERR_INTERNAL;
using kd::ERR_NAN;
using kd::MAXK;

constexpr int SEARCH_THREADS = 128;
constexpr int STACK_MAX = 64;  // a tree of at most 2^30 nodes is at most 31 levels deep

template <typename T>
__device__ __forceinline__ double abs_diff(T a, T b);
template <>
__device__ __forceinline__ double abs_diff<int32_t>(int32_t a, int32_t b) {
    const int64_t x = a, y = b;
    return __ull2double_rn(x > y ? (uint64_t)(x - y) : (uint64_t)(y - x));
}
template <>
__device__ __forceinline__ double abs_diff<int64_t>(int64_t a, int64_t b) {
    return __ull2double_rn(a > b ? (uint64_t)a - (uint64_t)b : (uint64_t)b - (uint64_t)a);
}
template <>
__device__ __forceinline__ double abs_diff<float>(float a, float b) {
    return fabs(__dsub_rn((double)a, (double)b));
}

template <typename T>
__device__ __forceinline__ bool is_nan(T) { return false; }
template <>
__device__ __forceinline__ bool is_nan<float>(float v) { return v != v; }

template <typename T>
__global__ void __launch_bounds__(256) k_index_gather(const T* __restrict__ coords, const int32_t* __restrict__ tuple,
                                                      int64_t m, int k, int64_t n, T* __restrict__ out,
                                                      int* __restrict__ err) {
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < m * k; e += (int64_t)gridDim.x * 256) {
        const int64_t a = e / k;
        const int d = (int)(e - a * k);
        const int32_t t = tuple[a];
        if (t < 0 || t >= n) {
            atomicOr(err, ERR_INTERNAL);
            continue;
        }
        out[e] = coords[(int64_t)t * k + d];
    }
}

struct KnnEntry {
    int32_t lo, hi, depth;
    double bound;
};

// Insert (d, t) into the sorted list best[0..kn) if it beats the last entry.
__device__ __forceinline__ void knn_insert(double* bd, int32_t* bi, int kn, double d, int32_t t) {
    int j = kn - 1;
    if (!(d < bd[j] || (d == bd[j] && (bi[j] < 0 || t < bi[j])))) return;
    while (j > 0 && (d < bd[j - 1] || (d == bd[j - 1] && (bi[j - 1] < 0 || t < bi[j - 1])))) {
        bd[j] = bd[j - 1];
        bi[j] = bi[j - 1];
        --j;
    }
    bd[j] = d;
    bi[j] = t;
}

// queries == nullptr: every node is a query (row = its address) and its own
// tuple is not a candidate.
template <typename T>
__global__ void __launch_bounds__(SEARCH_THREADS) k_knn(const T* __restrict__ nodes, const int32_t* __restrict__ tuple,
                                                        int32_t m, int k, const T* __restrict__ queries, int64_t nq,
                                                        int kn, int32_t* __restrict__ idx_out,
                                                        double* __restrict__ d_out, int* __restrict__ err) {
    const int64_t qi = (int64_t)blockIdx.x * SEARCH_THREADS + threadIdx.x;
    if (qi >= nq) return;
    const int32_t self = queries ? -1 : tuple[qi];
    if (!queries) queries = nodes;
    T q[MAXK];
    bool nan = false;
#pragma unroll
    for (int d = 0; d < MAXK; ++d) {
        q[d] = d < k ? queries[qi * k + d] : (T)0;
        nan |= d < k && is_nan(q[d]);
    }
    if (nan) {
        atomicOr(err, ERR_NAN);
        return;
    }
    double bd[KD_KNN_MAX];
    int32_t bi[KD_KNN_MAX];
    for (int j = 0; j < kn; ++j) {
        bd[j] = __longlong_as_double(0x7ff0000000000000ll);  // +inf
        bi[j] = -1;
    }
    KnnEntry st[STACK_MAX];
    int sp = 0;
    if (m > 0) st[sp++] = KnnEntry{0, m - 1, 0, 0.0};
    while (sp > 0) {
        const KnnEntry e = st[--sp];
        if (e.bound > bd[kn - 1]) continue;  // nothing in this subtree can enter the list
        const int32_t mid = e.lo + ((e.hi - e.lo) >> 1);
        const T* p = nodes + (int64_t)mid * k;
        double acc = 0.0;
        for (int d = 0; d < k; ++d) {
            const double u = abs_diff<T>(p[d], q[d]);
            acc = __dadd_rn(acc, __dmul_rn(u, u));
        }
        const int32_t tm = tuple[mid];
        if (tm != self) knn_insert(bd, bi, kn, acc, tm);
        const int dim = e.depth % k;
        T qd = q[0], pd = p[0];
#pragma unroll
        for (int d = 1; d < MAXK; ++d)
            if (d == dim) {
                qd = q[d];
                pd = p[dim];
            }
        const double u = abs_diff<T>(pd, qd);
        const double plane = __dmul_rn(u, u);
        const bool less = qd < pd;  // the query lies on the "less" side
        const double far = fmax(e.bound, plane);
        const KnnEntry lo_side{e.lo, mid - 1, e.depth + 1, less ? e.bound : far};
        const KnnEntry hi_side{mid + 1, e.hi, e.depth + 1, less ? far : e.bound};
        if (sp + 2 > STACK_MAX) {
            atomicOr(err, ERR_INTERNAL);
            break;
        }
        // far side below, near side on top
        if (less) {
            if (hi_side.lo <= hi_side.hi) st[sp++] = hi_side;
            if (lo_side.lo <= lo_side.hi) st[sp++] = lo_side;
        } else {
            if (lo_side.lo <= lo_side.hi) st[sp++] = lo_side;
            if (hi_side.lo <= hi_side.hi) st[sp++] = hi_side;
        }
    }
    for (int j = 0; j < kn; ++j) {
        idx_out[qi * kn + j] = bi[j];
        if (d_out) d_out[qi * kn + j] = bd[j];
    }
}

// Region search over box qi: count (out == nullptr) or write the indices
// of the tuples inside it at out[offs[qi] ...].
template <typename T>
__global__ void __launch_bounds__(SEARCH_THREADS) k_region(const T* __restrict__ nodes,
                                                           const int32_t* __restrict__ tuple, int32_t m, int k,
                                                           const T* __restrict__ lo, const T* __restrict__ hi,
                                                           int64_t nq, int64_t* __restrict__ counts,
                                                           const int64_t* __restrict__ offs, int32_t* __restrict__ out,
                                                           int* __restrict__ err) {
    const int64_t qi = (int64_t)blockIdx.x * SEARCH_THREADS + threadIdx.x;
    if (qi >= nq) return;
    T a[MAXK], b[MAXK];
    bool nan = false;
#pragma unroll
    for (int d = 0; d < MAXK; ++d) {
        a[d] = d < k ? lo[qi * k + d] : (T)0;
        b[d] = d < k ? hi[qi * k + d] : (T)0;
        nan |= d < k && (is_nan(a[d]) || is_nan(b[d]));
    }
    if (nan) {
        atomicOr(err, ERR_NAN);
        if (!out) counts[qi] = 0;
        return;
    }
    int64_t o = out ? offs[qi] : 0;
    const int64_t o_end = out ? offs[qi + 1] : 0;
    int64_t c = 0;
    int32_t st_lo[STACK_MAX], st_hi[STACK_MAX], st_dp[STACK_MAX];
    int sp = 0;
    if (m > 0) {
        st_lo[0] = 0;
        st_hi[0] = m - 1;
        st_dp[0] = 0;
        sp = 1;
    }
    while (sp > 0) {
        --sp;
        const int32_t l = st_lo[sp], h = st_hi[sp], depth = st_dp[sp];
        const int32_t mid = l + ((h - l) >> 1);
        const T* p = nodes + (int64_t)mid * k;
        bool in = true;
        for (int d = 0; d < k; ++d) {
            T ad = a[0], bdv = b[0];
#pragma unroll
            for (int x = 1; x < MAXK; ++x)
                if (x == d) {
                    ad = a[x];
                    bdv = b[x];
                }
            in = in && ad <= p[d] && p[d] <= bdv;
        }
        if (in) {
            if (out) {
                if (o < o_end) out[o++] = tuple[mid]; else atomicOr(err, ERR_INTERNAL);
            }
            ++c;
        }
        const int dim = depth % k;
        T ad = a[0], bdv = b[0];
#pragma unroll
        for (int x = 1; x < MAXK; ++x)
            if (x == dim) {
                ad = a[x];
                bdv = b[x];
            }
        const T pd = p[dim];
        if (sp + 2 > STACK_MAX) {
            atomicOr(err, ERR_INTERNAL);
            break;
        }
        if (mid + 1 <= h && pd <= bdv) {  // the greater side holds x_dim >= pd
            st_lo[sp] = mid + 1;
            st_hi[sp] = h;
            st_dp[sp] = depth + 1;
            ++sp;
        }
        if (l <= mid - 1 && ad <= pd) {  // the less side holds x_dim <= pd
            st_lo[sp] = l;
            st_hi[sp] = mid - 1;
            st_dp[sp] = depth + 1;
            ++sp;
        }
    }
    if (!out) counts[qi] = c;
}

// Reverse nearest neighbours: inv[tuple] = address, then per target
// address the number of nodes listing it, then the lists.
__global__ void __launch_bounds__(256) k_inv_map(const int32_t* __restrict__ tuple, int64_t m, int64_t n,
                                                 int32_t* __restrict__ inv, int* __restrict__ err) {
    for (int64_t a = (int64_t)blockIdx.x * 256 + threadIdx.x; a < m; a += (int64_t)gridDim.x * 256) {
        const int32_t t = tuple[a];
        if (t < 0 || t >= n) atomicOr(err, ERR_INTERNAL); else inv[t] = (int32_t)a;
    }
}
__global__ void __launch_bounds__(256) k_rev_count(const int32_t* __restrict__ nn, int64_t total,
                                                   const int32_t* __restrict__ inv, int64_t n,
                                                   int64_t* __restrict__ cnt, int* __restrict__ err) {
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < total; e += (int64_t)gridDim.x * 256) {
        const int32_t t = nn[e];
        if (t < 0) continue;
        const int32_t a = t < n ? inv[t] : -1;
        if (a < 0) atomicOr(err, ERR_INTERNAL); else atomicAdd((unsigned long long*)&cnt[a], 1ull);
    }
}
__global__ void __launch_bounds__(256) k_rev_fill(const int32_t* __restrict__ nn, int64_t total, int kn,
                                                  const int32_t* __restrict__ tuple, const int32_t* __restrict__ inv,
                                                  int64_t n, int64_t* __restrict__ cursor, int32_t* __restrict__ rev,
                                                  int* __restrict__ err) {
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < total; e += (int64_t)gridDim.x * 256) {
        const int32_t t = nn[e];
        if (t < 0) continue;
        const int32_t a = t < n ? inv[t] : -1;
        if (a < 0) {
            atomicOr(err, ERR_INTERNAL);
            continue;
        }
        const int64_t pos = (int64_t)atomicAdd((unsigned long long*)&cursor[a], 1ull);
        rev[pos] = tuple[e / kn];
    }
}

// offs[i] = sum of counts[0..i), offs[n] = total; one block.
__global__ void __launch_bounds__(1024) k_offsets(const int64_t* __restrict__ counts, int64_t n,
                                                 int64_t* __restrict__ offs) {
    __shared__ int64_t s_w[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t carry = 0;
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + tid;
        const int64_t v = i < n ? counts[i] : 0;
        int64_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int64_t w = s_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_w[lane] = w;
        }
        __syncthreads();
        const int64_t excl = carry + (warp ? s_w[warp - 1] : 0) + x - v;
        if (i < n) offs[i] = excl;
        carry += s_w[31];
        __syncthreads();
    }
    if (tid == 0) offs[n] = carry;
}

bool device_ptr(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t dtype_size(int dtype) { return dtype == KD_I64 ? 8 : 4; }

kd_status sfail(kd_ctx* ctx, kd_status code, const std::string& msg) {
    kd::ctx_set_error(ctx, msg);
    return code;
}

// Scratch owned by one call.
struct CallScratch {
    kd_ctx* ctx;
    std::vector<void*> ptrs;
    explicit CallScratch(kd_ctx* c) : ctx(c) {}
    ~CallScratch() {
        for (void* p : ptrs) kd::ctx_free(ctx, p);
    }
    kd_status get(void** p, size_t bytes) {
        kd_status s = kd::ctx_alloc(ctx, p, bytes);
        if (s == KD_OK) ptrs.push_back(*p);
        return s;
    }
};

// A device copy of host data (or the device pointer itself).
kd_status to_device(kd_ctx* ctx, CallScratch& S, const void* src, size_t bytes, int on_device, const void** out,
                    cudaStream_t s) {
    if (on_device || bytes == 0) {
        *out = src;
        return KD_OK;
    }
    void* d = nullptr;
    kd_status st = S.get(&d, bytes);
    if (st != KD_OK) return st;
    if (cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return sfail(ctx, KD_EDEVICE, "host to device copy failed");
    *out = d;
    return KD_OK;
}

kd_status read_err(kd_ctx* ctx, int* d_err, cudaStream_t s) {
    int h = 0;
    if (cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return sfail(ctx, KD_EDEVICE, std::string("search: ") + cudaGetErrorString(cudaGetLastError()));
    if (h & ERR_NAN) return sfail(ctx, KD_ENAN, "a query coordinate is NaN");
    if (h) return sfail(ctx, KD_EDEVICE, "inconsistent tree or index (device error flags " + std::to_string(h) + ")");
    return KD_OK;
}

int grid_of(int64_t n, int per) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, 1 << 20)); }

}  // namespace

extern "C" {

kd_status kd_index_create(kd_ctx* ctx, const kd_cloud* cloud, const kd_tree* tree, kd_index* out) {
    if (!ctx || !out) return KD_EINVAL;
    *out = nullptr;
    std::lock_guard<std::recursive_mutex> lk(kd::ctx_mutex(ctx));
    if (cudaSetDevice(kd::ctx_device(ctx)) != cudaSuccess) return sfail(ctx, KD_EDEVICE, "cudaSetDevice failed");
    if (!cloud || !tree) return sfail(ctx, KD_EINVAL, "cloud or tree is NULL");
    if (cloud->k < 1 || cloud->k > KD_MAX_K || cloud->n < 0 || cloud->n > KD_MAX_N ||
        (cloud->dtype != KD_I32 && cloud->dtype != KD_I64 && cloud->dtype != KD_F32))
        return sfail(ctx, KD_EINVAL, "bad cloud");
    if (tree->m < 0 || tree->m > cloud->n || (tree->m > 0 && (!tree->node_tuple || !cloud->coords)))
        return sfail(ctx, KD_EINVAL, "tree does not fit the cloud");
    cudaStream_t s = kd::ctx_stream(ctx);
    const size_t ts = dtype_size(cloud->dtype);
    std::unique_ptr<kd_index_s> ix(new kd_index_s());
    ix->ctx = ctx;
    ix->m = tree->m;
    ix->k = cloud->k;
    ix->dtype = cloud->dtype;
    if (ix->m == 0) {
        *out = ix.release();
        return KD_OK;
    }
    CallScratch S(ctx);
    const void* coords = nullptr;
    const void* tuple = nullptr;
    kd_status st = to_device(ctx, S, cloud->coords, (size_t)cloud->n * cloud->k * ts, cloud->on_device, &coords, s);
    if (st == KD_OK) st = to_device(ctx, S, tree->node_tuple, (size_t)ix->m * 4, tree->on_device, &tuple, s);
    if (st == KD_OK) st = kd::ctx_alloc(ctx, &ix->node_coords, (size_t)ix->m * ix->k * ts);
    if (st == KD_OK) st = kd::ctx_alloc(ctx, (void**)&ix->node_tuple, (size_t)ix->m * 4);
    int* d_err = nullptr;
    if (st == KD_OK) st = S.get((void**)&d_err, sizeof(int));
    if (st != KD_OK) {
        kd_index_destroy(ctx, ix.release());
        return st;
    }
    cudaMemsetAsync(d_err, 0, sizeof(int), s);
    cudaMemcpyAsync(ix->node_tuple, tuple, (size_t)ix->m * 4, cudaMemcpyDeviceToDevice, s);
    const int g = grid_of(ix->m * ix->k, 256);
    if (ix->dtype == KD_I32)
        k_index_gather<int32_t><<<g, 256, 0, s>>>((const int32_t*)coords, (const int32_t*)tuple, ix->m, ix->k,
                                                  cloud->n, (int32_t*)ix->node_coords, d_err);
    else if (ix->dtype == KD_I64)
        k_index_gather<int64_t><<<g, 256, 0, s>>>((const int64_t*)coords, (const int32_t*)tuple, ix->m, ix->k,
                                                  cloud->n, (int64_t*)ix->node_coords, d_err);
    else
        k_index_gather<float><<<g, 256, 0, s>>>((const float*)coords, (const int32_t*)tuple, ix->m, ix->k,
                                                cloud->n, (float*)ix->node_coords, d_err);
    kd::ctx_add_launches(ctx, 1);
    st = read_err(ctx, d_err, s);
    if (st != KD_OK) {
        kd_index_destroy(ctx, ix.release());
        return st;
    }
    *out = ix.release();
    return KD_OK;
}

kd_status kd_index_destroy(kd_ctx* ctx, kd_index ix) {
    if (!ctx || !ix) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(kd::ctx_mutex(ctx));
    cudaSetDevice(kd::ctx_device(ctx));
    if (ix->node_coords) kd::ctx_free(ctx, ix->node_coords);
    if (ix->node_tuple) kd::ctx_free(ctx, ix->node_tuple);
    delete ix;
    return KD_OK;
}

kd_status kd_knn(kd_ctx* ctx, kd_index ix, const void* queries, int64_t nq, int kn, int on_device, int32_t* idx_out,
                 double* dist_out) {
    if (!ctx || !ix) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(kd::ctx_mutex(ctx));
    if (cudaSetDevice(kd::ctx_device(ctx)) != cudaSuccess) return sfail(ctx, KD_EDEVICE, "cudaSetDevice failed");
    if (kn < 1 || kn > KD_KNN_MAX) return sfail(ctx, KD_EINVAL, "kn must be in [1, KD_KNN_MAX]");
    if (nq < 0 || (nq > 0 && (!queries || !idx_out))) return sfail(ctx, KD_EINVAL, "bad queries or outputs");
    if (nq == 0) return KD_OK;
    cudaStream_t s = kd::ctx_stream(ctx);
    const size_t ts = dtype_size(ix->dtype);
    CallScratch S(ctx);
    const void* q = nullptr;
    kd_status st = to_device(ctx, S, queries, (size_t)nq * ix->k * ts, on_device, &q, s);
    int32_t* di = idx_out;
    double* dd = dist_out;
    int* d_err = nullptr;
    if (st == KD_OK && !on_device) {
        st = S.get((void**)&di, (size_t)nq * kn * 4);
        if (st == KD_OK && dist_out) st = S.get((void**)&dd, (size_t)nq * kn * 8);
    }
    if (st == KD_OK) st = S.get((void**)&d_err, sizeof(int));
    if (st != KD_OK) return st;
    cudaMemsetAsync(d_err, 0, sizeof(int), s);
    const int g = grid_of(nq, SEARCH_THREADS);
    const int32_t m = (int32_t)ix->m;
    if (ix->dtype == KD_I32)
        k_knn<int32_t><<<g, SEARCH_THREADS, 0, s>>>((const int32_t*)ix->node_coords, ix->node_tuple, m, ix->k,
                                                    (const int32_t*)q, nq, kn, di, dd, d_err);
    else if (ix->dtype == KD_I64)
        k_knn<int64_t><<<g, SEARCH_THREADS, 0, s>>>((const int64_t*)ix->node_coords, ix->node_tuple, m, ix->k,
                                                    (const int64_t*)q, nq, kn, di, dd, d_err);
    else
        k_knn<float><<<g, SEARCH_THREADS, 0, s>>>((const float*)ix->node_coords, ix->node_tuple, m, ix->k,
                                                  (const float*)q, nq, kn, di, dd, d_err);
    kd::ctx_add_launches(ctx, 1);
    if (!on_device) {
        cudaMemcpyAsync(idx_out, di, (size_t)nq * kn * 4, cudaMemcpyDeviceToHost, s);
        if (dist_out) cudaMemcpyAsync(dist_out, dd, (size_t)nq * kn * 8, cudaMemcpyDeviceToHost, s);
    }
    return read_err(ctx, d_err, s);
}

// m nearest neighbours of every node (address order), its own tuple excluded.
static kd_status knn_all_device(kd_ctx* ctx, kd_index ix, int kn, int32_t* di, double* dd, int* d_err,
                                cudaStream_t s) {
    const int64_t m = ix->m;
    const int g = grid_of(m, SEARCH_THREADS);
    if (ix->dtype == KD_I32)
        k_knn<int32_t><<<g, SEARCH_THREADS, 0, s>>>((const int32_t*)ix->node_coords, ix->node_tuple, (int32_t)m,
                                                    ix->k, nullptr, m, kn, di, dd, d_err);
    else if (ix->dtype == KD_I64)
        k_knn<int64_t><<<g, SEARCH_THREADS, 0, s>>>((const int64_t*)ix->node_coords, ix->node_tuple, (int32_t)m,
                                                    ix->k, nullptr, m, kn, di, dd, d_err);
    else
        k_knn<float><<<g, SEARCH_THREADS, 0, s>>>((const float*)ix->node_coords, ix->node_tuple, (int32_t)m, ix->k,
                                                  nullptr, m, kn, di, dd, d_err);
    kd::ctx_add_launches(ctx, 1);
    return KD_OK;
}

kd_status kd_knn_all(kd_ctx* ctx, kd_index ix, int kn, int on_device, int32_t* idx_out, double* dist_out) {
    if (!ctx || !ix) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(kd::ctx_mutex(ctx));
    if (cudaSetDevice(kd::ctx_device(ctx)) != cudaSuccess) return sfail(ctx, KD_EDEVICE, "cudaSetDevice failed");
    if (kn < 1 || kn > KD_KNN_MAX) return sfail(ctx, KD_EINVAL, "kn must be in [1, KD_KNN_MAX]");
    if (ix->m > 0 && !idx_out) return sfail(ctx, KD_EINVAL, "idx_out is NULL");
    if (ix->m == 0) return KD_OK;
    cudaStream_t s = kd::ctx_stream(ctx);
    CallScratch S(ctx);
    int32_t* di = idx_out;
    double* dd = dist_out;
    int* d_err = nullptr;
    kd_status st = KD_OK;
    if (!on_device) {
        st = S.get((void**)&di, (size_t)ix->m * kn * 4);
        if (st == KD_OK && dist_out) st = S.get((void**)&dd, (size_t)ix->m * kn * 8);
    }
    if (st == KD_OK) st = S.get((void**)&d_err, sizeof(int));
    if (st != KD_OK) return st;
    cudaMemsetAsync(d_err, 0, sizeof(int), s);
    knn_all_device(ctx, ix, kn, di, dd, d_err, s);
    if (!on_device) {
        cudaMemcpyAsync(idx_out, di, (size_t)ix->m * kn * 4, cudaMemcpyDeviceToHost, s);
        if (dist_out) cudaMemcpyAsync(dist_out, dd, (size_t)ix->m * kn * 8, cudaMemcpyDeviceToHost, s);
    }
    return read_err(ctx, d_err, s);
}

kd_status kd_reverse_knn(kd_ctx* ctx, kd_index ix, int kn, int on_device, int64_t* offsets, int32_t* rev_out) {
    if (!ctx || !ix) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(kd::ctx_mutex(ctx));
    if (cudaSetDevice(kd::ctx_device(ctx)) != cudaSuccess) return sfail(ctx, KD_EDEVICE, "cudaSetDevice failed");
    if (kn < 1 || kn > KD_KNN_MAX) return sfail(ctx, KD_EINVAL, "kn must be in [1, KD_KNN_MAX]");
    if (!offsets || (ix->m > 0 && !rev_out)) return sfail(ctx, KD_EINVAL, "offsets or rev_out is NULL");
    cudaStream_t s = kd::ctx_stream(ctx);
    const int64_t m = ix->m, total = m * kn;
    CallScratch S(ctx);
    int32_t *nn = nullptr, *inv = nullptr, *rev = rev_out;
    int64_t *cnt = nullptr, *offs = offsets, *cursor = nullptr;
    int* d_err = nullptr;
    int64_t n = 0;  // tuple indices are below the largest one + 1; the inverse map spans them
    kd_status st = S.get((void**)&d_err, sizeof(int));
    if (st != KD_OK) return st;
    if (m == 0) {
        int64_t z = 0;
        if (on_device) cudaMemcpyAsync(offsets, &z, 8, cudaMemcpyHostToDevice, s); else offsets[0] = 0;
        return cudaStreamSynchronize(s) == cudaSuccess ? KD_OK : sfail(ctx, KD_EDEVICE, "synchronise failed");
    }
    // the inverse map needs the largest tuple index
    {
        std::vector<int32_t> tmp;
        int32_t mx = 0;
        tmp.resize((size_t)m);
        if (cudaMemcpyAsync(tmp.data(), ix->node_tuple, (size_t)m * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return sfail(ctx, KD_EDEVICE, "reading the index failed");
        for (int32_t t : tmp) mx = std::max(mx, t);
        n = (int64_t)mx + 1;
    }
    st = S.get((void**)&nn, (size_t)total * 4);
    if (st == KD_OK) st = S.get((void**)&inv, (size_t)n * 4);
    if (st == KD_OK) st = S.get((void**)&cnt, (size_t)m * 8);
    if (st == KD_OK) st = S.get((void**)&cursor, (size_t)(m + 1) * 8);
    if (st == KD_OK && !on_device) {
        st = S.get((void**)&offs, (size_t)(m + 1) * 8);
        if (st == KD_OK) st = S.get((void**)&rev, (size_t)std::max<int64_t>(total, 1) * 4);
    }
    if (st != KD_OK) return st;
    cudaMemsetAsync(d_err, 0, sizeof(int), s);
    cudaMemsetAsync(inv, 0xff, (size_t)n * 4, s);
    cudaMemsetAsync(cnt, 0, (size_t)m * 8, s);
    knn_all_device(ctx, ix, kn, nn, nullptr, d_err, s);
    k_inv_map<<<grid_of(m, 256), 256, 0, s>>>(ix->node_tuple, m, n, inv, d_err);
    k_rev_count<<<grid_of(total, 256), 256, 0, s>>>(nn, total, inv, n, cnt, d_err);
    k_offsets<<<1, 1024, 0, s>>>(cnt, m, offs);
    cudaMemcpyAsync(cursor, offs, (size_t)(m + 1) * 8, cudaMemcpyDeviceToDevice, s);
    k_rev_fill<<<grid_of(total, 256), 256, 0, s>>>(nn, total, kn, ix->node_tuple, inv, n, cursor, rev, d_err);
    kd::ctx_add_launches(ctx, 4);
    int64_t tot = 0;
    cudaMemcpyAsync(&tot, offs + m, 8, cudaMemcpyDeviceToHost, s);
    if (!on_device) {
        cudaMemcpyAsync(offsets, offs, (size_t)(m + 1) * 8, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(rev_out, rev, (size_t)total * 4, cudaMemcpyDeviceToHost, s);
    }
    return read_err(ctx, d_err, s);
}

kd_status kd_region(kd_ctx* ctx, kd_index ix, const void* lo, const void* hi, int64_t nq, int on_device,
                    int64_t* offsets, int32_t* idx_out, int64_t capacity) {
    if (!ctx || !ix) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(kd::ctx_mutex(ctx));
    if (cudaSetDevice(kd::ctx_device(ctx)) != cudaSuccess) return sfail(ctx, KD_EDEVICE, "cudaSetDevice failed");
    if (nq < 0 || !offsets || (nq > 0 && (!lo || !hi))) return sfail(ctx, KD_EINVAL, "bad boxes or offsets");
    cudaStream_t s = kd::ctx_stream(ctx);
    const size_t ts = dtype_size(ix->dtype);
    CallScratch S(ctx);
    const void *dlo = nullptr, *dhi = nullptr;
    kd_status st = to_device(ctx, S, lo, (size_t)nq * ix->k * ts, on_device, &dlo, s);
    if (st == KD_OK) st = to_device(ctx, S, hi, (size_t)nq * ix->k * ts, on_device, &dhi, s);
    int64_t *counts = nullptr, *doffs = offsets;
    int* d_err = nullptr;
    if (st == KD_OK) st = S.get((void**)&counts, (size_t)std::max<int64_t>(nq, 1) * 8);
    if (st == KD_OK && !on_device) st = S.get((void**)&doffs, (size_t)(nq + 1) * 8);
    if (st == KD_OK) st = S.get((void**)&d_err, sizeof(int));
    if (st != KD_OK) return st;
    cudaMemsetAsync(d_err, 0, sizeof(int), s);
    const int g = grid_of(nq, SEARCH_THREADS);
    const int32_t m = (int32_t)ix->m;
    auto launch = [&](const int64_t* offs, int32_t* out) {
        if (nq == 0) return;
        if (ix->dtype == KD_I32)
            k_region<int32_t><<<g, SEARCH_THREADS, 0, s>>>((const int32_t*)ix->node_coords, ix->node_tuple, m, ix->k,
                                                           (const int32_t*)dlo, (const int32_t*)dhi, nq, counts, offs,
                                                           out, d_err);
        else if (ix->dtype == KD_I64)
            k_region<int64_t><<<g, SEARCH_THREADS, 0, s>>>((const int64_t*)ix->node_coords, ix->node_tuple, m, ix->k,
                                                           (const int64_t*)dlo, (const int64_t*)dhi, nq, counts, offs,
                                                           out, d_err);
        else
            k_region<float><<<g, SEARCH_THREADS, 0, s>>>((const float*)ix->node_coords, ix->node_tuple, m, ix->k,
                                                         (const float*)dlo, (const float*)dhi, nq, counts, offs, out,
                                                         d_err);
        kd::ctx_add_launches(ctx, 1);
    };
    launch(nullptr, nullptr);
    k_offsets<<<1, 1024, 0, s>>>(counts, nq, doffs);
    kd::ctx_add_launches(ctx, 1);
    int64_t total = 0;
    cudaMemcpyAsync(&total, doffs + nq, 8, cudaMemcpyDeviceToHost, s);
    st = read_err(ctx, d_err, s);  // synchronises
    if (st != KD_OK) return st;
    if (!on_device) cudaMemcpyAsync(offsets, doffs, (size_t)(nq + 1) * 8, cudaMemcpyDeviceToHost, s);
    if (idx_out && total > 0) {
        if (total > capacity)
            return sfail(ctx, KD_EINVAL,
                         "capacity " + std::to_string(capacity) + " < " + std::to_string(total) + " results");
        int32_t* dout = idx_out;
        if (!on_device) {
            st = S.get((void**)&dout, (size_t)total * 4);
            if (st != KD_OK) return st;
        }
        launch(doffs, dout);
        if (!on_device) cudaMemcpyAsync(idx_out, dout, (size_t)total * 4, cudaMemcpyDeviceToHost, s);
    }
    return read_err(ctx, d_err, s);
}

}  // extern "C"

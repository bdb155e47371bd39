// kd_noalloc.cu -- presort of one small cloud that allocates no memory.
//
// kd_presort takes its workspace from the context's stream-ordered pool.
// Some callers cannot let a library allocate at call time: a process that
// has already handed all device memory to its own allocator (a call would
// then fail with KD_ENOMEM), or a latency-bound loop where a growing pool or
// a cudaFree would stall the device for every stream.  kd_presort_noalloc
// serves them for clouds of up to KD_NOALLOC_MAX_N tuples: its only
// workspace is one file-scope device array (1 MiB of key planes plus a
// status word), set up once per device, and its outputs go to buffers the
// caller owns.
//
// It computes what kd_presort + kd_handle_arrays compute (Section 2.1: the
// k index arrays sorted by the cyclic super keys x_d : x_{d+1} : ... and
// duplicate tuples removed, the smallest index of a run surviving) with two
// kernels sized for small clouds:
//   k_noalloc_keys  coordinates -> order-preserving unsigned key planes in
//                   the static array; a NaN sets the status word;
//   k_noalloc_sort  one block per super key d: the indices and their key
//                   x_d in shared memory, a bitonic sort whose comparisons
//                   fall back to x_{d+1}, ... (static array, L2-resident)
//                   and then to the index on ties, then an adjacent-compare
//                   and block-scan compaction dropping duplicate tuples.
//
// The one static array per device is shared by every call on that device:
// two calls whose kernels can overlap (different streams, or different
// threads without ordering between them) race on it.  Order such calls on
// one stream.
#include <mutex>
#include <string>

#include "kd_internal.cuh"
#include "kdtree.h"

namespace kd {
// Context access (kd_api.cu).
int ctx_device(const kd_ctx* ctx);
cudaStream_t ctx_stream(const kd_ctx* ctx);
void ctx_set_error(kd_ctx* ctx, const std::string& msg);
void ctx_add_launches(kd_ctx* ctx, int n);
}  // namespace kd

namespace {

constexpr int NA_MAX_N = KD_NOALLOC_MAX_N;
constexpr int NA_THREADS = 1024;
constexpr int NA_KEYS_THREADS = 256;
constexpr uint32_t NA_PAD = 0xffffffffu;  // index of a padding slot; sorts last

// Workspace: KD_MAX_K key planes of NA_MAX_N words, then the status word
// (nonzero once a NaN coordinate was seen).  The key planes are written in
// full for the cloud before they are read; only the status word must start
// at zero, and each call clears it on its stream before the first kernel.
constexpr size_t NA_STATUS_WORD = (size_t)KD_MAX_K * NA_MAX_N;
static __device__ __align__(256) uint64_t na_scratch[NA_STATUS_WORD + 32];

template <typename T>
__global__ void __launch_bounds__(NA_KEYS_THREADS) k_noalloc_keys(const T* __restrict__ coords, int n, int k,
                                                                  uint64_t* __restrict__ ws) {
    const int total = n * k;
    int nan = 0;
    for (int e = blockIdx.x * NA_KEYS_THREADS + threadIdx.x; e < total; e += gridDim.x * NA_KEYS_THREADS) {
        const int i = e / k, d = e - i * k;
        ws[(size_t)d * NA_MAX_N + i] = (uint64_t)kd::key_of(coords[e], &nan);
    }
    if (nan) atomicOr(reinterpret_cast<unsigned int*>(ws + NA_STATUS_WORD), 1u);
}

// Is (ka, ia) after (kb, ib) in super-key-d order?  ka, kb are the x_d keys.
__device__ __forceinline__ bool na_after(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib, int d, int k,
                                         const uint64_t* __restrict__ ws) {
    if (ka != kb) return ka > kb;
    if (ia == NA_PAD || ib == NA_PAD) return ia > ib;
    for (int r = 1; r < k; ++r) {
        const int dd = d + r < k ? d + r : d + r - k;
        const uint64_t xa = ws[(size_t)dd * NA_MAX_N + ia], xb = ws[(size_t)dd * NA_MAX_N + ib];
        if (xa != xb) return xa > xb;
    }
    return ia > ib;
}

// Block d sorts the indices by super key d and writes the deduplicated order
// to row d of out (row stride n).  Dynamic shared memory: npow2 keys (u64)
// then npow2 indices (u32).
__global__ void __launch_bounds__(NA_THREADS, 1) k_noalloc_sort(int n, int npow2, int k,
                                                                 const uint64_t* __restrict__ ws,
                                                                 int32_t* __restrict__ out, int32_t* m_out) {
    extern __shared__ __align__(16) unsigned char na_smem[];
    __shared__ int warp_tot[NA_THREADS / 32];
    uint64_t* sk = reinterpret_cast<uint64_t*>(na_smem);
    uint32_t* si = reinterpret_cast<uint32_t*>(sk + npow2);
    const int d = blockIdx.x, tid = threadIdx.x;
    if (*reinterpret_cast<const volatile unsigned int*>(ws + NA_STATUS_WORD)) {
        if (d == 0 && tid == 0) *m_out = KD_ENAN;
        return;
    }
    const uint64_t* xd = ws + (size_t)d * NA_MAX_N;
    for (int p = tid; p < npow2; p += NA_THREADS) {
        sk[p] = p < n ? xd[p] : ~0ull;
        si[p] = p < n ? (uint32_t)p : NA_PAD;
    }
    __syncthreads();
    // bitonic sort of npow2 slots; the order is total (ties end at the index)
    for (int size = 2; size <= npow2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = tid; t < (npow2 >> 1); t += NA_THREADS) {
                const int i = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));
                const int j = i + stride;
                const bool up = (i & size) == 0;
                const uint64_t ki = sk[i], kj = sk[j];
                const uint32_t ii = si[i], ij = si[j];
                if (na_after(ki, ii, kj, ij, d, k, ws) == up) {
                    sk[i] = kj;
                    sk[j] = ki;
                    si[i] = ij;
                    si[j] = ii;
                }
            }
            __syncthreads();
        }
    }
    // Duplicate removal: a slot whose tuple equals its predecessor's goes.
    // Each thread owns a contiguous chunk; a block scan of the kept counts
    // gives the chunk's output offset.
    const int chunk = (n + NA_THREADS - 1) / NA_THREADS;
    const int b = tid * chunk < n ? tid * chunk : n;
    const int e = b + chunk < n ? b + chunk : n;
    auto kept = [&](int p) -> bool {
        if (p == 0) return true;
        if (sk[p] != sk[p - 1]) return true;
        const uint32_t a = si[p], c = si[p - 1];
        for (int r = 1; r < k; ++r) {
            const int dd = d + r < k ? d + r : d + r - k;
            if (ws[(size_t)dd * NA_MAX_N + a] != ws[(size_t)dd * NA_MAX_N + c]) return true;
        }
        return false;
    };
    int cnt = 0;
    for (int p = b; p < e; ++p) cnt += kept(p);
    const int lane = tid & 31, warp = tid >> 5;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = warp_tot[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += v;
        }
        warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    int pos = (warp ? warp_tot[warp - 1] : 0) + incl - cnt;
    int32_t* row = out + (size_t)d * n;
    for (int p = b; p < e; ++p)
        if (kept(p)) row[pos++] = (int32_t)si[p];
    if (d == 0 && tid == NA_THREADS - 1) *m_out = warp_tot[31];
}

// Per-device set-up, once per device with that device current: the address
// of the static workspace and the shared-memory limit of the sort kernel.
std::mutex na_mu;
uint64_t* na_ws[64] = {};

cudaError_t noalloc_setup(int device, uint64_t** ws) {
    std::lock_guard<std::mutex> lk(na_mu);
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    if (!na_ws[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_noalloc_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 NA_MAX_N * (int)(sizeof(uint64_t) + sizeof(uint32_t)));
        if (e != cudaSuccess) return e;
        na_ws[device] = static_cast<uint64_t*>(p);
    }
    *ws = na_ws[device];
    return cudaSuccess;
}

// Device (or managed) memory owned by `device`: a buffer on another GPU
// would be read or written through peer access, which need not be enabled.
bool on_device_memory(const void* p, int device) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // the query's own error, raised just now
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}

// Launch with the error returned by the launch call itself, so that an
// error pending from the caller's earlier work is neither reported as this
// call's nor cleared.
template <typename... P>
cudaError_t na_launch(void (*kern)(P...), int grid, int block, size_t smem, cudaStream_t s, P... args) {
    void* argv[] = {static_cast<void*>(&args)...};
    return cudaLaunchKernel(reinterpret_cast<const void*>(kern), dim3(grid), dim3(block), argv, smem, s);
}

kd_status na_fail(kd_ctx* ctx, kd_status code, const std::string& msg) {
    kd::ctx_set_error(ctx, "kd_presort_noalloc: " + msg);
    return code;
}

}  // namespace

extern "C" kd_status kd_presort_noalloc(kd_ctx* ctx, const kd_cloud* cloud, int32_t* arrays_out, int32_t* m_out) {
    if (!ctx) return KD_EINVAL;
    if (!cloud || !m_out) return na_fail(ctx, KD_EINVAL, "null cloud or m_out");
    const int64_t n = cloud->n;
    const int k = cloud->k;
    if (k < 1 || k > KD_MAX_K) return na_fail(ctx, KD_EINVAL, "k must be in 1.." + std::to_string(KD_MAX_K));
    if (n < 0 || n > NA_MAX_N)
        return na_fail(ctx, KD_EINVAL,
                       "n = " + std::to_string(n) + " exceeds the static workspace limit of " +
                           std::to_string(NA_MAX_N) + " tuples (KD_NOALLOC_MAX_N); use kd_presort");
    if (cloud->dtype != KD_I32 && cloud->dtype != KD_I64 && cloud->dtype != KD_F32)
        return na_fail(ctx, KD_EINVAL, "bad dtype");
    if (!cloud->on_device) return na_fail(ctx, KD_EINVAL, "coordinates must be device memory (on_device = 1)");
    const int dev = kd::ctx_device(ctx);
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) return na_fail(ctx, KD_EDEVICE, cudaGetErrorString(e));
    if (!on_device_memory(m_out, dev))
        return na_fail(ctx, KD_EINVAL, "m_out must be device memory on the context's device");
    if (n > 0 && (!cloud->coords || !arrays_out || !on_device_memory(cloud->coords, dev) ||
                  !on_device_memory(arrays_out, dev)))
        return na_fail(ctx, KD_EINVAL, "coords and arrays_out must be non-null device memory on the context's device");
    uint64_t* ws = nullptr;
    e = noalloc_setup(dev, &ws);
    if (e != cudaSuccess) return na_fail(ctx, KD_EDEVICE, std::string("set-up: ") + cudaGetErrorString(e));
    cudaStream_t s = kd::ctx_stream(ctx);
    if (n == 0) {
        e = cudaMemsetAsync(m_out, 0, sizeof(int32_t), s);
        return e == cudaSuccess ? KD_OK : na_fail(ctx, KD_EDEVICE, cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(ws + NA_STATUS_WORD, 0, sizeof(uint64_t), s);
    if (e != cudaSuccess) return na_fail(ctx, KD_EDEVICE, cudaGetErrorString(e));
    const int ni = (int)n;
    int grid = (int)((n * k + NA_KEYS_THREADS - 1) / NA_KEYS_THREADS);
    if (grid > 1024) grid = 1024;
    switch (cloud->dtype) {
        case KD_I32:
            e = na_launch(k_noalloc_keys<int32_t>, grid, NA_KEYS_THREADS, 0, s,
                          static_cast<const int32_t*>(cloud->coords), ni, k, ws);
            break;
        case KD_I64:
            e = na_launch(k_noalloc_keys<int64_t>, grid, NA_KEYS_THREADS, 0, s,
                          static_cast<const int64_t*>(cloud->coords), ni, k, ws);
            break;
        default:
            e = na_launch(k_noalloc_keys<float>, grid, NA_KEYS_THREADS, 0, s, static_cast<const float*>(cloud->coords),
                          ni, k, ws);
            break;
    }
    if (e != cudaSuccess) return na_fail(ctx, KD_EDEVICE, std::string("launch: ") + cudaGetErrorString(e));
    int npow2 = 2;
    while (npow2 < ni) npow2 <<= 1;
    const size_t smem = (size_t)npow2 * (sizeof(uint64_t) + sizeof(uint32_t));
    e = na_launch(k_noalloc_sort, k, NA_THREADS, smem, s, ni, npow2, k, (const uint64_t*)ws, arrays_out, m_out);
    if (e != cudaSuccess) return na_fail(ctx, KD_EDEVICE, std::string("launch: ") + cudaGetErrorString(e));
    kd::ctx_add_launches(ctx, 2);
    return KD_OK;
}

// kd_api.cu -- host side of the C ABI declared in include/kdtree.h.
//
// Orders the presort and build kernels of one cloud or a batch of clouds on
// the context's stream, owns device workspace (a private stream-ordered
// memory pool with an optional byte budget), and runs the serving
// scheduler.  No arithmetic of the method happens here: every step of the
// path is a kernel in kd_presort.cu / kd_build.cu.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kd_internal.cuh"
#include "kdtree.h"

namespace kd {
cudaError_t launch_transform(int dtype, const void* coords, int64_t n, int k, void* keys, int64_t stride, void* tail,
                             const int64_t* cloud_start, int ncloud, uint32_t* cloud_plane, int cloud_digits,
                             uint32_t* hist, int* err, cudaStream_t s);
size_t sort_status_words(int64_t max_count);
cudaError_t launch_sort_pass(int key64, const int64_t* count_ptr, int64_t max_count, const void* key_src,
                             void* key_dst, const PayloadArgs& pay, const uint32_t* digit_base, int shift,
                             uint32_t* status, int* err, cudaStream_t s, uint32_t spin_limit = SPIN_LIMIT,
                             int withhold = 0);
cudaError_t launch_digit_bases(const uint32_t* hist, int nrows, uint32_t* bases, cudaStream_t s);
cudaError_t launch_pack_clouds(const PackDesc* d, int count, void* dst, cudaStream_t s);
cudaError_t launch_gather(int key64, const int64_t* count_ptr, int64_t max_count, const void* plane,
                          const uint32_t* ids, void* out, int* err, cudaStream_t s);
size_t dedup_scratch_words(int64_t n);
cudaError_t launch_dedup(int key64, int64_t n, const void* key0, const uint32_t* ids, const void* T, int64_t tstride,
                         int k, const uint32_t* cloud_plane, int cloud_digits, uint32_t* ids_out, void* y1_out,
                         void* y2_out, uint32_t* scratch, int64_t* m_out, uint32_t* hist, int32_t* mcloud, int* err,
                         cudaStream_t s);
cudaError_t launch_own_ranks(const int64_t* m_ptr, int64_t max_m, int k, const AllPlanes& rec, cudaStream_t s);
cudaError_t launch_run_stats(int key64, const int64_t* count_ptr, int64_t max_count, const void* key0, int tk,
                             uint2* range, uint2* cross_runs, uint32_t* run_meta, cudaStream_t s);
size_t run_tile_count(int64_t max_count);
cudaError_t launch_tail_gather(int key64, const int64_t* count_ptr, int64_t max_count, const uint32_t* ids,
                               const void* tail, int tk, void* T, int64_t tstride, int* err, cudaStream_t s);
cudaError_t launch_tie_runs(int key64, const int64_t* count_ptr, int64_t max_count, const void* key0, uint32_t* ids,
                            void* T, int64_t tstride, int tk, const uint2* range, const uint2* cross_runs,
                            const uint32_t* run_meta, int* err, cudaStream_t s);
cudaError_t launch_perm_bases(const int64_t* m_ptr, int shift, uint32_t* bases, cudaStream_t s);
cudaError_t launch_perm_scatter(const int64_t* m_ptr, int64_t max_m, const uint32_t* dest, const PayloadArgs& pa,
                                cudaStream_t s);
cudaError_t launch_arrays_out(const int64_t* m_ptr, int64_t max_m, int k, const AllPlanes& rec,
                              const uint32_t* perm0, int32_t* out, cudaStream_t s);
int level_tile(int k);
cudaError_t launch_shape(int32_t m, int k, int32_t* left, int32_t* right, uint8_t* dim, cudaStream_t s);
cudaError_t launch_tune_cloud(int dtype, void* coords, int64_t count, uint64_t seed, cudaStream_t s);
size_t sel_seg_bytes(int key64);
int sel_finish_tile(int key64, int k);
cudaError_t init_select_kernels();
cudaError_t launch_sel_level(int key64, void* const* id, void* const* key, int cur, int k, int32_t m, int L,
                             int tile, void* segs, uint32_t* ghist, int32_t* gany, uint32_t* unresolved, int32_t* node,
                             int64_t in_off, int* err, cudaStream_t s, int round_begin, int round_end, int phase);
cudaError_t launch_sel_finish(int key64, void* const* id, void* const* key, int cur, int k, int32_t m, int lam, int T,
                              int32_t* node, int32_t* left, int32_t* right, uint8_t* dim, int64_t in_off, int* err,
                              cudaStream_t s);
bool level_tile_supported(int k, int tile);
int level_status_stride(int k);
cudaError_t launch_level_pass(int k, int tile, const AllBufs& bufs, int q, const LevelJob* jobs, int njobs, int ntiles,
                              const CloudDev* clouds, uint32_t* medr, const uint32_t* perm0, uint32_t* status,
                              int* err, cudaStream_t s);
size_t level_status_words(int k, int ntiles);
size_t finish_smem(int k, int smax);
cudaError_t init_presort_kernels();
cudaError_t init_build_kernels();
int finish_kmax(int smax);
cudaError_t launch_finish(const AllBufs& bufs, int k, const int64_t* unit_prefix, int ncloud, int64_t unit_base,
                          int nunits, const CloudDev* clouds, const uint32_t* perm0, int smax, int* err,
                          unsigned long long* phase_ns, cudaStream_t s);
cudaError_t launch_top_nodes(const CloudDev* clouds, const int64_t* prefix, int ncloud, int64_t total, int k,
                             const uint32_t* perm0, uint32_t* medr, int all_nodes, cudaStream_t s);
}  // namespace kd

using namespace kd;

namespace {

// Array 0 by x_0 alone, then its runs of equal x_0 ordered on chip by
// compares, unless the runs of more than 32 tuples would cost more than this
// many compares per tuple (sum of their L^2 over n); then by the whole key.
constexpr uint64_t RUN_COST_PER_TUPLE = 128;

enum Family {
    F_TRANSFORM = 0, F_SORT, F_DEDUP, F_RECORDS, F_LEVEL, F_FINISH, F_TOP, F_OTHER, F_GATHER,
    F_SELECT,         // median-selection build: selection rounds and partitions of the levels
    F_SELECT_FINISH,  // median-selection build: on-chip finisher
    F_TIES,           // array 0: runs of equal x_0 ordered by the other coordinates
    F_COUNT
};

struct TimedLaunch {
    int family;
    cudaEvent_t a, b;
    double units;
    int64_t* units_dev;  // if set, units = *units_dev read after completion
    double bytes_per_unit;  // algorithmic bytes per element of this launch
};

struct Request;

}  // namespace

struct kd_presorted {
    int k = 0, dtype = 0, count = 0;
    int64_t N = 0, M = 0;
    std::vector<int64_t> n_c, in_off, m_c, m_off;
    uint32_t* perm0 = nullptr;
    AllPlanes rec{};
    void* rec_block = nullptr;
    void* sel_keys = nullptr;  // median-selection build: k key planes in array-0 order
    int64_t* d_m = nullptr;
    size_t bytes = 0;
};

struct kd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t pool = nullptr;
    size_t budget = 0;
    size_t in_use = 0;
    int debug = 0;
    int smax_override = 0;
    int level_tile_override = 0;
    // autotuner: the fastest (on-chip subtree size, level tile) measured per
    // (k, dtype, size bucket), and the cache file it is kept in
    struct Tuned {
        int smax, ltile;
        double ms;
    };
    std::map<uint32_t, Tuned> tuning;
    std::string tune_cache;
    int force_smax = 0, force_ltile = 0;  // the candidate kd_autotune is timing
    int schedule = KD_SCHEDULE_MULTI;     // level schedule (kd_config.schedule)
    int last_smax = 0, last_ltile = 0;    // what the last build used
    // Failure-detection tests (debug bit 8): the look-back polls are bounded
    // by a few thousand instead of 2^24, and the next presort's first sort
    // pass has its chunk 0 withhold its flag (once), so that the other
    // chunks' waits run out and the call reports KD_ETIMEOUT.
    uint32_t spin_limit = SPIN_LIMIT;
    bool inject_timeout = false;
    std::string last_error;
    std::recursive_mutex mu;
    std::unordered_map<void*, size_t> sizes;
    std::atomic<int64_t> launches{0};
    // kernel timing (debug bit 2)
    std::vector<TimedLaunch> timed;
    std::vector<cudaEvent_t> event_pool;
    double fam_ms[F_COUNT] = {0};
    double fam_units[F_COUNT] = {0};
    double fam_bytes[F_COUNT] = {0};
    double trace_ns[8] = {0};  // finisher phase block-time sums (debug bit 4)
    int64_t fam_launches[F_COUNT] = {0};
    // copies of host outputs overlapping the finisher (created on first use)
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> chunk_events;
    // pinned host scratch for small uploads
    void* pinned = nullptr;
    size_t pinned_bytes = 0;
    // serving (kd_submit / kd_wait): worker threads, each with a sub-context
    kd_config cfg{};
    std::vector<std::thread> workers;
    std::vector<kd_ctx*> worker_ctx;
    std::mutex qmu;
    std::condition_variable qcv, donecv;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<kd_ticket, std::shared_ptr<Request>> tickets;
    bool stopping = false;
    kd_ticket next_ticket = 1;
    std::vector<double> latencies_us;
    int64_t completed = 0;
};

namespace {

struct Request {
    kd_cloud cloud{};
    std::vector<unsigned char> coords;  // host copy
    kd_tree out{};
    kd_tree* user_out = nullptr;  // receives m and root when the request completes
    kd_status status = KD_OK;
    std::string error;
    bool done = false;
    std::chrono::steady_clock::time_point t_submit, t_done;
    size_t est_bytes = 0;
};

kd_status fail(kd_ctx* ctx, kd_status code, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t _e = (call);                                                                   \
        if (_e != cudaSuccess)                                                                     \
            return fail(ctx, KD_EDEVICE, std::string(#call) + ": " + cudaGetErrorString(_e));      \
    } while (0)

#define CKS(expr)                                                                                  \
    do {                                                                                           \
        kd_status _s = (expr);                                                                     \
        if (_s != KD_OK) return _s;                                                                \
    } while (0)

kd_status dev_alloc(kd_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return KD_OK;
    bytes = (bytes + 255) & ~(size_t)255;
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        return fail(ctx, KD_ENOMEM, "device memory budget exceeded (" + std::to_string(ctx->in_use + bytes) +
                                        " > " + std::to_string(ctx->budget) + " bytes)");
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ctx, KD_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    ctx->in_use += bytes;
    ctx->sizes[*p] = bytes;
    return KD_OK;
}

void dev_free(kd_ctx* ctx, void* p) {
    if (!p) return;
    auto it = ctx->sizes.find(p);
    if (it != ctx->sizes.end()) {
        ctx->in_use -= it->second;
        ctx->sizes.erase(it);
    }
    cudaFreeAsync(p, ctx->stream);
}

// Frees its allocations when it goes out of scope (temporaries of a call).
struct Scratch {
    kd_ctx* ctx;
    std::vector<void*> ptrs;
    explicit Scratch(kd_ctx* c) : ctx(c) {}
    ~Scratch() {
        for (void* p : ptrs) dev_free(ctx, p);
    }
    template <typename T>
    kd_status get(T** out, size_t bytes) {
        void* p = nullptr;
        kd_status s = dev_alloc(ctx, &p, bytes);
        if (s != KD_OK) return s;
        ptrs.push_back(p);
        *out = static_cast<T*>(p);
        return KD_OK;
    }
};

cudaEvent_t take_event(kd_ctx* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// Launch bookkeeping: count, and (timing mode) events around the launch.
struct LaunchTimer {
    kd_ctx* ctx;
    int fam;
    double units;
    int64_t* units_dev;
    double bpu;
    cudaEvent_t a = nullptr;
    LaunchTimer(kd_ctx* c, int f, double u, int64_t* ud = nullptr, double bytes_per_unit = 0)
        : ctx(c), fam(f), units(u), units_dev(ud), bpu(bytes_per_unit) {
        ctx->launches++;
        if (ctx->debug & 2) {
            a = take_event(ctx);
            cudaEventRecord(a, ctx->stream);
        }
    }
    ~LaunchTimer() {
        if (a) {
            cudaEvent_t b = take_event(ctx);
            cudaEventRecord(b, ctx->stream);
            ctx->timed.push_back(TimedLaunch{fam, a, b, units, units_dev, bpu});
        }
    }
};

void collect_timing(kd_ctx* ctx) {
    if (ctx->timed.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto& t : ctx->timed) {
        float ms = 0;
        cudaEventElapsedTime(&ms, t.a, t.b);
        double u = t.units;
        if (t.units_dev) {
            int64_t v = 0;
            cudaPointerAttributes pa{};
            if (cudaPointerGetAttributes(&pa, t.units_dev) == cudaSuccess && pa.type == cudaMemoryTypeDevice)
                cudaMemcpy(&v, t.units_dev, sizeof(v), cudaMemcpyDeviceToHost);
            else
                cudaGetLastError();
            u = (double)v;
        }
        ctx->fam_ms[t.family] += ms;
        ctx->fam_units[t.family] += u;
        ctx->fam_bytes[t.family] += u * t.bytes_per_unit;
        ctx->fam_launches[t.family] += 1;
        ctx->event_pool.push_back(t.a);
        ctx->event_pool.push_back(t.b);
    }
    ctx->timed.clear();
}

// The context's copy stream and at least nev events (created on first use).
kd_status ensure_copy_stream(kd_ctx* ctx, size_t nev) {
    if (!ctx->copy_stream && cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(ctx, KD_EDEVICE, "cannot create the copy stream");
    while (ctx->chunk_events.size() < nev) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return fail(ctx, KD_EDEVICE, "cannot create an event");
        ctx->chunk_events.push_back(e);
    }
    return KD_OK;
}

// Page-locked host memory (copies from and to it run asynchronously).
bool pinned_host(const void* p) {
    cudaPointerAttributes a{};
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

kd_status check_device_err(kd_ctx* ctx, int* d_err) {
    int err = 0;
    CK(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (err & ERR_NAN) return fail(ctx, KD_ENAN, "a float coordinate is NaN");
    if (err & ERR_TIMEOUT) return fail(ctx, KD_ETIMEOUT, "a device look-back wait exceeded its bound");
    if (err & ERR_INTERNAL) return fail(ctx, KD_EDEVICE, "internal consistency check failed on the device");
    return KD_OK;
}

size_t dtype_size(int dtype) { return dtype == KD_I64 ? 8 : 4; }

kd_status validate_cloud(kd_ctx* ctx, const kd_cloud* c) {
    if (!c) return fail(ctx, KD_EINVAL, "cloud is NULL");
    if (c->k < 1 || c->k > KD_MAX_K) return fail(ctx, KD_EINVAL, "k must be in [1, 8]");
    if (c->dtype != KD_I32 && c->dtype != KD_I64 && c->dtype != KD_F32)
        return fail(ctx, KD_EINVAL, "unknown dtype");
    if (c->n < 0 || c->n > KD_MAX_N) return fail(ctx, KD_EINVAL, "n out of range [0, 2^30 - 1]");
    if (c->n > 0 && !c->coords) return fail(ctx, KD_EINVAL, "coords is NULL");
    return KD_OK;
}

int bytes_for(int64_t v) {
    int b = 0;
    while (v > 0) {
        ++b;
        v >>= 8;
    }
    return b;
}

// ------------------------------------------------------------ presort
struct Pass {
    int plane;  // coordinate index, or -1 for the cloud-id plane
    int digit;
    int mode;
    int w;      // key word bytes of the plane
};

// Algorithmic bytes per element of one sort pass: the key word read (and
// written unless the next pass gathers a new plane), each payload word read
// and written (an iota plane is only written), plus the tuple id read for
// a gather.
double pass_bytes(const Pass& P, bool writes_key, int npay) {
    return (double)P.w * (writes_key ? 2 : 1) + 8.0 * npay + (P.mode == KEY_GATHER ? 4.0 : 0.0);
}

// all_arrays = false (median-selection build, single cloud): only array 0
// and its duplicate removal; the handle then holds the k key planes
// gathered into array-0 order instead of the other arrays and the rank
// records.
kd_status presort_batch(kd_ctx* ctx, const kd_cloud* clouds, int count, kd_presorted** out, bool all_arrays = true) {
    *out = nullptr;
    if (count < 1 || !clouds) return fail(ctx, KD_EINVAL, "no clouds");
    for (int i = 0; i < count; ++i) CKS(validate_cloud(ctx, &clouds[i]));
    const int k = clouds[0].k, dtype = clouds[0].dtype;
    for (int i = 1; i < count; ++i)
        if (clouds[i].k != k || clouds[i].dtype != dtype)
            return fail(ctx, KD_EINVAL, "all clouds of a batch must share k and dtype");
    std::unique_ptr<kd_presorted> H(new kd_presorted());
    H->k = k;
    H->dtype = dtype;
    H->count = count;
    H->n_c.resize(count);
    H->in_off.resize(count + 1);
    int64_t N = 0;
    for (int i = 0; i < count; ++i) {
        H->n_c[i] = clouds[i].n;
        H->in_off[i] = N;
        N += clouds[i].n;
    }
    H->in_off[count] = N;
    if (N > KD_MAX_N) return fail(ctx, KD_EINVAL, "total tuples of the batch exceed 2^30 - 1");
    H->N = N;
    const int key64 = dtype == KD_I64;
    const int w = key64 ? 8 : 4;
    const int D = w;
    const int cloud_digits = count > 1 ? std::max(1, bytes_for(count - 1)) : 0;
    const int nrows = k * D + cloud_digits;
    const size_t tsz = dtype_size(dtype);
    cudaStream_t s = ctx->stream;

    // persistent (handle-owned) allocations
    void* p = nullptr;
    CKS(dev_alloc(ctx, &p, sizeof(int64_t)));
    H->d_m = (int64_t*)p;
    CK(cudaMemsetAsync(H->d_m, 0, sizeof(int64_t), s));
    H->M = 0;
    H->m_c.assign(count, 0);
    H->m_off.assign(count + 1, 0);
    if (N == 0) {
        *out = H.release();
        return KD_OK;
    }
    CKS(dev_alloc(ctx, &p, (size_t)pad4(N) * 4 + 16));
    H->perm0 = (uint32_t*)p;
    if (!all_arrays && count != 1) return fail(ctx, KD_EINVAL, "internal: array-0-only presort of a batch");
    const size_t rec_planes = (k >= 2 && all_arrays) ? (size_t)k * k : 0;
    if (rec_planes) {
        kd_status st = dev_alloc(ctx, &H->rec_block, (rec_planes * pad4(N) + 4) * 4);
        if (st != KD_OK) {
            dev_free(ctx, H->perm0);
            dev_free(ctx, H->d_m);
            return st;
        }
        for (int d = 0; d < k; ++d)
            for (int q = 0; q < k; ++q) H->rec.p[d][q] = (uint32_t*)H->rec_block + ((size_t)d * k + q) * pad4(N);
    }
    H->bytes = (size_t)N * 4 + rec_planes * N * 4;
    struct Guard {
        kd_ctx* c;
        kd_presorted* h;
        bool armed = true;
        ~Guard() {
            if (armed && h) {
                dev_free(c, h->perm0);
                dev_free(c, h->rec_block);
                dev_free(c, h->sel_keys);
                dev_free(c, h->d_m);
            }
        }
    } guard{ctx, H.get()};

    Scratch S(ctx);
    // coordinates on the device, clouds back to back
    const void* coords = nullptr;
    // a single cloud in page-locked host memory is uploaded in chunks on the copy stream,
    // each transformed as soon as it has arrived
    const int up_chunks =
        (count == 1 && !clouds[0].on_device && N >= (1 << 20) && pinned_host(clouds[0].coords)) ? 8 : 1;
    if (count == 1 && clouds[0].on_device) {
        coords = clouds[0].coords;
    } else if (up_chunks > 1) {
        unsigned char* cb = nullptr;
        CKS(S.get(&cb, (size_t)N * k * tsz));
        coords = cb;
    } else {
        unsigned char* cb = nullptr;
        CKS(S.get(&cb, (size_t)N * k * tsz));
        // device clouds: one packing kernel over a descriptor table; host
        // clouds: one copy each
        std::vector<PackDesc> pk;
        for (int i = 0; i < count; ++i) {
            if (!clouds[i].n) continue;
            const size_t bytes = (size_t)clouds[i].n * k * tsz;
            if (clouds[i].on_device)
                pk.push_back(PackDesc{clouds[i].coords, (int64_t)(bytes / 4), (int64_t)(H->in_off[i] * k * tsz / 4)});
            else
                CK(cudaMemcpyAsync(cb + (size_t)H->in_off[i] * k * tsz, clouds[i].coords, bytes,
                                   cudaMemcpyHostToDevice, s));
        }
        if (!pk.empty()) {
            PackDesc* d_pk = nullptr;
            CKS(S.get(&d_pk, pk.size() * sizeof(PackDesc)));
            CK(cudaMemcpyAsync(d_pk, pk.data(), pk.size() * sizeof(PackDesc), cudaMemcpyHostToDevice, s));
            LaunchTimer lt(ctx, F_OTHER, 0.0);
            CK(launch_pack_clouds(d_pk, (int)pk.size(), cb, s));
        }
        coords = cb;  // (a copy from pageable memory has read pk by the time it returns)
    }
    unsigned char* keys = nullptr;
    uint32_t *cloud_plane = nullptr, *hist = nullptr;
    int64_t *cstart = nullptr, *d_n = nullptr;
    int32_t* mcloud = nullptr;
    int* d_err = nullptr;
    // every plane and sort buffer: stride padded to 16 bytes plus 16 bytes of
    // slack, for the 16-byte-aligned bulk copies of the sort passes
    const int64_t NS = pad4(N);
    CKS(S.get(&keys, (size_t)k * NS * w + 16));
    // tail records: keys x_1..x_{k-1} of each tuple side by side (duplicate
    // removal reads one record per tuple)
    unsigned char* tail = nullptr;
    if (k >= 2) CKS(S.get(&tail, (size_t)N * (k - 1) * w + 16));
    if (count > 1) {
        CKS(S.get(&cloud_plane, (size_t)NS * 4 + 16));
        CKS(S.get(&cstart, (size_t)(count + 1) * 8));
    }
    CKS(S.get(&hist, (size_t)nrows * RADIX * 4));
    uint32_t *bases_all = nullptr, *bases_kept = nullptr;  // digit bases over all / kept tuples
    CKS(S.get(&bases_all, (size_t)nrows * RADIX * 4));
    CKS(S.get(&bases_kept, (size_t)nrows * RADIX * 4));
    CKS(S.get(&d_n, 8));
    CKS(S.get(&mcloud, (size_t)count * 4));
    CKS(S.get(&d_err, 4));
    CK(cudaMemsetAsync(hist, 0, (size_t)nrows * RADIX * 4, s));
    CK(cudaMemsetAsync(d_err, 0, 4, s));
    std::vector<int32_t> nc32(count);
    for (int i = 0; i < count; ++i) nc32[i] = (int32_t)H->n_c[i];
    CK(cudaMemcpyAsync(d_n, &N, 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(mcloud, nc32.data(), (size_t)count * 4, cudaMemcpyHostToDevice, s));
    if (count > 1)
        CK(cudaMemcpyAsync(cstart, H->in_off.data(), (size_t)(count + 1) * 8, cudaMemcpyHostToDevice, s));
    if (up_chunks > 1) {
        CKS(ensure_copy_stream(ctx, up_chunks + 1));
        cudaStream_t cs = ctx->copy_stream;
        CK(cudaEventRecord(ctx->chunk_events[up_chunks], s));  // the upload buffer is ready on s
        CK(cudaStreamWaitEvent(cs, ctx->chunk_events[up_chunks], 0));
        const size_t row = (size_t)k * tsz;
        unsigned char* cb = (unsigned char*)coords;
        for (int c = 0; c < up_chunks; ++c) {
            const int64_t r0 = N * c / up_chunks, r1 = N * (c + 1) / up_chunks;
            CK(cudaMemcpyAsync(cb + r0 * row, (const unsigned char*)clouds[0].coords + r0 * row, (r1 - r0) * row,
                               cudaMemcpyHostToDevice, cs));
            CK(cudaEventRecord(ctx->chunk_events[c], cs));
        }
        for (int c = 0; c < up_chunks; ++c) {
            const int64_t r0 = N * c / up_chunks, r1 = N * (c + 1) / up_chunks;
            CK(cudaStreamWaitEvent(s, ctx->chunk_events[c], 0));
            LaunchTimer lt(ctx, F_TRANSFORM, (double)(r1 - r0), nullptr, (double)k * (tsz + w));
            CK(launch_transform(dtype, cb + r0 * row, r1 - r0, k, keys + r0 * w, NS,
                                tail ? tail + r0 * (k - 1) * w : nullptr, cstart, 1, cloud_plane, cloud_digits, hist,
                                d_err, s));
        }
    } else {
        LaunchTimer lt(ctx, F_TRANSFORM, (double)N, nullptr, (double)k * (tsz + w) + (count > 1 ? 4 : 0));
        CK(launch_transform(dtype, coords, N, k, keys, NS, tail, cstart, count, cloud_plane, cloud_digits, hist, d_err,
                            s));
    }
    {
        LaunchTimer lt(ctx, F_OTHER, 0.0);
        CK(launch_digit_bases(hist, nrows, bases_all, s));
    }
    std::vector<uint32_t> h_hist((size_t)nrows * RADIX);
    CK(cudaMemcpyAsync(h_hist.data(), hist, h_hist.size() * 4, cudaMemcpyDeviceToHost, s));
    CKS(check_device_err(ctx, d_err));  // synchronises
    auto trivial = [&](int row) {
        int nz = 0;
        for (int b = 0; b < RADIX; ++b) nz += h_hist[(size_t)row * RADIX + b] != 0;
        return nz <= 1;
    };
    auto row_of = [&](int plane, int digit) { return plane >= 0 ? plane * D + digit : k * D + digit; };

    // pass lists ------------------------------------------------------
    // a sort = its passes; the first pass of each plane always runs
    auto plane_passes = [&](std::vector<Pass>& v, int plane, int ndig, bool first_of_sort_direct) {
        for (int b = 0; b < ndig; ++b) {
            if (b > 0 && trivial(row_of(plane, b))) continue;
            int mode = b == 0 ? (first_of_sort_direct ? KEY_DIRECT : KEY_GATHER) : KEY_BUF;
            v.push_back(Pass{plane, b, mode, plane >= 0 ? w : 4});
        }
    };
    std::vector<Pass> s0;
    for (int c = k - 1; c >= 0; --c) plane_passes(s0, c, D, c == k - 1);
    std::vector<std::vector<Pass>> chain;  // chain[i] sorts array d = k-1-i
    for (int d = k - 1; d >= 1; --d) {
        std::vector<Pass> v;
        plane_passes(v, d, D, false);
        if (count > 1) plane_passes(v, -1, cloud_digits, false);
        chain.push_back(v);
    }
    std::vector<Pass> cloud_sort;
    if (count > 1) plane_passes(cloud_sort, -1, cloud_digits, false);

    // buffers
    // one status area serves every sort pass in turn (each pass clears what
    // it needs), followed by the dedup scratch
    uint32_t* status = nullptr;
    const size_t status_words = sort_status_words(N);
    const size_t dedup_words = dedup_scratch_words(N);
    CKS(S.get(&status, (status_words + dedup_words) * 4));
    unsigned char* kbuf[2];
    uint32_t* ibuf[2];
    const int maxpay = k + 1;
    uint32_t* pbuf[2][MAXPAY];
    CKS(S.get(&kbuf[0], (size_t)NS * w + 16));
    CKS(S.get(&kbuf[1], (size_t)NS * w + 16));
    CKS(S.get(&ibuf[0], (size_t)NS * 4 + 16));
    CKS(S.get(&ibuf[1], (size_t)NS * 4 + 16));
    if (k >= 2)
        for (int b = 0; b < 2; ++b)
            for (int j = 0; j < maxpay; ++j) CKS(S.get(&pbuf[b][j], (size_t)NS * 4 + 16));
    auto plane_ptr = [&](int plane) -> const void* {
        return plane >= 0 ? (const void*)(keys + (size_t)plane * NS * w) : (const void*)cloud_plane;
    };
    auto plane64 = [&](int plane) { return plane >= 0 ? key64 : 0; };

    // S_0: ids by super key 0 (all n tuples) ----------------------------
    // Array 0 is sorted by x_0 alone, and each run of equal x_0 is then
    // ordered by the remaining coordinates on chip (launch_tie_runs).  Only
    // if a run is too long for that does array 0 take the sort by the whole
    // super key, least significant coordinate first.  With 32-bit keys, the
    // passes of plane k-1 carry plane k-2 along as a second payload, so that
    // plane k-2's first pass reads its keys in order instead of gathering
    // them at random (a gather reads a few 32-byte sectors per 4-byte key;
    // the carry adds 8 streamed bytes per pass).
    int kc = 0, ic = 0;  // current key / id buffer
    auto sort_array0 = [&](const std::vector<Pass>& list, bool whole_key) -> kd_status {
        const int carry_plane = (whole_key && k >= 2 && !key64) ? k - 2 : -1;
        int cy = 0;                         // carried plane: current ping-pong buffer
        const uint32_t* carried = nullptr;  // plane k-2 in the current order, once carried
        kc = 0;
        ic = 0;
        for (size_t i = 0; i < list.size(); ++i) {
            const Pass& P = list[i];
            const bool last = i + 1 == list.size();
            const bool carry = carry_plane >= 0 && P.plane == k - 1;
            const bool from_carry = carry_plane >= 0 && P.plane == carry_plane && P.mode == KEY_GATHER;
            const bool next_gathers = !last && list[i + 1].mode != KEY_BUF;
            PayloadArgs pay{};
            pay.n = 1;
            pay.src[0] = P.mode == KEY_DIRECT ? nullptr : ibuf[ic];
            pay.dst[0] = ibuf[ic ^ 1];
            if (carry) {
                pay.n = 2;
                pay.src[1] = P.mode == KEY_DIRECT ? (const uint32_t*)plane_ptr(carry_plane) : pbuf[cy][0];
                pay.dst[1] = pbuf[cy ^ 1][0];
            }
            const void* ksrc = P.mode == KEY_BUF ? (const void*)kbuf[kc] : plane_ptr(P.plane);
            void* kdst = next_gathers ? nullptr : (void*)kbuf[kc ^ 1];
            if (from_carry) {
                if (!carried) return fail(ctx, KD_EINVAL, "internal: carried plane missing");
                ksrc = carried;
            } else if (P.mode == KEY_GATHER) {  // gather the new plane's keys into order first
                LaunchTimer lg(ctx, F_GATHER, (double)N, nullptr, 4.0 + 2.0 * P.w);
                CK(launch_gather(plane64(P.plane), d_n, N, plane_ptr(P.plane), ibuf[ic], kbuf[kc], d_err, s));
                ksrc = kbuf[kc];
            }
            const bool inject = ctx->inject_timeout && i == 0;
            {
                LaunchTimer lt(ctx, F_SORT, (double)N, nullptr, pass_bytes(P, kdst != nullptr, pay.n));
                ctx->launches += 2;  // count and scan kernels of the pass
                CK(launch_sort_pass(plane64(P.plane), d_n, N, ksrc, kdst, pay,
                                    bases_all + (size_t)row_of(P.plane, P.digit) * RADIX, 8 * P.digit, status, d_err, s,
                                    ctx->spin_limit, inject ? 1 : 0));
            }
            if (inject) {  // the injected wait: report it before anything else runs
                ctx->inject_timeout = false;
                CKS(check_device_err(ctx, d_err));
            }
            kc ^= 1;
            ic ^= 1;
            if (carry) {
                cy ^= 1;
                carried = pbuf[cy][0];
            }
        }
        return KD_OK;
    };
    std::vector<Pass> s0_x0;
    plane_passes(s0_x0, 0, D, true);
    const bool by_runs = k >= 2 && N >= 2;
    bool whole_key = !by_runs;
    CKS(sort_array0(by_runs ? s0_x0 : s0, whole_key));
    uint32_t* run_meta = nullptr;
    uint2 *run_range = nullptr, *cross_runs = nullptr;
    if (by_runs) {
        CKS(S.get(&run_meta, 4 * sizeof(uint32_t)));
        CKS(S.get(&run_range, run_tile_count(N) * sizeof(uint2)));
        CKS(S.get(&cross_runs, run_tile_count(N) * sizeof(uint2)));
        {
            LaunchTimer lt(ctx, F_TIES, (double)N, nullptr, (double)w);
            CK(launch_run_stats(key64, d_n, N, kbuf[kc], k - 1, run_range, cross_runs, run_meta, s));
        }
        uint32_t meta[4] = {0, 0, 0, 0};
        CK(cudaMemcpyAsync(meta, run_meta, sizeof(meta), cudaMemcpyDeviceToHost, s));
        CKS(check_device_err(ctx, d_err));  // synchronises
        // ordering the runs by compares costs sum(L^2) over the long ones;
        // above RUN_COST_PER_TUPLE per tuple the whole-key sort is cheaper
        const uint64_t cost = (uint64_t)meta[0] | ((uint64_t)meta[1] << 32);
        if (meta[2] || cost > (uint64_t)RUN_COST_PER_TUPLE * (uint64_t)N) {
            whole_key = true;
            CKS(sort_array0(s0, true));
        }
    }
    // x_1..x_{k-1} of every position of array 0, so that run ordering and
    // duplicate removal stream
    unsigned char* tplanes = nullptr;
    if (k >= 2) {
        CKS(S.get(&tplanes, (size_t)(k - 1) * NS * w + 16));
        LaunchTimer lg(ctx, F_GATHER, (double)N, nullptr, 4.0 + 2.0 * (k - 1) * w);
        CK(launch_tail_gather(key64, d_n, N, ibuf[ic], tail, k - 1, tplanes, NS, d_err, s));
    }
    if (!whole_key) {
        LaunchTimer lt(ctx, F_TIES, (double)N, nullptr, 2.0 * (4.0 + (k - 1) * w) + w);
        ctx->launches += 1;  // tiles, crossing runs
        CK(launch_tie_runs(key64, d_n, N, kbuf[kc], ibuf[ic], tplanes, NS, k - 1, run_range, cross_runs, run_meta,
                           d_err, s));
    }
    // dedup ---------------------------------------------------------------
    uint32_t* dedup_out = count == 1 ? H->perm0 : ibuf[ic ^ 1];
    // single cloud: duplicate removal also hands the chain x_{k-1} (into the
    // key buffer the chain's first sort reads) and, for 32-bit keys and
    // k >= 3, x_{k-2} (carried through that sort for the next one), both in
    // array-0 order, so neither needs a gather
    const bool y_first = count == 1 && k >= 2 && all_arrays;
    const bool y_second = y_first && k >= 3 && !key64;
    unsigned char* y2c = nullptr;
    if (y_second) CKS(S.get(&y2c, (size_t)NS * w + 16));
    {
        LaunchTimer lt(ctx, F_DEDUP, (double)N, nullptr, 2.0 * w + 8 + (k - 1) * w);
        ctx->launches += 2;  // flags, tile scan, compaction
        CK(launch_dedup(key64, N, kbuf[kc], ibuf[ic], tplanes, NS, k, cloud_plane, cloud_digits, dedup_out,
                        y_first ? (void*)kbuf[kc] : nullptr, y2c, status + status_words, H->d_m, hist, mcloud, d_err,
                        s));
    }
    ic ^= 1;
    {
        LaunchTimer lt(ctx, F_OTHER, 0.0);
        CK(launch_digit_bases(hist, nrows, bases_kept, s));
    }
    // cloud grouping of array 0 (batches) ----------------------------------
    for (size_t i = 0; i < cloud_sort.size(); ++i) {
        const Pass& P = cloud_sort[i];
        const bool last = i + 1 == cloud_sort.size();
        PayloadArgs pay{};
        pay.n = 1;
        pay.src[0] = ibuf[ic];
        pay.dst[0] = last ? H->perm0 : ibuf[ic ^ 1];
        const void* ksrc = P.mode == KEY_BUF ? (const void*)kbuf[kc] : plane_ptr(-1);
        if (P.mode == KEY_GATHER) {
            LaunchTimer lg(ctx, F_GATHER, 0.0, H->d_m, 12.0);
            CK(launch_gather(0, H->d_m, N, plane_ptr(-1), ibuf[ic], kbuf[kc], d_err, s));
            ksrc = kbuf[kc];
        }
        LaunchTimer lt(ctx, F_SORT, 0.0, H->d_m, pass_bytes(P, !last, 1));
        ctx->launches += 2;  // count and scan kernels of the pass
        CK(launch_sort_pass(0, H->d_m, N, ksrc, last ? nullptr : (void*)kbuf[kc ^ 1], pay,
                            bases_kept + (size_t)row_of(-1, P.digit) * RADIX, 8 * P.digit, status, d_err, s,
                            ctx->spin_limit));
        kc ^= 1;
        ic ^= 1;
    }
    // median-selection build: the key planes in array-0 order ----------------
    if (!all_arrays) {
        kd_status st = dev_alloc(ctx, &H->sel_keys, (size_t)k * NS * w + 16);
        if (st != KD_OK) return st;
        for (int d = 0; d < k; ++d) {
            LaunchTimer lg(ctx, F_GATHER, 0.0, H->d_m, 4.0 + 2.0 * w);
            CK(launch_gather(key64, H->d_m, N, plane_ptr(d), H->perm0,
                             (unsigned char*)H->sel_keys + (size_t)d * NS * w, d_err, s));
        }
    }
    // chain: array d = stable sort of array d+1 by x_d (then cloud) --------
    // payload plane list: [id (while a later gather needs it)], R_0, R_{k-1}, ..., R_{d+1}
    if (k >= 2 && all_arrays) {
        const uint32_t* id_src = H->perm0;  // array 0 order
        // the first sort's keys come from duplicate removal; the second's are
        // carried through the first sort (see above)
        auto gathers = [&](size_t ci, const Pass& P) {
            return P.mode == KEY_GATHER && !(ci == 0 && y_first) && !(ci == 1 && y_second);
        };
        int gathers_left = 0;
        for (size_t ci = 0; ci < chain.size(); ++ci)
            for (auto& P : chain[ci]) gathers_left += gathers(ci, P);
        std::vector<int> ranks_prev;  // rank planes carried by the previous array (R index list)
        const void* ysrc = y2c;       // x_{k-2} in the current order while it is carried
        for (size_t ci = 0; ci < chain.size(); ++ci) {
            const int d = k - 1 - (int)ci;
            const auto& v = chain[ci];
            // current sources of payload planes
            std::vector<int> ranks = ranks_prev;
            ranks.push_back((d + 1) % k);  // new plane: R_{d+1} = source position
            // source pointers for the first pass: from rec[d+1][r] or iota
            std::vector<const uint32_t*> rsrc(ranks.size());
            for (size_t j = 0; j < ranks.size(); ++j)
                rsrc[j] = (j + 1 == ranks.size()) ? nullptr : H->rec.p[(d + 1) % k][ranks[j]];
            const uint32_t* cur_id = id_src;
            int pb = 0;  // payload ping-pong
            for (size_t i = 0; i < v.size(); ++i) {
                const Pass& P = v[i];
                const bool last = i + 1 == v.size();
                const bool gather = gathers(ci, P);
                if (gather) --gathers_left;
                const bool carry_id = gathers_left > 0;
                const bool next_gathers = !last && v[i + 1].mode != KEY_BUF;
                PayloadArgs pay{};
                int np = 0;
                uint32_t* new_id = nullptr;
                if (carry_id) {
                    pay.src[np] = cur_id;
                    new_id = (cur_id == ibuf[0]) ? ibuf[1] : ibuf[0];
                    pay.dst[np] = new_id;
                    ++np;
                }
                for (size_t j = 0; j < ranks.size(); ++j) {
                    pay.src[np] = rsrc[j];
                    pay.dst[np] = last ? H->rec.p[d][ranks[j]] : pbuf[pb][j];
                    ++np;
                }
                // x_{k-2} for the next sort, ending in the key buffer it reads
                const bool carry_y = ci == 0 && y_second;
                if (carry_y) {
                    pay.src[np] = (const uint32_t*)ysrc;
                    pay.dst[np] = last ? (uint32_t*)kbuf[kc ^ 1] : pbuf[pb][maxpay - 1];
                    ++np;
                }
                pay.n = np;
                const void* ksrc = P.mode == KEY_BUF || !gather ? (const void*)kbuf[kc] : plane_ptr(P.plane);
                void* kdst = (last || next_gathers) ? nullptr : (void*)kbuf[kc ^ 1];
                if (gather) {
                    LaunchTimer lg(ctx, F_GATHER, 0.0, H->d_m, 4.0 + 2.0 * P.w);
                    CK(launch_gather(plane64(P.plane), H->d_m, N, plane_ptr(P.plane), cur_id, kbuf[kc], d_err, s));
                    ksrc = kbuf[kc];
                }
                LaunchTimer lt(ctx, F_SORT, 0.0, H->d_m, pass_bytes(P, kdst != nullptr, pay.n));
                ctx->launches += 2;  // count and scan kernels of the pass
                CK(launch_sort_pass(plane64(P.plane), H->d_m, N, ksrc, kdst, pay,
                                    bases_kept + (size_t)row_of(P.plane, P.digit) * RADIX, 8 * P.digit, status,
                                    d_err, s, ctx->spin_limit));
                kc ^= 1;
                if (carry_id) cur_id = new_id;
                for (size_t j = 0; j < ranks.size(); ++j) rsrc[j] = last ? H->rec.p[d][ranks[j]] : pbuf[pb][j];
                if (carry_y) ysrc = pbuf[pb][maxpay - 1];
                pb ^= 1;
            }
            id_src = cur_id;
            ranks_prev = ranks;
        }
        // Remaining rank planes: array d (d != 1) lacks the ranks R_p of the
        // planes the chain did not carry; they are a permutation of array 1's
        // planes by destination R_d.  Each is done as one grouping pass on the
        // top bits of R_d (ranges that fit in L2) and an in-range scatter.
        uint32_t* pbases = nullptr;
        CKS(S.get(&pbases, RADIX * 4));
        uint64_t present = 0;  // 8 bits per array: planes already written
        for (int d = 0; d < k; ++d) {
            if (d == 1) {
                uint64_t bits = 0;
                for (int q = 0; q < k; ++q) bits |= (q != 1) ? (1u << q) : 0u;
                present |= bits << (d * MAXK);
                continue;
            }
            uint64_t bits = (d >= 2) ? 1u : 0u;  // chain output carries R_0 and R_{d+1..k-1}
            if (d >= 2)
                for (int q = d + 1; q < k; ++q) bits |= 1u << q;
            std::vector<int> miss;
            for (int q = 0; q < k; ++q)
                if (q != d && !((bits >> q) & 1u)) miss.push_back(q);
            if (!miss.empty()) {
                const int nv = (int)miss.size();
                // destination ranges of about 16 MB of scattered words: the
                // scatter's random 4-byte writes then merge in L2 (2^26
                // tuples: 1.92 ms for the records against 2.01 ms with 48 MB
                // ranges, 1.92 with 8 MB)
                int shift = 0;
                while (((int64_t)1 << shift) * nv * 4 < ((int64_t)16 << 20) && shift < 30) ++shift;
                while ((((int64_t)N - 1) >> shift) > 255) ++shift;
                {
                    LaunchTimer lt(ctx, F_OTHER, 0.0);
                    CK(launch_perm_bases(H->d_m, shift, pbases, s));
                }
                PayloadArgs pay{};
                pay.n = nv;
                for (int j = 0; j < nv; ++j) {
                    pay.src[j] = miss[j] == 1 ? nullptr : H->rec.p[1][miss[j]];  // R_1 of array 1 = position
                    pay.dst[j] = pbuf[0][j];
                }
                uint32_t* gdest = ibuf[0];
                {
                    LaunchTimer lt(ctx, F_RECORDS, 0.0, H->d_m, 4.0 + 8.0 * nv + 4.0);
                    ctx->launches += 2;  // count and scan kernels of the pass
                    CK(launch_sort_pass(0, H->d_m, N, H->rec.p[1][d], gdest, pay, pbases, shift, status, d_err, s,
                                        ctx->spin_limit));
                }
                PayloadArgs sc{};
                sc.n = nv;
                for (int j = 0; j < nv; ++j) {
                    sc.src[j] = pbuf[0][j];
                    sc.dst[j] = H->rec.p[d][miss[j]];
                }
                LaunchTimer lt(ctx, F_RECORDS, 0.0, H->d_m, 4.0 + 8.0 * nv);
                CK(launch_perm_scatter(H->d_m, N, gdest, sc, s));
                for (int q : miss) bits |= 1u << q;
            }
            present |= bits << (d * MAXK);
        }
        if (present != 0) {
            LaunchTimer lt(ctx, F_RECORDS, 0.0, H->d_m, 4.0);
            CK(launch_own_ranks(H->d_m, N, k, H->rec, s));
        }
    }
    // learn m ----------------------------------------------------------------
    int64_t M = 0;
    CK(cudaMemcpyAsync(&M, H->d_m, 8, cudaMemcpyDeviceToHost, s));
    std::vector<int32_t> mc(count);
    CK(cudaMemcpyAsync(mc.data(), mcloud, (size_t)count * 4, cudaMemcpyDeviceToHost, s));
    CKS(check_device_err(ctx, d_err));
    H->M = M;
    int64_t acc = 0;
    for (int i = 0; i < count; ++i) {
        H->m_c[i] = mc[i];
        H->m_off[i] = acc;
        acc += mc[i];
    }
    H->m_off[count] = acc;
    if (acc != M) return fail(ctx, KD_EDEVICE, "per-cloud counts do not add up to m");
    if (ctx->debug & 1) CK(cudaStreamSynchronize(s));
    guard.armed = false;
    *out = H.release();
    return KD_OK;
}

void release_handle(kd_ctx* ctx, kd_presorted* h) {
    if (!h) return;
    dev_free(ctx, h->perm0);
    dev_free(ctx, h->rec_block);
    dev_free(ctx, h->sel_keys);
    dev_free(ctx, h->d_m);
    delete h;
}

// ---------------------------------------------------------------- build
int64_t max_seg(int64_t m, int L) {
    for (int l = 0; l < L; ++l) m /= 2;
    return m;
}
int nlevels(int64_t m) {
    int L = 0;
    while (((int64_t)1 << L) <= m) ++L;
    return L;  // ceil(log2(m + 1))
}

// ---------------------------------------------------------- tuned parameters
// Size bucket: floor(log2 n) of the largest cloud.
uint32_t tune_key(int k, int dtype, int64_t n) {
    int b = 0;
    while (b < 62 && ((int64_t)2 << b) <= n) ++b;
    return ((uint32_t)k << 16) | ((uint32_t)dtype << 8) | (uint32_t)b;
}

// The on-chip subtree size and the level-step tile a build of clouds of at
// most nmax tuples uses: the candidate being timed by kd_autotune, else the
// context's fixed settings, else the tuned entry for (k, dtype, bucket),
// else the defaults (1024; 2048 for k <= 4, 1024 above).
void choose_params(kd_ctx* ctx, int k, int dtype, int64_t nmax, int* smax_out, int* ltile_out) {
    const auto it = ctx->tuning.find(tune_key(k, dtype, nmax));
    const bool tuned = it != ctx->tuning.end();
    int want = ctx->force_smax ? ctx->force_smax
                               : (ctx->smax_override ? ctx->smax_override : (tuned ? it->second.smax : 1024));
    int smax = 1024;
    while (smax < want && smax < 4096) smax *= 2;
    while (smax > 1024 && k > finish_kmax(smax)) smax /= 2;
    int lt = ctx->force_ltile ? ctx->force_ltile
                              : (ctx->level_tile_override ? ctx->level_tile_override
                                                          : (tuned ? it->second.ltile : level_tile(std::max(k, 2))));
    if (!level_tile_supported(std::max(k, 2), lt)) lt = level_tile(std::max(k, 2));
    *smax_out = smax;
    *ltile_out = lt;
}

// Tuning cache file: one line per entry, "k dtype bucket smax level_tile ms".
void tuning_load(kd_ctx* ctx) {
    if (ctx->tune_cache.empty()) return;
    FILE* f = fopen(ctx->tune_cache.c_str(), "r");
    if (!f) return;
    int k, dt, b, sm, lt;
    double ms;
    while (fscanf(f, "%d %d %d %d %d %lf", &k, &dt, &b, &sm, &lt, &ms) == 6) {
        if (k < 1 || k > KD_MAX_K || dt < 0 || dt > 2 || b < 0 || b > 62) continue;
        if (sm != 1024 && sm != 2048 && sm != 4096) continue;
        ctx->tuning[((uint32_t)k << 16) | ((uint32_t)dt << 8) | (uint32_t)b] = kd_ctx::Tuned{sm, lt, ms};
    }
    fclose(f);
}

bool tuning_save(kd_ctx* ctx) {
    if (ctx->tune_cache.empty()) return true;
    const std::string tmp = ctx->tune_cache + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    for (const auto& e : ctx->tuning)
        fprintf(f, "%u %u %u %d %d %.6f\n", e.first >> 16, (e.first >> 8) & 255u, e.first & 255u, e.second.smax,
                e.second.ltile, e.second.ms);
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), ctx->tune_cache.c_str()) == 0;
}

kd_status build_batch(kd_ctx* ctx, kd_presorted* H, kd_tree* outs) {
    const int k = H->k, count = H->count;
    const int64_t M = H->M;
    cudaStream_t s = ctx->stream;
    for (int i = 0; i < count; ++i) {
        if (!outs[i].node_tuple && H->m_c[i] > 0) return fail(ctx, KD_EINVAL, "node_tuple output is NULL");
        outs[i].m = (int32_t)H->m_c[i];
        outs[i].root = H->m_c[i] > 0 ? (int32_t)((H->m_c[i] - 1) / 2) : -1;
    }
    if (M == 0) return KD_OK;
    Scratch S(ctx);
    int* d_err = nullptr;
    CKS(S.get(&d_err, 4));
    CK(cudaMemsetAsync(d_err, 0, 4, s));
    // subtree size finished on chip (a power of two in [1024, 4096]) and
    // level-step tile (1024 or 2048 positions; a tile may touch at most 4
    // segments, so segments above the finisher need at least tile / 3):
    // tuned per (k, dtype, size bucket), else 1024 and the larger tile
    int smax = 1024, tile = level_tile(std::max(k, 2));
    {
        int64_t nmax = 0;
        for (int i = 0; i < count; ++i) nmax = std::max(nmax, H->n_c[i]);
        choose_params(ctx, k, H->dtype, nmax, &smax, &tile);
    }
    ctx->last_smax = smax;
    ctx->last_ltile = tile;
    if (k >= 2 && smax * 3 < tile + 3) return fail(ctx, KD_EINVAL, "switch threshold too small");

    // outputs: user device arrays, or staging for host arrays
    bool any_host = false, want_l = false, want_r = false, want_d = false;
    for (int i = 0; i < count; ++i) {
        any_host |= !outs[i].on_device;
        want_l |= outs[i].left != nullptr;
        want_r |= outs[i].right != nullptr;
        want_d |= outs[i].dim != nullptr;
    }
    int32_t *st_node = nullptr, *st_left = nullptr, *st_right = nullptr;
    uint8_t* st_dim = nullptr;
    if (any_host) {
        CKS(S.get(&st_node, (size_t)M * 4));
        if (want_l) CKS(S.get(&st_left, (size_t)M * 4));
        if (want_r) CKS(S.get(&st_right, (size_t)M * 4));
        if (want_d) CKS(S.get(&st_dim, (size_t)M));
    }
    std::vector<CloudDev> cd(count);
    std::vector<int> lam(count);
    int64_t medr_total = 0;
    int maxlam = 0;
    for (int i = 0; i < count; ++i) {
        CloudDev& c = cd[i];
        memset(&c, 0, sizeof(c));
        c.off = H->m_off[i];
        c.in_off = H->in_off[i];
        c.m = (int32_t)H->m_c[i];
        const int64_t m = H->m_c[i];
        int L = 0;
        if (k == 1) {
            L = nlevels(m);
        } else {
            while (max_seg(m, L) > smax) ++L;
        }
        lam[i] = L;
        c.lam = L;
        c.medr_off = medr_total;
        if (k >= 2 && L >= 1) medr_total += ((int64_t)1 << L) - 1;
        maxlam = std::max(maxlam, L);
        if (outs[i].on_device) {
            c.node = outs[i].node_tuple;
            c.left = outs[i].left;
            c.right = outs[i].right;
            c.dim = outs[i].dim;
        } else {
            c.node = st_node + c.off;
            c.left = outs[i].left ? st_left + c.off : nullptr;
            c.right = outs[i].right ? st_right + c.off : nullptr;
            c.dim = outs[i].dim ? st_dim + c.off : nullptr;
        }
    }
    uint32_t* medr = nullptr;
    if (medr_total) CKS(S.get(&medr, (size_t)medr_total * 4));

    // schedule of level passes -------------------------------------------
    std::vector<std::vector<LevelJob>> step_jobs;
    std::vector<int64_t> step_ntiles;
    std::vector<double> step_elems;
    std::vector<int> step_q;
    std::vector<std::array<int, MAXK>> moves(count), level(count);
    for (int i = 0; i < count; ++i) {
        moves[i].fill(0);
        level[i].fill(0);
    }
    bool need_bufs = false;
    if (k >= 2) {
        // Level schedule.  Array q lies sorted within the segments of some
        // level; a step moves it from level lin to level lout (applying the
        // splits of levels lin .. lout-1 around their medians).  At its
        // primary level its halves are in place (a free split).
        //   KD_SCHEDULE_MULTI (default): step t moves array t mod k to level
        //     t, through up to k-1 levels at once: each array is partitioned
        //     only when it is about to become primary, one pass per level.
        //   KD_SCHEDULE_DEFERRED (Appendix "Deferred Merge Sort and
        //     Partitioning"): array d first appears at level d, already split
        //     by levels 0 .. d-1 (one pass); from then on every non-primary
        //     array is partitioned at every level, one level per pass.
        //   KD_SCHEDULE_EVERY_LEVEL (Section 2.1): every non-primary array is
        //     partitioned at every level, one level per pass.
        const int sched = ctx->schedule;
        int lmax = 0;
        for (int i = 0; i < count; ++i) lmax = std::max(lmax, lam[i]);
        std::vector<std::pair<int, int>> steps;  // (t, q): move array q to level t
        if (sched == KD_SCHEDULE_MULTI) {
            for (int t = 1; t <= lmax + k - 2; ++t) steps.push_back({t, t % k});
        } else {
            for (int t = 1; t <= lmax; ++t)
                for (int q = 0; q < k; ++q)
                    if (!(sched == KD_SCHEDULE_DEFERRED && q >= 1 && t < q)) steps.push_back({t, q});
        }
        for (const auto& tq : steps) {
            const int t = tq.first, q = tq.second;
            std::vector<LevelJob> jl;
            int64_t ntl = 0;
            double el = 0;
            for (int i = 0; i < count; ++i) {
                if (lam[i] < 1) continue;
                const int cur = level[i][q];
                int lin = cur;
                if (cur % k == q && cur < lam[i]) lin = cur + 1;
                const int lout = std::min(t, lam[i]);
                if (lin >= lout) {
                    level[i][q] = std::max(cur, std::min(lin, lam[i]));
                    continue;
                }
                if (lout - lin > k - 1) return fail(ctx, KD_EDEVICE, "internal: level pass spans too many levels");
                if (max_seg(H->m_c[i], lin) - 1 < (tile + 2) / 3)
                    return fail(ctx, KD_EDEVICE, "internal: segments too small for a level-pass tile");
                LevelJob J{};
                J.cloud = i;
                J.lev_in = lin;
                J.lev_out = lout;
                J.src_buf = buf_after(moves[i][q]);
                J.dst_buf = buf_after(moves[i][q] + 1);
                J.write_med = (lout % k == q) && (lout < lam[i]) ? LEVEL_MED : 0;
                J.tile_begin = ntl;
                jl.push_back(J);
                ntl += (H->m_c[i] + tile - 1) / tile;
                el += (double)H->m_c[i];
                moves[i][q] += 1;
                level[i][q] = lout;
                need_bufs = true;
            }
            if (!jl.empty()) {
                step_jobs.push_back(std::move(jl));
                step_ntiles.push_back(ntl);
                step_elems.push_back(el);
                step_q.push_back(q);
            }
        }
        for (int i = 0; i < count; ++i) {
            if (lam[i] < 1) continue;
            for (int q = 0; q < k; ++q) {
                int lv = level[i][q];
                if (lv < lam[i] && lv % k == q && lv + 1 == lam[i]) lv = lam[i];
                if (lv != lam[i]) return fail(ctx, KD_EDEVICE, "internal: schedule did not reach the finisher level");
            }
        }
    }
    for (int i = 0; i < count; ++i)
        for (int q = 0; q < k && q < MAXK; ++q) cd[i].buf[q] = (uint8_t)buf_after(moves[i][q]);
    // an array's last move before the finisher writes rank 0 alone: the
    // finisher reads no other plane
    {
        std::vector<uint8_t> seen((size_t)count * k, 0);
        for (size_t st = step_jobs.size(); st-- > 0;)
            for (auto& J : step_jobs[st]) {
                uint8_t& f = seen[(size_t)J.cloud * k + step_q[st]];
                if (!f) {
                    J.write_med |= LEVEL_FINAL;
                    f = 1;
                }
            }
    }

    AllBufs bufs{};
    for (int d = 0; d < k && k >= 2; ++d)
        for (int p = 0; p < k; ++p) bufs.p[d][0][p] = H->rec.p[d][p];
    if (need_bufs) {
        uint32_t* blk = nullptr;
        // plane strides padded to 16 bytes, and 16 bytes of slack at the end:
        // the level passes stage tiles with 16-byte-aligned bulk copies
        CKS(S.get(&blk, ((size_t)2 * k * k * pad4(M) + 4) * 4));
        for (int b = 1; b <= 2; ++b)
            for (int d = 0; d < k; ++d)
                for (int p = 0; p < k; ++p) bufs.p[d][b][p] = blk + (((size_t)(b - 1) * k + d) * k + p) * pad4(M);
    }

    // upload tables -------------------------------------------------------
    std::vector<int64_t> top_prefix(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        int64_t e = 0;
        if (cd[i].m > 0 && (k == 1 || lam[i] >= 1)) e = ((int64_t)1 << lam[i]) - 1;
        top_prefix[i + 1] = top_prefix[i] + e;
    }
    std::vector<int64_t> unit_prefix(count + 1, 0);  // finisher units: 2^lam segments per cloud
    for (int i = 0; i < count; ++i)
        unit_prefix[i + 1] = unit_prefix[i] + ((k >= 2 && cd[i].m > 0) ? ((int64_t)1 << lam[i]) : 0);
    const int64_t nunits = unit_prefix[count];
    // A single cloud with page-locked host outputs: the children and split
    // dimensions (pure functions of m) are computed first and copied back on
    // a second stream while the level passes run; the finisher then runs in
    // chunks of units and each chunk's node tuples are copied back while the
    // next chunk runs.
    const bool overlap_copy = any_host && count == 1 && nunits >= 64 && !(ctx->debug & 4) && !outs[0].on_device &&
                              pinned_host(outs[0].node_tuple) && (!outs[0].left || pinned_host(outs[0].left)) &&
                              (!outs[0].right || pinned_host(outs[0].right)) &&
                              (!outs[0].dim || pinned_host(outs[0].dim));
    const int nchunks = overlap_copy ? 8 : 1;
    if (overlap_copy) {
        CKS(ensure_copy_stream(ctx, nchunks + 2));
        const int32_t mm = cd[0].m;
        {
            LaunchTimer lt(ctx, F_OTHER, 0.0);
            CK(launch_shape(mm, k, cd[0].left, cd[0].right, cd[0].dim, s));
        }
        CK(cudaEventRecord(ctx->chunk_events[nchunks + 1], s));
        CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->chunk_events[nchunks + 1], 0));
        cudaStream_t cs = ctx->copy_stream;
        if (outs[0].left) CK(cudaMemcpyAsync(outs[0].left, st_left, (size_t)mm * 4, cudaMemcpyDeviceToHost, cs));
        if (outs[0].right) CK(cudaMemcpyAsync(outs[0].right, st_right, (size_t)mm * 4, cudaMemcpyDeviceToHost, cs));
        if (outs[0].dim) CK(cudaMemcpyAsync(outs[0].dim, st_dim, (size_t)mm, cudaMemcpyDeviceToHost, cs));
        cd[0].left = cd[0].right = nullptr;  // the level kernels and the finisher write node tuples only
        cd[0].dim = nullptr;
    }
    std::vector<LevelJob> flat;
    std::vector<size_t> job_off;
    for (auto& v : step_jobs) {
        job_off.push_back(flat.size());
        flat.insert(flat.end(), v.begin(), v.end());
    }
    CloudDev* d_cd = nullptr;
    int64_t *d_prefix = nullptr, *d_uprefix = nullptr;
    LevelJob* d_jobs = nullptr;
    uint32_t* d_status = nullptr;
    CKS(S.get(&d_cd, sizeof(CloudDev) * count));
    CKS(S.get(&d_prefix, sizeof(int64_t) * (count + 1)));
    CKS(S.get(&d_uprefix, sizeof(int64_t) * (count + 1)));
    CK(cudaMemcpyAsync(d_cd, cd.data(), sizeof(CloudDev) * count, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_prefix, top_prefix.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_uprefix, unit_prefix.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
    // per step: tile counts, their segmented scan and head flags (no zeroing needed)
    size_t st_words = 0;
    for (size_t st = 0; st < step_jobs.size(); ++st)
        st_words = std::max(st_words, level_status_words(std::max(k, 2), (int)step_ntiles[st]));
    if (!flat.empty()) {
        CKS(S.get(&d_jobs, sizeof(LevelJob) * flat.size()));
        CK(cudaMemcpyAsync(d_jobs, flat.data(), sizeof(LevelJob) * flat.size(), cudaMemcpyHostToDevice, s));
        CKS(S.get(&d_status, st_words * 4));
    }
    // launches ----------------------------------------------------------------
    {
        LaunchTimer lt(ctx, F_TOP, (double)top_prefix[count], nullptr, 13.0);
        CK(launch_top_nodes(d_cd, d_prefix, count, top_prefix[count], k, H->perm0, medr, k == 1, s));
    }
    for (size_t st = 0; st < step_jobs.size(); ++st) {
        const int F = step_jobs[st][0].lev_out - step_jobs[st][0].lev_in;
        // array q moves k planes (array 0) or k - 1 (its own rank is not carried)
        LaunchTimer lt(ctx, F_LEVEL, step_elems[st], nullptr, 8.0 * (k - (step_q[st] != 0)) + 4.0 * F);
        ctx->launches += 3;  // tile records, count pass and scan
        CK(launch_level_pass(k, tile, bufs, step_q[st], d_jobs + job_off[st], (int)step_jobs[st].size(),
                             (int)step_ntiles[st], d_cd, medr, H->perm0, d_status, d_err, s));
    }
    if (nunits > 0) {
        unsigned long long* phase = nullptr;
        if (ctx->debug & 4) {
            CKS(S.get(&phase, sizeof(unsigned long long) * 8));
            CK(cudaMemsetAsync(phase, 0, sizeof(unsigned long long) * 8, s));
        }
        const int64_t m0 = cd[0].m;
        const double fin_bytes = 4.0 * (2 * k - 1) + 8.0;
        for (int c = 0; c < nchunks; ++c) {
            const int64_t u0 = nunits * c / nchunks, u1 = nunits * (c + 1) / nchunks;
            {
                LaunchTimer lt(ctx, F_FINISH, (double)M * (u1 - u0) / nunits, nullptr,
                               fin_bytes + (want_l ? 4 : 0) + (want_r ? 4 : 0) + (want_d ? 1 : 0));
                CK(launch_finish(bufs, k, d_uprefix, count, u0, (int)(u1 - u0), d_cd, H->perm0, smax, d_err, phase,
                                 s));
            }
            if (overlap_copy) {
                // addresses [a0, a1): from the first unit's start (0 for the
                // first chunk) to the next chunk's first unit (m for the last)
                auto unit_lo = [&](int64_t u) {
                    int32_t lo = 0, hi = (int32_t)m0 - 1;
                    for (int l = lam[0] - 1; l >= 0; --l) {
                        const int32_t mid = lo + ((hi - lo) >> 1);
                        if ((u >> l) & 1) lo = mid + 1; else hi = mid - 1;
                    }
                    return (int64_t)lo;
                };
                const int64_t a0 = c == 0 ? 0 : unit_lo(u0), a1 = c + 1 == nchunks ? m0 : unit_lo(u1);
                CK(cudaEventRecord(ctx->chunk_events[c], s));
                CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->chunk_events[c], 0));
                // (the chunk's address range also holds the nodes above the
                // finisher level between its units, final by now)
                if (a1 > a0)
                    CK(cudaMemcpyAsync(outs[0].node_tuple + a0, st_node + a0, (size_t)(a1 - a0) * 4,
                                       cudaMemcpyDeviceToHost, ctx->copy_stream));
            }
        }
        if (phase) {
            unsigned long long h[8];
            CK(cudaMemcpyAsync(h, phase, sizeof(h), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int i = 0; i < 8; ++i) ctx->trace_ns[i] += (double)h[i];
        }
    }
    if (overlap_copy) {
        // the caller's stream completes only after the copies
        CK(cudaEventRecord(ctx->chunk_events[nchunks], ctx->copy_stream));
        CK(cudaStreamWaitEvent(s, ctx->chunk_events[nchunks], 0));
    }
    CKS(check_device_err(ctx, d_err));
    if (overlap_copy) return KD_OK;  // check_device_err synchronised the stream after the copies
    if (any_host) {
        for (int i = 0; i < count; ++i) {
            if (outs[i].on_device || cd[i].m == 0) continue;
            const size_t mi = (size_t)cd[i].m;
            CK(cudaMemcpyAsync(outs[i].node_tuple, st_node + cd[i].off, mi * 4, cudaMemcpyDeviceToHost, s));
            if (outs[i].left) CK(cudaMemcpyAsync(outs[i].left, st_left + cd[i].off, mi * 4, cudaMemcpyDeviceToHost, s));
            if (outs[i].right)
                CK(cudaMemcpyAsync(outs[i].right, st_right + cd[i].off, mi * 4, cudaMemcpyDeviceToHost, s));
            if (outs[i].dim) CK(cudaMemcpyAsync(outs[i].dim, st_dim + cd[i].off, mi, cudaMemcpyDeviceToHost, s));
        }
        CK(cudaStreamSynchronize(s));
    }
    return KD_OK;
}

// ------------------------------------------------- median-selection build
// The O(n log n) build of the paper's "Comparative Performance" section:
// one index array (array 0, presorted by super key 0 and deduplicated) with
// its key planes; every level selects each segment's median in the level's
// super key (kd_select.cu) and partitions the segment around it.
kd_status select_build(kd_ctx* ctx, kd_presorted* H, kd_tree* out) {
    const int k = H->k;
    const int64_t M = H->M;
    cudaStream_t s = ctx->stream;
    if (!out->node_tuple && M > 0) return fail(ctx, KD_EINVAL, "node_tuple output is NULL");
    out->m = (int32_t)M;
    out->root = M > 0 ? (int32_t)((M - 1) / 2) : -1;
    if (M == 0) return KD_OK;
    if (k == 1) return build_batch(ctx, H, out);  // one dimension: the sorted array is the tree
    const int key64 = H->dtype == KD_I64;
    const int w = key64 ? 8 : 4;
    const int64_t NS = pad4(H->N);
    Scratch S(ctx);
    int* d_err = nullptr;
    CKS(S.get(&d_err, 4));
    CK(cudaMemsetAsync(d_err, 0, 4, s));
    // outputs: the caller's device arrays or staging for host arrays
    int32_t *node = out->node_tuple, *left = out->left, *right = out->right;
    uint8_t* dim = out->dim;
    if (!out->on_device) {
        CKS(S.get(&node, (size_t)M * 4));
        if (out->left) CKS(S.get(&left, (size_t)M * 4));
        if (out->right) CKS(S.get(&right, (size_t)M * 4));
        if (out->dim) CKS(S.get(&dim, (size_t)M));
    }
    // planes: buffer 0 is the handle's (array 0 and its key planes), buffer 1 new
    void* ids[2];
    void* keys[2 * MAXK] = {};
    ids[0] = H->perm0;
    CKS(S.get(&ids[1], (size_t)NS * 4 + 16));
    unsigned char* k1 = nullptr;
    CKS(S.get(&k1, (size_t)k * NS * w + 16));
    for (int d = 0; d < k; ++d) {
        keys[d] = (unsigned char*)H->sel_keys + (size_t)d * NS * w;
        keys[MAXK + d] = k1 + (size_t)d * NS * w;
    }
    const int T = sel_finish_tile(key64, k);
    const int stile = T >= 1024 ? 2048 : 1024;  // a level tile touches at most 4 segments of >= T tuples
    int lam = 0;
    while (max_seg(M, lam) > T) ++lam;
    void* segs = nullptr;
    uint32_t *ghist = nullptr, *unresolved = nullptr;
    int32_t* gany = nullptr;
    const int64_t nsegmax = lam > 0 ? ((int64_t)1 << (lam - 1)) : 1;
    CKS(S.get(&segs, (size_t)nsegmax * sel_seg_bytes(key64)));
    CKS(S.get(&ghist, (size_t)nsegmax * RADIX * 4));
    CKS(S.get(&gany, (size_t)nsegmax * RADIX * 4));
    CKS(S.get(&unresolved, 16));
    const int nbytes = k * w;
    int cur = 0;
    for (int L = 0; L < lam; ++L) {
        LaunchTimer lt(ctx, F_SELECT, (double)M, nullptr, 0.0);
        CK(launch_sel_level(key64, ids, keys, cur, k, (int32_t)M, L, stile, segs, ghist, gany, unresolved, node, 0, d_err, s,
                            0, 0, 0));
        // the leading bytes each segment shares are skipped: selection starts
        // at the first byte where some segment's elements differ; then two
        // rounds, then rounds until no segment is open
        int32_t r0 = 0;
        {
            const int32_t init = nbytes;
            CK(cudaMemcpyAsync(unresolved, &init, 4, cudaMemcpyHostToDevice, s));
            CK(launch_sel_level(key64, ids, keys, cur, k, (int32_t)M, L, stile, segs, ghist, gany, unresolved, node, 0,
                                d_err, s, 0, 0, 3));
            ctx->launches += 2;
            CK(cudaMemcpyAsync(&r0, unresolved, 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            r0 = std::max(0, std::min(r0, nbytes - 1));
        }
        CK(launch_sel_level(key64, ids, keys, cur, k, (int32_t)M, L, stile, segs, ghist, gany, unresolved, node, 0, d_err, s,
                            r0, std::min(r0 + 2, nbytes), 1));
        ctx->launches += 2 * (std::min(r0 + 2, nbytes) - r0);
        for (int r = r0 + 2; r < nbytes; ++r) {
            uint32_t open = 0;
            CK(cudaMemsetAsync(unresolved, 0, 4, s));
            CK(launch_sel_level(key64, ids, keys, cur, k, (int32_t)M, L, stile, segs, ghist, gany, unresolved, node, 0,
                                d_err, s, r, r + 1, 1));
            ctx->launches += 2;
            CK(cudaMemcpyAsync(&open, unresolved, 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (open == 0) break;
        }
        CK(launch_sel_level(key64, ids, keys, cur, k, (int32_t)M, L, stile, segs, ghist, gany, unresolved, node, 0, d_err, s,
                            0, 0, 2));
        cur ^= 1;
    }
    // children and split dimension of the nodes above the finisher level
    CloudDev cd{};
    cd.off = 0;
    cd.in_off = 0;
    cd.m = (int32_t)M;
    cd.lam = lam;
    cd.medr_off = 0;
    cd.node = node;
    cd.left = left;
    cd.right = right;
    cd.dim = dim;
    const int64_t top = lam > 0 ? ((int64_t)1 << lam) - 1 : 0;
    if (top > 0) {
        CloudDev* d_cd = nullptr;
        int64_t* d_prefix = nullptr;
        CKS(S.get(&d_cd, sizeof(CloudDev)));
        CKS(S.get(&d_prefix, 2 * sizeof(int64_t)));
        const int64_t prefix[2] = {0, top};
        CK(cudaMemcpyAsync(d_cd, &cd, sizeof(CloudDev), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_prefix, prefix, sizeof(prefix), cudaMemcpyHostToDevice, s));
        LaunchTimer lt(ctx, F_TOP, (double)top, nullptr, 13.0);
        CK(launch_top_nodes(d_cd, d_prefix, 1, top, k, H->perm0, nullptr, 0, s));
        CK(cudaStreamSynchronize(s));  // the host copies of cd and prefix go out of scope
    }
    {
        LaunchTimer lt(ctx, F_SELECT_FINISH, (double)M, nullptr, 0.0);
        CK(launch_sel_finish(key64, ids, keys, cur, k, (int32_t)M, lam, T, node, left, right, dim, 0, d_err, s));
    }
    CKS(check_device_err(ctx, d_err));
    if (!out->on_device) {
        CK(cudaMemcpyAsync(out->node_tuple, node, (size_t)M * 4, cudaMemcpyDeviceToHost, s));
        if (out->left) CK(cudaMemcpyAsync(out->left, left, (size_t)M * 4, cudaMemcpyDeviceToHost, s));
        if (out->right) CK(cudaMemcpyAsync(out->right, right, (size_t)M * 4, cudaMemcpyDeviceToHost, s));
        if (out->dim) CK(cudaMemcpyAsync(out->dim, dim, (size_t)M, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return KD_OK;
}

// ---------------------------------------------------------------- serving
constexpr size_t SERVE_QUEUE_MAX = 1 << 20;
constexpr int SERVE_WORKERS = 2;              // batches in flight on the device at once
constexpr int64_t SERVE_BATCH_POINTS = 1 << 26;
constexpr int SERVE_BATCH_CLOUDS = 8192;

// Device bytes a request needs while it is built (presort buffers, rank
// records and the build's ping-pong copies), with slack for status words.
size_t serve_estimate(int64_t n, int k, int dtype) {
    const size_t s = dtype_size(dtype), w = dtype == KD_I64 ? 8 : 4;
    const size_t per = k * s + k * w + 2 * w + 8 + 8 * (k + 1) + 4 + 12 * (size_t)k * k + 64;
    return (size_t)n * per + (1u << 16);
}

void serve_worker(kd_ctx* ctx, kd_ctx* wctx) {
    const size_t budget = wctx->budget;
    for (;;) {
        std::vector<std::shared_ptr<Request>> batch;
        {
            std::unique_lock<std::mutex> lk(ctx->qmu);
            ctx->qcv.wait(lk, [&] { return ctx->stopping || !ctx->queue.empty(); });
            if (ctx->stopping && ctx->queue.empty()) return;
            // admit from the queue head: same k and dtype, within this
            // worker's memory budget and the batch caps
            const int k = ctx->queue.front()->cloud.k, dt = ctx->queue.front()->cloud.dtype;
            size_t bytes = 0;
            int64_t pts = 0;
            for (auto it = ctx->queue.begin(); it != ctx->queue.end();) {
                const auto& r = *it;
                if (r->cloud.k != k || r->cloud.dtype != dt) {
                    ++it;
                    continue;
                }
                if (!batch.empty() && ((budget && bytes + r->est_bytes > budget) ||
                                       pts + r->cloud.n > SERVE_BATCH_POINTS ||
                                       (int)batch.size() >= SERVE_BATCH_CLOUDS))
                    break;
                bytes += r->est_bytes;
                pts += r->cloud.n;
                batch.push_back(r);
                it = ctx->queue.erase(it);
            }
        }
        std::vector<kd_cloud> clouds;
        std::vector<kd_tree> outs;
        for (auto& r : batch) {
            clouds.push_back(r->cloud);
            outs.push_back(r->out);
        }
        kd_status st = kd_build_batch(wctx, clouds.data(), (int)clouds.size(), outs.data());
        const std::string err = st == KD_OK ? std::string() : std::string(kd_last_error(wctx));
        const auto now = std::chrono::steady_clock::now();
        {
            std::lock_guard<std::mutex> lk(ctx->qmu);
            for (size_t i = 0; i < batch.size(); ++i) {
                auto& r = batch[i];
                r->status = st;
                r->error = err;
                if (st == KD_OK) {
                    r->out.m = outs[i].m;
                    r->out.root = outs[i].root;
                    r->user_out->m = outs[i].m;
                    r->user_out->root = outs[i].root;
                }
                r->t_done = now;
                r->done = true;
                ctx->latencies_us.push_back(
                    std::chrono::duration<double, std::micro>(now - r->t_submit).count());
                ctx->completed++;
            }
        }
        ctx->donecv.notify_all();
    }
}

kd_status start_serving(kd_ctx* ctx) {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!ctx->workers.empty()) return KD_OK;
    for (int i = 0; i < SERVE_WORKERS; ++i) {
        kd_config c = ctx->cfg;
        c.cuda_stream = nullptr;  // each worker orders its batches on its own stream
        c.debug = 0;
        c.mem_budget_bytes = ctx->budget ? ctx->budget / SERVE_WORKERS : 0;
        kd_ctx* w = nullptr;
        kd_status st = kd_create(&w, &c);
        if (st != KD_OK) return fail(ctx, st, "cannot create a serving worker context");
        ctx->worker_ctx.push_back(w);
    }
    for (kd_ctx* w : ctx->worker_ctx) ctx->workers.emplace_back(serve_worker, ctx, w);
    return KD_OK;
}

}  // namespace

// Context access for the entry points in kd_noalloc.cu and kd_search.cu.
namespace kd {
int ctx_device(const kd_ctx* ctx) { return ctx->device; }
cudaStream_t ctx_stream(const kd_ctx* ctx) { return ctx->stream; }
void ctx_set_error(kd_ctx* ctx, const std::string& msg) { ctx->last_error = msg; }
void ctx_add_launches(kd_ctx* ctx, int n) { ctx->launches += n; }
kd_status ctx_alloc(kd_ctx* ctx, void** p, size_t bytes) { return dev_alloc(ctx, p, bytes); }
void ctx_free(kd_ctx* ctx, void* p) { dev_free(ctx, p); }
std::recursive_mutex& ctx_mutex(kd_ctx* ctx) { return ctx->mu; }
}  // namespace kd

// =================================================================== C ABI
extern "C" {

kd_status kd_create(kd_ctx** out, const kd_config* cfg) {
    if (!out) return KD_EINVAL;
    *out = nullptr;
    kd_config c{};
    if (cfg) c = *cfg;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return KD_EDEVICE;
    }
    if (c.device < 0 || c.device >= ndev) return KD_EINVAL;
    std::unique_ptr<kd_ctx> ctx(new kd_ctx());
    ctx->cfg = c;
    ctx->device = c.device;
    ctx->budget = c.mem_budget_bytes;
    ctx->debug = c.debug;
    ctx->smax_override = c.switch_threshold;
    if (c.level_tile != 0 && c.level_tile != 1024 && c.level_tile != 2048) return KD_EINVAL;
    if (c.schedule < KD_SCHEDULE_MULTI || c.schedule > KD_SCHEDULE_EVERY_LEVEL) return KD_EINVAL;
    ctx->schedule = c.schedule;
    ctx->level_tile_override = c.level_tile;
    if (c.tune_cache) ctx->tune_cache = c.tune_cache;
    ctx->cfg.tune_cache = ctx->tune_cache.empty() ? nullptr : ctx->tune_cache.c_str();  // owned copy for workers
    tuning_load(ctx.get());
    if (c.debug & 8) {
        ctx->spin_limit = 4096;
        ctx->inject_timeout = true;
    }
    if (cudaSetDevice(c.device) != cudaSuccess) return KD_EDEVICE;
    // kernel attributes are per device: set them once for each device used
    static std::mutex init_mu;
    static bool init_done[64] = {false};
    {
        std::lock_guard<std::mutex> lk(init_mu);
        if (c.device < 64 && !init_done[c.device]) {
            if (init_presort_kernels() != cudaSuccess || init_build_kernels() != cudaSuccess ||
                init_select_kernels() != cudaSuccess) {
                cudaGetLastError();
                return KD_EDEVICE;
            }
            init_done[c.device] = true;
        }
    }
    if (c.cuda_stream) {
        ctx->stream = (cudaStream_t)c.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return KD_EDEVICE;
        ctx->own_stream = true;
    }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c.device;
    if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess) return KD_EDEVICE;
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    *out = ctx.release();
    return KD_OK;
}

kd_status kd_presort(kd_ctx* ctx, const kd_cloud* cloud, kd_handle* out) {
    if (!ctx || !out) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    ctx->last_error.clear();
    kd_status st = presort_batch(ctx, cloud, 1, out);
    if (st == KD_OK && (ctx->debug & 2)) collect_timing(ctx);
    return st;
}

kd_status kd_handle_info(kd_handle h, int64_t* n, int32_t* m, int* k) {
    if (!h) return KD_EINVAL;
    if (n) *n = h->N;
    if (m) *m = (int32_t)h->M;
    if (k) *k = h->k;
    return KD_OK;
}

kd_status kd_handle_arrays(kd_ctx* ctx, kd_handle h, int32_t* out, int on_device) {
    if (!ctx || !h || (!out && h->M > 0)) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    if (h->count != 1) return fail(ctx, KD_EINVAL, "index arrays are available for single-cloud handles only");
    if (h->M == 0) return KD_OK;
    const size_t bytes = (size_t)h->M * h->k * 4;
    Scratch S(ctx);
    int32_t* dst = out;
    if (!on_device) CKS(S.get(&dst, bytes));
    if (h->k == 1) {
        CK(cudaMemcpyAsync(dst, h->perm0, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
        LaunchTimer lt(ctx, F_OTHER, (double)h->M);
        CK(launch_arrays_out(h->d_m, h->M, h->k, h->rec, h->perm0, dst, ctx->stream));
    }
    if (!on_device) CK(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return KD_OK;
}

kd_status kd_build(kd_ctx* ctx, kd_handle h, kd_tree* out) {
    if (!ctx || !h) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    ctx->last_error.clear();
    kd_status st = out ? build_batch(ctx, h, out) : fail(ctx, KD_EINVAL, "tree output is NULL");
    if (st == KD_OK && (ctx->debug & 2)) collect_timing(ctx);
    release_handle(ctx, h);
    return st;
}

kd_status kd_build_select(kd_ctx* ctx, const kd_cloud* cloud, kd_tree* out) {
    if (!ctx || !cloud || !out) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    ctx->last_error.clear();
    kd_presorted* h = nullptr;
    kd_status st = presort_batch(ctx, cloud, 1, &h, /*all_arrays=*/false);
    if (st != KD_OK) return st;
    st = select_build(ctx, h, out);
    if (st == KD_OK && (ctx->debug & 2)) collect_timing(ctx);
    release_handle(ctx, h);
    return st;
}

kd_status kd_release(kd_ctx* ctx, kd_handle h) {
    if (!ctx || !h) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    release_handle(ctx, h);
    return KD_OK;
}

kd_status kd_build_batch(kd_ctx* ctx, const kd_cloud* clouds, int count, kd_tree* outs) {
    if (!ctx || !clouds || !outs || count < 1) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    ctx->last_error.clear();
    kd_presorted* h = nullptr;
    kd_status st = presort_batch(ctx, clouds, count, &h);
    if (st != KD_OK) return st;
    st = build_batch(ctx, h, outs);
    // timing first: presort launches read their element counts from the
    // handle's device memory
    if (st == KD_OK && (ctx->debug & 2)) collect_timing(ctx);
    release_handle(ctx, h);
    return st;
}

kd_status kd_submit(kd_ctx* ctx, const kd_cloud* cloud, kd_tree* out, kd_ticket* ticket) {
    if (!ctx || !cloud || !out || !ticket) return KD_EINVAL;
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        CKS(validate_cloud(ctx, cloud));
        if (out->on_device) return fail(ctx, KD_EINVAL, "served trees are returned in host memory");
        if (cloud->n > 0 && !out->node_tuple) return fail(ctx, KD_EINVAL, "node_tuple output is NULL");
    }
    auto r = std::make_shared<Request>();
    r->cloud = *cloud;
    const size_t bytes = (size_t)cloud->n * cloud->k * dtype_size(cloud->dtype);
    r->coords.resize(bytes);
    if (bytes) {
        if (cloud->on_device) {
            std::lock_guard<std::recursive_mutex> lk(ctx->mu);
            cudaSetDevice(ctx->device);
            CK(cudaMemcpyAsync(r->coords.data(), cloud->coords, bytes, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
        } else {
            memcpy(r->coords.data(), cloud->coords, bytes);
        }
    }
    r->cloud.coords = r->coords.data();
    r->cloud.on_device = 0;
    r->out = *out;
    r->user_out = out;
    r->est_bytes = serve_estimate(cloud->n, cloud->k, cloud->dtype);
    r->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(ctx->qmu);
        if (ctx->queue.size() >= SERVE_QUEUE_MAX) return fail(ctx, KD_EBUSY, "serving queue is full");
        *ticket = ctx->next_ticket++;
        ctx->tickets[*ticket] = r;
        ctx->queue.push_back(r);
    }
    kd_status st = start_serving(ctx);
    if (st != KD_OK) return st;
    ctx->qcv.notify_one();
    return KD_OK;
}

kd_status kd_wait(kd_ctx* ctx, kd_ticket ticket, int timeout_ms) {
    if (!ctx) return KD_EINVAL;
    std::unique_lock<std::mutex> lk(ctx->qmu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(ctx, KD_EINVAL, "unknown ticket");
    std::shared_ptr<Request> r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0)
        ctx->donecv.wait(lk, ready);
    else if (!ctx->donecv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return fail(ctx, KD_ETIMEOUT, "request still pending");
    ctx->tickets.erase(ticket);
    if (r->status != KD_OK) ctx->last_error = r->error;
    return r->status;
}

kd_status kd_serving_stats(kd_ctx* ctx, int64_t* completed, double* p50_us, double* p99_us) {
    if (!ctx) return KD_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->qmu);
    std::vector<double> v = ctx->latencies_us;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
        if (v.empty()) return 0.0;
        size_t i = (size_t)std::min<double>(v.size() - 1, std::floor(p * (v.size() - 1) + 0.5));
        return v[i];
    };
    if (completed) *completed = ctx->completed;
    if (p50_us) *p50_us = pct(0.50);
    if (p99_us) *p99_us = pct(0.99);
    return KD_OK;
}

kd_status kd_autotune(kd_ctx* ctx, int k, kd_dtype dtype, int64_t n, int reps, int* smax_out, int* ltile_out) {
    if (!ctx) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    ctx->last_error.clear();
    if (k < 1 || k > KD_MAX_K || n < 1 || n > KD_MAX_N || reps < 1 || reps > 100 ||
        (dtype != KD_I32 && dtype != KD_I64 && dtype != KD_F32))
        return fail(ctx, KD_EINVAL, "kd_autotune: k, n, dtype or reps out of range");
    const uint32_t key = tune_key(k, dtype, n);
    if (k >= 2) {
        Scratch S(ctx);
        void* coords = nullptr;
        CKS(S.get(&coords, (size_t)n * k * dtype_size(dtype)));
        {
            LaunchTimer lt(ctx, F_OTHER, 0.0);
            CK(launch_tune_cloud(dtype, coords, n * k, (uint64_t)key * 0x9E3779B97F4A7C15ull, ctx->stream));
        }
        kd_cloud cl{coords, n, k, dtype, 1};
        kd_presorted* H = nullptr;
        CKS(presort_batch(ctx, &cl, 1, &H));
        struct Release {
            kd_ctx* c;
            kd_presorted* h;
            ~Release() { release_handle(c, h); }
        } rel{ctx, H};
        int32_t *node = nullptr, *left = nullptr, *right = nullptr;
        uint8_t* dim = nullptr;
        CKS(S.get(&node, (size_t)n * 4));
        CKS(S.get(&left, (size_t)n * 4));
        CKS(S.get(&right, (size_t)n * 4));
        CKS(S.get(&dim, (size_t)n));
        cudaEvent_t e0 = take_event(ctx), e1 = take_event(ctx);
        double best = 1e30;
        int bsm = 1024, blt = level_tile(k);
        for (int sm : {1024, 2048, 4096}) {
            if (k > finish_kmax(sm)) continue;
            for (int lt : {1024, 2048}) {
                if (!level_tile_supported(k, lt) || sm * 3 < lt + 3) continue;
                ctx->force_smax = sm;
                ctx->force_ltile = lt;
                std::vector<float> ms;
                kd_status st = KD_OK;
                for (int r = 0; r <= reps && st == KD_OK; ++r) {  // the first run is a warm-up
                    kd_tree t{0, -1, node, left, right, dim, 1};
                    cudaEventRecord(e0, ctx->stream);
                    st = build_batch(ctx, H, &t);
                    cudaEventRecord(e1, ctx->stream);
                    if (st == KD_OK && r > 0) {
                        cudaEventSynchronize(e1);
                        float x = 0;
                        cudaEventElapsedTime(&x, e0, e1);
                        ms.push_back(x);
                    }
                }
                ctx->force_smax = ctx->force_ltile = 0;
                if (st != KD_OK) {
                    ctx->event_pool.push_back(e0);
                    ctx->event_pool.push_back(e1);
                    return st;
                }
                std::sort(ms.begin(), ms.end());
                const double med = ms[ms.size() / 2];
                if (med < best) {
                    best = med;
                    bsm = sm;
                    blt = lt;
                }
            }
        }
        ctx->event_pool.push_back(e0);
        ctx->event_pool.push_back(e1);
        ctx->tuning[key] = kd_ctx::Tuned{bsm, blt, best};
        if (!tuning_save(ctx)) return fail(ctx, KD_EINVAL, "kd_autotune: cannot write " + ctx->tune_cache);
    }
    if (ctx->debug & 2) collect_timing(ctx);
    int sm = 0, lt = 0;
    choose_params(ctx, k, dtype, n, &sm, &lt);
    if (smax_out) *smax_out = sm;
    if (ltile_out) *ltile_out = lt;
    return KD_OK;
}

kd_status kd_tuning_get(kd_ctx* ctx, int k, kd_dtype dtype, int64_t n, int* smax_out, int* ltile_out) {
    if (!ctx || k < 1 || k > KD_MAX_K || n < 0) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    int sm = 0, lt = 0;
    choose_params(ctx, k, dtype, n, &sm, &lt);
    if (smax_out) *smax_out = sm;
    if (ltile_out) *ltile_out = lt;
    return KD_OK;
}

kd_status kd_destroy(kd_ctx* ctx) {
    if (!ctx) return KD_EINVAL;
    {
        std::lock_guard<std::mutex> lk(ctx->qmu);
        ctx->stopping = true;
    }
    ctx->qcv.notify_all();
    for (auto& t : ctx->workers)
        if (t.joinable()) t.join();
    for (kd_ctx* w : ctx->worker_ctx) kd_destroy(w);
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        for (auto& t : ctx->timed) {
            cudaEventDestroy(t.a);
            cudaEventDestroy(t.b);
        }
        for (auto e : ctx->event_pool) cudaEventDestroy(e);
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
        for (cudaEvent_t e : ctx->chunk_events) cudaEventDestroy(e);
    }
    delete ctx;
    return KD_OK;
}

const char* kd_last_error(kd_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

int64_t kd_launch_count(kd_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

kd_status kd_kernel_stats(kd_ctx* ctx, int family, double* ms, int64_t* launches, double* units,
                          double* bytes) {
    if (!ctx || family < 0 || family >= F_COUNT) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    collect_timing(ctx);
    if (ms) *ms = ctx->fam_ms[family];
    if (launches) *launches = ctx->fam_launches[family];
    if (units) *units = ctx->fam_units[family];
    if (bytes) *bytes = ctx->fam_bytes[family];
    return KD_OK;
}

kd_status kd_trace_counters(kd_ctx* ctx, double* out, int n) {
    if (!ctx || !out || n < 0) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    for (int i = 0; i < n && i < 8; ++i) out[i] = ctx->trace_ns[i];
    return KD_OK;
}

kd_status kd_kernel_stats_reset(kd_ctx* ctx) {
    if (!ctx) return KD_EINVAL;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    collect_timing(ctx);
    for (int f = 0; f < F_COUNT; ++f) {
        ctx->fam_ms[f] = 0;
        ctx->fam_units[f] = 0;
        ctx->fam_bytes[f] = 0;
        ctx->fam_launches[f] = 0;
    }
    return KD_OK;
}

}  // extern "C"

/*
 * kdtree.h -- C ABI of the GB300 presorting k-d tree builder.
 *
 * The library builds the balanced k-d tree of Brown, "Building a Balanced
 * k-d Tree in O(kn log n) Time", Section 2.1: n tuples of k coordinates in,
 * a balanced binary tree of tuple indices with "less than" / "greater than"
 * children out, duplicate tuples removed.  Every step runs in CUDA kernels
 * on one GB300 (sm_103a); the calls below only marshal arguments, order
 * work on a CUDA stream and report status.
 *
 * Conventions (all calls):
 *  - Every call returns a kd_status; none throws or aborts.  After an
 *    error the context stays usable and kd_last_error() describes it.
 *  - Input coordinates are borrowed for the duration of the call (kd_submit
 *    copies them before it returns).  Outputs are allocated by the caller.
 *  - Pointers flagged "on_device" are CUDA device pointers on the context's
 *    device; otherwise they are host pointers (page-locked memory gives the
 *    fastest copies, pageable memory works).
 *  - 0 <= n <= KD_MAX_N tuples per cloud; 1 <= k <= KD_MAX_K; the sum of
 *    tuples over a batch is also at most KD_MAX_N.
 *
 * Output layout (in-order addresses).  Node address a in [0, m) holds the
 * tuple chosen as the median of the sub-range whose median address is a;
 * the root is at (m - 1) / 2; the children of node a with range [lo, hi]
 * are the medians of [lo, a - 1] and [a + 1, hi] (-1 when empty); the split
 * dimension of a node at depth t is t mod k.  Medians are lower medians,
 * lo + (hi - lo) / 2 (the paper uses only odd sizes).  Of a run of identical
 * tuples the one with the smallest index survives.  Floats compare
 * numerically (-0.0 equals +0.0); a NaN coordinate is an error.
 */
#ifndef KDTREE_H
#define KDTREE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KD_MAX_K 8
#define KD_MAX_N 1073741823LL /* 2^30 - 1: the range the kernels' 32-bit positions and counts are sized for */

typedef enum {
    KD_OK = 0,
    KD_EINVAL = -1,   /* bad argument: null pointer, n or k out of range, bad dtype */
    KD_ENOMEM = -2,   /* device allocation failed or the memory budget is exceeded */
    KD_EDEVICE = -3,  /* a CUDA call failed (message in kd_last_error) */
    KD_ETIMEOUT = -4, /* a bounded device wait or kd_wait ran out of time */
    KD_EBUSY = -5,    /* the serving queue is full */
    KD_ENAN = -6      /* a float coordinate is NaN */
} kd_status;

typedef enum { KD_I32 = 0, KD_I64 = 1, KD_F32 = 2 } kd_dtype;

typedef struct {
    int device;              /* CUDA device ordinal */
    void *cuda_stream;       /* cudaStream_t to order work on; NULL: the library makes its own */
    size_t mem_budget_bytes; /* cap on the library's device workspace; 0: no cap */
    int level_tile;          /* positions per level-step tile: 1024, or 2048 (k <= 4); 0: tuned, else 2048 for
                                k <= 4 and 1024 above */
    int switch_threshold;    /* subtree size finished on chip (rounded up to 1024, 2048 or 4096, capped by k);
                                0: tuned, else 1024 */
    int debug;               /* bit 1: synchronise after the presort; bit 2: time every launch
                                (kd_kernel_stats); bit 4: finisher phase counters; bit 8
                                (failure-detection tests): bound the device waits to a few
                                thousand polls and make the next presort's first look-back
                                wait run out once, which it reports as KD_ETIMEOUT */
    const char *tune_cache;  /* autotuner cache file (read by kd_create, rewritten by kd_autotune); NULL: none */
    int schedule;            /* level schedule of kd_build (same tree under each):
                                KD_SCHEDULE_MULTI (0, default): an array is partitioned only when it is
                                  about to become primary, through up to k-1 levels in one pass;
                                KD_SCHEDULE_DEFERRED: Appendix "Deferred Merge Sort and Partitioning":
                                  array d first appears at level d, then every non-primary array is
                                  partitioned at every level;
                                KD_SCHEDULE_EVERY_LEVEL: Section 2.1: every non-primary array is
                                  partitioned at every level */
} kd_config;

#define KD_SCHEDULE_MULTI 0
#define KD_SCHEDULE_DEFERRED 1
#define KD_SCHEDULE_EVERY_LEVEL 2

typedef struct {
    const void *coords; /* row-major n x k array of dtype; borrowed for the call */
    int64_t n;
    int k;
    kd_dtype dtype;
    int on_device; /* coords is a device pointer */
} kd_cloud;

typedef struct {
    int32_t m;           /* out: tuples after duplicate removal (= nodes) */
    int32_t root;        /* out: root address, (m - 1) / 2, or -1 when m = 0 */
    int32_t *node_tuple; /* caller-allocated, capacity n: tuple index per address */
    int32_t *left;       /* optional (NULL to skip), capacity n: child addresses */
    int32_t *right;      /* optional, capacity n */
    uint8_t *dim;        /* optional, capacity n: split dimension per address */
    int on_device;       /* the four arrays are device pointers */
} kd_tree;

typedef struct kd_ctx kd_ctx;
typedef struct kd_presorted *kd_handle;
typedef int64_t kd_ticket;

/*
 * Create a context on cfg->device.  *out receives the context; it owns a
 * stream-ordered device memory pool and, if cfg->cuda_stream is NULL, a
 * stream.  cfg may be NULL for defaults (device 0).
 */
kd_status kd_create(kd_ctx **out, const kd_config *cfg);

/*
 * Presort (Section 2.1, first paragraphs; duplicates paragraph): transform
 * the coordinates to order-preserving unsigned keys, sort index arrays by
 * the k cyclic super keys x_d : x_{d+1} : ... : x_{d-1}, and remove
 * duplicate tuples.  *out receives a handle owning the device arrays
 * (the k index orders and their rank vectors); pass it to kd_build or
 * release it with kd_release.  Errors: KD_EINVAL, KD_ENAN, KD_ENOMEM,
 * KD_EDEVICE, KD_ETIMEOUT.  Synchronises the stream three times: to read
 * the key-byte histograms (constant digits are skipped), the run lengths of
 * array 0 after its sort by x_0 (k >= 2: long or costly runs take the
 * whole-key sort), and m.
 */
kd_status kd_presort(kd_ctx *ctx, const kd_cloud *cloud, kd_handle *out);

/* m (tuples after duplicate removal), n and k of a presorted handle. */
kd_status kd_handle_info(kd_handle h, int64_t *n, int32_t *m, int *k);

/*
 * Copy the k presorted, deduplicated index arrays of a handle (array d in
 * super-key-d order, tuple indices local to the cloud) into out, k rows of
 * m int32 each, row-major.  For checking the presort on its own.
 */
kd_status kd_handle_arrays(kd_ctx *ctx, kd_handle h, int32_t *out, int on_device);

/*
 * Build (Section 2.1, partition and recursion paragraphs; Appendix
 * "Optimized Partitioning" for partitioning only the k-1 non-primary
 * arrays): level by level, the median of each segment of the primary array
 * becomes a node and the other arrays are partitioned around it in address
 * order, keeping their sorted order.  Consumes and releases the handle
 * (also on error).  out->node_tuple must hold n entries.
 */
kd_status kd_build(kd_ctx *ctx, kd_handle h, kd_tree *out);

/*
 * The O(n log n) build of the paper's "Comparative Performance" section
 * ("The O(n log n) Algorithm"): one index array sorted by super key 0 and
 * deduplicated, then at every level the median of each sub-array in the
 * level's super key is found by selection (a most-significant-byte radix
 * selection, linear per level) and the sub-array is partitioned around it.
 * No other super-key order is presorted.  The tree equals kd_presort +
 * kd_build's for the same cloud (every median is unique).  cloud and out as
 * for kd_presort / kd_build; errors as theirs.
 */
kd_status kd_build_select(kd_ctx *ctx, const kd_cloud *cloud, kd_tree *out);

/* Release a handle that will not be built. */
kd_status kd_release(kd_ctx *ctx, kd_handle h);

/*
 * Presort and build `count` independent clouds (same k and dtype) as one
 * batch: the clouds share every launch.  outs[i] receives cloud i's tree;
 * the result of each cloud equals its plain kd_presort + kd_build result.
 */
kd_status kd_build_batch(kd_ctx *ctx, const kd_cloud *clouds, int count, kd_tree *outs);

/*
 * Serving: enqueue one build request.  The coordinates are copied before
 * the call returns.  *out (host arrays; on_device must be 0) must stay
 * valid until kd_wait reports the ticket done: the arrays receive the tree
 * and out->m / out->root are set on completion.  Two worker threads, each
 * with its own stream and half of cfg->mem_budget_bytes, take batches from
 * the queue head (requests of equal k and dtype, within the budget): work
 * admitted while another batch runs overlaps it on the device.  KD_EBUSY
 * when the queue is full.  Each served tree equals the tree of the same
 * cloud built alone.
 */
kd_status kd_submit(kd_ctx *ctx, const kd_cloud *cloud, kd_tree *out, kd_ticket *ticket);

/*
 * Wait up to timeout_ms (negative: forever) for a ticket.  Returns the
 * request's own status, or KD_ETIMEOUT if it is still pending.  A finished
 * ticket is forgotten once it has been reported.
 */
kd_status kd_wait(kd_ctx *ctx, kd_ticket ticket, int timeout_ms);

/* Serving statistics: completed requests and their admission-to-result
 * latency percentiles (microseconds). */
kd_status kd_serving_stats(kd_ctx *ctx, int64_t *completed, double *p50_us, double *p99_us);

/*
 * Autotuner.  The on-chip subtree size (1024, 2048 or 4096 tuples, as k
 * allows) and the level-step tile (1024 or 2048 positions) are chosen per
 * (k, dtype, size bucket = floor(log2 n) of the largest cloud of a build).
 * kd_autotune presorts a synthetic cloud of n tuples (uniform coordinates,
 * generated on the device), times kd_build with every candidate pair (reps
 * runs each, median of CUDA-event times on the context's stream), records
 * the fastest for the bucket in the context, rewrites cfg->tune_cache when
 * one was given, and returns it.  Later builds whose bucket has an entry use
 * it unless cfg->switch_threshold or cfg->level_tile fix a value.  Every
 * candidate builds the same tree.  Errors: KD_EINVAL (k, n, dtype or reps
 * out of range), KD_ENOMEM, KD_EDEVICE.  Synchronises the stream.
 */
kd_status kd_autotune(kd_ctx *ctx, int k, kd_dtype dtype, int64_t n, int reps, int *switch_threshold_out,
                      int *level_tile_out);

/* The subtree size and level tile a build of clouds of at most n tuples
 * (k, dtype) would use on this context now. */
kd_status kd_tuning_get(kd_ctx *ctx, int k, kd_dtype dtype, int64_t n, int *switch_threshold_out,
                        int *level_tile_out);

/* Stop serving, free every device resource and the context. */
kd_status kd_destroy(kd_ctx *ctx);

/* Text of the last error on this context ("" if none).  Valid until the
 * next call on the context. */
const char *kd_last_error(kd_ctx *ctx);

/*
 * kd_presort_noalloc -- what kd_presort + kd_handle_arrays compute, for one
 * small cloud, without allocating any memory.  The paper has no
 * counterpart: it exists for callers that cannot let a library allocate
 * during a call, such as a process whose device memory is all owned by its
 * own allocator, or a latency-bound loop that cannot absorb a pool growth
 * or a device-wide synchronising free.  Its workspace is one static device
 * array of about 1 MiB per device, sized for KD_NOALLOC_MAX_N tuples of up
 * to KD_MAX_K coordinates.
 *
 *  cloud       coordinates in device memory on the context's device
 *              (cloud->on_device must be 1), n <= KD_NOALLOC_MAX_N; larger
 *              clouds return KD_EINVAL with the limit in kd_last_error (use
 *              kd_presort for them).
 *  arrays_out  device memory on the context's device, k rows of n int32
 *              (row stride n): row d receives the deduplicated super-key-d
 *              order, the same values kd_handle_arrays gives for the same
 *              cloud, in its first m entries; the rest of the row is left
 *              untouched.
 *  m_out       device memory on the context's device, one int32: m, or
 *              KD_ENAN if a float coordinate is NaN (arrays_out is then
 *              left untouched).
 *
 * Asynchronous: the work is ordered on the context's stream and the call
 * returns without waiting; read *m_out after the stream.  Argument errors
 * (KD_EINVAL) are found on the host before anything is enqueued.  The first
 * call on a device does a one-time set-up (the address of the static
 * workspace and a kernel attribute), so a caller that records its stream
 * into a graph should make one call before it starts recording.  All calls
 * on a device share the one workspace: calls whose work can overlap on the
 * device (different streams, or threads without ordering between them)
 * race and give wrong results; order them on one stream.
 */
#define KD_NOALLOC_MAX_N 16384
kd_status kd_presort_noalloc(kd_ctx *ctx, const kd_cloud *cloud, int32_t *arrays_out, int32_t *m_out);

/*
 * Searches over a built tree ("Nearest Neighbors" subsection of the paper,
 * and the hyper-rectangular region search of its source-code subsection).
 *
 * kd_index_create: a search index for tree `tree` built from `cloud` (the
 * same coordinates, host or device; the tree's node_tuple array host or
 * device).  The index keeps the tuples in the tree's address order on the
 * device (m x k coordinates and m tuple indices), allocated from the
 * context; destroy it with kd_index_destroy before destroying the context.
 */
typedef struct kd_index_s *kd_index;
kd_status kd_index_create(kd_ctx *ctx, const kd_cloud *cloud, const kd_tree *tree, kd_index *out);
kd_status kd_index_destroy(kd_ctx *ctx, kd_index index);

/*
 * kd_knn: for each of nq query points (row-major nq x k, the index's dtype),
 * its kn nearest tuples (1 <= kn <= KD_KNN_MAX) by squared Euclidean
 * distance, nearest first, equal distances by the smaller tuple index.
 * Distances are exact per dimension (integers: |a - b| as an unsigned
 * 64-bit value, rounded to double; floats: the double difference), squared
 * and summed in double in dimension order without fused multiply-add.
 * idx_out: nq x kn tuple indices (-1 past the tree's m tuples); dist_out
 * (optional): nq x kn squared distances (+inf past m).  on_device: queries
 * and outputs are device pointers.  A NaN query coordinate gives KD_ENAN.
 * Synchronises the stream.
 */
#define KD_KNN_MAX 32
kd_status kd_knn(kd_ctx *ctx, kd_index index, const void *queries, int64_t nq, int kn, int on_device,
                 int32_t *idx_out, double *dist_out);

/*
 * kd_knn_all: the kn nearest neighbours of every tuple of the tree among
 * the others (its own tuple excluded), as the first step of the paper's
 * reverse-nearest-neighbours search.  Row a of idx_out (m x kn) belongs to
 * the tuple at tree address a (node_tuple[a]); ordering and distances as
 * kd_knn.  on_device: outputs are device pointers.
 */
kd_status kd_knn_all(kd_ctx *ctx, kd_index index, int kn, int on_device, int32_t *idx_out, double *dist_out);

/*
 * kd_reverse_knn: the reverse nearest neighbours of every tuple of the
 * tree: for the tuple at address a, the tuples whose kn nearest neighbours
 * (kd_knn_all) include it.  offsets (m + 1 int64) is the exclusive prefix
 * of the list lengths; the tuple indices of list a are
 * rev_out[offsets[a] .. offsets[a+1]), in no particular order (rev_out
 * needs m * kn entries).  on_device: outputs are device pointers.
 */
kd_status kd_reverse_knn(kd_ctx *ctx, kd_index index, int kn, int on_device, int64_t *offsets, int32_t *rev_out);

/*
 * kd_region: for each of nq boxes [lo[i], hi[i]] (row-major nq x k,
 * inclusive in every dimension), the indices of the tuples inside it.
 * offsets (nq + 1 int64) receives the exclusive prefix of the per-box
 * counts; box i's indices are idx_out[offsets[i] .. offsets[i+1]) in the
 * order the walk meets them.  idx_out may be NULL (counts only); a
 * capacity below the total gives KD_EINVAL (offsets are still written).
 * on_device: boxes, offsets and idx_out are device pointers.  Synchronises
 * the stream.
 */
kd_status kd_region(kd_ctx *ctx, kd_index index, const void *lo, const void *hi, int64_t nq, int on_device,
                    int64_t *offsets, int32_t *idx_out, int64_t capacity);

/* Kernels launched by this context since creation (instrumentation). */
int64_t kd_launch_count(kd_ctx *ctx);

/*
 * Kernel timing (instrumentation; active when cfg->debug & 2): CUDA events
 * recorded on the context's stream around every launch, summed per kernel
 * family (0 transform, 1 sort pass, 2 dedup, 3 records, 4 level pass,
 * 5 finisher, 6 top nodes, 7 other, 8 key gathers, 9 median selection and
 * partition of kd_build_select, 10 its finisher, 11 ordering the runs of
 * equal x_0 in array 0).  *ms: device time, *launches: launch count, *units: elements the launches processed, *bytes: the algorithmic
 * bytes those launches must move (reads + writes per element of each kernel,
 * summed over launches).  Any output pointer may be NULL.  Synchronises the
 * stream.
 */
kd_status kd_kernel_stats(kd_ctx *ctx, int family, double *ms, int64_t *launches, double *units,
                          double *bytes);

/* Zero the kernel timing sums and trace counters. */
kd_status kd_kernel_stats_reset(kd_ctx *ctx);

/*
 * Trace counters (instrumentation; active when cfg->debug & 4): the
 * on-chip finisher's phases, summed over its thread blocks in nanoseconds
 * (block time, not wall time): [0] loading a subtree's rank table and
 * index arrays, [1] levels with segments above 32 tuples, [2] levels
 * finished one warp per segment, [3] resolving node tuples, [4] ordering
 * every array within the segments the warps finish.  Copies min(n, 8)
 * values into out.
 */
kd_status kd_trace_counters(kd_ctx *ctx, double *out, int n);

#ifdef __cplusplus
}
#endif

#endif /* KDTREE_H */

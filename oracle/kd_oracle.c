/*
 * kd_oracle.c -- CPU oracle for the presorting k-d tree build.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * restatement of the O(kn log n) algorithm of Brown, "Building a Balanced
 * k-d Tree in O(kn log n) Time" (Section 2.1), against which the CUDA path
 * is checked.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg may load it.  It shares no code, header or constant
 * with the CUDA library: it compares coordinates natively (no key
 * transform), sorts by merge sort, and recurses exactly as Section 2.1
 * describes.
 *
 * Steps and the passages they follow:
 *   super key     Section 2.1: the key of dimension d is the cyclic
 *                 concatenation x_d : x_{d+1} : ... : x_{d-1}; compared
 *                 most-significant part first (Appendix "Optimized Super
 *                 Key Comparison" tests that part before the loop).
 *   presort       Section 2.1: k merge sorts of index arrays, one per super
 *                 key; the tuples array is never moved.
 *   dedup         Section 2.1 (duplicates paragraph): one pass per sorted
 *                 index array discards all but one index of each run of
 *                 identical tuples.
 *   build         Section 2.1: the median of the primary index array
 *                 becomes the node; the other k-1 arrays are partitioned in
 *                 address order around the median's super key, equal keys
 *                 skipped; the temporary-array rotation (primary copied to
 *                 temp, array j partitioned into array j-1's storage, temp
 *                 copied to the last array) cycles the primary dimension.
 *                 Recursion ends at one, two or three elements as the
 *                 Section 2.1 termination paragraph states.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - even-length segments take the lower median lo + (hi - lo) / 2;
 *   - of a run of identical tuples the smallest original index survives
 *     (merge sort is stable and starts from the identity order);
 *   - floats compare numerically, so -0.0 equals +0.0; NaN is rejected;
 *   - the split dimension of depth t is t mod k, starting at x.
 *
 * Output layout: node address a holds the tuple chosen as the median at a;
 * children are the medians of the left/right sub-ranges (-1 if empty);
 * dim[a] = depth mod k; root = (m - 1) / 2.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* KDO_MUTANT plants one deliberate mistake (tests only, never the default
 * build): 1 upper median, 2 super key reduced to its first part, 3 dedup keeps
 * the last of a run, 4 no role rotation, 5 partition in the wrong dimension,
 * 6 merge sort not stable, 7 the median's own index kept in the lower half. */
#ifndef KDO_MUTANT
#define KDO_MUTANT 0
#endif

#define KDO_I32 0
#define KDO_I64 1
#define KDO_F32 2

#define KDO_OK 0
#define KDO_EINVAL (-1)
#define KDO_ENOMEM (-2)
#define KDO_ENAN (-6)

typedef struct {
    const void *coords; /* row-major n x k */
    int64_t n;
    int k;
    int dtype;
} tuples_t;

/* Compare coordinate d of tuples a and b: -1, 0, +1. */
static int coord_cmp(const tuples_t *t, int32_t a, int32_t b, int d)
{
    int64_t ia = (int64_t)a * t->k + d, ib = (int64_t)b * t->k + d;
    switch (t->dtype) {
    case KDO_I32: {
        int32_t x = ((const int32_t *)t->coords)[ia], y = ((const int32_t *)t->coords)[ib];
        return (x > y) - (x < y);
    }
    case KDO_I64: {
        int64_t x = ((const int64_t *)t->coords)[ia], y = ((const int64_t *)t->coords)[ib];
        return (x > y) - (x < y);
    }
    default: {
        float x = ((const float *)t->coords)[ia], y = ((const float *)t->coords)[ib];
        return (x > y) - (x < y);
    }
    }
}

/* Super key comparison for dimension p: x_p, then x_{p+1}, ... cyclically. */
static int superkey_cmp(const tuples_t *t, int32_t a, int32_t b, int p)
{
    int c = coord_cmp(t, a, b, p);
    if (c != 0 || KDO_MUTANT == 2)
        return c;
    for (int i = 1; i < t->k; i++) {
        c = coord_cmp(t, a, b, (p + i) % t->k);
        if (c != 0)
            return c;
    }
    return 0;
}

/* Top-down merge sort of idx[lo..hi] by super key p; stable (ties keep the
 * left run first). */
static void merge_sort(const tuples_t *t, int32_t *idx, int32_t *tmp, int64_t lo, int64_t hi, int p)
{
    if (hi <= lo)
        return;
    int64_t mid = lo + (hi - lo) / 2;
    merge_sort(t, idx, tmp, lo, mid, p);
    merge_sort(t, idx, tmp, mid + 1, hi, p);
    int64_t i = lo, j = mid + 1, o = lo;
    while (i <= mid && j <= hi)
        tmp[o++] = (superkey_cmp(t, idx[j], idx[i], p) < (KDO_MUTANT == 6 ? 1 : 0)) ? idx[j++] : idx[i++];
    while (i <= mid)
        tmp[o++] = idx[i++];
    while (j <= hi)
        tmp[o++] = idx[j++];
    memcpy(idx + lo, tmp + lo, (size_t)(hi - lo + 1) * sizeof(int32_t));
}

/* One pass over a sorted index array keeping the first index of each run of
 * identical tuples.  Returns the new length. */
static int64_t remove_duplicates(const tuples_t *t, int32_t *idx, int64_t n)
{
    if (n == 0)
        return 0;
    int64_t w = 1;
    for (int64_t r = 1; r < n; r++) {
        if (superkey_cmp(t, idx[r], idx[w - 1], 0) != 0)
            idx[w++] = idx[r];
        else if (KDO_MUTANT == 3)
            idx[w - 1] = idx[r];
    }
    return w;
}

static int check_input(const tuples_t *t)
{
    if (t->n < 0 || t->n > 0x7FFFFFFF || t->k < 1 || t->k > 64)
        return KDO_EINVAL;
    if (t->dtype != KDO_I32 && t->dtype != KDO_I64 && t->dtype != KDO_F32)
        return KDO_EINVAL;
    if (t->dtype == KDO_F32) {
        const float *f = (const float *)t->coords;
        for (int64_t i = 0; i < t->n * t->k; i++)
            if (f[i] != f[i])
                return KDO_ENAN;
    }
    return KDO_OK;
}

/* Presort + dedup: arrays_out holds k arrays of *m_out indices each
 * (array d sorted by super key d), stored back to back with stride n. */
int kdo_presort(const void *coords, int64_t n, int k, int dtype, int32_t *arrays_out, int64_t *m_out)
{
    tuples_t t = {coords, n, k, dtype};
    int rc = check_input(&t);
    if (rc != KDO_OK)
        return rc;
    int32_t *tmp = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!tmp)
        return KDO_ENOMEM;
    int64_t m = n;
    for (int d = 0; d < k; d++) {
        int32_t *a = arrays_out + (int64_t)d * n;
        for (int64_t i = 0; i < n; i++)
            a[i] = (int32_t)i;
        merge_sort(&t, a, tmp, 0, n - 1, d);
        int64_t md = remove_duplicates(&t, a, n);
        if (d > 0 && md != m) {
            free(tmp);
            return KDO_EINVAL; /* cannot happen: identical tuples are adjacent in every order */
        }
        m = md;
    }
    free(tmp);
    *m_out = m;
    return KDO_OK;
}

typedef struct {
    const tuples_t *t;
    int32_t **arr;   /* k pointers into the index storage; arr[0] is the primary */
    int32_t *temp;
    int32_t *temp2;  /* used only by mutant 4 */
    int32_t *node;   /* node[a] = tuple index at address a */
    int32_t *left, *right;
    uint8_t *dim;
    int terminate_small; /* 1: end recursion at <= 3 elements as Section 2.1 states */
} build_t;

static void set_node(build_t *b, int64_t a, int32_t tuple, int depth, int64_t l, int64_t r)
{
    b->node[a] = tuple;
    if (b->left)
        b->left[a] = (int32_t)l;
    if (b->right)
        b->right[a] = (int32_t)r;
    if (b->dim)
        b->dim[a] = (uint8_t)(depth % b->t->k);
}

static int64_t median_addr(int64_t lo, int64_t hi)
{
    return KDO_MUTANT == 1 ? lo + (hi - lo + 1) / 2 : lo + (hi - lo) / 2;
}

static int64_t child_addr(int64_t lo, int64_t hi)
{
    return hi < lo ? -1 : median_addr(lo, hi);
}

/* Partition arrays[1..k-1][lo..hi] around the median of arrays[0] and
 * rotate the array roles (Section 2.1, temporary index array paragraph). */
static void split_level(build_t *b, int64_t lo, int64_t hi, int depth)
{
    const tuples_t *t = b->t;
    int k = t->k, p = (depth + (KDO_MUTANT == 5 ? 1 : 0)) % k;
    int64_t mid = median_addr(lo, hi);
    int32_t med = b->arr[0][mid];
    memcpy(b->temp + lo, b->arr[0] + lo, (size_t)(hi - lo + 1) * sizeof(int32_t));
    for (int j = 1; j < k; j++) {
        int32_t *src = b->arr[j], *dst = b->arr[j - 1];
        int64_t lower = lo, upper = mid + 1;
        if (KDO_MUTANT == 4)
            dst = b->temp2;
        for (int64_t i = lo; i <= hi; i++) {
            int c = superkey_cmp(t, src[i], med, p);
            if (c < 0 || (KDO_MUTANT == 7 && c == 0))
                dst[lower++] = src[i];
            else if (c > 0)
                dst[upper++] = src[i];
        }
        if (KDO_MUTANT == 4)
            memcpy(src + lo, b->temp2 + lo, (size_t)(hi - lo + 1) * sizeof(int32_t));
    }
    if (KDO_MUTANT != 4)
        memcpy(b->arr[k - 1] + lo, b->temp + lo, (size_t)(hi - lo + 1) * sizeof(int32_t));
}

static void build_rec(build_t *b, int64_t lo, int64_t hi, int depth)
{
    if (hi < lo)
        return;
    int64_t n = hi - lo + 1;
    int32_t *A = b->arr[0];
    if (b->terminate_small && n <= 3) {
        if (n == 1) {
            set_node(b, lo, A[lo], depth, -1, -1);
        } else if (n == 2) {
            /* lower element is the node, the other its "greater" child */
            set_node(b, lo, A[lo], depth, -1, lo + 1);
            set_node(b, lo + 1, A[lo + 1], depth + 1, -1, -1);
        } else {
            set_node(b, lo + 1, A[lo + 1], depth, lo, lo + 2);
            set_node(b, lo, A[lo], depth + 1, -1, -1);
            set_node(b, lo + 2, A[lo + 2], depth + 1, -1, -1);
        }
        return;
    }
    int64_t mid = median_addr(lo, hi);
    set_node(b, mid, A[mid], depth, child_addr(lo, mid - 1), child_addr(mid + 1, hi));
    if (n > 1) {
        /* After the rotation, storage j holds the array sorted by super key
         * (depth + 1 + j) mod k within each half, so the role table is the
         * same for the children. */
        split_level(b, lo, hi, depth);
        build_rec(b, lo, mid - 1, depth + 1);
        build_rec(b, mid + 1, hi, depth + 1);
    }
}

/*
 * Full build: presort, dedup, then the recursive partition.  Outputs
 * (capacity n each): node_tuple, and optionally left/right/dim (NULL to
 * skip).  terminate_small selects the Section 2.1 termination at <= 3
 * elements (1) or plain recursion to single elements (0); both give the
 * same tree, which the tests check.  arrays_out, if not NULL, receives the
 * k presorted deduplicated index arrays (stride n) as kdo_presort does.
 */
int kdo_build(const void *coords, int64_t n, int k, int dtype, int terminate_small,
              int32_t *node_tuple, int32_t *left, int32_t *right, uint8_t *dim,
              int64_t *m_out, int32_t *arrays_out)
{
    tuples_t t = {coords, n, k, dtype};
    int rc = check_input(&t);
    if (rc != KDO_OK)
        return rc;
    size_t cap = (size_t)(n > 0 ? n : 1);
    int32_t *store = (int32_t *)malloc(cap * (size_t)k * sizeof(int32_t));
    int32_t *temp = (int32_t *)malloc(cap * sizeof(int32_t));
    int32_t *temp2 = (int32_t *)malloc(cap * sizeof(int32_t));
    if (!store || !temp || !temp2) {
        free(store);
        free(temp);
        free(temp2);
        return KDO_ENOMEM;
    }
    int64_t m = 0;
    rc = kdo_presort(coords, n, k, dtype, store, &m);
    if (rc != KDO_OK) {
        free(store);
        free(temp);
        free(temp2);
        return rc;
    }
    if (arrays_out)
        memcpy(arrays_out, store, cap * (size_t)k * sizeof(int32_t));
    int32_t *roles[64];
    for (int d = 0; d < k; d++)
        roles[d] = store + (int64_t)d * n;
    build_t b = {&t, roles, temp, temp2, node_tuple, left, right, dim, terminate_small};
    build_rec(&b, 0, m - 1, 0);
    free(store);
    free(temp);
    free(temp2);
    *m_out = m;
    return KDO_OK;
}

/*
 * The first split only (Section 2.1, "After First Split"): presort, dedup,
 * partition arrays 1..k-1 around the median of array 0 over [0, m-1].
 * Writes the k arrays in dimension order (array d still sorted by super
 * key d within each half; address mid of arrays 1..k-1 is left as -1 since
 * the median is dropped there).  Returns the median tuple in *median.
 */
int kdo_first_split(const void *coords, int64_t n, int k, int dtype,
                    int32_t *arrays_out, int64_t *m_out, int32_t *median)
{
    tuples_t t = {coords, n, k, dtype};
    int64_t m = 0;
    int rc = kdo_presort(coords, n, k, dtype, arrays_out, &m);
    if (rc != KDO_OK)
        return rc;
    *m_out = m;
    if (m == 0)
        return KDO_OK;
    int32_t *tmp = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    if (!tmp)
        return KDO_ENOMEM;
    int64_t mid = median_addr(0, m - 1);
    int32_t med = arrays_out[mid];
    *median = med;
    for (int d = 1; d < k; d++) {
        int32_t *a = arrays_out + (int64_t)d * n;
        int64_t lower = 0, upper = mid + 1;
        for (int64_t i = 0; i < m; i++) {
            int c = superkey_cmp(&t, a[i], med, 0);
            if (c < 0)
                tmp[lower++] = a[i];
            else if (c > 0)
                tmp[upper++] = a[i];
        }
        tmp[mid] = -1;
        memcpy(a, tmp, (size_t)m * sizeof(int32_t));
    }
    free(tmp);
    return KDO_OK;
}

/*
 * The paper's parallel execution scheme (Section "Parallel Execution"),
 * a host baseline rather than a reference: the merge sorts and the
 * recursive build split their ranges as above, and at the first `levels`
 * levels of recursion the parent thread hands the lower half to a child
 * thread, processes the upper half itself and then joins the child
 * (2^levels threads).  Deeper levels run in the calling thread.  The result
 * is the single-threaded result: the halves never overlap.
 */
typedef struct {
    const tuples_t *t;
    int32_t *idx, *tmp;
    int64_t lo, hi;
    int p, levels;
} msort_job;

static void merge_sort_mt(const tuples_t *t, int32_t *idx, int32_t *tmp, int64_t lo, int64_t hi, int p, int levels);

static void *msort_thread(void *arg)
{
    msort_job *j = (msort_job *)arg;
    merge_sort_mt(j->t, j->idx, j->tmp, j->lo, j->hi, j->p, j->levels);
    return NULL;
}

static void merge_sort_mt(const tuples_t *t, int32_t *idx, int32_t *tmp, int64_t lo, int64_t hi, int p, int levels)
{
    if (levels <= 0 || hi - lo < 4096) {
        merge_sort(t, idx, tmp, lo, hi, p);
        return;
    }
    int64_t mid = lo + (hi - lo) / 2;
    msort_job child = {t, idx, tmp, lo, mid, p, levels - 1};
    pthread_t th;
    int forked = pthread_create(&th, NULL, msort_thread, &child) == 0;
    if (!forked)
        merge_sort_mt(t, idx, tmp, lo, mid, p, levels - 1);
    merge_sort_mt(t, idx, tmp, mid + 1, hi, p, levels - 1);
    if (forked)
        pthread_join(th, NULL);
    int64_t i = lo, j = mid + 1, o = lo;
    while (i <= mid && j <= hi)
        tmp[o++] = (superkey_cmp(t, idx[j], idx[i], p) < 0) ? idx[j++] : idx[i++];
    while (i <= mid)
        tmp[o++] = idx[i++];
    while (j <= hi)
        tmp[o++] = idx[j++];
    memcpy(idx + lo, tmp + lo, (size_t)(hi - lo + 1) * sizeof(int32_t));
}

typedef struct {
    build_t *b;
    int64_t lo, hi;
    int depth, levels;
} build_job;

static void build_rec_mt(build_t *b, int64_t lo, int64_t hi, int depth, int levels);

static void *build_thread(void *arg)
{
    build_job *j = (build_job *)arg;
    build_rec_mt(j->b, j->lo, j->hi, j->depth, j->levels);
    return NULL;
}

static void build_rec_mt(build_t *b, int64_t lo, int64_t hi, int depth, int levels)
{
    if (levels <= 0 || hi - lo < 4096) {
        build_rec(b, lo, hi, depth);
        return;
    }
    int32_t *A = b->arr[0];
    int64_t mid = median_addr(lo, hi);
    set_node(b, mid, A[mid], depth, child_addr(lo, mid - 1), child_addr(mid + 1, hi));
    split_level(b, lo, hi, depth);
    build_job child = {b, lo, mid - 1, depth + 1, levels - 1};
    pthread_t th;
    int forked = pthread_create(&th, NULL, build_thread, &child) == 0;
    if (!forked)
        build_rec_mt(b, lo, mid - 1, depth + 1, levels - 1);
    build_rec_mt(b, mid + 1, hi, depth + 1, levels - 1);
    if (forked)
        pthread_join(th, NULL);
}

int kdo_build_parallel(const void *coords, int64_t n, int k, int dtype, int levels, int32_t *node_tuple,
                       int32_t *left, int32_t *right, uint8_t *dim, int64_t *m_out)
{
    tuples_t t = {coords, n, k, dtype};
    int rc = check_input(&t);
    if (rc != KDO_OK)
        return rc;
    size_t cap = (size_t)(n > 0 ? n : 1);
    int32_t *store = (int32_t *)malloc(cap * (size_t)k * sizeof(int32_t));
    int32_t *temp = (int32_t *)malloc(cap * sizeof(int32_t));
    if (!store || !temp) {
        free(store);
        free(temp);
        return KDO_ENOMEM;
    }
    int64_t m = n;
    for (int d = 0; d < k && rc == KDO_OK; d++) {
        int32_t *a = store + (int64_t)d * n;
        for (int64_t i = 0; i < n; i++)
            a[i] = (int32_t)i;
        merge_sort_mt(&t, a, temp, 0, n - 1, d, levels);
        int64_t md = remove_duplicates(&t, a, n);
        if (d > 0 && md != m)
            rc = KDO_EINVAL;
        m = md;
    }
    if (rc == KDO_OK) {
        int32_t *roles[64];
        for (int d = 0; d < k; d++)
            roles[d] = store + (int64_t)d * n;
        build_t b = {&t, roles, temp, NULL, node_tuple, left, right, dim, 1};
        build_rec_mt(&b, 0, m - 1, 0, levels);
        *m_out = m;
    }
    free(store);
    free(temp);
    return rc;
}

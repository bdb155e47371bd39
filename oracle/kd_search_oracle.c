/*
 * kd_search_oracle.c -- CPU oracle for searches over a k-d tree.
 *
 * TEST INFRASTRUCTURE ONLY, like kd_oracle.c: only tests/,
 * __graft_entry__.smoke() and bench.py's baseline legs load it, and it shares
 * no code with the CUDA library.  The searches the paper lists for a built
 * tree (the "Nearest Neighbors" subsection and the region search of the
 * source-code subsection) are defined here by brute force over the set of
 * distinct tuples, so that a tree search on the GPU can be checked against
 * their definitions rather than against another tree walk.
 *
 *   m nearest neighbours  of a query point q: the m distinct tuples with the
 *                         smallest squared Euclidean distance to q, ordered
 *                         by distance, ties by smaller tuple index.
 *   region search         of a box [lo, hi] (inclusive in every dimension):
 *                         every distinct tuple inside it.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - distance: per dimension the exact difference of the two coordinates
 *     (integers: |a - b| as an unsigned 64-bit value, then rounded to
 *     double; floats: the double-precision difference of the two values),
 *     squared and summed in double precision in dimension order, each
 *     operation rounded separately (no fused multiply-add);
 *   - distance ties are broken by the smaller tuple index; with fewer than m
 *     distinct tuples the remaining slots hold index -1 and distance +inf;
 *   - the distinct tuples are the duplicate-removal survivors (the smallest
 *     index of each run of identical tuples), passed in by the caller.
 */
#include <math.h>
#include <stdint.h>

#define KDS_I32 0
#define KDS_I64 1
#define KDS_F32 2

/* |a - b| of coordinate d between tuple row x and query row q, as double. */
static double coord_diff(const void *coords, int64_t row, const void *queries, int64_t qrow, int k, int d,
                         int dtype)
{
    switch (dtype) {
    case KDS_I32: {
        int64_t a = ((const int32_t *)coords)[row * k + d], b = ((const int32_t *)queries)[qrow * k + d];
        uint64_t u = a > b ? (uint64_t)(a - b) : (uint64_t)(b - a);
        return (double)u;
    }
    case KDS_I64: {
        int64_t a = ((const int64_t *)coords)[row * k + d], b = ((const int64_t *)queries)[qrow * k + d];
        uint64_t u = a > b ? (uint64_t)a - (uint64_t)b : (uint64_t)b - (uint64_t)a;
        return (double)u;
    }
    default: {
        double a = ((const float *)coords)[row * k + d], b = ((const float *)queries)[qrow * k + d];
        double v = a - b;
        return v < 0 ? -v : v;
    }
    }
}

static double dist2(const void *coords, int64_t row, const void *queries, int64_t qrow, int k, int dtype)
{
    double acc = 0.0;
    for (int d = 0; d < k; d++) {
        double u = coord_diff(coords, row, queries, qrow, k, d, dtype);
        double sq = u * u;
        acc = acc + sq;
    }
    return acc;
}

/* m nearest neighbours of each query among the candidate tuples cand[0..nc)
 * (tuple indices into coords).  idx_out / d_out: nq x kn, row-major. */
int kdo_knn(const void *coords, int64_t n, int k, int dtype, const int32_t *cand, int64_t nc, const void *queries,
            int64_t nq, int kn, int32_t *idx_out, double *d_out)
{
    if (k < 1 || kn < 1 || n < 0 || nc < 0 || nq < 0)
        return -1;
    for (int64_t q = 0; q < nq; q++) {
        int32_t *bi = idx_out + q * kn;
        double *bd = d_out + q * kn;
        for (int j = 0; j < kn; j++) {
            bi[j] = -1;
            bd[j] = INFINITY;
        }
        for (int64_t c = 0; c < nc; c++) {
            const int32_t t = cand[c];
            const double d = dist2(coords, t, queries, q, k, dtype);
            /* insertion into the sorted list (distance, then index) */
            int j = kn - 1;
            if (!(d < bd[j] || (d == bd[j] && (bi[j] < 0 || t < bi[j]))))
                continue;
            while (j > 0 && (d < bd[j - 1] || (d == bd[j - 1] && (bi[j - 1] < 0 || t < bi[j - 1])))) {
                bd[j] = bd[j - 1];
                bi[j] = bi[j - 1];
                j--;
            }
            bd[j] = d;
            bi[j] = t;
        }
    }
    return 0;
}

static int coord_in(const void *coords, int64_t row, const void *lo, const void *hi, int64_t qrow, int k, int d,
                    int dtype)
{
    switch (dtype) {
    case KDS_I32: {
        int32_t x = ((const int32_t *)coords)[row * k + d];
        return ((const int32_t *)lo)[qrow * k + d] <= x && x <= ((const int32_t *)hi)[qrow * k + d];
    }
    case KDS_I64: {
        int64_t x = ((const int64_t *)coords)[row * k + d];
        return ((const int64_t *)lo)[qrow * k + d] <= x && x <= ((const int64_t *)hi)[qrow * k + d];
    }
    default: {
        float x = ((const float *)coords)[row * k + d];
        return ((const float *)lo)[qrow * k + d] <= x && x <= ((const float *)hi)[qrow * k + d];
    }
    }
}

/* Region search: for each box q, the candidate tuples inside it, in
 * candidate order.  counts[q] receives the number; the indices of box q
 * follow those of boxes 0..q-1 in idx_out (capacity cap).  Returns the
 * total, or -1 if cap is too small. */
int64_t kdo_region(const void *coords, int64_t n, int k, int dtype, const int32_t *cand, int64_t nc,
                   const void *lo, const void *hi, int64_t nq, int64_t *counts, int32_t *idx_out, int64_t cap)
{
    (void)n;
    int64_t total = 0;
    for (int64_t q = 0; q < nq; q++) {
        int64_t c0 = total;
        for (int64_t c = 0; c < nc; c++) {
            const int32_t t = cand[c];
            int in = 1;
            for (int d = 0; d < k && in; d++)
                in = coord_in(coords, t, lo, hi, q, k, d, dtype);
            if (in) {
                if (total >= cap)
                    return -1;
                idx_out[total++] = t;
            }
        }
        counts[q] = total - c0;
    }
    return total;
}

/*
 * mf_oracle.c -- CPU oracle for the sliding-window median filter.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline / reference arm may load this file's library.  The CUDA library
 * shares no code with it: no header, no helper, no table.
 *
 * What it computes (paper Section 1, "Median filter"; Section 2, the trivial
 * algorithm that finds the median of every window separately):
 *
 *   input  x[0 .. n-1], odd window size k = 2h + 1, 1 <= k <= n
 *   output y[i] = median of (x[i], ..., x[i+k-1]) for i = 0 .. n-k
 *
 * The paper prints the output vector as (y_1, ..., x_{n-k+1}); the last entry
 * is a typo for y_{n-k+1}: there are n-k+1 outputs, one per full window.
 *
 * The median is the element of rank h (0-based) in the window under the total
 * order
 *
 *     a < b  <=>  key(x_a) < key(x_b)  or  (key(x_a) == key(x_b) and a < b)
 *
 * i.e. values compared first and ties broken by the element's index.  This is
 * the order the paper's method works in: its piecewise sort is stable
 * (Section 5.2, sorting the pairs (alpha[i], i) lexicographically) and, on
 * ties between the two blocks, elements of the older block count as smaller
 * (Section 6.3).  Because equal keys mean equal bits, y is unique; the index
 * tie-break fixes only argmed, the index of the median element.
 *
 * Values: int32 and int64 are compared as signed integers.  float32 and
 * float64 are compared by the IEEE 754-2008 totalOrder predicate (Section 5.10
 * of that standard): -NaN < -inf < negative numbers < -0 < +0 < positive
 * numbers < +inf < +NaN, NaNs ordered by payload.  The paper's experiments
 * use 32-bit and 64-bit inputs (Section 7.3).  The paper only uses integers (Section 7.2); IEEE "<"
 * would make -0 and +0 equal and let the result's bits depend on which of the
 * two was picked, so the oracle never uses it.
 *
 * Method, per window: copy the k (value, index) pairs, sort them with the C
 * library's qsort under the order above, output the element at rank h.  That
 * is O(n k log k): slow and plain on purpose.
 *
 * Rank filter (mfo_rank_filter / mfo_rank_windows): the same per-window sort,
 * output the element at a given 0-based rank r, 0 <= r < k, for any k >= 1.
 * The paper defines the median for odd k = 2h + 1 (Section 1, Section 3);
 * for even k the lower median is the element of rank k/2 - 1 (the k/2-th
 * smallest), the upper median that of rank k/2.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { MFO_INT32 = 0, MFO_FLOAT32 = 1, MFO_INT64 = 2, MFO_FLOAT64 = 3 };

typedef struct {
    uint64_t bits;   /* the element's raw bits (32-bit types zero-extended) */
    int64_t index;   /* its position in x */
} elem_t;

static int elem_bytes(int dtype) { return dtype >= MFO_INT64 ? 8 : 4; }

/* IEEE 754 totalOrder on binary32 bit patterns: returns <0, 0, >0. */
static int float_total_order(uint32_t a, uint32_t b)
{
    int neg_a = (int)(a >> 31), neg_b = (int)(b >> 31);
    if (neg_a != neg_b)
        return neg_a ? -1 : 1;              /* every negative precedes every positive */
    if (a == b)
        return 0;
    if (!neg_a)                             /* both non-negative: larger magnitude is larger */
        return a < b ? -1 : 1;
    return a > b ? -1 : 1;                  /* both negative: larger magnitude is smaller */
}

static int int32_order(uint32_t a, uint32_t b)
{
    int32_t sa = (int32_t)a, sb = (int32_t)b;
    return sa < sb ? -1 : (sa > sb ? 1 : 0);
}

/* IEEE 754 totalOrder on binary64 bit patterns, the same rule as above. */
static int double_total_order(uint64_t a, uint64_t b)
{
    int neg_a = (int)(a >> 63), neg_b = (int)(b >> 63);
    if (neg_a != neg_b)
        return neg_a ? -1 : 1;
    if (a == b)
        return 0;
    if (!neg_a)
        return a < b ? -1 : 1;
    return a > b ? -1 : 1;
}

static int int64_order(uint64_t a, uint64_t b)
{
    int64_t sa = (int64_t)a, sb = (int64_t)b;
    return sa < sb ? -1 : (sa > sb ? 1 : 0);
}

static int cmp_int32(const void* pa, const void* pb)
{
    const elem_t* a = (const elem_t*)pa;
    const elem_t* b = (const elem_t*)pb;
    int c = int32_order((uint32_t)a->bits, (uint32_t)b->bits);
    if (c) return c;
    return a->index < b->index ? -1 : (a->index > b->index ? 1 : 0);
}

static int cmp_float32(const void* pa, const void* pb)
{
    const elem_t* a = (const elem_t*)pa;
    const elem_t* b = (const elem_t*)pb;
    int c = float_total_order((uint32_t)a->bits, (uint32_t)b->bits);
    if (c) return c;
    return a->index < b->index ? -1 : (a->index > b->index ? 1 : 0);
}

static int cmp_int64(const void* pa, const void* pb)
{
    const elem_t* a = (const elem_t*)pa;
    const elem_t* b = (const elem_t*)pb;
    int c = int64_order(a->bits, b->bits);
    if (c) return c;
    return a->index < b->index ? -1 : (a->index > b->index ? 1 : 0);
}

static int cmp_float64(const void* pa, const void* pb)
{
    const elem_t* a = (const elem_t*)pa;
    const elem_t* b = (const elem_t*)pb;
    int c = double_total_order(a->bits, b->bits);
    if (c) return c;
    return a->index < b->index ? -1 : (a->index > b->index ? 1 : 0);
}

typedef int (*cmp_fn)(const void*, const void*);

static cmp_fn comparator(int dtype)
{
    switch (dtype) {
        case MFO_INT32: return cmp_int32;
        case MFO_FLOAT32: return cmp_float32;
        case MFO_INT64: return cmp_int64;
        default: return cmp_float64;
    }
}

/* Element of rank r of the window that starts at x[start]; scratch holds k
 * elements. */
static void window_select(int dtype, const void* x, int64_t start, int32_t k, int32_t r,
                          elem_t* scratch, void* y, int64_t yi, int64_t* arg_out)
{
    const int wide = elem_bytes(dtype) == 8;
    for (int32_t t = 0; t < k; ++t) {
        scratch[t].bits = wide ? ((const uint64_t*)x)[start + t] : ((const uint32_t*)x)[start + t];
        scratch[t].index = start + t;
    }
    qsort(scratch, (size_t)k, sizeof(elem_t), comparator(dtype));
    if (wide) ((uint64_t*)y)[yi] = scratch[r].bits;
    else ((uint32_t*)y)[yi] = (uint32_t)scratch[r].bits;
    if (arg_out) *arg_out = scratch[r].index;
}

/* Median (rank h of an odd window k = 2h + 1). */
static void window_median(int dtype, const void* x, int64_t start, int32_t k,
                          elem_t* scratch, void* y, int64_t yi, int64_t* arg_out)
{
    window_select(dtype, x, start, k, (k - 1) / 2, scratch, y, yi, arg_out);
}

static int check_args(int dtype, const void* x, int64_t n, int32_t k)
{
    if (dtype < MFO_INT32 || dtype > MFO_FLOAT64) return -1;
    if (!x || n < 1) return -2;
    if (k < 1 || (k % 2) == 0 || (int64_t)k > n) return -3;
    return 0;
}

/*
 * Full filter: y[0 .. n-k] (raw 32-bit patterns), argmed optional (may be NULL).
 * nthreads <= 0 lets OpenMP pick.  Returns 0, or a negative code on bad args.
 */
int mfo_filter(int dtype, const void* x, int64_t n, int32_t k,
               void* y, int64_t* argmed, int nthreads)
{
    int rc = check_args(dtype, x, n, k);
    if (rc) return rc;
    int64_t m = n - k + 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        elem_t* scratch = (elem_t*)malloc(sizeof(elem_t) * (size_t)k);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t i = 0; i < m; ++i)
            window_median(dtype, x, i, k, scratch, y, i, argmed ? &argmed[i] : NULL);
        free(scratch);
    }
    return 0;
}

/*
 * Sampled windows: for each requested start s = starts[j] (0 <= s <= n-k),
 * y[j] = median of x[s .. s+k-1].  Used to check outputs of huge inputs one
 * by one.  Returns -4 if a start is out of range.
 */
int mfo_windows(int dtype, const void* x, int64_t n, int32_t k,
                const int64_t* starts, int64_t count,
                void* y, int64_t* argmed, int nthreads)
{
    int rc = check_args(dtype, x, n, k);
    if (rc) return rc;
    for (int64_t j = 0; j < count; ++j)
        if (starts[j] < 0 || starts[j] > n - k) return -4;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        elem_t* scratch = (elem_t*)malloc(sizeof(elem_t) * (size_t)k);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t j = 0; j < count; ++j)
            window_median(dtype, x, starts[j], k, scratch, y, j, argmed ? &argmed[j] : NULL);
        free(scratch);
    }
    return 0;
}

static int check_rank_args(int dtype, const void* x, int64_t n, int32_t k, int32_t r)
{
    if (dtype < MFO_INT32 || dtype > MFO_FLOAT64) return -1;
    if (!x || n < 1) return -2;
    if (k < 1 || (int64_t)k > n) return -3;
    if (r < 0 || r >= k) return -5;
    return 0;
}

/* Rank filter: y[i] = element of rank r in x[i .. i+k-1], i = 0 .. n-k. */
int mfo_rank_filter(int dtype, const void* x, int64_t n, int32_t k, int32_t r,
                    void* y, int64_t* arg, int nthreads)
{
    int rc = check_rank_args(dtype, x, n, k, r);
    if (rc) return rc;
    int64_t m = n - k + 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        elem_t* scratch = (elem_t*)malloc(sizeof(elem_t) * (size_t)k);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t i = 0; i < m; ++i)
            window_select(dtype, x, i, k, r, scratch, y, i, arg ? &arg[i] : NULL);
        free(scratch);
    }
    return 0;
}

/* Rank filter on sampled windows (see mfo_windows). */
int mfo_rank_windows(int dtype, const void* x, int64_t n, int32_t k, int32_t r,
                     const int64_t* starts, int64_t count, void* y, int64_t* arg,
                     int nthreads)
{
    int rc = check_rank_args(dtype, x, n, k, r);
    if (rc) return rc;
    for (int64_t j = 0; j < count; ++j)
        if (starts[j] < 0 || starts[j] > n - k) return -4;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        elem_t* scratch = (elem_t*)malloc(sizeof(elem_t) * (size_t)k);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t j = 0; j < count; ++j)
            window_select(dtype, x, starts[j], k, r, scratch, y, j, arg ? &arg[j] : NULL);
        free(scratch);
    }
    return 0;
}

/* Number of threads an OpenMP parallel region would use (1 without OpenMP). */
int mfo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * mf.h -- C ABI of the GB300 (sm_103a) sliding-window median filter.
 *
 * The operation (paper "Median Filtering is Equivalent to Sorting", Section 1,
 * "Median filter"): given x[0 .. n-1] and an odd window size k = 2h + 1,
 * output y[i] = median(x[i], ..., x[i+k-1]) for i = 0 .. n-k ("valid" windows
 * only, n-k+1 outputs; the paper defines no boundary padding).
 *
 * The median is the element of rank h under the order "value first, then
 * index", so it is always one of the input elements and y carries its exact
 * bits.  int32 values compare as signed integers; float32 values compare by
 * IEEE 754 totalOrder on their bit patterns (-0 < +0, NaNs at the ends by
 * sign), never by IEEE "<".  argmed[i] is the index of the median element in
 * the signal (ties between equal values resolve to the lower index, which is
 * what the paper's stable piecewise sort and its "older block first" rule in
 * Section 6.3 give).
 *
 * Method (paper Sections 3-6): phase 1 sorts each block X_j = x[jk .. jk+k)
 * stably (Section 3 "Piecewise Sorting", Section 5.2); phase 2 walks each
 * adjacent block pair with two sorted doubly-linked lists, deleting the old
 * block's elements and undoing the deletions of the new block's elements
 * (Knuth's dancing links, Section 4 equations del / undo-del), and prints the
 * smaller of the two lists' first large elements (Section 6.2).  Both phases
 * run fused in CUDA kernels; there is no CPU fallback.
 *
 * Conventions for every call below:
 *  - "device pointer" means memory of the handle's device (cudaMalloc, torch
 *    CUDA tensors, ...); "host pointer" means CPU memory.  The caller owns every
 *    buffer it passes; the library owns only its handle and an internal
 *    workspace inside the handle.
 *  - Arrays are dense and contiguous, element type given by mf_dtype.
 *  - Calls that take device pointers are asynchronous on the handle's stream
 *    and return after enqueueing; errors raised while kernels run surface at
 *    the next mf_sync (or any later call that synchronises).
 *  - Arguments are checked before anything is enqueued; on a bad argument
 *    nothing is launched and no output is written.
 *  - A handle is not thread-safe: use one handle per host thread.
 */
#ifndef MF_H
#define MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mf_ctx* mf_handle;

typedef enum {
    MF_OK = 0,
    MF_ERR_NULL = 1,         /* a required pointer or the handle is NULL            */
    MF_ERR_BAD_N = 2,        /* n < 1, or n too large for the requested outputs     */
    MF_ERR_EVEN_K = 3,       /* k is even: the paper assumes k = 2h + 1 (Section 3) */
    MF_ERR_K_GT_N = 4,       /* k < 1 or k > n: no full window                      */
    MF_ERR_DTYPE = 5,        /* unknown mf_dtype                                    */
    MF_ERR_OOM = 6,          /* workspace above max_workspace_bytes, or malloc fail */
    MF_ERR_CUDA = 7,         /* a CUDA runtime call or kernel failed                */
    MF_ERR_UNSUPPORTED = 8,  /* valid request this library variant does not serve  */
    MF_ERR_OVERLAP = 9,      /* an output buffer overlaps an input buffer           */
    MF_ERR_DEVICE = 10,      /* device index invalid or not an sm_103 GPU           */
    MF_ERR_BAD_SEGMENT = 11, /* a batched segment descriptor is invalid             */
    MF_ERR_TOO_LARGE = 12,   /* request needs more scratch than mf_filter_noalloc's
                                fixed array holds                                   */
    MF_ERR_BAD_RANK = 13     /* mf_filter_rank: rank outside 0 .. k-1               */
} mf_status;

/* Element types.  Keys are compared as signed integers (int32, int64) or by
 * IEEE 754-2008 totalOrder (float32, float64; Section 5.10 of that standard);
 * the paper's experiments use 32-bit and 64-bit inputs (Section 7.3). */
typedef enum { MF_INT32 = 0, MF_FLOAT32 = 1, MF_INT64 = 2, MF_FLOAT64 = 3 } mf_dtype;

/* One signal of a batch.  Offsets are in elements from the x / y base
 * pointers passed to mf_filter_batched; the signal is x[x_off .. x_off+n) and
 * its n-k+1 outputs go to y[y_off ..].  pad must be 0. */
typedef struct {
    int64_t x_off;
    int64_t n;
    int64_t y_off;
    int32_t k;
    int32_t pad;
} mf_segment;

/* Create a handle bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  max_workspace_bytes
 * caps the device workspace the handle may hold (0 = no cap).
 * Errors: MF_ERR_NULL (out NULL), MF_ERR_DEVICE (no such device, or not
 * compute capability 10.3), MF_ERR_CUDA.  On error *out is set to NULL. */
mf_status mf_create(mf_handle* out, int device, void* cuda_stream, size_t max_workspace_bytes);

/* Rebind the handle to another stream of the same device. */
mf_status mf_set_stream(mf_handle h, void* cuda_stream);

/* Median filter of one signal (paper Section 1; method Sections 3-6).
 *  x       device pointer, n elements of `dtype` (input, not modified)
 *  n       signal length, n >= k
 *  k       odd window size, 1 <= k <= n and k <= 262,143.  Below 3001
 *          (the handle's tier threshold, see mf_set_tier_threshold; at most
 *          9,344 for 4-byte and about 5,800 for 8-byte elements, one block
 *          pair in shared memory) the shared-memory pipeline runs; from it
 *          the large-k tier: global-memory merge tiers for the
 *          block sort and the post-processing chain of each block pair split
 *          into up to 32 segments, each started from a state rebuilt with the
 *          invariant of Section 6.3 (workspace about 52 + 16 * segments bytes
 *          per sample)
 *  y       device pointer, n-k+1 elements of `dtype` (output, overwritten)
 *  argmed  device pointer to n-k+1 int32 (output) or NULL; needs n <= 2^31-1
 * y and argmed must not overlap x.
 * Errors: MF_ERR_NULL, MF_ERR_DTYPE, MF_ERR_BAD_N, MF_ERR_EVEN_K,
 * MF_ERR_K_GT_N, MF_ERR_OVERLAP, MF_ERR_UNSUPPORTED (k above the limit),
 * MF_ERR_CUDA (launch failed). */
mf_status mf_filter(mf_handle h, mf_dtype dtype, const void* x, int64_t n, int32_t k,
                    void* y, int32_t* argmed);

/* Rank (order-statistic) filter: y[i] = the element of 0-based rank `rank`
 * among x[i .. i+k-1] under the (value, index) order of mf_filter, for
 * i = 0 .. n-k; argmed[i] its index.  The paper's method works unchanged for
 * any rank h in 0 .. k-1: the post-processing invariant (Section 6.3) keeps
 * the h smallest elements of the window "small" and prints the smallest
 * large one.  rank = (k-1)/2 with odd k is mf_filter; any k >= 1 is accepted
 * here, so even k gives the lower median with rank = k/2 - 1 (the upper
 * median with k/2), rank 0 a running minimum and rank k-1 a running maximum.
 * Arguments, ownership, limits and errors as mf_filter, plus MF_ERR_BAD_RANK;
 * MF_ERR_EVEN_K is never returned. */
mf_status mf_filter_rank(mf_handle h, mf_dtype dtype, const void* x, int64_t n, int32_t k,
                         int32_t rank, void* y, int32_t* argmed);

/* Same as mf_filter, but x, y and argmed are HOST pointers.  The call copies
 * x to the handle's device workspace, filters, copies y (and argmed) back and
 * waits: it is synchronous.  Signals of more than 2^20 outputs run in up to
 * eight chunks of outputs (each with its k-1 input halo) as a pipeline on
 * three streams: copies in on a stream of the handle, the filter on the
 * handle's stream, copies out on a third, chained by events, with three
 * chunk buffers in flight; so one chunk's copies overlap the filtering of
 * the others, and copies in overlap copies out.  The results equal one whole
 * call.  Pinned host memory gives the fastest copies; pageable memory works.
 * Errors: as mf_filter, plus MF_ERR_OOM (workspace). */
mf_status mf_filter_host(mf_handle h, mf_dtype dtype, const void* x_host, int64_t n, int32_t k,
                         void* y_host, int32_t* argmed_host);

/* Filter many independent signals in one call (all of one dtype).
 *  x, y       device base pointers; signal s is x[segs[s].x_off ..+n) and
 *             writes y[segs[s].y_off ..+ n-k+1)
 *  segs_host  HOST array of nseg descriptors (read before return)
 *  argmed     device pointer parallel to y (index within each signal) or NULL
 * Output ranges must not overlap each other or x.
 * The signals are grouped by window size into at most six classes and each
 * class runs as one launch per kernel (at most 24 launches per call,
 * whatever nseg is).  Signals whose k is above the shared-memory pipeline's
 * limit follow, one large-k launch sequence each (7 + log2(k / 1024)
 * launches), in the same workspace.  The call can be captured into a CUDA graph: make one
 * uncaptured call with the same sizes first (it allocates the workspace and
 * a pinned descriptor buffer; during capture nothing may be allocated and
 * such calls return MF_ERR_OOM).  A captured call's descriptors stay with
 * its graph; later calls on the handle use a new buffer.
 * Errors: as mf_filter, plus MF_ERR_BAD_SEGMENT (naming no segment index:
 * any invalid descriptor rejects the whole call), MF_ERR_OOM. */
mf_status mf_filter_batched(mf_handle h, mf_dtype dtype, const void* x, void* y,
                            const mf_segment* segs_host, int32_t nseg, int32_t* argmed);

/* Backward pass of y = median_filter(x): gx[j] = sum of gy[i] over the
 * outputs i whose median element is j (argmed[i] == j), summed in ascending
 * i, so the result is deterministic.  This is the gradient of y with respect
 * to x wherever the window values are distinct.
 *  gy      device pointer, n-k+1 float32 (upstream gradient)
 *  argmed  device pointer, n-k+1 int32 from mf_filter of the same (n, k)
 *  gx      device pointer, n float32 (output, overwritten)
 * Errors: as mf_filter. */
mf_status mf_filter_backward(mf_handle h, const float* gy, const int32_t* argmed,
                             int64_t n, int32_t k, float* gx);

/* mf_filter_backward for `rows` independent signals of the same n and k in
 * one launch (the backward pass of a batched call on equal rows).
 *  gy      device pointer, rows x (n-k+1) float32, row-major
 *  argmed  device pointer, rows x (n-k+1) int32, each row's indices local to
 *          that row (as mf_filter_batched reports them)
 *  gx      device pointer, rows x n float32 (output, overwritten)
 * Row r of gx is mf_filter_backward of row r of gy and argmed, bit for bit.
 * Errors: as mf_filter_backward; rows < 1 is MF_ERR_BAD_N. */
mf_status mf_filter_backward_rows(mf_handle h, const float* gy, const int32_t* argmed,
                                  int64_t rows, int64_t n, int32_t k, float* gx);

/* The median filter of mf_filter for callers that cannot call cudaMalloc.
 * The paper has no counterpart: this entry point exists because some callers
 * may not allocate device memory -- programs whose device memory is handed
 * out only by their own pool or arena (which must see no allocation made
 * behind its back), and real-time loops that cannot take an allocation's
 * unbounded latency.  It needs no handle and allocates nothing: its scratch
 * is a fixed 32 MiB device array inside the library, present on every GPU
 * that loads libmf.so until the process exits.
 *  x, n, k, y, argmed  as mf_filter (device pointers of the current device;
 *                      MF_INT32 or MF_FLOAT32 only, else MF_ERR_DTYPE)
 *  cuda_stream         cudaStream_t to run on (NULL = legacy default stream)
 * Limits: k <= 9,344 (larger windows return MF_ERR_UNSUPPORTED).  The call
 * always runs the shared-memory pipeline: the tier threshold of
 * mf_set_tier_threshold does not apply, so for 3,001 <= k <= 9,344, where
 * mf_filter uses the large-k tier by default, the results are the same but
 * the time and the scratch differ.  The scratch a call needs is the larger
 * of 12 * kp bytes per block of k samples plus 6 * kp per block pair, and
 * 8 * kw + 2 * kp per block pair (kp = k rounded up to a multiple of 8,
 * kw = k + 3 rounded up to a multiple of 8): about 18 bytes per input
 * sample for k >= 31, so n is limited to about 1.8 million (1,805,843 at
 * k = 31, 1,850,849 at k = 1001).  Small k costs more per sample because
 * kp rounds up: 48 bytes at k = 3 (n <= 699,027), 144 at k = 1
 * (n <= 233,009).  Larger requests return MF_ERR_TOO_LARGE and launch
 * nothing.
 * The first call on a device, with that device current, looks up the
 * array's device address and sets the kernels' limits; make that first call
 * before any stream capture.  All calls share the one array: calls whose
 * kernels overlap on the GPU (different streams, different host threads)
 * race on it and must be serialised by the caller.  The array keeps the
 * previous call's contents; the kernels write every scratch element before
 * reading it, so nothing needs clearing.
 * Errors: as mf_filter for the arguments, plus MF_ERR_UNSUPPORTED
 * (k > 9,344), MF_ERR_TOO_LARGE and MF_ERR_DEVICE. */
mf_status mf_filter_noalloc(mf_dtype dtype, const void* x, int64_t n, int32_t k,
                            void* y, int32_t* argmed, void* cuda_stream);

/* Wait for the handle's stream; returns MF_ERR_CUDA if any enqueued work failed. */
mf_status mf_sync(mf_handle h);

/* Number of kernels this handle has launched since creation (for accounting). */
mf_status mf_launch_count(mf_handle h, uint64_t* count);

/* Debug build only (libmf_debug.so, compiled with -DMF_DEBUG; the Python
 * binding loads it when the environment sets MF_DEBUG=1).  Its kernels check
 * their indices and the invariants of the block data structures (Section 5:
 * link fields name a slot or a sentinel, 0 <= s <= h, m a live node of its
 * list whose cached word is current; Section 6.3: s_A + s_B = h after every
 * step of the large-k tier; a printed node is an element, not a sentinel).
 * A failed check does not fault: it is counted, the first one's site and
 * value are kept, and the kernel continues with the index clamped into
 * range.  mf_debug_take waits for all work on the handle's device, then
 * returns and clears the records of every kernel file: *count failed checks
 * in all, *site / *value of the first (sites 1xx fused sort kernel, 2xx chain
 * and store kernels, 3xx large-k tier, 999 the self-test).  The records are
 * per process and device, not per handle.  mf_debug_selftest enqueues one
 * thread that fails one check (site 999, value 42) on the handle's stream,
 * so a test can see the record reach the host.  Errors: MF_ERR_NULL,
 * MF_ERR_CUDA; in the normal build both return MF_ERR_UNSUPPORTED (and
 * mf_debug_take zeroes its outputs). */
mf_status mf_debug_take(mf_handle h, uint32_t* count, uint32_t* site, uint64_t* value);
mf_status mf_debug_selftest(mf_handle h);

/* Launch-plan tuning for the window-size class that contains k (classes
 * k <= 64, <= 256, <= 1021, <= 2047, <= 4093, larger): block pairs per CTA
 * of the sort+merge kernel and of the store kernel (0 = built-in choice;
 * values above the built-in choice, which fills shared memory, are capped).
 * Used by the autotuner in paper_1406_1717_gb300/tune.py. */
mf_status mf_set_tuning(mf_handle h, int32_t k, int32_t sort_pairs_per_cta,
                        int32_t store_pairs_per_cta);

/* Block-sort variant for the window-size class that contains k (the classes
 * of mf_set_tuning).  Section 3 leaves the piecewise sort open ("any sorting
 * algorithm"); both variants give the same stable order, so the results do
 * not change, only the time:
 *  0  built-in choice;
 *  1  merge-sort tiles: a warp sorts 1024-element tiles (odd-even network per
 *     lane, merge-path rounds) in the same kernel that builds both lists
 *     (k <= 1021; elsewhere variant 2 is used); 8-byte elements are sorted
 *     twice, on the low then the high half of their 64-bit key;
 *  2  warp LSD radix sort (8-bit digits) in a kernel of its own, followed by
 *     separate unwind, chain and store kernels;
 *  3  as 1, but every tile is first tested for blocks that are already in
 *     order (ascending, or strictly descending) and those tiles are not
 *     sorted (Section 1: an adaptive sort gives an adaptive median filter);
 *     the test costs a few percent on unordered input (4-byte elements;
 *     for 8-byte elements 3 acts as 1).
 * Used by the autotuner.  Errors: MF_ERR_NULL, MF_ERR_K_GT_N (k < 1),
 * MF_ERR_UNSUPPORTED (variant outside 0 .. 3). */
mf_status mf_set_sort_variant(mf_handle h, int32_t k, int32_t variant);

/* Device workspace (bytes) that mf_filter_batched with these descriptors
 * needs on this handle (host-only computation; the request server admits
 * work by it).  Errors: MF_ERR_NULL, MF_ERR_BAD_SEGMENT. */
mf_status mf_batched_workspace_bytes(mf_handle h, mf_dtype dtype, const mf_segment* segs_host,
                                     int32_t nseg, size_t* bytes);

/* Bytes of device workspace the handle currently holds. */
mf_status mf_workspace_size(mf_handle h, size_t* bytes);

/* Wait for the handle's stream and free its device workspace (the next call
 * allocates again).  Errors: MF_ERR_NULL, MF_ERR_UNSUPPORTED (stream being
 * captured), MF_ERR_CUDA. */
mf_status mf_release_workspace(mf_handle h);

/* Window size from which calls on this handle use the large-k tier instead
 * of the shared-memory pipeline (k >= k_large_from; k above the pipeline's
 * limit of 9,344 always uses it).  0 restores the built-in crossover (3001,
 * measured on GB300); values above the pipeline's limit are capped to it.  Both tiers give the same results; the threshold only
 * chooses the faster one (the autotuner in paper_1406_1717_gb300/tune.py
 * measures the crossover).  Errors: MF_ERR_NULL, MF_ERR_K_GT_N (k < 0). */
mf_status mf_set_tier_threshold(mf_handle h, int32_t k_large_from);

/* The handle's current threshold: calls with k >= *k_large_from use the
 * large-k tier. */
mf_status mf_get_tier_threshold(mf_handle h, int32_t* k_large_from);

/* Per-kernel timing for measurement.  With timing enabled, every mf_filter /
 * mf_filter_host call records CUDA events on the handle's stream around its
 * four kernel groups (sort, unwind, post-processing chains, store), in a ring
 * of the last 128 calls; enabling resets the ring.  The groups per path:
 *   k <= 1021: the fused sort kernel (block sort, joint
 *     ranks, unwind links, list words) / nothing / chains / store;
 *   other windows of the shared-memory pipeline: sort + joint ranks /
 *     unwind links / chains / store;
 *   large-k tier: chunk sort, merge tiers and joint ranks / unwind /
 *     segment states and chains / store. */
mf_status mf_set_timing(mf_handle h, int enable);

/* Sum of each kernel's duration (ms) over the last `ncalls` timed calls
 * (at most 128): ms[0] sort, ms[1] unwind, ms[2] chains, ms[3] store.
 * Waits for those calls to finish. */
mf_status mf_kernel_times(mf_handle h, int32_t ncalls, float* ms);

/* Static string naming a status code (never NULL). */
const char* mf_status_str(mf_status s);

/* Release the handle and its workspace (waits for its stream first). */
mf_status mf_destroy(mf_handle h);

#ifdef __cplusplus
}
#endif

#endif /* MF_H */

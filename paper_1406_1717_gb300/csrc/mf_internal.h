// mf_internal.h -- declarations shared by the library's translation units
// (kernel parameter blocks and host launchers).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace mf {

constexpr int kMaxSmemBytes = 227 * 1024;          // opt-in dynamic shared memory per CTA

// ---- multi-kernel pipeline (mf_pipeline.cu) --------------------------------
constexpr int kPipeThreads = 256;

struct PipeParams {
    const void* x;            // n elements of 4 bytes (int32, float32) or 8 (int64, float64)
    void* y;
    int32_t* argmed;
    int64_t n, nblocks, npairs;
    int k, h, kp;             // kp: k rounded up to a multiple of 8 (16-byte rows)
    bool is_float;
    uint16_t* perm;           // [nblocks][kp] position of the t-th smallest
    uint16_t* rnk;            // [nblocks][kp] rank of position p
    uint32_t* slink;          // [nblocks][kp] sorted-order prev:16|next:16, sentinel k
    uint32_t* ulink;          // [nblocks][kp] unwind-time prev:16|next:16, sentinel k+1
    uint16_t* ja;             // [npairs][kp] joint rank of A's position p
    uint16_t* jb;             // [npairs][kp] joint rank of B's position p
    uint16_t* out;            // [npairs][kp] printed node at step i: isB << 15 | slot
    // fused path (sortlist_kernel; k <= kFusedMaxK)
    uint32_t* wA;             // [npairs][kw] list words of construct(A): slots 0..k+1, m_A in slot k+2
    uint32_t* wB;             // [npairs][kw] undelete(B, i) word of every position i of B
    int kw;                   // row stride of wA / wB in words: >= k + 3, multiple of 4
    int lG;                   // block pairs per sortlist CTA
    int bpw;                  // blocks per warp tile (kTileElems / k)
    uint64_t kmagic, bmagic;  // ceil(2^32 / k), ceil(2^32 / bpw): exact division of tile indices
    int eG;                   // block pairs per epilogue CTA
    int64_t start[4];         // batched launches: this signal's first item per kernel
};

// The signals of one launch: one descriptor by value, or a device table
// (segs != nullptr) sorted by first item.
struct SegTable {
    const PipeParams* segs;
    int nseg;
    PipeParams one;
};

// Optional per-handle tuning of the launch plans (0 = built-in choice).
struct Tuning {
    int sort_G;               // pairs per sortmerge CTA
    int epi_G;                // pairs per epilogue CTA
    int variant;              // block sort: 0 built-in, 1 merge-sort tiles (fused path,
                              // k <= kFusedMaxK), 2 warp radix sort (four-kernel
                              // path), 3 merge-sort tiles that skip tiles of
                              // ordered blocks (4-byte elements; 8-byte: as 1)
};
struct SortPlan {
    uint32_t off_keyA, off_keyB, off_valA, off_valB, off_hist;
    int G;
};
struct UnwindPlan {
    int segs, seglen;         // runs per block (1, 2, 4) and positions per run (multiple of 8)
    int nw, ns;               // bitset words; summary words (0: one summary word in a register)
    uint32_t words_per_warp;
    int64_t items;            // warp groups in the launch
};
// Fused path: one kernel sorts the blocks (warp merge sort of 1024-element
// tiles), merges the pairs and makes B's unwind links; the chain kernel reads
// its list words.  Packed chain format only (slots fit in 10 bits).
constexpr int kFusedMaxK = 1021;
constexpr int kMidMaxK = 4093;                   // 12-bit slot numbers: slots 0 .. k+1 <= 4094
constexpr int kTileElems = 1024;                 // elements per warp tile
constexpr int kSortListWarps = 8;          // warps (tiles) per sortlist CTA
struct ChainPlan {
    int fmt;                  // list node format: packed (k <= 1021), mid (k <= kMidMaxK), wide
    int nwarps;
    int pairs_per_cta;
    uint32_t lanes_log2;      // 3 bits per warp: warp w handles 1 << field pairs
    uint32_t lane_words;      // shared-memory words per pair
    uint32_t rec_words;       // k + 2
    uint32_t info_off;        // byte offset of the per-pair descriptors of the CTA-wide construct
    int64_t items;            // pairs in the launch
};

// Launch accounting of a handle: kernel count and, when timing is on, CUDA
// events around the four kernels of each of the last kRing calls.
struct LaunchStats {
    static constexpr int kRing = 128;
    uint64_t launches = 0;
    bool timing = false;
    uint64_t ring_pos = 0;
    cudaEvent_t ev[kRing][5];
    const Tuning* tune = nullptr;      // per launch class, kNumTuneClasses entries
};

constexpr int kNumTuneClasses = 6;     // classes of k: <= 64, 256, 1021, 2047, 4095, larger
int tune_class_of(int k);

// Element type of a call: float or integer, 4 or 8 bytes.
struct Elem {
    bool is_float;
    bool wide;                // 8-byte elements
    int bytes() const { return wide ? 8 : 4; }
};

int pipeline_max_k(bool wide = false);
size_t sortlist_smem_bytes(int warps);
cudaError_t sortlist_setup();
cudaError_t launch_sortlist(const SegTable& tab, int64_t items, int warps, bool adaptive, bool wide,
                            cudaStream_t stream);
size_t pipeline_workspace_bytes(int64_t n, int k);
cudaError_t pipeline_setup();
// rank: 0-based order statistic printed for every window (the median of an
// odd window is (k - 1) / 2)
cudaError_t launch_pipeline(const void* x, int64_t n, int k, int rank, Elem el,
                            void* y, int32_t* argmed, void* ws, size_t ws_bytes,
                            int num_sms, cudaStream_t stream, LaunchStats* stats);
size_t pipeline_batched_workspace_bytes(const int64_t* n, const int32_t* k, int nseg);
// Batched: `stage` is host memory (pinned for graph capture) of at least
// nseg * sizeof(PipeParams) bytes that must stay unchanged until the copy ran.
cudaError_t launch_pipeline_batched(const void* x, void* y, int32_t* argmed, Elem el,
                                    const int64_t* x_off, const int64_t* n, const int64_t* y_off,
                                    const int32_t* k, int nseg, void* ws, size_t ws_bytes,
                                    void* stage, size_t stage_bytes, int num_sms,
                                    cudaStream_t stream, LaunchStats* stats);

// ---- large-k tier (mf_large.cu): pipeline_max_k() < k <= kLargeMaxK -------
constexpr int kLargeMaxK = (1 << 18) - 1;      // window-rank bitsets fit in shared memory
constexpr int kLargeSegSteps = 1024;   // target steps per chain segment
constexpr int kLargeMaxSegs = 32;      // segments per block pair at most
// Default tier crossover, measured on GB300 (float32 random walk, ms,
// pipeline / large-k tier): n = 10^7: k = 3001 2.01 / 2.08, 3501 2.18 /
// 2.21, 4001 2.64 / 2.20; n = 10^6: 3001 0.69 / 0.56; n = 10^5: 3001 0.59 /
// 0.43.  A batch of 4096 signals with k up to 4095 took 12.24 ms with the
// crossover at 3001 and 12.60 ms at 5001.
constexpr int kLargeFromK = 3001;
cudaError_t large_setup();
size_t large_workspace_bytes(int64_t n, int k, bool wide);
cudaError_t launch_large(const void* x, int64_t n, int k, int rank, Elem el, void* y,
                         int32_t* argmed, void* ws, size_t ws_bytes, cudaStream_t stream,
                         LaunchStats* stats);
// Every large-k signal of a batch in one launch sequence (median rank of each
// signal): descriptors staged in `stage` (host memory of at least
// nseg * large_descriptor_bytes(), unchanged until the copy ran), workspace
// large_batched_workspace_bytes().
size_t large_descriptor_bytes();
size_t large_batched_workspace_bytes(const int64_t* n, const int32_t* k, int nseg, bool wide);
cudaError_t launch_large_batched(const void* x, void* y, int32_t* argmed, Elem el,
                                 const int64_t* x_off, const int64_t* n, const int64_t* y_off,
                                 const int32_t* k, int nseg, void* ws, size_t ws_bytes,
                                 void* stage, size_t stage_bytes, cudaStream_t stream,
                                 LaunchStats* stats);

cudaError_t backward_setup();
cudaError_t launch_backward(const float* gy, const int32_t* argmed, int64_t rows, int64_t n, int k,
                            float* gx, cudaStream_t stream, uint64_t* launches);

#ifdef MF_DEBUG
// Debug build: each translation unit's record of failed device checks (read
// and cleared), and a one-thread kernel that fails one check on purpose
// (site 999, value 42) so that the recording itself can be tested.
cudaError_t debug_take_sortlist(uint32_t* count, uint32_t* site, uint64_t* value);
cudaError_t debug_take_pipeline(uint32_t* count, uint32_t* site, uint64_t* value);
cudaError_t debug_take_large(uint32_t* count, uint32_t* site, uint64_t* value);
cudaError_t debug_selftest(cudaStream_t stream);
#endif

}  // namespace mf

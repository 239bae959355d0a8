// mf_large.cu -- the median filter for window sizes too large for the
// shared-memory pipeline (pipeline_max_k() < k <= kLargeMaxK).
//
// Paper: "Median Filtering is Equivalent to Sorting" (Suomela).  The method
// of mf_pipeline.cu (comparisons by joint rank in A u B, A first on ties)
// with 32-bit indices and the data in global memory:
//
//   large_chunk_sort  a warp sorts each 1024-element chunk of a block in
//                     shared memory, stably (Section 5.2), by the warp tile
//                     merge sort of key : index composites (8-byte keys: on
//                     their top 44 bits, the chunk sorted again on the whole
//                     key when two of them tie there)
//   large_merge       global merge-path tiers: sorted runs of R -> 2R until a
//                     run covers the block, left run first on equal keys
//   large_ranks       rank of each position in its block
//   large_jrank       joint ranks of each pair by a merge of its two sorted
//                     blocks (A first on equal keys): ja / jb by position,
//                     jrs by B's sorted order and M = the merged order
//   large_unwind      unwind(B)'s links (Section 4: after unwind, undelete(B, i)
//                     relinks i between its nearest smaller and larger
//                     elements among positions < i); one CTA per eight runs
//                     of positions, seeded with a rank bitset of the
//                     positions before its first run
//   large_seginit     rebuilds the lists before step i0 of a pair (Section 6.3
//                     invariant: S_A u S_B are the h smallest of the window)
//                     in one coalesced pass over the pair's merged order
//   large_chain       the steps i0 .. i1-1 of Section 6.2 from that state,
//                     one thread per (pair, segment), lists in global memory,
//                     one level of independent node loads per step
//   large_epilogue    node -> input element, y / argmed
//
// Nodes are numbered by joint rank: the element of joint rank r is node r,
// A's sentinel is 2k and B's 2k+1.  A node's number is its rank, so "is
// small" and peek(A) <= peek(B) compare node numbers, and list neighbours are
// rank neighbours: the walks of the two m pointers stay within a few cache
// lines, and the only random load of a step (the deleted node, known in
// advance) is prefetched into L2.
// The serial depth of one pair is k steps; splitting the k steps of a pair
// into S independent segments, each starting from a state rebuilt with O(k)
// parallel work, cuts the depth to k / S at the price of S private copies of
// the pair's links (8 bytes per node, 2k + 2 nodes).
#include <cuda_runtime.h>
#include <cstdint>
#include "mf_device.cuh"
#include "mf_internal.h"
#include "mf_tilesort.cuh"

namespace mf {

constexpr int kChunk = 1024;                     // elements per warp sort
constexpr int kUnwindRun = 1024;                 // positions per unwind run
constexpr int kUnwindRunsPerCta = 8;             // consecutive runs of one unwind CTA
constexpr uint32_t kBFlag = 0x80000000u;          // node id of B's element

struct LargeParams {
    const void* x;                               // 4- or 8-byte elements
    void* y;
    int32_t* argmed;
    int64_t n, nblocks, npairs;
    int k, h;
    int64_t kp;                                  // row stride (k rounded up to 32)
    bool is_float;
    int S, L;                                    // segments per pair, steps per segment
    int64_t LN;                                  // list stride: 2k + 2 rounded up to 32
    void *keyA, *keyB;                           // [nblocks][kp] sort keys (4 or 8 bytes)
    uint32_t *valA, *valB;                       // [nblocks][kp] positions (ping-pong)
    uint32_t* rnk;                               // [nblocks][kp] rank of position p
    uint2* ulink;                                // [nblocks][kp] unwind (prev, next), sentinel k+1
    uint32_t* ja;                                // [npairs][kp] joint rank of A's position p
    uint32_t* jb;                                // [npairs][kp] joint rank of B's position p
    uint32_t* jrs;                               // [npairs][kp] joint rank of B's t-th smallest
    uint32_t* M;                                 // [npairs][2 kp] node at joint rank r
    uint32_t* out;                               // [npairs][kp] printed node at step i
    int4* seg;                                   // [npairs][S] (mA, mB, sA, sB) before step i0
    uint2* lists;                                // [npairs][S][LN] (next, prev) per rank node
    int cpb;                                     // 1024-element chunks per block
    int ntier;                                   // merge tiers (runs of 1024 -> one run per block)
    const void* ksort;                           // keyA or keyB: the sorted keys after the tiers
    const uint32_t* vsort;                       // valA or valB: the sorted positions
    int64_t start[15];                           // this signal's first item in each launch
};

// Launches of the tier and their work items.  One launch serves every signal
// of a call (one signal, or the large-k signals of a batch): an item finds its
// signal by binary search over the signals' first items.
enum {
    kLChunk = 0,          // warp: (block, chunk)
    kLMerge0 = 1,         // thread: 4 outputs of merge tier t (kLMerge0 + t)
    kLRanks = 9,          // thread: (block, sorted index)
    kLJrank = 10,         // thread: (pair, run of kJrankRun merged outputs)
    kLUnwind = 11,        // CTA: (block >= 1, run of kUnwindRun positions)
    kLSeg = 12,           // CTA: (pair, segment)
    kLChain = 13,         // thread: (pair, segment)
    kLEpi = 14            // thread: output
};
constexpr int kLMaxTiers = 8;                    // 1024 << 8 > kLargeMaxK

struct LargeTable {
    const LargeParams* segs;                     // device table (nullptr: `one`)
    int nseg;
    LargeParams one;
};

__device__ __forceinline__ LargeParams find_large(const LargeTable& t, int kind, int64_t item,
                                                  int64_t* local)
{
    if (t.segs == nullptr) { *local = item; return t.one; }
    int lo = 0, hi = t.nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.segs[mid].start[kind] <= item) lo = mid; else hi = mid - 1;
    }
    *local = item - t.segs[lo].start[kind];      // indexed in global memory, not in the copy
    return t.segs[lo];
}

__device__ __forceinline__ int block_len(const LargeParams& p, int64_t b) {
    const int64_t r = p.n - b * (int64_t)p.k;
    return (int)(r < p.k ? r : p.k);
}

// Two-level bitsets in shared memory: W[w] bit b = element 32w+b, summary
// W1[s] bit c set iff W[32s+c] != 0.
__device__ __forceinline__ int bits_first_from(const uint32_t* W, const uint32_t* W1,
                                               int nw, int ns, int r)
{
    if (r < 0) r = 0;
    const int w = r >> 5;
    if (w >= nw) return -1;
    const uint32_t m = W[w] & (0xffffffffu << (r & 31));
    if (m) return (w << 5) + __ffs(m) - 1;
    const int w1 = w + 1;
    if (w1 >= nw) return -1;
    int s = w1 >> 5;
    uint32_t sm = W1[s] & (0xffffffffu << (w1 & 31));
    while (true) {
        if (sm) {
            const int ww = (s << 5) + __ffs(sm) - 1;
            return (ww << 5) + __ffs(W[ww]) - 1;
        }
        if (++s >= ns) return -1;
        sm = W1[s];
    }
}

// largest element < r, or -1
__device__ __forceinline__ int bits_last_before(const uint32_t* W, const uint32_t* W1,
                                                int nw, int r)
{
    if (r > (nw << 5)) r = nw << 5;
    if (r <= 0) return -1;
    const int t = r - 1;
    const int w = t >> 5;
    const uint32_t m = W[w] & (0xffffffffu >> (31 - (t & 31)));
    if (m) return (w << 5) + 31 - __clz(m);
    const int w1 = w - 1;
    if (w1 < 0) return -1;
    int s = w1 >> 5;
    uint32_t sm = W1[s] & (0xffffffffu >> (31 - (w1 & 31)));
    while (true) {
        if (sm) {
            const int ww = (s << 5) + 31 - __clz(sm);
            return (ww << 5) + 31 - __clz(W[ww]);
        }
        if (--s < 0) return -1;
        sm = W1[s];
    }
}

// ---------------------------------------------------------------------------
// a warp's shared memory: the padded tile of composites, plus 4 KB of
// permutation scratch for the whole-key re-sort of 8-byte chunks
template <typename KeyT>
__host__ __device__ constexpr size_t chunk_warp_bytes() { return 8ull * kTileU64 + (sizeof(KeyT) == 8 ? 4096 : 0); }
static_assert(kChunk == kTileElems, "a chunk is one warp tile of composites");

template <typename KeyT>
__global__ void __launch_bounds__(256, 2)
large_chunk_sort(LargeTable tab, int64_t items)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (gw >= items) return;
    int64_t id;
    const LargeParams p = find_large(tab, kLChunk, gw, &id);
    const int64_t b = id / p.cpb;
    const int c = (int)(id - b * p.cpb);
    const int NB = block_len(p, b);
    const int lo = c * kChunk;
    const int cnt = min(kChunk, NB - lo);
    if (cnt <= 0) return;
    unsigned char* ws = smem + (size_t)warp * chunk_warp_bytes<KeyT>();
    const KeyT* xs = reinterpret_cast<const KeyT*>(p.x) + b * (int64_t)p.k + lo;
    if constexpr (sizeof(KeyT) == 4) {
        // 4-byte keys: the warp merge sort of composites key : index in the
        // chunk (10 bits), which orders equal keys by position
        uint64_t* T = reinterpret_cast<uint64_t*>(ws);
        uint64_t v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {                  // coalesced: the network takes any 32
            const int t = lane + 32 * i;
            v[i] = t < cnt ? ((uint64_t)to_key(__ldg(xs + t), p.is_float) << 10) | (uint32_t)t : kPadComp;
        }
        tile_sort(T, v, lane);
        const int64_t o = b * p.kp + lo;
        KeyT* keys = reinterpret_cast<KeyT*>(p.keyA);
#pragma unroll 4
        for (int i = 0; i < 32; ++i) {
            const int t = lane + 32 * i;
            if (t < cnt) {
                const uint64_t cp = T[tix(t)];
                keys[o + t] = (KeyT)(cp >> 10);
                p.valA[o + t] = (uint32_t)lo + (uint32_t)(cp & 1023u);
            }
        }
    } else {
        // 8-byte keys: the same sort on the top 44 bits of the key; a chunk
        // with ties in them is sorted again on the whole key (perm scratch:
        // 4 KB after the tile)
        uint64_t* T = reinterpret_cast<uint64_t*>(ws);
        uint64_t v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {                  // coalesced: the network takes any 32
            const int t = lane + 32 * i;
            v[i] = t < cnt ? ((to_key(__ldg(xs + t), p.is_float) >> 20) << 10) | (uint64_t)t : kPadComp;
        }
        tile_sort(T, v, lane);
        // one "block" of kChunk elements: block field 0 (x / kChunk by magic 2^22)
        if (tile_has_wide_ties(T, cnt, lane))
            tile_resort_wide(T, xs, p.is_float, cnt, kChunk, 1ull << 22,
                             reinterpret_cast<uint16_t*>(ws + 8 * kTileU64), lane);
        const int64_t o = b * p.kp + lo;
        KeyT* keys = reinterpret_cast<KeyT*>(p.keyA);
#pragma unroll 4
        for (int i = 0; i < 32; ++i) {
            const int t = lane + 32 * i;
            if (t < cnt) {
                const uint32_t e = (uint32_t)(T[tix(t)] & 1023u);
                keys[o + t] = (KeyT)to_key(__ldg(xs + e), p.is_float);
                p.valA[o + t] = (uint32_t)lo + e;
            }
        }
    }
}

// sorted runs [l0, l0+R) and [l0+R, l0+2R) of every block -> one run; each
// thread writes kMergeOut consecutive outputs after a merge-path search (2 was
// slower too)
constexpr int kMergeOut = 4;             // 8, 16, 32 measured slower (GB300, k = 100,001)
template <typename KeyT>
__global__ void __launch_bounds__(256)
large_merge(LargeTable tab, int tier, int64_t items)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= items) return;
    int64_t gid;
    const LargeParams p = find_large(tab, kLMerge0 + tier, g, &gid);
    // tier t reads the buffers tier t-1 wrote (A for even t, B for odd t)
    const bool odd = (tier & 1) != 0;
    const KeyT* __restrict__ kin = reinterpret_cast<const KeyT*>(odd ? p.keyB : p.keyA);
    KeyT* __restrict__ kout = reinterpret_cast<KeyT*>(odd ? p.keyA : p.keyB);
    const uint32_t* __restrict__ vin = odd ? p.valB : p.valA;
    uint32_t* __restrict__ vout = odd ? p.valA : p.valB;
    const int R = kChunk << tier;
    const int per_block = (int)(p.kp / kMergeOut);
    const int64_t b = gid / per_block;
    const int o = (int)(gid - b * per_block) * kMergeOut;
    const int NB = block_len(p, b);
    if (o >= NB) return;
    const int64_t base = b * p.kp;
    const int l0 = (o / (2 * R)) * 2 * R, r0 = min(l0 + R, NB);
    const int lenL = r0 - l0, lenR = min(l0 + 2 * R, NB) - r0;
    const int d = o - l0;
    const KeyT* KL = kin + base + l0;
    const KeyT* KR = kin + base + r0;
    int lo = max(0, d - lenR), hi = min(d, lenL);
    while (lo < hi) {                              // ia = #left elements among the first d
        const int mid = (lo + hi) >> 1;
        if (KL[mid] <= KR[d - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    int ia = lo, ib = d - lo;
    const int oend = min(o + kMergeOut, NB);
    for (int q = o; q < oend; ++q) {
        const bool takeL = ib >= lenR || (ia < lenL && KL[ia] <= KR[ib]);
        if (takeL) { kout[base + q] = KL[ia]; vout[base + q] = vin[base + l0 + ia]; ++ia; }
        else       { kout[base + q] = KR[ib]; vout[base + q] = vin[base + r0 + ib]; ++ib; }
    }
}

__global__ void __launch_bounds__(256)
large_ranks(LargeTable tab, int64_t items)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= items) return;
    int64_t gid;
    const LargeParams p = find_large(tab, kLRanks, g, &gid);
    const uint32_t* __restrict__ vs = p.vsort;
    const int64_t b = gid / p.kp;
    const int t = (int)(gid - b * p.kp);
    if (t >= block_len(p, b)) return;
    p.rnk[b * p.kp + vs[b * p.kp + t]] = (uint32_t)t;
}

// Joint ranks of pair q (A = block q, B = block q+1) by a merge of the two
// sorted blocks, A first on equal keys: A's t-th smallest gets t + #{B keys
// < key}, B's u-th u + #{A keys <= key}.  A thread takes kJrankRun
// consecutive outputs of the merged order: one merge-path search for where
// they start (Green, McColl & Bader 2012), then a sequential merge.
constexpr int kJrankRun = 4;             // 8 and 16 measured slower (GB300, k = 100,001)
template <typename KeyT>
__global__ void __launch_bounds__(256)
large_jrank(LargeTable tab, int64_t items)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= items) return;
    int64_t gid;
    const LargeParams p = find_large(tab, kLJrank, g, &gid);
    const KeyT* __restrict__ ks = reinterpret_cast<const KeyT*>(p.ksort);
    const uint32_t* __restrict__ vs = p.vsort;
    const int64_t per_pair = 2 * p.kp / kJrankRun;
    const int64_t q = gid / per_pair;
    const int NA = p.k, NB = block_len(p, q + 1), tot = NA + NB;
    const int o0 = (int)(gid - q * per_pair) * kJrankRun;
    if (o0 >= tot) return;
    const int o1 = min(o0 + kJrankRun, tot);
    const KeyT* KA = ks + q * p.kp;
    const KeyT* KB = ks + (q + 1) * p.kp;
    int lo = max(0, o0 - NB), hi = min(o0, NA);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (KA[mid] <= KB[o0 - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    int ia = lo, ib = o0 - lo;
    uint32_t* M = p.M + q * 2 * p.kp;
    for (int o = o0; o < o1; ++o) {
        if (ib >= NB || (ia < NA && KA[ia] <= KB[ib])) {
            const uint32_t pos = vs[q * p.kp + ia];
            M[o] = pos;
            p.ja[q * p.kp + pos] = (uint32_t)o;
            ++ia;
        } else {
            const uint32_t pos = vs[(q + 1) * p.kp + ib];
            M[o] = kBFlag | pos;
            p.jb[q * p.kp + pos] = (uint32_t)o;
            p.jrs[q * p.kp + ib] = (uint32_t)o;
            ++ib;
        }
    }
}

// Unwind links of block b >= 1 (Section 4, "Unwind": the links of position
// p are the nearest smaller and larger ranks among the positions before p).
// One CTA takes kUnwindRunsPerCta consecutive runs of kUnwindRun positions
// (item = (b - 1) * groups + group).  It keeps the bitset W of the ranks of
// all positions before the current run (built once from the sorted order,
// then grown run by run) and, for each run, takes the better of two
// candidates per position:
//  * among the positions before the run: a query of W (all threads);
//  * among the earlier positions of the run: the run's ranks are numbered
//    0 .. len-1 in sorted order ("local ranks", prefix popcounts of the bitset
//    R of the run's ranks), and warp 0 walks the run as 32 lanes of 32
//    positions, each lane's 1024-bit local bitset seeded with the local ranks
//    of the lanes before it (an exclusive OR-scan over lanes), as the fused
//    sort kernel does for a whole block.
// The ranks are then turned into nodes.
// Three CTAs per SM (80 registers; shared memory allows three): a CTA's
// run-by-run phases leave most of its warps at barriers while warp 0 walks,
// so a third CTA fills the SM (GB300, n = 10^7, k = 100,001: 0.95 -> 0.72 ms,
// despite 200 bytes of spills).
__global__ void __launch_bounds__(256, 3)
large_unwind(LargeTable tab)
{
    extern __shared__ __align__(16) uint32_t sw[];
    int64_t id;
    const LargeParams p = find_large(tab, kLUnwind, blockIdx.x, &id);
    const uint32_t* __restrict__ vs = p.vsort;
    const int runs = (p.k + kUnwindRun - 1) / kUnwindRun;
    const int groups = (runs + kUnwindRunsPerCta - 1) / kUnwindRunsPerCta;
    const int nw = (p.k + 31) / 32, ns = (nw + 31) / 32;
    const int64_t b = 1 + id / groups;
    const int NB = block_len(p, b);
    const int run0 = (int)(id - (b - 1) * groups) * kUnwindRunsPerCta;
    const int run1 = min(run0 + kUnwindRunsPerCta, (NB + kUnwindRun - 1) / kUnwindRun);
    if (run0 >= run1) return;
    int2* pp = reinterpret_cast<int2*>(sw);       // kUnwindRun (pred, succ) ranks
    uint32_t* rr = sw + 2 * kUnwindRun;            // kUnwindRun ranks of the run
    uint32_t* srt = rr + kUnwindRun;               // kUnwindRun: rank of local rank j
    uint32_t* lrk = srt + kUnwindRun;              // kUnwindRun: local rank of position t
    uint32_t* lb = lrk + kUnwindRun;               // 32 x 32 local bitsets (word w of lane L at 32 w + L)
    uint32_t* cs = lb + 32 * 32;                   // 256 per-thread counts (scan)
    uint32_t* W = cs + 256;                        // nw words: ranks of positions before the run
    uint32_t* W1 = W + nw;                         // ns words: summary of W
    uint32_t* R = W1 + ns;                         // nw words: ranks of the run
    uint32_t* Rc = R + nw;                         // nw words: popcount of R before word w
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const int64_t base = b * p.kp;
    const uint32_t sentB = 2u * (uint32_t)p.k + 1u;
    const uint32_t* jrs = p.jrs + (b - 1) * p.kp;
    {
        // eight words per warp at a time: their loads in flight together
        const int first = run0 * kUnwindRun;
        for (int w0 = warp; w0 < nw; w0 += 8 * nwarp) {
            uint32_t pos[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int r = ((w0 + j * nwarp) << 5) + lane;
                pos[j] = w0 + j * nwarp < nw && r < NB ? __ldg(vs + base + r) : 0xffffffffu;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t word = __ballot_sync(kFull, pos[j] < (uint32_t)first);
                if (lane == 0 && w0 + j * nwarp < nw) W[w0 + j * nwarp] = word;
            }
        }
        __syncthreads();
        for (int sI = tid; sI < ns; sI += blockDim.x) {
            uint32_t sm = 0;
            for (int c = 0; c < 32 && (sI << 5) + c < nw; ++c)
                if (W[(sI << 5) + c]) sm |= 1u << c;
            W1[sI] = sm;
        }
    }
    const int per = (nw + (int)blockDim.x - 1) / (int)blockDim.x;
    const int w0 = min(nw, tid * per), w1 = min(nw, w0 + per);
    for (int run = run0; run < run1; ++run) {
        const int i0 = run * kUnwindRun;
        const int len = min(kUnwindRun, NB - i0);
        for (int w = w0; w < w1; ++w) R[w] = 0u;
        for (int t = tid; t < len; t += blockDim.x) rr[t] = __ldg(p.rnk + base + i0 + t);
        __syncthreads();
        for (int t = tid; t < len; t += blockDim.x) atomicOr(&R[rr[t] >> 5], 1u << (rr[t] & 31));
        __syncthreads();
        // exclusive prefix popcount of R: thread t sums words [w0, w1)
        uint32_t cnt = 0;
        for (int w = w0; w < w1; ++w) cnt += __popc(R[w]);
        cs[tid] = cnt;
        __syncthreads();
        if (warp == 0) {                           // scan of the 256 counts, 8 per lane
            uint32_t c8[8], sum = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) { c8[q] = cs[8 * lane + q]; sum += c8[q]; }
            uint32_t incl = sum;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t v = __shfl_up_sync(kFull, incl, off);
                if (lane >= off) incl += v;
            }
            uint32_t acc = incl - sum;
#pragma unroll
            for (int q = 0; q < 8; ++q) { cs[8 * lane + q] = acc; acc += c8[q]; }
        }
        __syncthreads();
        cnt = cs[tid];
        for (int w = w0; w < w1; ++w) { Rc[w] = cnt; cnt += __popc(R[w]); }
        __syncthreads();
        // local ranks, sorted run; candidates among the positions before the run
        for (int t = tid; t < len; t += blockDim.x) {
            const uint32_t r = rr[t];
            const uint32_t lr = Rc[r >> 5] + __popc(R[r >> 5] & ((1u << (r & 31)) - 1u));
            lrk[t] = lr;
            srt[lr] = r;
            int2 q = make_int2(-1, -1);
            if (i0 > 0)
                q = make_int2(bits_last_before(W, W1, nw, (int)r), bits_first_from(W, W1, nw, ns, (int)r + 1));
            pp[t] = q;
        }
        __syncthreads();
        if (warp == 0) {
            // lane L: positions [32 L, 32 L + 32) of the run; bitsets over local ranks
            const int q0 = min(32 * lane, len), q1 = min(q0 + 32, len);
            uint32_t* bw = lb + lane;
            for (int w = 0; w < 32; ++w) bw[32 * w] = 0u;
            for (int t = q0; t < q1; ++t) bw[32 * (lrk[t] >> 5)] |= 1u << (lrk[t] & 31);
            __syncwarp();
            {
                // exclusive OR-scan over lanes, transposed: lane w scans word w
                // of all 32 lanes' bitsets (rotated order, bank (i + w) % 32)
                uint32_t* col = lb + 32 * lane;
                uint32_t c[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) c[i] = col[(i + lane) & 31];
                uint32_t low = 0u;
#pragma unroll
                for (int i = 0; i < 32; ++i) low |= (i >= 32 - lane) ? c[i] : 0u;
                uint32_t acc_hi = 0u, acc_lo = 0u;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const bool hi_part = i < 32 - lane;
                    const uint32_t pre = hi_part ? (low | acc_hi) : acc_lo;
                    acc_hi |= hi_part ? c[i] : 0u;
                    acc_lo |= hi_part ? 0u : c[i];
                    col[(i + lane) & 31] = pre;
                }
            }
            __syncwarp();
            uint32_t summ = 0;                      // bit w: word w non-empty
            for (int w = 0; w < 32; ++w) summ |= bw[32 * w] ? (1u << w) : 0u;
            for (int t = q0; t < q1; ++t) {
                const int lr = (int)lrk[t];
                const int w = lr >> 5, bb = lr & 31;
                const uint32_t word = bw[32 * w];
                const uint32_t mlo = word & ((1u << bb) - 1u);
                const uint32_t mhi = word & ~((2u << bb) - 1u);       // bb = 31: 0
                const uint32_t slo = summ & ((1u << w) - 1u);
                const uint32_t shi = summ & ~((2u << w) - 1u);
                int pl = -1, sl = -1;
                if (mlo) pl = (w << 5) | (31 - __clz(mlo));
                else if (slo) { const int ww = 31 - __clz(slo); pl = (ww << 5) | (31 - __clz(bw[32 * ww])); }
                if (mhi) sl = (w << 5) | (__ffs(mhi) - 1);
                else if (shi) { const int ww = __ffs(shi) - 1; sl = (ww << 5) | (__ffs(bw[32 * ww]) - 1); }
                bw[32 * w] = word | (1u << bb);
                summ |= 1u << w;
                int2 q = pp[t];
                if (pl >= 0) q.x = max(q.x, (int)srt[pl]);
                if (sl >= 0) { const int r = (int)srt[sl]; q.y = q.y < 0 ? r : min(q.y, r); }
                pp[t] = q;
            }
        }
        __syncthreads();
        // ranks -> rank nodes of pair b-1 (B's t-th smallest is node jrs[t]);
        // the run's ranks join W for the next run
        static_assert(kUnwindRun <= 4 * 256, "four positions per thread cover a run");
        {
            uint2 o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {                // loads first, four positions in flight
                const int t = tid + u * (int)blockDim.x;
                o[u] = make_uint2(sentB, sentB);
                if (t < len) {
                    const int2 q = pp[t];
                    if (q.x >= 0) o[u].x = __ldg(jrs + q.x);
                    if (q.y >= 0) o[u].y = __ldg(jrs + q.y);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = tid + u * (int)blockDim.x;
                if (t < len) {
                    p.ulink[base + i0 + t] = o[u];
                    const uint32_t r = rr[t];
                    atomicOr(&W[r >> 5], 1u << (r & 31));
                    atomicOr(&W1[r >> 10], 1u << ((r >> 5) & 31));
                }
            }
        }
        __syncthreads();
    }
}

// One CTA per (pair q, segment s): the state before step i0 = s L (Section
// 6.3: S_A u S_B are the h smallest elements of the window A[i0 .. k) u
// B[0 .. i0)), from the pair's merged order M in one coalesced pass.  Joint
// rank r is kept in A's list if it is an element of A at a position >= i0,
// in B's list if it is an element of B at a position < i0; a kept node's
// neighbours are the nearest kept ranks of its own list (sentinels SA = 2k,
// SB = 2k + 1).  Each warp takes a range of ranks, 32 per ballot: a kept
// node's prev is the highest kept rank of its list below it in the same 32,
// else the last one in the warp's earlier ranks, and the node writes itself
// as that node's next.  The first kept node of each list in a warp's range
// is linked after a barrier, to the last one of the warps before it.  Every
// 32 ballots a warp saves its counts and last kept nodes; the warp whose
// ranks hold the window's element of rank h then finds it by rescanning at
// most 32 ballots from a saved point, and with it s_A and the last kept node
// of each list below it.  Eight loads of M are in flight per lane.
__global__ void __launch_bounds__(256)
large_seginit(LargeTable tab)
{
    constexpr int kW = 8;                          // warps per CTA
    constexpr int kAhead = 8;                      // chunks of 32 ranks loaded at once
    constexpr int kCk = 32;                        // chunks between saved points
    constexpr int kMaxCk = (2 * kLargeMaxK + 2 + 32 * kW * kCk - 1) / (32 * kW * kCk);
    constexpr uint32_t kNone = 0xffffffffu;        // past the window: neither list
    __shared__ int s_cnt[2][kW], s_last[2][kW];
    __shared__ int4 s_ck[kW][kMaxCk];              // before chunk c0 + 32 j: (#A, #both, last A, last B)
    __shared__ int s_res[3];                       // s_A, last kept A / B rank below T
    int64_t sid;
    const LargeParams p = find_large(tab, kLSeg, blockIdx.x, &sid);
    const int64_t q = sid / p.S;
    const int s = (int)(sid - q * p.S);
    const int NB = block_len(p, q + 1);
    const int i0 = s * p.L;
    if (i0 >= NB) return;
    const int k = p.k, h = p.h, tot = k + NB;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t* M = p.M + q * 2 * p.kp;
    const int nch = (tot + 31) >> 5;
    const int per = (nch + kW - 1) / kW;
    const int c0 = min(nch, warp * per), c1 = min(nch, c0 + per);
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t SA = 2u * (uint32_t)k, SB = SA + 1u;
    uint32_t* NX = reinterpret_cast<uint32_t*>(p.lists + sid * p.LN);   // next of r at [2r], prev at [2r+1]
    auto load = [&](int cb, uint32_t (&ids)[kAhead]) {
#pragma unroll
        for (int j = 0; j < kAhead; ++j) {
            const int r = ((cb + j) << 5) + lane;
            ids[j] = cb + j < c1 && r < tot ? __ldg(M + r) : kNone;
        }
    };
    auto kept = [&](uint32_t id, int l) {
        const bool isB = (id & kBFlag) != 0;
        const int pos = (int)(id & ~kBFlag);
        return l == 0 ? (!isB && pos >= i0) : (isB && pos < i0);
    };

    // ---- the pass: links within the warp's ranks, counts, saved points ----
    int run[2] = {-1, -1}, first[2] = {-1, -1};
    int nA = 0, nU = 0;                                // kept nodes before the chunk (this warp)
    for (int cb = c0; cb < c1; cb += kAhead) {
        uint32_t ids[kAhead];
        load(cb, ids);
#pragma unroll
        for (int j = 0; j < kAhead; ++j) {
            const int c = cb + j;
            if (c >= c1) break;
            if (((c - c0) & (kCk - 1)) == 0 && lane == 0)
                s_ck[warp][(c - c0) / kCk] = make_int4(nA, nU, run[0], run[1]);
            const int r = (c << 5) + lane;
            const uint32_t kb[2] = {__ballot_sync(kFull, kept(ids[j], 0)), __ballot_sync(kFull, kept(ids[j], 1))};
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                if (!kb[l]) continue;
                const uint32_t m = kb[l] & below;
                const int pv = m ? (c << 5) + 31 - __clz(m) : run[l];
                if (((kb[l] >> lane) & 1u) && pv >= 0) {
                    NX[2 * r + 1] = (uint32_t)pv;         // prev of r
                    NX[2 * pv] = (uint32_t)r;             // next of its predecessor
                }
                if (first[l] < 0) first[l] = (c << 5) + __ffs(kb[l]) - 1;
                run[l] = (c << 5) + 31 - __clz(kb[l]);
            }
            nA += __popc(kb[0]);
            nU += __popc(kb[0] | kb[1]);
        }
    }
    if (lane == 0) {
        s_cnt[0][warp] = nA;
        s_cnt[1][warp] = nU;
        s_last[0][warp] = run[0];
        s_last[1][warp] = run[1];
    }
    __syncthreads();
    // ---- links across warps and to the sentinels (lane 0 of each warp) ----
    int baseA = 0, baseU = 0, carry[2] = {-1, -1};
    for (int w = 0; w < warp; ++w) {
        baseA += s_cnt[0][w];
        baseU += s_cnt[1][w];
#pragma unroll
        for (int l = 0; l < 2; ++l)
            if (s_last[l][w] >= 0) carry[l] = s_last[l][w];
    }
    if (lane == 0) {
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const uint32_t sent = l == 0 ? SA : SB;
            if (first[l] >= 0) {                         // this warp's first kept node
                const uint32_t pr = carry[l] >= 0 ? (uint32_t)carry[l] : sent;
                NX[2 * first[l] + 1] = pr;
                NX[2 * pr] = (uint32_t)first[l];
            }
            if (warp == kW - 1) {                         // the list's last node, the sentinel's prev
                int lastAll = carry[l];
                if (run[l] >= 0) lastAll = run[l];
                if (lastAll >= 0) NX[2 * lastAll] = sent;
                NX[2 * sent + 1] = lastAll >= 0 ? (uint32_t)lastAll : sent;
                if (lastAll < 0) NX[2 * sent] = sent;
            }
        }
    }
    // ---- the window's element of rank h: the warp holding it rescans ------
    if (baseU <= h && h < baseU + nU) {                 // warp-uniform
        int j = 0;
        const int nck = (c1 - c0 + kCk - 1) / kCk;
        while (j + 1 < nck && s_ck[warp][j + 1].y <= h - baseU) ++j;
        const int4 ck = s_ck[warp][j];
        int cA = ck.x, cU = ck.y, rl[2] = {ck.z, ck.w};
        bool found = false;
        for (int c = c0 + j * kCk; c < c1 && !found; ++c) {
            const int r = (c << 5) + lane;
            const uint32_t id = r < tot ? __ldg(M + r) : kNone;
            const uint32_t kb0 = __ballot_sync(kFull, kept(id, 0)), kb1 = __ballot_sync(kFull, kept(id, 1));
            const uint32_t u = kb0 | kb1;
            const int cu = __popc(u);
            if (h - baseU < cU + cu) {                    // warp-uniform: T is in this chunk
                if (((u >> lane) & 1u) && __popc(u & below) == h - baseU - cU) {
                    s_res[0] = baseA + cA + __popc(kb0 & below);   // s_A: kept A ranks below T
                    const uint32_t m0 = kb0 & below, m1 = kb1 & below;
                    const int pA = m0 ? (c << 5) + 31 - __clz(m0) : rl[0];
                    const int pB = m1 ? (c << 5) + 31 - __clz(m1) : rl[1];
                    s_res[1] = pA >= 0 ? pA : carry[0];             // last kept A rank below T
                    s_res[2] = pB >= 0 ? pB : carry[1];
                }
                found = true;
            }
            if (kb0) rl[0] = (c << 5) + 31 - __clz(kb0);
            if (kb1) rl[1] = (c << 5) + 31 - __clz(kb1);
            cA += __popc(kb0);
            cU += cu;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // m_A / m_B: the first kept node of each list at or above T, i.e. the
        // next of the last kept node below T (or the sentinel's next)
        const volatile uint32_t* vx = NX;
        const int sA = s_res[0], pA = s_res[1], pB = s_res[2];
        const uint32_t fa = vx[2 * (pA >= 0 ? (uint32_t)pA : SA)];
        const uint32_t fb = vx[2 * (pB >= 0 ? (uint32_t)pB : SB)];
        p.seg[sid] = make_int4((int)fa, (int)fb, sA, h - sA);
    }
}

__device__ __forceinline__ void prefetch_l2(const void* ptr)
{
    asm volatile("prefetch.global.L2 [%0];" :: "l"(ptr));
}

// Section 6.2, steps i0 .. i1-1 of pair q: delete(A, i), undelete(B, i),
// advance if s_A + s_B < h, print min(peek A, peek B).  Node numbers are
// joint ranks, so "is small" and the peek comparison compare node numbers;
// the sentinels 2k (A) and 2k+1 (B) rank above every element.
// The thread keeps m_A and m_B with their nodes (next, prev) in registers.
// Every node a step can move an m pointer to is m or one of its neighbours
// at the start of the step, or the relinked node b itself (Section 5.3:
// delete moves m to prev(m), or to next(m) when m itself goes; undelete
// moves m to prev(m), which is b when b is relinked just before m; advance
// moves m to next(m)).  So a step first stores its unlink and relink
// (equations del / undo-del of Section 4), then loads the nodes of m_A, m_B
// and their four neighbours, and the node the next step deletes: the loads
// see the new links, their addresses depend only on the state at the start
// of the step, and they form a single level of independent loads.
__global__ void __launch_bounds__(32)
large_chain(LargeTable tab, int64_t items)
{
    constexpr int kAhead = 8;                      // L2 prefetch distance in steps
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= items) return;
    int64_t sid;
    const LargeParams p = find_large(tab, kLChain, g, &sid);
    const int64_t q = sid / p.S;
    const int s = (int)(sid - q * p.S);
    const int NB = block_len(p, q + 1);
    const int i0 = s * p.L;
    if (i0 >= NB) return;
    const int i1 = min(i0 + p.L, NB);
    uint2* Lq = p.lists + sid * p.LN;
    uint32_t* NXp = reinterpret_cast<uint32_t*>(Lq);       // next of node r at [2r], prev at [2r+1]
    const uint32_t* JA = p.ja + q * p.kp;
    const uint32_t* JB = p.jb + q * p.kp;
    const uint2* UL = p.ulink + (q + 1) * p.kp;
    uint32_t* OUT = p.out + q * p.kp;
    const int4 st = p.seg[sid];
#ifdef MF_DEBUG
    const uint32_t nmax = 2u * (uint32_t)p.k + 1u;          // sentinel B, the largest node
    auto node = [&](uint32_t r, uint32_t site) { return MF_CHECK(r <= nmax, site, r) ? r : nmax; };
#else
    auto node = [](uint32_t r, uint32_t) { return r; };
#endif
    uint32_t mA = node((uint32_t)st.x, 301), mB = node((uint32_t)st.y, 301);
    int sA = st.z;                                 // s_B = h - s_A at every step boundary
    for (int t = i0; t < min(i0 + kAhead, i1); ++t) prefetch_l2(Lq + __ldg(JA + t));
    uint2 wmA = Lq[mA], wmB = Lq[mB];
    uint32_t a = node(__ldg(JA + i0), 301);
    uint2 La = Lq[a];
    for (int i = i0; i < i1; ++i) {
        const uint32_t b = node(__ldg(JB + i), 301);
        const uint2 u = __ldg(UL + i);
        const uint32_t pb = node(u.x, 301), nb = node(u.y, 301);   // b's unwind links
        const uint32_t an = i + 1 < i1 ? node(__ldg(JA + i + 1), 301) : a;
        if (i + kAhead < i1) prefetch_l2(Lq + __ldg(JA + i + kAhead));
        const uint32_t pm = node(wmA.y, 301), nm = node(wmA.x, 301);
        const uint32_t pmB = node(wmB.y, 301), nmB = node(wmB.x, 301);
        // -------- relinks: delete(A, i) unlinks a, undelete(B, i) relinks b ----
        const uint32_t na = node(La.x, 301), pa = node(La.y, 301);
        NXp[2 * pa] = na;                                   // next[prev[a]] <- next[a]
        NXp[2 * na + 1] = pa;                               // prev[next[a]] <- prev[a]
        const uint2 wb = make_uint2(nb, pb);
        Lq[b] = wb;
        NXp[2 * pb] = b;                                    // next[prev[b]] <- b
        NXp[2 * nb + 1] = b;                                // prev[next[b]] <- b
        // -------- the candidates' nodes, after the relinks ------------------------
        const uint2 wA0 = Lq[mA], wpm = Lq[pm], wnm = Lq[nm];
        const uint2 wB0 = Lq[mB], wpmB = Lq[pmB], wnmB = Lq[nmB];
        const uint2 Lan = Lq[an];
        // -------- delete(A, i): the m pointer and s -------------------------------
        const bool small = a < mA;
        const bool isM = a == mA;
        const bool sApos = sA > 0;
        const bool toP = !small && sApos, toN = !small && !sApos && isM;
        const uint32_t mA1 = toP ? pm : (toN ? nm : mA);
        const uint2 wA1 = toP ? wpm : (toN ? wnm : wA0);
        sA -= (small || sApos) ? 1 : 0;                     // s <- max(0, s - 1)
        const bool nxtOld = toP && !isM;                    // next of prev(m) is m itself
        const uint32_t aNode = nxtOld ? mA : nm;
        const uint2 aWord = nxtOld ? wA0 : wnm;
        // -------- undelete(B, i): the m pointer -------------------------------------
        const bool smallB = b < mB;                         // small: m <- prev[m]
        const bool justB = nb == mB;                        // b relinked just before m
        const uint32_t mB1 = smallB ? (justB ? b : pmB) : mB;
        const uint2 wB1 = smallB ? (justB ? wb : wpmB) : wB0;
        const bool afterB = pb == mB;                       // b relinked just after m
        const uint32_t bNode = smallB ? mB : (afterB ? b : nmB);
        const uint2 bWord = smallB ? wB0 : (afterB ? wb : wnmB);
        // -------- advance the list whose first large element is smaller -------------
        const bool aA = mA1 < mB1;
        const bool advA = sApos && aA, advB = sApos && !aA;
        mA = advA ? aNode : mA1;
        wmA = advA ? aWord : wA1;
        mB = advB ? bNode : mB1;
        wmB = advB ? bWord : wB1;
        sA += advA ? 1 : 0;
        // Section 6.3: 0 <= s_A <= h after every step; the median is an element
        (void)MF_CHECK(sA >= 0 && sA <= p.h, 302, sA);
        (void)MF_CHECK((mA < mB ? mA : mB) < 2u * (uint32_t)p.k, 303, mA < mB ? mA : mB);
        OUT[i] = mA < mB ? mA : mB;                        // joint rank of the median
        a = an;
        La = Lan;
    }
}

template <typename ValT>
__global__ void __launch_bounds__(256)
large_epilogue(LargeTable tab, int64_t items)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= items) return;
    int64_t o;
    const LargeParams p = find_large(tab, kLEpi, g, &o);
    const uint32_t* __restrict__ vs = p.vsort;
    int64_t src;
    if (o == 0) {
        src = vs[p.h];                           // y[0] = X_0[P_0[h]]
    } else {
        const int64_t q = (o - 1) / p.k, i = (o - 1) - q * p.k;
        const uint32_t r = p.out[q * p.kp + i];                 // joint rank in pair q
        const uint32_t id = __ldg(p.M + q * 2 * p.kp + r);
        src = (q + (id >> 31)) * (int64_t)p.k + (id & ~kBFlag);
    }
    if (!MF_CHECK(src >= 0 && src < p.n, 304, src)) src = 0;
    reinterpret_cast<ValT*>(p.y)[o] = __ldg(reinterpret_cast<const ValT*>(p.x) + src);
    if (p.argmed) p.argmed[o] = (int32_t)src;
}

// ---------------------------------------------------------------------------
static inline uint64_t a256(uint64_t v) { return (v + 255) & ~uint64_t(255); }

struct LargeShape {
    int64_t nblocks, npairs, kp, LN;
    int S, L;
};

static LargeShape large_shape(int64_t n, int k)
{
    LargeShape s;
    s.nblocks = (n + k - 1) / k;
    s.npairs = s.nblocks - 1;
    s.kp = ((int64_t)k + 31) & ~int64_t(31);
    s.LN = (2 * (int64_t)k + 2 + 31) & ~int64_t(31);
    int S = (k + kLargeSegSteps - 1) / kLargeSegSteps;
    S = S < 1 ? 1 : (S > kLargeMaxSegs ? kLargeMaxSegs : S);
    s.S = S;
    s.L = (k + S - 1) / S;
    return s;
}

// shared memory of the unwind and segment-init CTAs
static size_t unwind_smem(int k, int* nw, int* ns)
{
    *nw = (k + 31) / 32;
    *ns = (*nw + 31) / 32;
    // pp (8 B), rr, srt, lrk (4 B each) per run position; 32 x 32 local
    // bitset words; 256 scan counts; W, R, Rc (nw each) and W1 (ns)
    return 20ull * kUnwindRun + 4ull * (32 * 32 + 256) + 4ull * (3 * (size_t)*nw + *ns);
}

size_t large_workspace_bytes(int64_t n, int k, bool wide)
{
    const LargeShape s = large_shape(n, k);
    const uint64_t nb = (uint64_t)s.nblocks, kp = (uint64_t)s.kp;
    const uint64_t np1 = (uint64_t)(s.npairs > 0 ? s.npairs : 1);
    const uint64_t kb = wide ? 8 : 4;
    uint64_t b = a256(kb * nb * kp) * 2;                     // keyA keyB
    b += a256(4ull * nb * kp) * 3;                           // valA valB rnk
    b += a256(8ull * nb * kp);                               // ulink
    b += a256(4ull * np1 * kp) * 3;                          // ja jb out
    b += a256(8ull * np1 * kp);                              // M
    b += a256(16ull * np1 * s.S);                            // seg
    b += a256(4ull * np1 * kp);                              // jrs
    b += a256(8ull * np1 * s.S * (uint64_t)s.LN);            // lists
    return (size_t)b;
}

cudaError_t large_setup()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(large_chunk_sort<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(8 * chunk_warp_bytes<uint32_t>())))) return e;
    if ((e = cudaFuncSetAttribute(large_chunk_sort<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(8 * chunk_warp_bytes<uint64_t>())))) return e;
    return cudaFuncSetAttribute(large_unwind, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kMaxSmemBytes);
}

// The launch sequence of one call, for every signal of `tab`: chunk sort,
// ntier merge tiers, ranks, joint ranks, unwind, segment states, chains,
// store.  tot[kind] = items of each launch over all signals; the shared
// memory of the unwind and segment-state CTAs is sized for the largest k.
// KeyT = uint32_t or uint64_t (key and element width).
template <typename KeyT>
static cudaError_t run_large(const LargeTable& tab, const int64_t* tot, int ntier, int kmax,
                             cudaStream_t stream, LaunchStats* stats)
{
    auto launched = [&]() -> cudaError_t {
        if (stats) stats->launches += 1;
        return cudaGetLastError();
    };
    // per-call timing marks, as in the pipeline: [sort + joint ranks, unwind,
    // segment states + chains, store]
    cudaEvent_t* evs = nullptr;
    if (stats && stats->timing) {
        evs = stats->ev[stats->ring_pos % LaunchStats::kRing];
        stats->ring_pos += 1;
    }
    auto mark = [&](int idx) { if (evs) cudaEventRecord(evs[idx], stream); };
    auto grid = [](int64_t items, int per) { return (unsigned)((items + per - 1) / per); };
    int unw, uns;
    const size_t usmem = unwind_smem(kmax, &unw, &uns);
    cudaError_t e;
    mark(0);
    // phase 1: chunks, then merge tiers (ping-pong between the A and B buffers)
    large_chunk_sort<KeyT><<<grid(tot[kLChunk], 8), 256, 8 * chunk_warp_bytes<KeyT>(), stream>>>(tab, tot[kLChunk]);
    if ((e = launched()) != cudaSuccess) return e;
    for (int t = 0; t < ntier; ++t) {
        large_merge<KeyT><<<grid(tot[kLMerge0 + t], 256), 256, 0, stream>>>(tab, t, tot[kLMerge0 + t]);
        if ((e = launched()) != cudaSuccess) return e;
    }
    if (tot[kLChain] > 0) {
        // phase 2: ranks, joint ranks, unwind links, segment states, chains
        large_ranks<<<grid(tot[kLRanks], 256), 256, 0, stream>>>(tab, tot[kLRanks]);
        if ((e = launched()) != cudaSuccess) return e;
        large_jrank<KeyT><<<grid(tot[kLJrank], 256), 256, 0, stream>>>(tab, tot[kLJrank]);
        if ((e = launched()) != cudaSuccess) return e;
        mark(1);
        large_unwind<<<(unsigned)tot[kLUnwind], 256, usmem, stream>>>(tab);
        if ((e = launched()) != cudaSuccess) return e;
        mark(2);
        large_seginit<<<(unsigned)tot[kLSeg], 256, 0, stream>>>(tab);
        if ((e = launched()) != cudaSuccess) return e;
        // chains per CTA: the fewest (a power of two up to 32) that keep the
        // CTAs within 24 per SM.  A chain's node accesses do not coalesce with
        // other chains', so spreading them over every SM and over more warps
        // spreads their L1 traffic (GB300, n = 10^7: k = 100,001, 3,168
        // chains, 4.49 ms with 32 per CTA, 3.99 ms with one; k = 20,001,
        // 9,980 chains, best with 4 per CTA)
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int cpc = 1;
        while (cpc < 32 && (tot[kLChain] + cpc - 1) / cpc > 24ll * sms) cpc <<= 1;
        large_chain<<<grid(tot[kLChain], cpc), cpc, 0, stream>>>(tab, tot[kLChain]);
        if ((e = launched()) != cudaSuccess) return e;
    } else {
        mark(1);
        mark(2);
    }
    mark(3);
    large_epilogue<KeyT><<<grid(tot[kLEpi], 256), 256, 0, stream>>>(tab, tot[kLEpi]);
    if ((e = launched()) != cudaSuccess) return e;
    mark(4);
    return cudaSuccess;
}

// Descriptor of one signal carved from `w` (advanced past its workspace);
// its items are appended to the running totals tot[].
static bool large_prepare(LargeParams& p, const void* x, int64_t n, int k, int rank, Elem el,
                          void* y, int32_t* argmed, char*& w, int64_t* tot)
{
    if (k < 1 || k > kLargeMaxK || n < k || rank < 0 || rank >= k) return false;
    int unw, uns;
    if (unwind_smem(k, &unw, &uns) > (size_t)kMaxSmemBytes) return false;
    const LargeShape sh = large_shape(n, k);
    p = LargeParams{};
    p.x = x; p.y = y; p.argmed = argmed;
    p.n = n; p.k = k; p.h = rank;
    p.nblocks = sh.nblocks; p.npairs = sh.npairs; p.kp = sh.kp;
    p.is_float = el.is_float;
    p.S = sh.S; p.L = sh.L; p.LN = sh.LN;
    const uint64_t nb = (uint64_t)sh.nblocks, kp = (uint64_t)sh.kp;
    const uint64_t np1 = (uint64_t)(sh.npairs > 0 ? sh.npairs : 1);
    const uint64_t kb = (uint64_t)el.bytes();
    char* const w0 = w;
    p.keyA = w;            w += a256(kb * nb * kp);
    p.keyB = w;            w += a256(kb * nb * kp);
    p.valA = (uint32_t*)w; w += a256(4ull * nb * kp);
    p.valB = (uint32_t*)w; w += a256(4ull * nb * kp);
    p.rnk = (uint32_t*)w;  w += a256(4ull * nb * kp);
    p.ulink = (uint2*)w;   w += a256(8ull * nb * kp);
    p.ja = (uint32_t*)w;   w += a256(4ull * np1 * kp);
    p.jb = (uint32_t*)w;   w += a256(4ull * np1 * kp);
    p.jrs = (uint32_t*)w;  w += a256(4ull * np1 * kp);
    p.out = (uint32_t*)w;  w += a256(4ull * np1 * kp);
    p.M = (uint32_t*)w;    w += a256(8ull * np1 * kp);
    p.seg = (int4*)w;      w += a256(16ull * np1 * sh.S);
    p.lists = (uint2*)w;
    w = w0 + large_workspace_bytes(n, k, el.wide);
    p.cpb = (k + kChunk - 1) / kChunk;
    p.ntier = 0;
    while ((kChunk << p.ntier) < k) ++p.ntier;
    if (p.ntier > kLMaxTiers) return false;
    p.ksort = p.ntier & 1 ? p.keyB : p.keyA;
    p.vsort = p.ntier & 1 ? p.valB : p.valA;
    int64_t cnt[15] = {0};
    cnt[kLChunk] = sh.nblocks * p.cpb;
    for (int t = 0; t < p.ntier; ++t) cnt[kLMerge0 + t] = sh.nblocks * (sh.kp / kMergeOut);
    if (sh.npairs > 0) {
        cnt[kLRanks] = sh.nblocks * sh.kp;
        cnt[kLJrank] = sh.npairs * 2 * sh.kp / kJrankRun;
        cnt[kLUnwind] = (sh.nblocks - 1) *
                        (((k + kUnwindRun - 1) / kUnwindRun + kUnwindRunsPerCta - 1) / kUnwindRunsPerCta);
        cnt[kLSeg] = sh.npairs * sh.S;
        cnt[kLChain] = sh.npairs * sh.S;
    }
    cnt[kLEpi] = n - k + 1;
    for (int i = 0; i < 15; ++i) { p.start[i] = tot[i]; tot[i] += cnt[i]; }
    return true;
}

cudaError_t launch_large(const void* x, int64_t n, int k, int rank, Elem el, void* y,
                         int32_t* argmed, void* ws, size_t ws_bytes, cudaStream_t stream,
                         LaunchStats* stats)
{
    if (k < 1 || k > kLargeMaxK || n < k) return cudaErrorInvalidValue;
    if (ws_bytes < large_workspace_bytes(n, k, el.wide)) return cudaErrorInvalidValue;
    LargeTable tab{};
    tab.segs = nullptr;
    tab.nseg = 1;
    int64_t tot[15] = {0};
    char* w = (char*)ws;
    if (!large_prepare(tab.one, x, n, k, rank, el, y, argmed, w, tot)) return cudaErrorInvalidValue;
    if (el.wide) return run_large<uint64_t>(tab, tot, tab.one.ntier, k, stream, stats);
    return run_large<uint32_t>(tab, tot, tab.one.ntier, k, stream, stats);
}

size_t large_batched_workspace_bytes(const int64_t* n, const int32_t* k, int nseg, bool wide)
{
    uint64_t b = a256((uint64_t)nseg * sizeof(LargeParams));
    for (int s = 0; s < nseg; ++s) b += large_workspace_bytes(n[s], k[s], wide);
    return (size_t)b;
}

size_t large_descriptor_bytes() { return sizeof(LargeParams); }

cudaError_t launch_large_batched(const void* x, void* y, int32_t* argmed, Elem el,
                                 const int64_t* x_off, const int64_t* n, const int64_t* y_off,
                                 const int32_t* k, int nseg, void* ws, size_t ws_bytes,
                                 void* stage, size_t stage_bytes, cudaStream_t stream,
                                 LaunchStats* stats)
{
    if (nseg <= 0) return cudaSuccess;
    if (ws_bytes < large_batched_workspace_bytes(n, k, nseg, el.wide)) return cudaErrorInvalidValue;
    if (stage_bytes < (size_t)nseg * sizeof(LargeParams)) return cudaErrorInvalidValue;
    LargeParams* host = (LargeParams*)stage;
    LargeParams* dev = (LargeParams*)ws;
    char* w = (char*)ws + a256((uint64_t)nseg * sizeof(LargeParams));
    int64_t tot[15] = {0};
    int ntier = 0, kmax = 1;
    const int eb = el.bytes();
    for (int s = 0; s < nseg; ++s) {
        if (!large_prepare(host[s], (const char*)x + x_off[s] * eb, n[s], k[s], (k[s] - 1) / 2, el,
                           (char*)y + y_off[s] * eb, argmed ? argmed + y_off[s] : nullptr, w, tot))
            return cudaErrorInvalidValue;
        ntier = max(ntier, host[s].ntier);
        kmax = max(kmax, k[s]);
    }
    cudaError_t e = cudaMemcpyAsync(dev, host, (size_t)nseg * sizeof(LargeParams),
                                    cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return e;
    LargeTable tab{};
    tab.segs = dev;
    tab.nseg = nseg;
    if (el.wide) return run_large<uint64_t>(tab, tot, ntier, kmax, stream, stats);
    return run_large<uint32_t>(tab, tot, ntier, kmax, stream, stats);
}

MF_DEBUG_TAKE_FN(large)

}  // namespace mf

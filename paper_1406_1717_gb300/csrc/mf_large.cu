// mf_large.cu -- the median filter for window sizes too large for the
// shared-memory pipeline (pipeline_max_k() < k <= kLargeMaxK).
//
// Paper: "Median Filtering is Equivalent to Sorting" (Suomela).  The method
// of mf_pipeline.cu (comparisons by joint rank in A u B, A first on ties)
// with 32-bit indices and the data in global memory:
//
//   large_chunk_sort  a warp sorts each 1024-element chunk of a block in
//                     shared memory (stable LSD radix, Section 6.1)
//   large_merge       global merge-path tiers: sorted runs of R -> 2R until a
//                     run covers the block, left run first on equal keys
//   large_ranks       rank of each position in its block
//   large_jrank       joint ranks of each pair by binary search in the other
//                     block: ja / jb by position, jrs by B's sorted order and
//                     M = the merged order
//   large_unwind      unwind(B)'s links (Section 4: after unwind, undelete(B, i)
//                     relinks i between its nearest smaller and larger
//                     elements among positions < i); one CTA per run of
//                     positions, seeded with a rank bitset of the positions
//                     before the run
//   large_seginit     rebuilds the lists before step i0 of a pair (Section 6.3
//                     invariant: S_A u S_B are the h smallest of the window)
//                     from bitsets of the window's joint ranks
//   large_chain       the steps i0 .. i1-1 of Section 6.2 from that state,
//                     one thread per (pair, segment), lists in global memory
//   large_epilogue    node -> input element, y / argmed
//
// Nodes are numbered by joint rank: the element of joint rank r is node r,
// A's sentinel is 2k and B's 2k+1.  A node's number is its rank, so "is
// small" and peek(A) <= peek(B) compare node numbers, and list neighbours are
// rank neighbours: the walks of the two m pointers stay within a few cache
// lines, and the only random load of a step (the deleted node, known in
// advance) is prefetched.
// The serial depth of one pair is k steps; splitting the k steps of a pair
// into S independent segments, each starting from a state rebuilt with O(k)
// parallel work, cuts the depth to k / S at the price of S private copies of
// the pair's links (8 bytes per node, 2k + 2 nodes).
#include <cuda_runtime.h>
#include <cstdint>
#include "mf_device.cuh"
#include "mf_internal.h"

namespace mf {

constexpr int kChunk = 1024;                     // elements per warp sort
constexpr int kUnwindRun = 1024;                 // positions per unwind CTA
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
};

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
template <typename KeyT>
__host__ __device__ constexpr size_t chunk_warp_bytes() { return (size_t)kChunk * (2 * sizeof(KeyT) + 4) + 1024; }

template <typename KeyT>
__global__ void __launch_bounds__(256)
large_chunk_sort(LargeParams p, int chunks_per_block)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t id = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (id >= p.nblocks * chunks_per_block) return;
    const int64_t b = id / chunks_per_block;
    const int c = (int)(id - b * chunks_per_block);
    const int NB = block_len(p, b);
    const int lo = c * kChunk;
    const int cnt = min(kChunk, NB - lo);
    if (cnt <= 0) return;
    unsigned char* ws = smem + (size_t)warp * chunk_warp_bytes<KeyT>();
    KeyT* ka = reinterpret_cast<KeyT*>(ws);
    KeyT* kb = ka + kChunk;
    uint16_t* va = reinterpret_cast<uint16_t*>(kb + kChunk);
    uint16_t* vb = va + kChunk;
    uint32_t* hist = reinterpret_cast<uint32_t*>(vb + kChunk);
    const KeyT* xs = reinterpret_cast<const KeyT*>(p.x) + b * (int64_t)p.k + lo;
    for (int t = lane; t < cnt; t += 32) { ka[t] = to_key(__ldg(xs + t), p.is_float); va[t] = (uint16_t)t; }
    __syncwarp();
    warp_sort_group<KeyT>(ka, va, kb, vb, cnt, 0, kChunk, 1, hist);
    const int64_t o = b * p.kp + lo;
    KeyT* keys = reinterpret_cast<KeyT*>(p.keyA);
    for (int t = lane; t < cnt; t += 32) { keys[o + t] = ka[t]; p.valA[o + t] = (uint32_t)lo + va[t]; }
}

// sorted runs [l0, l0+R) and [l0+R, l0+2R) of every block -> one run; each
// thread writes 4 consecutive outputs after a merge-path search
template <typename KeyT>
__global__ void __launch_bounds__(256)
large_merge(LargeParams p, const KeyT* __restrict__ kin, const uint32_t* __restrict__ vin,
            KeyT* __restrict__ kout, uint32_t* __restrict__ vout, int R, int per_block)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b = gid / per_block;
    if (b >= p.nblocks) return;
    const int o = (int)(gid - b * per_block) * 4;
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
    const int oend = min(o + 4, NB);
    for (int q = o; q < oend; ++q) {
        const bool takeL = ib >= lenR || (ia < lenL && KL[ia] <= KR[ib]);
        if (takeL) { kout[base + q] = KL[ia]; vout[base + q] = vin[base + l0 + ia]; ++ia; }
        else       { kout[base + q] = KR[ib]; vout[base + q] = vin[base + r0 + ib]; ++ib; }
    }
}

__global__ void __launch_bounds__(256)
large_ranks(LargeParams p, const uint32_t* __restrict__ vs)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b = gid / p.kp;
    if (b >= p.nblocks) return;
    const int t = (int)(gid - b * p.kp);
    if (t >= block_len(p, b)) return;
    p.rnk[b * p.kp + vs[b * p.kp + t]] = (uint32_t)t;
}

// joint rank of every element of pair q (A = block q, B = block q+1):
// A's t-th smallest -> t + #{B keys < key}; B's u-th -> u + #{A keys <= key}
template <typename KeyT>
__global__ void __launch_bounds__(256)
large_jrank(LargeParams p, const KeyT* __restrict__ ks, const uint32_t* __restrict__ vs)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per_pair = 2 * p.kp;
    const int64_t q = gid / per_pair;
    if (q >= p.npairs) return;
    const int e = (int)(gid - q * per_pair);
    const int NA = p.k, NB = block_len(p, q + 1);
    const int64_t abase = q * p.kp, bbase = (q + 1) * p.kp;
    uint32_t* M = p.M + q * per_pair;
    if (e < NA) {
        const KeyT key = ks[abase + e];
        int lo = 0, hi = NB;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (ks[bbase + mid] < key) lo = mid + 1; else hi = mid; }
        const uint32_t pos = vs[abase + e];
        M[e + lo] = pos;
        p.ja[q * p.kp + pos] = (uint32_t)(e + lo);
    } else if (e >= (int)p.kp && e - (int)p.kp < NB) {
        const int u = e - (int)p.kp;
        const KeyT key = ks[bbase + u];
        int lo = 0, hi = NA;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (ks[abase + mid] <= key) lo = mid + 1; else hi = mid; }
        const uint32_t pos = vs[bbase + u];
        M[u + lo] = kBFlag | pos;
        p.jb[q * p.kp + pos] = (uint32_t)(u + lo);
        p.jrs[q * p.kp + u] = (uint32_t)(u + lo);
    }
}

// Unwind links of block b >= 1 (blockIdx.x = b - 1), positions
// [i0, i0 + kUnwindRun) (blockIdx.y = run).  The bitset of the ranks of all
// positions < i0 is built from the sorted order; then one thread inserts the
// run's ranks in position order, recording for each its nearest set ranks
// below and above; the CTA turns those ranks into nodes.
__global__ void __launch_bounds__(256)
large_unwind(LargeParams p, const uint32_t* __restrict__ vs, int nw, int ns)
{
    extern __shared__ __align__(16) uint32_t sw[];
    const int64_t b = 1 + (int64_t)blockIdx.x;
    const int NB = block_len(p, b);
    const int i0 = blockIdx.y * kUnwindRun;
    if (i0 >= NB) return;
    const int len = min(kUnwindRun, NB - i0);
    int2* pp = reinterpret_cast<int2*>(sw);       // kUnwindRun (pred, succ) ranks
    uint32_t* rr = sw + 2 * kUnwindRun;            // kUnwindRun ranks of the run
    uint32_t* W = rr + kUnwindRun;                 // nw words
    uint32_t* W1 = W + nw;                         // ns words
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int64_t base = b * p.kp;
    for (int w = warp; w < nw; w += nwarp) {
        const int r = (w << 5) + lane;
        const bool set = r < NB && (int)__ldg(vs + base + r) < i0;
        const uint32_t word = __ballot_sync(kFull, set);
        if (lane == 0) W[w] = word;
    }
    for (int t = threadIdx.x; t < len; t += blockDim.x) rr[t] = __ldg(p.rnk + base + i0 + t);
    __syncthreads();
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        uint32_t sm = 0;
        for (int c = 0; c < 32 && (s << 5) + c < nw; ++c)
            if (W[(s << 5) + c]) sm |= 1u << c;
        W1[s] = sm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 0; t < len; ++t) {
            const int r = (int)rr[t];
            pp[t] = make_int2(bits_last_before(W, W1, nw, r), bits_first_from(W, W1, nw, ns, r + 1));
            W[r >> 5] |= 1u << (r & 31);
            W1[r >> 10] |= 1u << ((r >> 5) & 31);
        }
    }
    __syncthreads();
    // block ranks -> rank nodes of pair b-1 (B's t-th smallest is node jrs[t])
    const uint32_t sentB = 2u * (uint32_t)p.k + 1u;
    const uint32_t* jrs = p.jrs + (b - 1) * p.kp;
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
        const int2 q = pp[t];
        const uint32_t pv = q.x >= 0 ? __ldg(jrs + q.x) : sentB;
        const uint32_t nx = q.y >= 0 ? __ldg(jrs + q.y) : sentB;
        p.ulink[base + i0 + t] = make_uint2(pv, nx);
    }
}

// One CTA per (pair q, segment s), i0 = s * L: the lists before step i0.
// The window is A's positions >= i0 and B's positions < i0.  KA / KB mark
// the joint ranks of its A and B elements; a node's list neighbours are the
// nearest marked ranks of its own block, and the small elements are the
// window's h smallest (Section 6.3 invariant), found by a prefix count.
__global__ void __launch_bounds__(256)
large_seginit(LargeParams p, int nw, int ns)
{
    extern __shared__ __align__(16) uint32_t sw[];
    const int64_t sid = blockIdx.x;
    const int64_t q = sid / p.S;
    const int s = (int)(sid - q * p.S);
    const int NB = block_len(p, q + 1);
    const int i0 = s * p.L;
    if (i0 >= NB) return;
    const int k = p.k, h = p.h, tot = k + NB;
    uint32_t* KA = sw;
    uint32_t* KB = KA + nw;
    uint32_t* KA1 = KB + nw;
    uint32_t* KB1 = KA1 + ns;
    int* scan = reinterpret_cast<int*>(KB1 + ns); // 2 * blockDim.x
    int* sh_state = scan + 2 * blockDim.x;        // T, s_A
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const uint32_t* M = p.M + q * 2 * p.kp;
    for (int w = warp; w < nw; w += nwarp) {
        const int r = (w << 5) + lane;
        const uint32_t id = r < tot ? __ldg(M + r) : 0u;
        const bool isB = (id & kBFlag) != 0;
        const uint32_t pos = id & ~kBFlag;
        const uint32_t a = __ballot_sync(kFull, r < tot && !isB && pos >= (uint32_t)i0);
        const uint32_t bb = __ballot_sync(kFull, r < tot && isB && pos < (uint32_t)i0);
        if (lane == 0) { KA[w] = a; KB[w] = bb; }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ns; t += blockDim.x) {
        uint32_t sa = 0, sb = 0;
        for (int c = 0; c < 32 && (t << 5) + c < nw; ++c) {
            if (KA[(t << 5) + c]) sa |= 1u << c;
            if (KB[(t << 5) + c]) sb |= 1u << c;
        }
        KA1[t] = sa;
        KB1[t] = sb;
    }
    // window rank h: thread t counts the marks of words [w0, w1)
    const int per = (nw + blockDim.x - 1) / blockDim.x;
    const int w0 = min(nw, (int)threadIdx.x * per), w1 = min(nw, w0 + per);
    int ca = 0, cb = 0;
    for (int w = w0; w < w1; ++w) { ca += __popc(KA[w]); cb += __popc(KB[w]); }
    scan[threadIdx.x] = ca + cb;
    scan[blockDim.x + threadIdx.x] = ca;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0, acca = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int c = scan[t], a = scan[blockDim.x + t];
            scan[t] = acc; scan[blockDim.x + t] = acca;
            acc += c; acca += a;
        }
    }
    __syncthreads();
    {
        int before = scan[threadIdx.x], beforeA = scan[blockDim.x + threadIdx.x];
        if (before <= h && h < before + ca + cb) {
            // the element of window rank h lies in this thread's words
            for (int w = w0; w < w1; ++w) {
                const uint32_t any = KA[w] | KB[w];
                const int c = __popc(any);
                if (before + c > h) {
                    uint32_t m = any;
                    for (int j = h - before; j > 0; --j) m &= m - 1;   // drop the lower ones
                    const int bit = __ffs(m) - 1;
                    const int T = (w << 5) + bit;
                    const int sA = beforeA + __popc(KA[w] & ((1u << bit) - 1u));
                    sh_state[0] = T;
                    sh_state[1] = sA;
                    break;
                }
                before += c;
                beforeA += __popc(KA[w]);
            }
        }
    }
    __syncthreads();
    // lists of the window in rank-node space: a kept node's neighbours are the
    // nearest kept ranks of its own block; sentinels SA = 2k, SB = 2k+1
    uint2* Lq = p.lists + sid * p.LN;
    const uint32_t SA = 2u * (uint32_t)k, SB = SA + 1u;
    if (threadIdx.x == 0) {
        const int T = sh_state[0], sA = sh_state[1];
        const int fa = bits_first_from(KA, KA1, nw, ns, T), fb = bits_first_from(KB, KB1, nw, ns, T);
        p.seg[sid] = make_int4(fa >= 0 ? fa : (int)SA, fb >= 0 ? fb : (int)SB, sA, h - sA);
        const int a0 = bits_first_from(KA, KA1, nw, ns, 0), a1 = bits_last_before(KA, KA1, nw, tot);
        const int b0 = bits_first_from(KB, KB1, nw, ns, 0), b1 = bits_last_before(KB, KB1, nw, tot);
        Lq[SA] = make_uint2(a0 >= 0 ? (uint32_t)a0 : SA, a1 >= 0 ? (uint32_t)a1 : SA);
        Lq[SB] = make_uint2(b0 >= 0 ? (uint32_t)b0 : SB, b1 >= 0 ? (uint32_t)b1 : SB);
    }
    for (int r = threadIdx.x; r < tot; r += blockDim.x) {
        const uint32_t bit = 1u << (r & 31);
        const bool inA = (KA[r >> 5] & bit) != 0, inB = (KB[r >> 5] & bit) != 0;
        if (!inA && !inB) continue;                  // not in the window: never read
        const uint32_t* W = inA ? KA : KB;
        const uint32_t* W1 = inA ? KA1 : KB1;
        const uint32_t sent = inA ? SA : SB;
        const int nx = bits_first_from(W, W1, nw, ns, r + 1);
        const int pv = bits_last_before(W, W1, nw, r);
        Lq[r] = make_uint2(nx >= 0 ? (uint32_t)nx : sent, pv >= 0 ? (uint32_t)pv : sent);
    }
}

__device__ __forceinline__ void prefetch_l2(const void* ptr)
{
    asm volatile("prefetch.global.L2 [%0];" :: "l"(ptr));
}

// Section 6.2, steps i0 .. i1-1 of pair q: delete(A, i), undelete(B, i),
// advance while s_A + s_B < h, print min(peek A, peek B).  Node numbers are
// joint ranks, so "is small" and the peek comparison compare node numbers;
// the sentinels 2k (A) and 2k+1 (B) rank above every element.
__global__ void __launch_bounds__(32)
large_chain(LargeParams p)
{
    constexpr int kAhead = 8;                      // prefetch distance in steps
    const int64_t sid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (sid >= p.npairs * p.S) return;
    const int64_t q = sid / p.S;
    const int s = (int)(sid - q * p.S);
    const int NB = block_len(p, q + 1);
    const int i0 = s * p.L;
    if (i0 >= NB) return;
    const int i1 = min(i0 + p.L, NB);
    const int h = p.h;
    uint2* Lq = p.lists + sid * p.LN;
    uint32_t* NXp = reinterpret_cast<uint32_t*>(Lq);       // next of node r at [2r], prev at [2r+1]
    const uint32_t* JA = p.ja + q * p.kp;
    const uint32_t* JB = p.jb + q * p.kp;
    const uint2* UL = p.ulink + (q + 1) * p.kp;
    uint32_t* OUT = p.out + q * p.kp;
    const int4 st = p.seg[sid];
    uint32_t mA = (uint32_t)st.x, mB = (uint32_t)st.y;
    int sA = st.z, sB = st.w;
    for (int t = i0; t < min(i0 + kAhead, i1); ++t) prefetch_l2(Lq + __ldg(JA + t));
    for (int i = i0; i < i1; ++i) {
        const uint32_t a = __ldg(JA + i), b = __ldg(JB + i);
        const uint2 u = __ldg(UL + i);
        if (i + kAhead < i1) prefetch_l2(Lq + __ldg(JA + i + kAhead));
        const uint2 La = Lq[a];
        const uint2 LmA = Lq[mA];
        const uint2 LmB = Lq[mB];
        // delete(A, i): unlink node a, then keep s_A and m consistent
        const uint32_t na = La.x, pa = La.y;
        NXp[2 * pa] = na;
        NXp[2 * na + 1] = pa;
        if (a < mA) {
            --sA;
        } else {
            uint32_t pvm = (mA == na) ? pa : LmA.y;        // prev of m after the unlink
            if (mA == a) { mA = na; pvm = pa; }
            if (sA > 0) { mA = pvm; --sA; }
        }
        // undelete(B, i): relink node b between its unwind links
        Lq[b] = make_uint2(u.y, u.x);
        NXp[2 * u.x] = b;
        NXp[2 * u.y + 1] = b;
        if (b < mB) mB = (mB == u.y) ? b : LmB.y;
        // advance the smaller peek while s_A + s_B < h
        if (sA + sB < h) {
            if (mA < mB) { mA = Lq[mA].x; ++sA; }
            else         { mB = Lq[mB].x; ++sB; }
        }
        OUT[i] = mA < mB ? mA : mB;                        // joint rank of the median
    }
}

template <typename ValT>
__global__ void __launch_bounds__(256)
large_epilogue(LargeParams p, const uint32_t* __restrict__ vs)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t m = p.n - p.k + 1;
    if (o >= m) return;
    int64_t src;
    if (o == 0) {
        src = vs[p.h];                           // y[0] = X_0[P_0[h]]
    } else {
        const int64_t q = (o - 1) / p.k, i = (o - 1) - q * p.k;
        const uint32_t r = p.out[q * p.kp + i];                 // joint rank in pair q
        const uint32_t id = __ldg(p.M + q * 2 * p.kp + r);
        src = (q + (id >> 31)) * (int64_t)p.k + (id & ~kBFlag);
    }
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
    return 4ull * (size_t)(*nw + *ns) + 12ull * kUnwindRun;
}
static size_t seginit_smem(int k, int* nw, int* ns)
{
    *nw = (2 * k + 31) / 32;
    *ns = (*nw + 31) / 32;
    return 8ull * (size_t)(*nw + *ns) + 2 * 4 * 256 + 16;
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
    if ((e = cudaFuncSetAttribute(large_unwind, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kMaxSmemBytes))) return e;
    return cudaFuncSetAttribute(large_seginit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kMaxSmemBytes);
}

// All launches of one call; KeyT = uint32_t or uint64_t (key and element width).
template <typename KeyT>
static cudaError_t run_large(LargeParams& p, const LargeShape& sh, size_t usmem, int unw, int uns,
                             size_t ssmem, int snw, int sns, cudaStream_t stream,
                             LaunchStats* stats)
{
    const int k = p.k;
    const uint64_t kp = (uint64_t)sh.kp;
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
    cudaError_t e;
    mark(0);
    // phase 1: chunks, then merge tiers (ping-pong between the A and B buffers)
    const int cpb = (k + kChunk - 1) / kChunk;
    const int64_t warps = sh.nblocks * cpb;
    large_chunk_sort<KeyT><<<(unsigned)((warps + 7) / 8), 256, 8 * chunk_warp_bytes<KeyT>(), stream>>>(p, cpb);
    if ((e = launched()) != cudaSuccess) return e;
    KeyT *ks = (KeyT*)p.keyA, *kt = (KeyT*)p.keyB;
    uint32_t *vs = p.valA, *vt = p.valB;
    const int per_block4 = (int)(kp / 4);
    for (int R = kChunk; R < k; R *= 2) {
        const int64_t threads = sh.nblocks * per_block4;
        large_merge<KeyT><<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(p, ks, vs, kt, vt, R, per_block4);
        if ((e = launched()) != cudaSuccess) return e;
        KeyT* t1 = ks; ks = kt; kt = t1;
        uint32_t* t2 = vs; vs = vt; vt = t2;
    }
    if (sh.npairs > 0) {
        // phase 2: ranks, joint ranks, unwind links, segment states, chains
        const int64_t tr = sh.nblocks * sh.kp;
        large_ranks<<<(unsigned)((tr + 255) / 256), 256, 0, stream>>>(p, vs);
        if ((e = launched()) != cudaSuccess) return e;
        const int64_t tj = sh.npairs * 2 * sh.kp;
        large_jrank<KeyT><<<(unsigned)((tj + 255) / 256), 256, 0, stream>>>(p, ks, vs);
        if ((e = launched()) != cudaSuccess) return e;
        mark(1);
        const dim3 ug((unsigned)(sh.nblocks - 1), (unsigned)((k + kUnwindRun - 1) / kUnwindRun));
        large_unwind<<<ug, 256, usmem, stream>>>(p, vs, unw, uns);
        if ((e = launched()) != cudaSuccess) return e;
        mark(2);
        const int64_t nseg = sh.npairs * sh.S;
        large_seginit<<<(unsigned)nseg, 256, ssmem, stream>>>(p, snw, sns);
        if ((e = launched()) != cudaSuccess) return e;
        large_chain<<<(unsigned)((nseg + 31) / 32), 32, 0, stream>>>(p);
        if ((e = launched()) != cudaSuccess) return e;
    } else {
        mark(1);
        mark(2);
    }
    mark(3);
    const int64_t m = p.n - k + 1;
    large_epilogue<KeyT><<<(unsigned)((m + 255) / 256), 256, 0, stream>>>(p, vs);
    if ((e = launched()) != cudaSuccess) return e;
    mark(4);
    return cudaSuccess;
}

cudaError_t launch_large(const void* x, int64_t n, int k, int rank, Elem el, void* y,
                         int32_t* argmed, void* ws, size_t ws_bytes, cudaStream_t stream,
                         LaunchStats* stats)
{
    if (k < 1 || k > kLargeMaxK || n < k || rank < 0 || rank >= k) return cudaErrorInvalidValue;
    if (ws_bytes < large_workspace_bytes(n, k, el.wide)) return cudaErrorInvalidValue;
    int unw, uns, snw, sns;
    const size_t usmem = unwind_smem(k, &unw, &uns);
    const size_t ssmem = seginit_smem(k, &snw, &sns);
    if (usmem > (size_t)kMaxSmemBytes || ssmem > (size_t)kMaxSmemBytes) return cudaErrorInvalidValue;
    const LargeShape sh = large_shape(n, k);
    LargeParams p{};
    p.x = x; p.y = y; p.argmed = argmed;
    p.n = n; p.k = k; p.h = rank;
    p.nblocks = sh.nblocks; p.npairs = sh.npairs; p.kp = sh.kp;
    p.is_float = el.is_float;
    p.S = sh.S; p.L = sh.L; p.LN = sh.LN;
    const uint64_t nb = (uint64_t)sh.nblocks, kp = (uint64_t)sh.kp;
    const uint64_t np1 = (uint64_t)(sh.npairs > 0 ? sh.npairs : 1);
    const uint64_t kb = (uint64_t)el.bytes();
    char* w = (char*)ws;
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
    if (el.wide) return run_large<uint64_t>(p, sh, usmem, unw, uns, ssmem, snw, sns, stream, stats);
    return run_large<uint32_t>(p, sh, usmem, unw, uns, ssmem, snw, sns, stream, stats);
}

}  // namespace mf

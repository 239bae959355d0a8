// mf_large.cu -- the median filter for window sizes too large for the
// shared-memory pipeline (pipeline_max_k() < k <= kLargeMaxK).
//
// Paper: "Median Filtering is Equivalent to Sorting" (Suomela).  Same method
// and node numbering as mf_pipeline.cu (slot i = A's position i until step i,
// then B's position i; sentinels k and k+1; comparisons by joint rank in
// A u B, A first on ties), with 32-bit indices and the data in global memory:
//
//   large_chunk_sort  a warp sorts each 1024-element chunk of a block in
//                     shared memory (stable LSD radix, Section 5.1)
//   large_merge       global merge-path tiers: sorted runs of R -> 2R until a
//                     run covers the block, left run first on equal keys
//   large_ranks       rank of each position in its block
//   large_jrank       joint ranks of each pair by binary search in the other
//                     block; M = the pair's merged order, jb = B's ranks
//   large_unwind      unwind(B)'s links (Section 4: after unwind, undelete(B, i)
//                     relinks i between its nearest smaller and larger
//                     elements among positions < i), by a rank bitset per run
//   large_seginit     rebuilds the state before step i0 of a pair (Section 5.3
//                     invariant: S_A u S_B are the h smallest of the window)
//   large_chain       the steps i0 .. i1-1 of Section 5.2 from that state,
//                     one thread per (pair, segment), lists in global memory
//   large_epilogue    node -> input element, y / argmed
//
// The serial depth of one pair is k steps; splitting the k steps of a pair
// into S independent segments, each starting from a state rebuilt with O(k)
// parallel work, cuts the depth to k / S at the price of S private copies of
// the pair's lists.
#include <cuda_runtime.h>
#include <cstdint>
#include "mf_device.cuh"
#include "mf_internal.h"

namespace mf {

constexpr int kChunk = 1024;                     // elements per warp sort
constexpr uint32_t kBFlag = 0x80000000u;          // node id of B's element
constexpr uint32_t kInf = 0xffffffffu;           // joint rank of the sentinels

struct LargeParams {
    const uint32_t* x;
    uint32_t* y;
    int32_t* argmed;
    int64_t n, nblocks, npairs;
    int k, h;
    int64_t kp;                                  // row stride (k rounded up to 32)
    bool is_float;
    int S, L;                                    // segments per pair, steps per segment
    int64_t LS;                                  // list stride: k + 2 rounded up to 32
    uint32_t *keyA, *valA, *keyB, *valB;         // [nblocks][kp] sort ping-pong
    uint32_t* rnk;                               // [nblocks][kp] rank of position p
    uint2* ulink;                                // [nblocks][kp] unwind (prev, next), sentinel k+1
    uint32_t* jb;                                // [npairs][kp] joint rank of B's position p
    uint32_t* M;                                 // [npairs][2 kp] node at joint rank r
    uint32_t* out;                               // [npairs][kp] printed node at step i
    int4* seg;                                   // [npairs][S] (mA, mB, sA, sB) before step i0
    uint32_t* lists;                             // [npairs][S][3][LS] next, prev, joint rank
};

__device__ __forceinline__ int block_len(const LargeParams& p, int64_t b) {
    const int64_t r = p.n - b * (int64_t)p.k;
    return (int)(r < p.k ? r : p.k);
}

// ---------------------------------------------------------------------------
constexpr size_t kChunkWarpBytes = (size_t)kChunk * 12 + 1024;

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
    unsigned char* ws = smem + (size_t)warp * kChunkWarpBytes;
    uint32_t* ka = reinterpret_cast<uint32_t*>(ws);
    uint32_t* kb = ka + kChunk;
    uint16_t* va = reinterpret_cast<uint16_t*>(kb + kChunk);
    uint16_t* vb = va + kChunk;
    uint32_t* hist = reinterpret_cast<uint32_t*>(vb + kChunk);
    const uint32_t* xs = p.x + b * (int64_t)p.k + lo;
    for (int t = lane; t < cnt; t += 32) { ka[t] = to_key(__ldg(xs + t), p.is_float); va[t] = (uint16_t)t; }
    __syncwarp();
    warp_sort_group(ka, va, kb, vb, cnt, 0, kChunk, 1, hist);
    const int64_t o = b * p.kp + lo;
    for (int t = lane; t < cnt; t += 32) { p.keyA[o + t] = ka[t]; p.valA[o + t] = (uint32_t)lo + va[t]; }
}

// sorted runs [l0, l0+R) and [l0+R, l0+2R) of every block -> one run; each
// thread writes 4 consecutive outputs after a merge-path search
__global__ void __launch_bounds__(256)
large_merge(LargeParams p, const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
            uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int R, int per_block)
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
    const uint32_t* KL = kin + base + l0;
    const uint32_t* KR = kin + base + r0;
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
__global__ void __launch_bounds__(256)
large_jrank(LargeParams p, const uint32_t* __restrict__ ks, const uint32_t* __restrict__ vs)
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
        const uint32_t key = ks[abase + e];
        int lo = 0, hi = NB;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (ks[bbase + mid] < key) lo = mid + 1; else hi = mid; }
        M[e + lo] = vs[abase + e];
    } else if (e >= (int)p.kp && e - (int)p.kp < NB) {
        const int u = e - (int)p.kp;
        const uint32_t key = ks[bbase + u];
        int lo = 0, hi = NA;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (ks[abase + mid] <= key) lo = mid + 1; else hi = mid; }
        const uint32_t pos = vs[bbase + u];
        M[u + lo] = kBFlag | pos;
        p.jb[q * p.kp + pos] = (uint32_t)(u + lo);
    }
}

// unwind links of block b >= 1, lane = run of positions [i0, i1): the run's
// bitset starts with the ranks of all positions < i0; for each position, the
// nearest set ranks below and above its own give (prev, next)
__global__ void __launch_bounds__(64)
large_unwind(LargeParams p, const uint32_t* __restrict__ vs, int seglen, int nw, int ns)
{
    extern __shared__ __align__(16) uint32_t sw[];
    const int lane = threadIdx.x, S = blockDim.x;
    const int64_t b = 1 + blockIdx.x;
    if (b >= p.nblocks) return;
    const int NB = block_len(p, b);
    const int i0 = lane * seglen, i1 = min(i0 + seglen, NB);
    if (i0 >= i1) return;
    uint32_t* W0 = sw + lane;                     // word x at W0[x * S]
    uint32_t* W1 = sw + (size_t)nw * S + lane;
    for (int w = 0; w < nw; ++w) W0[(size_t)w * S] = 0u;
    for (int s = 0; s < ns; ++s) W1[(size_t)s * S] = 0u;
    const int64_t base = b * p.kp;
    const uint32_t* rk = p.rnk + base;
    for (int i = 0; i < i0; ++i) {
        const uint32_t r = rk[i];
        W0[(size_t)(r >> 5) * S] |= 1u << (r & 31);
        W1[(size_t)(r >> 10) * S] |= 1u << ((r >> 5) & 31);
    }
    const uint32_t sentB = (uint32_t)p.k + 1;
    for (int i = i0; i < i1; ++i) {
        const int r = (int)rk[i];
        const int w = r >> 5, bb = r & 31;
        const uint32_t word = W0[(size_t)w * S];
        int pred = -1, succ = -1;
        const uint32_t mlo = word & ((1u << bb) - 1u);
        const uint32_t mhi = word & ~((2u << bb) - 1u);
        if (mlo) {
            pred = (w << 5) | (31 - __clz(mlo));
        } else {
            int s = w >> 5;
            uint32_t sm = W1[(size_t)s * S] & ((1u << (w & 31)) - 1u);
            while (true) {
                if (sm) {
                    const int ww = (s << 5) | (31 - __clz(sm));
                    pred = (ww << 5) | (31 - __clz(W0[(size_t)ww * S]));
                    break;
                }
                if (--s < 0) break;
                sm = W1[(size_t)s * S];
            }
        }
        if (mhi) {
            succ = (w << 5) | (__ffs(mhi) - 1);
        } else {
            int s = w >> 5;
            uint32_t sm = W1[(size_t)s * S] & ~((2u << (w & 31)) - 1u);
            while (true) {
                if (sm) {
                    const int ww = (s << 5) | (__ffs(sm) - 1);
                    succ = (ww << 5) | (__ffs(W0[(size_t)ww * S]) - 1);
                    break;
                }
                if (++s >= ns) break;
                sm = W1[(size_t)s * S];
            }
        }
        W0[(size_t)w * S] = word | (1u << bb);
        W1[(size_t)(w >> 5) * S] |= 1u << (w & 31);
        const uint32_t pv = pred >= 0 ? vs[base + pred] : sentB;
        const uint32_t nx = succ >= 0 ? vs[base + succ] : sentB;
        p.ulink[base + i] = make_uint2(pv, nx);
    }
}

// One warp per (pair q, segment s), i0 = s * L: the state before step i0.
// The window is A's positions >= i0 and B's positions < i0; walking the
// pair's merged order M, the kept elements of each block come out in sorted
// order (their links), and the first h kept elements are the small ones.
__global__ void __launch_bounds__(256)
large_seginit(LargeParams p)
{
    const int lane = threadIdx.x & 31;
    const int64_t sid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (sid >= p.npairs * p.S) return;
    const int64_t q = sid / p.S;
    const int s = (int)(sid - q * p.S);
    const int NB = block_len(p, q + 1);
    const int i0 = s * p.L;
    if (i0 >= NB) return;
    const int k = p.k, h = p.h;
    const uint32_t SA = (uint32_t)k, SB = (uint32_t)k + 1;
    uint32_t* NX = p.lists + sid * 3 * p.LS;
    uint32_t* PV = NX + p.LS;
    uint32_t* JR = PV + p.LS;
    const uint32_t* M = p.M + q * 2 * p.kp;
    const int tot = k + NB;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t lastA = SA, lastB = SB, mA = SA, mB = SB;
    int wcount = 0, sA = 0, sB = 0;
    bool foundA = false, foundB = false;
    for (int r0 = 0; r0 < tot; r0 += 32) {
        const int r = r0 + lane;
        const bool valid = r < tot;
        const uint32_t id = valid ? M[r] : 0u;
        const bool isB = (id & kBFlag) != 0;
        const uint32_t pos = id & ~kBFlag;
        const bool keepA = valid && !isB && pos >= (uint32_t)i0;
        const bool keepB = valid && isB && pos < (uint32_t)i0;
        const uint32_t bA = __ballot_sync(kFull, keepA);
        const uint32_t bB = __ballot_sync(kFull, keepB);
        const uint32_t bK = bA | bB;
        const bool small = wcount + __popc(bK & lt) < h;
        const uint32_t loA = bA & lt, loB = bB & lt;
        const uint32_t pA = __shfl_sync(kFull, pos, loA ? 31 - __clz(loA) : lane);
        const uint32_t pB = __shfl_sync(kFull, pos, loB ? 31 - __clz(loB) : lane);
        if (keepA) {
            const uint32_t prev = loA ? pA : lastA;
            PV[pos] = prev; NX[prev] = pos; JR[pos] = (uint32_t)r;
        }
        if (keepB) {
            const uint32_t prev = loB ? pB : lastB;
            PV[pos] = prev; NX[prev] = pos; JR[pos] = (uint32_t)r;
        }
        const uint32_t smA = __ballot_sync(kFull, keepA && small);
        const uint32_t smB = __ballot_sync(kFull, keepB && small);
        sA += __popc(smA);
        sB += __popc(smB);
        const uint32_t bigA = bA & ~smA, bigB = bB & ~smB;
        const uint32_t cA = __shfl_sync(kFull, pos, bigA ? __ffs(bigA) - 1 : 0);
        const uint32_t cB = __shfl_sync(kFull, pos, bigB ? __ffs(bigB) - 1 : 0);
        if (!foundA && bigA) { mA = cA; foundA = true; }
        if (!foundB && bigB) { mB = cB; foundB = true; }
        const uint32_t tA = __shfl_sync(kFull, pos, bA ? 31 - __clz(bA) : 0);
        const uint32_t tB = __shfl_sync(kFull, pos, bB ? 31 - __clz(bB) : 0);
        if (bA) lastA = tA;
        if (bB) lastB = tB;
        wcount += __popc(bK);
    }
    if (lane == 0) {
        NX[lastA] = SA; PV[SA] = lastA;
        NX[lastB] = SB; PV[SB] = lastB;
        JR[SA] = kInf; JR[SB] = kInf;
        p.seg[sid] = make_int4((int)mA, (int)mB, sA, sB);
    }
}

// Section 5.2, steps i0 .. i1-1 of pair q: delete(A, i), undelete(B, i),
// advance while s_A + s_B < h, print min(peek A, peek B)
__global__ void __launch_bounds__(128)
large_chain(LargeParams p)
{
    const int64_t sid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (sid >= p.npairs * p.S) return;
    const int64_t q = sid / p.S;
    const int s = (int)(sid - q * p.S);
    const int NB = block_len(p, q + 1);
    const int i0 = s * p.L;
    if (i0 >= NB) return;
    const int i1 = min(i0 + p.L, NB);
    const int h = p.h;
    uint32_t* NX = p.lists + sid * 3 * p.LS;
    uint32_t* PV = NX + p.LS;
    uint32_t* JR = PV + p.LS;
    const int4 st = p.seg[sid];
    uint32_t mA = (uint32_t)st.x, mB = (uint32_t)st.y;
    int sA = st.z, sB = st.w;
    const uint2* UL = p.ulink + (q + 1) * p.kp;
    const uint32_t* JB = p.jb + q * p.kp;
    uint32_t* OUT = p.out + q * p.kp;
    for (int i = i0; i < i1; ++i) {
        const uint32_t ui = (uint32_t)i;
        // delete(A, i)
        const uint32_t pa = PV[i], na = NX[i], ra = JR[i];
        const bool was_small = ra < JR[mA];
        NX[pa] = na;
        PV[na] = pa;
        if (was_small) {
            --sA;
        } else {
            if (mA == ui) mA = na;
            if (sA > 0) { mA = PV[mA]; --sA; }
        }
        // undelete(B, i): slot i now holds B's element i
        const uint2 u = UL[i];
        const uint32_t rb = JB[i];
        PV[i] = u.x; NX[i] = u.y; JR[i] = rb;
        NX[u.x] = ui;
        PV[u.y] = ui;
        if (rb < JR[mB]) mB = PV[mB];
        // advance the smaller peek while s_A + s_B < h
        uint32_t jA = JR[mA], jB = JR[mB];
        if (sA + sB < h) {
            if (jA < jB) { mA = NX[mA]; ++sA; jA = JR[mA]; }
            else         { mB = NX[mB]; ++sB; jB = JR[mB]; }
        }
        OUT[i] = jA < jB ? mA : (kBFlag | mB);
    }
}

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
        const uint32_t id = p.out[q * p.kp + i];
        src = (q + (id >> 31)) * (int64_t)p.k + (id & ~kBFlag);
    }
    p.y[o] = __ldg(p.x + src);
    if (p.argmed) p.argmed[o] = (int32_t)src;
}

// ---------------------------------------------------------------------------
static inline uint64_t a256(uint64_t v) { return (v + 255) & ~uint64_t(255); }

struct LargeShape {
    int64_t nblocks, npairs, kp, LS;
    int S, L;
};

static LargeShape large_shape(int64_t n, int k)
{
    LargeShape s;
    s.nblocks = (n + k - 1) / k;
    s.npairs = s.nblocks - 1;
    s.kp = ((int64_t)k + 31) & ~int64_t(31);
    s.LS = ((int64_t)k + 2 + 31) & ~int64_t(31);
    int S = (k + kLargeSegSteps - 1) / kLargeSegSteps;
    S = S < 1 ? 1 : (S > kLargeMaxSegs ? kLargeMaxSegs : S);
    s.S = S;
    s.L = (k + S - 1) / S;
    return s;
}

size_t large_workspace_bytes(int64_t n, int k)
{
    const LargeShape s = large_shape(n, k);
    const uint64_t nb = (uint64_t)s.nblocks, kp = (uint64_t)s.kp;
    const uint64_t np1 = (uint64_t)(s.npairs > 0 ? s.npairs : 1);
    uint64_t b = a256(4ull * nb * kp) * 5;                   // keyA valA keyB valB rnk
    b += a256(8ull * nb * kp);                               // ulink
    b += a256(4ull * np1 * kp) * 2;                          // jb out
    b += a256(8ull * np1 * kp);                              // M
    b += a256(16ull * np1 * s.S);                            // seg
    b += a256(12ull * np1 * s.S * (uint64_t)s.LS);           // lists
    return (size_t)b;
}

cudaError_t large_setup()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(large_chunk_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(8 * kChunkWarpBytes)))) return e;
    return cudaFuncSetAttribute(large_unwind, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes);
}

cudaError_t launch_large(const uint32_t* x, int64_t n, int k, bool is_float, uint32_t* y,
                         int32_t* argmed, void* ws, size_t ws_bytes, cudaStream_t stream,
                         LaunchStats* stats)
{
    if (k < 1 || (k & 1) == 0 || k > kLargeMaxK || n < k) return cudaErrorInvalidValue;
    if (ws_bytes < large_workspace_bytes(n, k)) return cudaErrorInvalidValue;
    const LargeShape sh = large_shape(n, k);
    LargeParams p{};
    p.x = x; p.y = y; p.argmed = argmed;
    p.n = n; p.k = k; p.h = (k - 1) / 2;
    p.nblocks = sh.nblocks; p.npairs = sh.npairs; p.kp = sh.kp;
    p.is_float = is_float;
    p.S = sh.S; p.L = sh.L; p.LS = sh.LS;
    const uint64_t nb = (uint64_t)sh.nblocks, kp = (uint64_t)sh.kp;
    const uint64_t np1 = (uint64_t)(sh.npairs > 0 ? sh.npairs : 1);
    char* w = (char*)ws;
    p.keyA = (uint32_t*)w; w += a256(4ull * nb * kp);
    p.valA = (uint32_t*)w; w += a256(4ull * nb * kp);
    p.keyB = (uint32_t*)w; w += a256(4ull * nb * kp);
    p.valB = (uint32_t*)w; w += a256(4ull * nb * kp);
    p.rnk = (uint32_t*)w;  w += a256(4ull * nb * kp);
    p.ulink = (uint2*)w;   w += a256(8ull * nb * kp);
    p.jb = (uint32_t*)w;   w += a256(4ull * np1 * kp);
    p.out = (uint32_t*)w;  w += a256(4ull * np1 * kp);
    p.M = (uint32_t*)w;    w += a256(8ull * np1 * kp);
    p.seg = (int4*)w;      w += a256(16ull * np1 * sh.S);
    p.lists = (uint32_t*)w;
    auto launched = [&]() -> cudaError_t {
        if (stats) stats->launches += 1;
        return cudaGetLastError();
    };
    cudaError_t e;
    // phase 1: chunks, then merge tiers (ping-pong between the A and B buffers)
    const int cpb = (k + kChunk - 1) / kChunk;
    const int64_t warps = sh.nblocks * cpb;
    large_chunk_sort<<<(unsigned)((warps + 7) / 8), 256, 8 * kChunkWarpBytes, stream>>>(p, cpb);
    if ((e = launched()) != cudaSuccess) return e;
    uint32_t *ks = p.keyA, *vs = p.valA, *kt = p.keyB, *vt = p.valB;
    const int per_block4 = (int)(kp / 4);
    for (int R = kChunk; R < k; R *= 2) {
        const int64_t threads = sh.nblocks * per_block4;
        large_merge<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(p, ks, vs, kt, vt, R, per_block4);
        if ((e = launched()) != cudaSuccess) return e;
        uint32_t* t1 = ks; ks = kt; kt = t1;
        uint32_t* t2 = vs; vs = vt; vt = t2;
    }
    if (sh.npairs > 0) {
        // phase 2: ranks, joint ranks, unwind links, segment states, chains
        const int64_t tr = sh.nblocks * sh.kp;
        large_ranks<<<(unsigned)((tr + 255) / 256), 256, 0, stream>>>(p, vs);
        if ((e = launched()) != cudaSuccess) return e;
        const int64_t tj = sh.npairs * 2 * sh.kp;
        large_jrank<<<(unsigned)((tj + 255) / 256), 256, 0, stream>>>(p, ks, vs);
        if ((e = launched()) != cudaSuccess) return e;
        const int nw = (k + 31) / 32, ns = (nw + 31) / 32;
        const size_t per_lane = 4ull * (size_t)(nw + ns);
        int S = (int)((size_t)kMaxSmemBytes / per_lane);
        S = S > 64 ? 64 : (S < 1 ? 1 : S);
        const int seglen = (k + S - 1) / S;
        large_unwind<<<(unsigned)(sh.nblocks - 1), S, per_lane * S, stream>>>(p, vs, seglen, nw, ns);
        if ((e = launched()) != cudaSuccess) return e;
        const int64_t nseg = sh.npairs * sh.S;
        large_seginit<<<(unsigned)((nseg * 32 + 255) / 256), 256, 0, stream>>>(p);
        if ((e = launched()) != cudaSuccess) return e;
        large_chain<<<(unsigned)((nseg + 127) / 128), 128, 0, stream>>>(p);
        if ((e = launched()) != cudaSuccess) return e;
    }
    const int64_t m = n - k + 1;
    large_epilogue<<<(unsigned)((m + 255) / 256), 256, 0, stream>>>(p, vs);
    return launched();
}

}  // namespace mf

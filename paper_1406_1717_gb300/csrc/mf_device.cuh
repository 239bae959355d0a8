// mf_device.cuh -- device building blocks shared by the median-filter kernels.
//
// Paper: "Median Filtering is Equivalent to Sorting" (Suomela).
//  * order keys ............ Section 5.2 (the stable sort compares (alpha[i], i))
//  * warp radix sort ....... Section 3 "Piecewise Sorting" / Section 6.1 (the
//                            four-kernel path: 8-byte elements, k > 1021)
//  * signal / work-item lookup of batched launches
//  * pair merge ............ joint ranks of the two blocks of a pair: the
//                            rank-space form of the comparisons of Section 5.3
//                            ("(alpha[i], i) < (alpha[m], m)") and of the
//                            post-processing (peek(A) <= peek(B), Section 6.2)
#pragma once
#include <cstdint>
#include "mf_internal.h"

namespace mf {

constexpr uint32_t kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Debug build (compiled with -DMF_DEBUG): the kernels check their indices and
// the block data structures' invariants (Section 5: link fields name a slot
// or a sentinel, 0 <= s <= h, m is a live node of its list).  A failed check
// counts itself, keeps the first site and value in this translation unit's
// record, and the kernel carries on with the index clamped into range, so no
// check faults, traps or waits.  mf_debug_take (mf_api.cu) reads and clears
// the records of all translation units.  In the normal build MF_CHECK is the
// constant true and its arguments are not evaluated.
// Sites: 1xx fused sort kernel, 2xx chain and store kernels, 3xx large-k
// tier, 999 the self-test.
// ---------------------------------------------------------------------------
#ifdef MF_DEBUG
namespace {
__device__ unsigned int g_dbg_count;
__device__ unsigned int g_dbg_site;
__device__ unsigned long long g_dbg_value;
__device__ __noinline__ bool debug_check(bool ok, uint32_t site, uint64_t value)
{
    if (!ok && atomicAdd(&g_dbg_count, 1u) == 0u) {
        g_dbg_site = site;
        g_dbg_value = value;
    }
    return ok;
}
}  // namespace
#define MF_CHECK(cond, site, value) ::mf::debug_check((cond), (site), (uint64_t)(value))
// Host side of this translation unit's record: read it, then clear it.
#define MF_DEBUG_TAKE_FN(name)                                                              \
    cudaError_t debug_take_##name(uint32_t* count, uint32_t* site, uint64_t* value)         \
    {                                                                                       \
        cudaError_t e = cudaMemcpyFromSymbol(count, g_dbg_count, sizeof(uint32_t));         \
        if (e == cudaSuccess) e = cudaMemcpyFromSymbol(site, g_dbg_site, sizeof(uint32_t)); \
        if (e == cudaSuccess) e = cudaMemcpyFromSymbol(value, g_dbg_value, sizeof(uint64_t)); \
        const uint32_t z32 = 0u;                                                            \
        const uint64_t z64 = 0ull;                                                          \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_dbg_count, &z32, sizeof(uint32_t));  \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_dbg_site, &z32, sizeof(uint32_t));   \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_dbg_value, &z64, sizeof(uint64_t));  \
        return e;                                                                           \
    }
#else
#define MF_CHECK(cond, site, value) true
#define MF_DEBUG_TAKE_FN(name)
#endif

// ---------------------------------------------------------------------------
// Order keys.  int32: flipping the sign bit turns signed order into unsigned
// order.  float32: IEEE 754 totalOrder on bit patterns becomes unsigned order
// after flipping all bits of negatives and the sign bit of non-negatives.
// Both maps are bijections, so from_key recovers the exact input bits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t to_key(uint32_t bits, bool is_float) {
    if (is_float) return (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
    return bits ^ 0x80000000u;
}
__device__ __forceinline__ uint32_t from_key(uint32_t key, bool is_float) {
    if (is_float) return (key & 0x80000000u) ? (key & 0x7fffffffu) : ~key;
    return key ^ 0x80000000u;
}
// 64-bit elements (int64, float64): the same two maps on 64-bit patterns.
__device__ __forceinline__ uint64_t to_key(uint64_t bits, bool is_float) {
    const uint64_t s = 0x8000000000000000ull;
    if (is_float) return (bits & s) ? ~bits : (bits | s);
    return bits ^ s;
}

__device__ __forceinline__ uint32_t warp_max_u32(uint32_t v) {
    for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(kFull, v, off));
    return v;
}

// ---------------------------------------------------------------------------
// Warp-level stable LSD radix sort of one group of consecutive blocks held in
// shared memory (phase 1, piecewise sort).  The group holds `cnt` elements:
// keys kin[0..cnt) and values vin[0..cnt) = CTA-local element indices, which
// start in ascending order, so LSD stability orders equal keys by index --
// the stable sort of (alpha[i], i) of Section 5.2.  Four 8-bit key passes;
// when the group holds more than one block, a final pass on the block number
// (vin - e0) / k regroups the elements block by block.  A pass whose digits
// are all equal is skipped (common for the high bytes of smooth signals).
// kt / vt are scratch of the same size.  On return kin / vin hold the result.
// hist is this warp's private 256-entry counter array.
// Adaptive step (Section 1: adaptive sorting algorithms give adaptive median
// filters): before any pass the warp checks the adjacent pairs inside each
// block; blocks that are all ascending keep the identity permutation and
// need no pass, blocks that are all strictly descending are reversed.  The
// check stops after the first 32 pairs that rule out both orders, so
// unordered inputs pay one vote.
// ---------------------------------------------------------------------------
template <typename KeyT>
__device__ __forceinline__ uint32_t sort_digit(int pass, KeyT key, uint32_t val, int e0, int k) {
    if (pass < (int)sizeof(KeyT)) return (uint32_t)(key >> (8 * pass)) & 0xffu;
    return (val - (uint32_t)e0) / (uint32_t)k;
}

// KeyT: uint32_t (4 key passes) or uint64_t (8 key passes).
template <typename KeyT>
inline __device__ void warp_sort_group(KeyT* kin, uint16_t* vin, KeyT* kt, uint16_t* vt,
                                int cnt, int e0, int k, int nblk, uint32_t* hist)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    {
        bool asc = true, desc = true;
        int pib = nblk > 1 ? lane % k : lane;          // position of pair start in its block
        for (int base = 0; base + 1 < cnt; base += 32) {
            const int idx = base + lane;
            if (idx + 1 < cnt && (nblk == 1 || pib + 1 < k)) {
                const KeyT a = kin[idx], b = kin[idx + 1];
                asc = asc && a <= b;
                desc = desc && a > b;
            }
            if (nblk > 1) { pib += 32; while (pib >= k) pib -= k; }
            const bool asc_out = __any_sync(kFull, !asc), desc_out = __any_sync(kFull, !desc);
            if (asc_out && desc_out) break;             // neither order can hold
        }
        const bool all_asc = __all_sync(kFull, asc), all_desc = __all_sync(kFull, desc);
        if (all_asc) { __syncwarp(); return; }
        if (all_desc) {
            for (int idx = lane; idx < cnt; idx += 32) {
                const int s = (idx / k) * k, len = min(k, cnt - s);
                const int dst = s + (len - 1 - (idx - s));
                kt[dst] = kin[idx];
                vt[dst] = vin[idx];
            }
            __syncwarp();
            for (int idx = lane; idx < cnt; idx += 32) { kin[idx] = kt[idx]; vin[idx] = vt[idx]; }
            __syncwarp();
            return;
        }
    }
    KeyT* ks = kin; uint16_t* vs = vin;
    KeyT* kd = kt;  uint16_t* vd = vt;
    const int nkey = (int)sizeof(KeyT);
    const int npass = nblk > 1 ? nkey + 1 : nkey;
    for (int pass = 0; pass < npass; ++pass) {
        for (int d = lane; d < 256; d += 32) hist[d] = 0;
        __syncwarp();
        for (int idx = lane; idx < cnt; idx += 32)
            atomicAdd(&hist[sort_digit<KeyT>(pass, ks[idx], vs[idx], e0, k)], 1u);
        __syncwarp();
        // exclusive scan of the 256 counters: lane owns entries 8*lane .. 8*lane+7
        uint32_t c[8], s = 0, mx = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) { c[q] = hist[lane * 8 + q]; s += c[q]; mx = max(mx, c[q]); }
        uint32_t incl = s;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t t = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += t;
        }
        uint32_t run = incl - s;
#pragma unroll
        for (int q = 0; q < 8; ++q) { hist[lane * 8 + q] = run; run += c[q]; }
        mx = warp_max_u32(mx);
        __syncwarp();
        if (mx == (uint32_t)cnt) continue;          // one digit only: order unchanged
        for (int base = 0; base < cnt; base += 32) {
            const int idx = base + lane;
            const bool valid = idx < cnt;
            KeyT key = 0;
            uint32_t val = 0, d = 0x100u + (uint32_t)lane;           // unique for idle lanes
            if (valid) { key = ks[idx]; val = vs[idx]; d = sort_digit<KeyT>(pass, key, val, e0, k); }
            const uint32_t peers = __match_any_sync(kFull, d);
            const int leader = __ffs(peers) - 1;
            uint32_t b = 0;
            if (valid && lane == leader) { b = hist[d]; hist[d] = b + __popc(peers); }
            b = __shfl_sync(kFull, b, leader);
            if (valid) {
                const uint32_t dst = b + __popc(peers & lt_mask);
                kd[dst] = key;
                vd[dst] = (uint16_t)val;
            }
            __syncwarp();
        }
        KeyT* tk = ks; ks = kd; kd = tk;
        uint16_t* tv = vs; vs = vd; vd = tv;
    }
    if (ks != kin) {
        for (int idx = lane; idx < cnt; idx += 32) { kin[idx] = ks[idx]; vin[idx] = vs[idx]; }
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Joint ranks of one block pair (A = older block, B = newer block): merging
// the two sorted blocks, with A first on equal keys, gives every element of
// A u B its rank in the window order; "alpha[i] is small" (Section 5.3) and
// peek(A) <= peek(B) (Section 6.2) become comparisons of these ranks.
// Warp-cooperative merge path: lane L emits merged positions
// [L*per, (L+1)*per).  Results are stored by position (jposA / jposB).
// ---------------------------------------------------------------------------
template <typename KeyT>
inline __device__ void warp_merge_ranks(const KeyT* kA, const uint16_t* vA, int NA, int eA0,
                                 const KeyT* kB, const uint16_t* vB, int NB, int eB0,
                                 uint16_t* jposA, uint16_t* jposB)
{
    const int lane = threadIdx.x & 31;
    const int total = NA + NB;
    const int per = (total + 31) >> 5;
    const int o0 = min(lane * per, total);
    const int o1 = min(o0 + per, total);
    int lo = max(0, o0 - NB), hi = min(o0, NA);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (kA[mid] <= kB[o0 - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    int ia = lo, ib = o0 - lo;
    // heads of both runs in registers
    KeyT a = ia < NA ? kA[ia] : KeyT(0);
    KeyT b = ib < NB ? kB[ib] : KeyT(0);
    for (int o = o0; o < o1; ++o) {
        if (ib >= NB || (ia < NA && a <= b)) {
            jposA[vA[ia] - eA0] = (uint16_t)o;
            ++ia;
            if (ia < NA) a = kA[ia];
        } else {
            jposB[vB[ib] - eB0] = (uint16_t)o;
            ++ib;
            if (ib < NB) b = kB[ib];
        }
    }
}

// ===========================================================================
// Signals and work items.  Every kernel works on items (sortmerge,
// sortlist and epilogue: CTAs of G consecutive block pairs; unwind: warp groups of blocks;
// chain: block pairs).  A launch covers one signal (descriptor passed by
// value) or a batch of signals (device table; each descriptor carries the
// index of its first item in every kernel, and an item finds its signal by
// binary search).
// ===========================================================================
enum { kItemSort = 0, kItemUnwind = 1, kItemChain = 2, kItemEpilogue = 3 };

__device__ __forceinline__ PipeParams find_signal(const SegTable& t, int kern, int64_t item,
                                                  int64_t* local)
{
    if (t.segs == nullptr) { *local = item; return t.one; }
    int lo = 0, hi = t.nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.segs[mid].start[kern] <= item) lo = mid; else hi = mid - 1;
    }
    const PipeParams p = t.segs[lo];
    *local = item - p.start[kern];
    return p;
}


}  // namespace mf

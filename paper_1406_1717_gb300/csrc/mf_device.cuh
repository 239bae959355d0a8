// mf_device.cuh -- device building blocks of the fused median-filter kernels.
//
// Paper: "Median Filtering is Equivalent to Sorting" (Suomela).
//  * order keys ............ Section 4.2 (the stable sort compares (alpha[i], i))
//  * warp radix sort ....... Section 3 "Piecewise Sorting" / Section 5.1
//  * pair merge ............ joint ranks of the two blocks of a pair: the
//                            rank-space form of the comparisons of Section 4.3
//                            ("(alpha[i], i) < (alpha[m], m)") and of the
//                            post-processing (peek(A) <= peek(B), Section 5.2)
//  * list build / unwind ... Section 4.3 construct, Section 3 "Unwind"
//  * pair chain ............ Section 5.2 post-processing, with delete /
//                            undelete / advance of Section 4.3
#pragma once
#include <cstdint>

namespace mf {

constexpr uint32_t kFull = 0xffffffffu;

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

__device__ __forceinline__ uint32_t warp_max_u32(uint32_t v) {
    for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(kFull, v, off));
    return v;
}

// ---------------------------------------------------------------------------
// Warp-level stable LSD radix sort of one group of consecutive blocks held in
// shared memory (phase 1, piecewise sort).  The group holds `cnt` elements:
// keys kin[0..cnt) and values vin[0..cnt) = CTA-local element indices, which
// start in ascending order, so LSD stability orders equal keys by index --
// the stable sort of (alpha[i], i) of Section 4.2.  Four 8-bit key passes;
// when the group holds more than one block, a final pass on the block number
// (vin - e0) / k regroups the elements block by block.  A pass whose digits
// are all equal is skipped (common for the high bytes of smooth signals).
// kt / vt are scratch of the same size.  On return kin / vin hold the result.
// hist is this warp's private 256-entry counter array.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t sort_digit(int pass, uint32_t key, uint32_t val, int e0, int k) {
    if (pass < 4) return (key >> (8 * pass)) & 0xffu;
    return (val - (uint32_t)e0) / (uint32_t)k;
}

__device__ void warp_sort_group(uint32_t* kin, uint16_t* vin, uint32_t* kt, uint16_t* vt,
                                int cnt, int e0, int k, int nblk, uint32_t* hist)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t* ks = kin; uint16_t* vs = vin;
    uint32_t* kd = kt;  uint16_t* vd = vt;
    const int npass = nblk > 1 ? 5 : 4;
    for (int pass = 0; pass < npass; ++pass) {
        for (int d = lane; d < 256; d += 32) hist[d] = 0;
        __syncwarp();
        for (int idx = lane; idx < cnt; idx += 32)
            atomicAdd(&hist[sort_digit(pass, ks[idx], vs[idx], e0, k)], 1u);
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
            uint32_t key = 0, val = 0, d = 0x100u + (uint32_t)lane;   // unique for idle lanes
            if (valid) { key = ks[idx]; val = vs[idx]; d = sort_digit(pass, key, val, e0, k); }
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
        uint32_t* tk = ks; ks = kd; kd = tk;
        uint16_t* tv = vs; vs = vd; vd = tv;
    }
    if (ks != kin) {
        for (int idx = lane; idx < cnt; idx += 32) { kin[idx] = ks[idx]; vin[idx] = vs[idx]; }
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Joint ranks of one block pair (A = older block, B = newer block).
// Merging the two sorted blocks, with A first on equal keys, numbers every
// element of A u B by its rank in the window order; these numbers are the
// node ids of both linked lists.  Then "is alpha[i] small" (Section 4.3) is
// "node < m", peek(A) <= peek(B) (Section 5.2) is "mA < mB", and the printed
// min is the node min(mA, mB).  Warp-cooperative merge path: lane L emits
// merged positions [L*per, (L+1)*per).
//   kA/vA, kB/vB : sorted keys and CTA-local element indices of A and B
//   eA0, eB0     : CTA-local element index of each block's first element
//   jsA, jsB     : out, node id of the t-th smallest element of A / B
//   jposA, jposB : out, node id of the element at position i of A / B
//   info         : out, node -> (isB << 15) | sorted index within its block
// ---------------------------------------------------------------------------
__device__ void warp_merge_pair(const uint32_t* kA, const uint16_t* vA, int NA, int eA0,
                                const uint32_t* kB, const uint16_t* vB, int NB, int eB0,
                                uint16_t* jsA, uint16_t* jsB,
                                uint16_t* jposA, uint16_t* jposB, uint16_t* info)
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
    for (int o = o0; o < o1; ++o) {
        const bool takeA = (ib >= NB) || (ia < NA && kA[ia] <= kB[ib]);
        if (takeA) {
            jsA[ia] = (uint16_t)o;
            jposA[vA[ia] - eA0] = (uint16_t)o;
            info[o] = (uint16_t)ia;
            ++ia;
        } else {
            jsB[ib] = (uint16_t)o;
            jposB[vB[ib] - eB0] = (uint16_t)o;
            info[o] = (uint16_t)(0x8000u | (uint32_t)ib);
            ++ib;
        }
    }
}

// Link the nodes js[0..cnt) (ascending) into one sorted list through
// sentinel `sent` (Section 4.3 construct: next[k] = p_0, prev[k] = p_{c-1}).
// rec[r] packs prev(r) in the high and next(r) in the low 16 bits.
__device__ void warp_link_list(uint32_t* rec, const uint16_t* js, int cnt, uint32_t sent)
{
    const int lane = threadIdx.x & 31;
    for (int t = lane; t < cnt; t += 32) {
        const uint32_t p = t > 0 ? js[t - 1] : sent;
        const uint32_t q = t + 1 < cnt ? js[t + 1] : sent;
        rec[js[t]] = (p << 16) | q;
    }
    if (lane == 0) rec[sent] = ((uint32_t)js[cnt - 1] << 16) | js[0];
}

// 16-bit halves of a list record (little endian: next is the low half).
__device__ __forceinline__ void set_next(uint32_t* rec, uint32_t r, uint32_t v) {
    reinterpret_cast<uint16_t*>(rec)[2 * r] = (uint16_t)v;
}
__device__ __forceinline__ void set_prev(uint32_t* rec, uint32_t r, uint32_t v) {
    reinterpret_cast<uint16_t*>(rec)[2 * r + 1] = (uint16_t)v;
}
__device__ __forceinline__ uint32_t rec_prev(uint32_t w) { return w >> 16; }
__device__ __forceinline__ uint32_t rec_next(uint32_t w) { return w & 0xffffu; }

// ---------------------------------------------------------------------------
// Post-processing of one block pair (Section 5.2), run by one thread.
//   rec    : lists of A and B in joint node space (A linked through SA, B's
//            full list linked through SB)
//   jposA/B: node of the element at position i of A / B
//   out    : node printed at step i (may alias jposA: step i reads jposA[i]
//            before writing out[i])
//   NB     : elements in B (k, or r < k for the last block)
//   h      : half window
//   mA0    : node of A's element of rank h (construct sets m = pi[h], s = h)
// ---------------------------------------------------------------------------
__device__ void pair_chain(uint32_t* rec, const uint16_t* jposA, const uint16_t* jposB,
                           uint16_t* out, int NB, int h, uint32_t mA0,
                           uint32_t SA, uint32_t SB)
{
    // unwind(B): delete B's elements from position NB-1 down to 0 (Section 3,
    // "Unwind"); each deleted node keeps its own prev/next, which later lets
    // undelete put it back (equation undo-del).  m_B = sentinel, s_B = 0.
    for (int i = NB - 1; i >= 0; --i) {
        const uint32_t b = jposB[i];
        const uint32_t w = rec[b];
        set_next(rec, rec_prev(w), rec_next(w));
        set_prev(rec, rec_next(w), rec_prev(w));
    }
    uint32_t mA = mA0, mB = SB;
    int sA = h, sB = 0;
    for (int i = 0; i < NB; ++i) {
        const uint32_t a = jposA[i];
        const uint32_t b = jposB[i];
        // delete(A, i): unlink (equation del); s_A <- max(0, s_A - 1)
        const uint32_t wa = rec[a];
        const uint32_t pa = rec_prev(wa), na = rec_next(wa);
        set_next(rec, pa, na);
        set_prev(rec, na, pa);
        if (a < mA) {                       // a was small (or A's list is at its end)
            --sA;
        } else {                            // a was large
            if (mA == a) mA = na;           // a's retained pointer names its successor
            if (sA > 0) { mA = rec_prev(rec[mA]); --sA; }
        }
        // undelete(B, i): relink (equation undo-del); if small, m_B <- prev[m_B]
        const uint32_t wb = rec[b];
        set_next(rec, rec_prev(wb), b);
        set_prev(rec, rec_next(wb), b);
        if (b < mB) mB = rec_prev(rec[mB]);
        // advance the list whose first large element is smaller (A on ties)
        if (sA + sB < h) {
            if (mA < mB) { mA = rec_next(rec[mA]); ++sA; }
            else         { mB = rec_next(rec[mB]); ++sB; }
        }
        out[i] = (uint16_t)min(mA, mB);     // print min(peek(A), peek(B))
    }
    (void)SA;
}

}  // namespace mf

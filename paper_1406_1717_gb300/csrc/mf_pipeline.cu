// mf_pipeline.cu -- the median filter as a pipeline of four kernels.
//
// Paper: "Median Filtering is Equivalent to Sorting" (Suomela).
//
// The post-processing of a block pair (Section 6.2) is a chain of k dependent
// steps whose lists must sit in shared memory; how many chains an SM can run
// at once -- shared-memory bytes per chain -- sets the speed.  So everything
// that is not the chain runs in separate, fully parallel kernels, and the
// chain kernel keeps nothing in shared memory but the lists:
//
//   sortmerge_kernel  load x, stable sort of every block (Section 5.2), and
//                     per block: perm (pi), rank (pi^-1) and the sorted-order
//                     links in position space (construct, Section 5.3); per
//                     pair: the rank of every element in the merged order of
//                     the pair's two blocks ("joint rank", A first on ties).
//   unwind_kernel     per block used as B: the links unwind(B) leaves behind
//                     (Section 4, "Unwind"); one lane per block.
//   chain_kernel      one lane per pair: delete(A, i), undelete(B, i),
//                     advance, print min(peek) for every step (Section 6.2),
//                     lists in shared memory (built by the whole CTA first
//                     when k > 256).
//   epilogue_kernel   node -> input element, coalesced stores of y / argmed.
//
// For 4-byte elements and k <= kFusedMaxK, sortlist_kernel (mf_sortlist.cu)
// replaces the first two kernels and writes the list words themselves; the
// chain kernel then copies them (chain_body_words).
//
// Node numbering ("slots"): node i of the pair's lists is position i of A
// until step i deletes it, and position i of B from the moment step i
// undeletes it (A only ever holds positions > i, B only positions <= i), plus
// two sentinels k (A) and k+1 (B) -- the paper's arrays of length k+1
// (Section 5.3), shared by A and B.  Comparisons use the joint rank of the
// node's element (the pi^-1 form of Section 5.2, extended across the pair),
// so "alpha[i] is small" is jr(i) < jr(m) and peek(A) <= peek(B) is
// jr(mA) < jr(mB); the sentinels have the largest rank the node format holds
// (all ones), above every element.
#include <cuda_runtime.h>
#include <cstdint>
#include "mf_device.cuh"
#include "mf_internal.h"

namespace mf {


// ===========================================================================
// sortmerge_kernel
// ===========================================================================
// One merge round over the parts of every block of the CTA: within a block
// (start b k, length min(k, E - b k)) the runs [g, g + w) and [g + w, g + 2w),
// g a multiple of 2w, are merged, the left run first on equal keys.  Thread t
// writes a contiguous span of the CTA's outputs, split where a merge ends;
// each piece finds its start by a merge-path search.
template <typename KeyT>
__device__ void merge_runs(const KeyT* ks, const uint16_t* vs, KeyT* kd, uint16_t* vd,
                           int E, int k, int w)
{
    const int C = (E + (int)blockDim.x - 1) / (int)blockDim.x;
    int e = (int)threadIdx.x * C;
    const int eend = min(e + C, E);
    while (e < eend) {
        const int bstart = (e / k) * k;
        const int blen = min(k, E - bstart);
        const int off = e - bstart;
        const int g0 = off - off % (2 * w);
        const int L1 = min(g0 + w, blen), R1 = min(g0 + 2 * w, blen);
        const int na = L1 - g0, nb = R1 - L1;
        const int pend = min(eend, bstart + R1);
        const int d = off - g0;
        const KeyT* A = ks + bstart + g0;
        const KeyT* B = ks + bstart + L1;
        const uint16_t* VA = vs + bstart + g0;
        const uint16_t* VB = vs + bstart + L1;
        int lo = max(0, d - nb), hi = min(d, na);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= B[d - 1 - mid]) lo = mid + 1; else hi = mid;
        }
        int ia = lo, ib = d - lo;
        for (int o = e; o < pend; ++o) {
            if (ib >= nb || (ia < na && A[ia] <= B[ib])) { kd[o] = A[ia]; vd[o] = VA[ia]; ++ia; }
            else { kd[o] = B[ib]; vd[o] = VB[ib]; ++ib; }
        }
        e = pend;
    }
}

// KeyT: uint32_t for 4-byte elements, uint64_t for 8-byte elements.
template <typename KeyT>
__global__ void __launch_bounds__(kPipeThreads)
sortmerge_kernel(SegTable tab, SortPlan sp)
{
    int64_t cta;
    const PipeParams p = find_signal(tab, kItemSort, blockIdx.x, &cta);
    extern __shared__ __align__(16) unsigned char smem[];
    KeyT* keyA = reinterpret_cast<KeyT*>(smem + sp.off_keyA);
    KeyT* keyB = reinterpret_cast<KeyT*>(smem + sp.off_keyB);
    const KeyT* xp = reinterpret_cast<const KeyT*>(p.x);
    uint16_t* valA = reinterpret_cast<uint16_t*>(smem + sp.off_valA);
    uint16_t* valB = reinterpret_cast<uint16_t*>(smem + sp.off_valB);
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + sp.off_hist);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int W = blockDim.x >> 5;
    const int k = p.k;
    const int64_t j0 = 1 + cta * sp.G;
    const int64_t left = p.npairs - (j0 - 1);
    const int npair = (int)(left < sp.G ? (left > 0 ? left : 0) : sp.G);
    const int nblk = npair + 1;
    const int64_t ebase = (j0 - 1) * (int64_t)k;
    const int64_t rem = p.n - ebase;
    const int E = (int)((int64_t)nblk * k < rem ? (int64_t)nblk * k : rem);
    // blocks sorted per warp: enough blocks for all warps, at most ~2048 elements
    int bpg = (nblk + W - 1) / W;
    const int cap = min(255, max(1, 2048 / k));
    bpg = max(1, min(bpg, cap));

    for (int e = tid; e < E; e += blockDim.x) {
        keyA[e] = to_key(__ldg(xp + ebase + e), p.is_float);
        valA[e] = (uint16_t)e;
    }
    __syncthreads();

    // Long blocks, fewer than half as many as warps: each block is split into
    // H position-contiguous parts (H = 2 or 4), a warp sorts each part and
    // merge rounds of all threads join them.  Still a stable sort: the parts
    // are in position order and a merge takes the left run first on ties.
    int H = 1;
    if (k >= 512)
        while (H < 4 && nblk * H * 2 <= W) H <<= 1;
    if (H == 1) {
        const int ngroups = (nblk + bpg - 1) / bpg;
        for (int gi = warp; gi < ngroups; gi += W) {
            const int b0 = gi * bpg;
            const int b1 = min(b0 + bpg, nblk);
            const int e0 = b0 * k;
            const int e1 = min(b1 * k, E);
            warp_sort_group<KeyT>(keyA + e0, valA + e0, keyB + e0, valB + e0,
                            max(0, e1 - e0), e0, k, b1 - b0, hist + warp * 256);
        }
        __syncthreads();
    } else {
        const int part = (k + H - 1) / H;
        for (int gi = warp; gi < nblk * H; gi += W) {
            const int b = gi / H, hp = gi - b * H;
            const int bstart = b * k;
            const int blen = min(k, E - bstart);
            const int s0 = min(hp * part, blen), s1 = min(s0 + part, blen);
            if (s1 > s0)
                warp_sort_group<KeyT>(keyA + bstart + s0, valA + bstart + s0, keyB + bstart + s0,
                                      valB + bstart + s0, s1 - s0, bstart + s0, k, 1,
                                      hist + warp * 256);
        }
        __syncthreads();
        KeyT* ks = keyA;  uint16_t* vs = valA;
        KeyT* kd = keyB;  uint16_t* vd = valB;
        for (int w = part; w < k; w <<= 1) {
            merge_runs<KeyT>(ks, vs, kd, vd, E, k, w);
            __syncthreads();
            KeyT* tk = ks; ks = kd; kd = tk;
            uint16_t* tv = vs; vs = vd; vd = tv;
        }
        if (ks != keyA) {
            for (int e = tid; e < E; e += blockDim.x) { keyA[e] = ks[e]; valA[e] = vs[e]; }
            __syncthreads();
        }
    }

    // inverse permutation (rank of each position) into valB, block by block
    for (int blk = 0, bstart = 0; bstart < E; ++blk, bstart += k) {
        const int NBb = min(k, E - bstart);
        for (int t = tid; t < NBb; t += blockDim.x)
            valB[valA[bstart + t]] = (uint16_t)t;
    }
    __syncthreads();

    // per block owned by this CTA: perm, rank, sorted-order links (sentinel k)
    const int lb0 = (j0 == 1) ? 0 : 1;
    for (int blk = lb0, bstart = lb0 * k; bstart < E; ++blk, bstart += k) {
        const int NBb = min(k, E - bstart);
        const size_t ob = (size_t)(j0 - 1 + blk) * p.kp;
        for (int pos = tid; pos < NBb; pos += blockDim.x) {
            const int e = bstart + pos;
            p.perm[ob + pos] = (uint16_t)(valA[e] - bstart);       // e = bstart + t
            const int t = valB[e];
            p.rnk[ob + pos] = (uint16_t)t;
            const uint32_t pv = t > 0 ? (uint32_t)(valA[bstart + t - 1] - bstart) : (uint32_t)k;
            const uint32_t nx = t + 1 < NBb ? (uint32_t)(valA[bstart + t + 1] - bstart) : (uint32_t)k;
            p.slink[ob + pos] = (pv << 16) | nx;
        }
    }

    // per pair: joint ranks by position (scratch in keyB, free after the sort)
    uint16_t* jp = reinterpret_cast<uint16_t*>(keyB);
    for (int g = warp; g < npair; g += W) {
        const int NB = min(k, E - (g + 1) * k);
        warp_merge_ranks<KeyT>(keyA + g * k, valA + g * k, k, g * k,
                         keyA + (g + 1) * k, valA + (g + 1) * k, NB, (g + 1) * k,
                         jp + (size_t)g * 2 * k, jp + (size_t)g * 2 * k + k);
    }
    __syncthreads();
    for (int g = 0; g < npair; ++g) {
        const int NB = min(k, E - (g + 1) * k);
        const size_t q = (size_t)(j0 - 1 + g) * p.kp;
        for (int i = tid; i < k; i += blockDim.x) p.ja[q + i] = jp[(size_t)g * 2 * k + i];
        for (int i = tid; i < NB; i += blockDim.x) p.jb[q + i] = jp[(size_t)g * 2 * k + k + i];
    }
}

// ===========================================================================
// unwind_kernel: links of every block j >= 1 (block j is B of pair j).
// unwind(B) (Section 4, "Unwind") deletes positions NB-1 .. 0; when position
// i is deleted its list holds exactly positions 0..i, so the prev / next it
// keeps are the nearest smaller / larger element among positions < i.
// Walking positions upward with a bitset of the ranks seen so far gives the
// same links: prev = predecessor, next = successor of rank(i) in the set,
// mapped back to positions through the block's perm; missing -> B's
// sentinel k+1.
// A block's positions are split into S runs of seglen (a multiple of 8); run
// s starts with the ranks of all positions before it already in its bitset,
// so the S lanes of a block work independently and share one copy of the
// block's perm in shared memory.  Lane l of a warp serves block slot l / S,
// run l % S.  For k <= 1024 the summary of non-empty bitset words is one
// register and the search has no branches.
// ===========================================================================
template <bool SMALL>
__global__ void __launch_bounds__(kPipeThreads)
unwind_kernel(SegTable tab, UnwindPlan up)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int S = up.segs, BPW = 32 / S;
    const int bslot = lane / S, sg = lane - bslot * S;
    const int64_t wg = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;   // warp group
    if (wg >= up.items) return;                                           // warp-uniform
    int64_t lwg;
    const PipeParams p = find_signal(tab, kItemUnwind, wg, &lwg);
    const int k = p.k;
    const int64_t gb = 1 + lwg * BPW + bslot;
    uint32_t* ws = reinterpret_cast<uint32_t*>(smem) + warp * up.words_per_warp;
    uint32_t* W0 = ws + lane;                                   // bitset word x at W0[x * 32]
    uint32_t* W1 = ws + up.nw * 32 + lane;                      // summary words (when !SMALL)
    uint32_t* PMW = ws + (up.nw + up.ns) * 32 + bslot;          // perm word x at PMW[x * BPW]
    const bool live = gb < p.nblocks;
    const int NB = live ? (int)min((int64_t)k, p.n - gb * (int64_t)k) : 0;
    const uint16_t* perm = p.perm + (live ? gb : 0) * (int64_t)p.kp;
    const uint16_t* rnk = p.rnk + (live ? gb : 0) * (int64_t)p.kp;
    // ---- the block's perm into shared memory, split over its S lanes -------
    {
        const uint4* pm4 = reinterpret_cast<const uint4*>(perm);
        const int nch = (NB + 7) >> 3;
        for (int c = sg; c < nch; c += S) {
            const uint4 v = __ldg(pm4 + c);
            PMW[(4 * c + 0) * BPW] = v.x;
            PMW[(4 * c + 1) * BPW] = v.y;
            PMW[(4 * c + 2) * BPW] = v.z;
            PMW[(4 * c + 3) * BPW] = v.w;
        }
    }
    __syncwarp();
    const int i0 = sg * up.seglen;
    const int i1 = min(i0 + up.seglen, NB);
    if (i0 >= i1) return;
    for (int w = 0; w < up.nw; ++w) W0[w * 32] = 0;
    if (!SMALL) for (int s = 0; s < up.ns; ++s) W1[s * 32] = 0;
    const uint4* rk4 = reinterpret_cast<const uint4*>(rnk);
    uint32_t summ = 0;                                          // SMALL: non-empty words
    // ---- seed: ranks of positions 0 .. i0-1 (independent updates) ----------
    for (int c = 0; c < (i0 >> 3); ++c) {
        const uint4 v = __ldg(rk4 + c);
        const uint32_t rw[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t r = (t & 1) ? rw[t >> 1] >> 16 : rw[t >> 1] & 0xffffu;
            atomicOr(&W0[(r >> 5) * 32], 1u << (r & 31));
            if (SMALL) summ |= 1u << (r >> 5);
            else atomicOr(&W1[(r >> 10) * 32], 1u << ((r >> 5) & 31));
        }
    }
    const uint32_t sentB = (uint32_t)k + 1;
    uint4* ul4 = reinterpret_cast<uint4*>(p.ulink + gb * (int64_t)p.kp);
    // ---- the run, 8 positions per round (rank chunk prefetched one ahead) ---
    uint4 rn = __ldg(rk4 + (i0 >> 3));
    for (int c0 = i0; c0 < i1; c0 += 8) {
        const uint4 rv = rn;
        if (c0 + 8 < i1) rn = __ldg(rk4 + (c0 >> 3) + 1);
        const uint32_t rw[4] = {rv.x, rv.y, rv.z, rv.w};
        uint32_t uo[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            uo[t] = 0u;
            if (c0 + t < i1) {
                const int r = (int)((t & 1) ? rw[t >> 1] >> 16 : rw[t >> 1] & 0xffffu);
                const int w = r >> 5, b = r & 31;
                const uint32_t word = W0[w * 32];
                const uint32_t mlo = word & ((1u << b) - 1u);
                const uint32_t mhi = word & ~((2u << b) - 1u);   // b = 31: 2u << 31 == 0, ~(0 - 1) == 0
                int pred = -1, succ = -1;
                if (SMALL) {
                    const uint32_t slo = summ & ((1u << w) - 1u);
                    const uint32_t shi = summ & ~((2u << w) - 1u);
                    const int wlo = slo ? 31 - __clz(slo) : 0;
                    const int whi = shi ? __ffs(shi) - 1 : 0;
                    const uint32_t xlo = W0[wlo * 32], xhi = W0[whi * 32];
                    pred = mlo ? ((w << 5) | (31 - __clz(mlo))) : (slo ? ((wlo << 5) | (31 - __clz(xlo))) : -1);
                    succ = mhi ? ((w << 5) | (__ffs(mhi) - 1)) : (shi ? ((whi << 5) | (__ffs(xhi) - 1)) : -1);
                    summ |= 1u << w;
                } else {
                    if (mlo) {
                        pred = (w << 5) | (31 - __clz(mlo));
                    } else {
                        int s = w >> 5;
                        uint32_t sm = W1[s * 32] & ((1u << (w & 31)) - 1u);
                        while (true) {
                            if (sm) {
                                const int ww = (s << 5) | (31 - __clz(sm));
                                pred = (ww << 5) | (31 - __clz(W0[ww * 32]));
                                break;
                            }
                            if (--s < 0) break;
                            sm = W1[s * 32];
                        }
                    }
                    if (mhi) {
                        succ = (w << 5) | (__ffs(mhi) - 1);
                    } else {
                        int s = w >> 5;
                        uint32_t sm = W1[s * 32] & ~((2u << (w & 31)) - 1u);
                        while (true) {
                            if (sm) {
                                const int ww = (s << 5) | (__ffs(sm) - 1);
                                succ = (ww << 5) | (__ffs(W0[ww * 32]) - 1);
                                break;
                            }
                            if (++s >= up.ns) break;
                            sm = W1[s * 32];
                        }
                    }
                    W1[(w >> 5) * 32] |= 1u << (w & 31);
                }
                W0[w * 32] = word | (1u << b);
                uint32_t pv = sentB, nx = sentB;
                if (pred >= 0) { const uint32_t pw = PMW[(pred >> 1) * BPW]; pv = (pred & 1) ? pw >> 16 : pw & 0xffffu; }
                if (succ >= 0) { const uint32_t nw2 = PMW[(succ >> 1) * BPW]; nx = (succ & 1) ? nw2 >> 16 : nw2 & 0xffffu; }
                uo[t] = (pv << 16) | nx;
            }
        }
        // runs start on multiples of 8, so these two 16-byte groups are ours
        ul4[c0 >> 2] = make_uint4(uo[0], uo[1], uo[2], uo[3]);
        if (c0 + 4 < i1) ul4[(c0 >> 2) + 1] = make_uint4(uo[4], uo[5], uo[6], uo[7]);
    }
}

// ===========================================================================
// chain_kernel: the post-processing of Section 6.2, one lane per block pair.
// Shared memory per lane (bank-private, word index x * NL + lane):
//   rec[0 .. k+1]   the list word of every node (node numbers = slots, see top)
//   jr [0 .. k+1]   wide format only: joint rank of the node's current element
//                   (u16, two per word)
// Each list keeps m, m's word and m's rank in registers (patched in place
// when a relink touches m), so a step loads only the words m moves to.
// ===========================================================================
// Per-lane view of the lists in shared memory.  Slot e's word sits at word
// index e * NL + lane of the warp's slice, so every lane owns one bank.
//   packed (k <= 1021): next:10 | prev:10 | joint rank:11 in one word
//   mid    (k <= 4093): next:12 | prev:12 | joint rank bits 12..5 in one word,
//                       rank bits 4..0 in a byte array (5 bytes per node)
//   wide             : next:16 | prev:16, joint rank in a separate u16 array
// The side arrays are bank-private too: the 4 bytes or 2 halves of the word
// at word index (e / 4 or e / 2) * NL + lane.
// Relinks never read the word: when delete(A, i) unlinks i, next(prev(i)) is
// i and prev(next(i)) is i; when undelete(B, i) relinks i between p and n,
// next(p) is n and prev(n) is p.  So in the packed and mid formats each
// relink is one XOR of old ^ new into the field; in the wide format it is a
// 16-bit store (equations del / undo-del of Section 4).
enum { kFmtPacked = 0, kFmtMid = 1, kFmtWide = 2 };

template <int FMT>
struct Lists {
    static constexpr bool PACKED = FMT == kFmtPacked, MID = FMT == kFmtMid;
    static constexpr int PSH = PACKED ? 10 : (MID ? 12 : 16);
    static constexpr uint32_t FM = (1u << PSH) - 1u;
    static constexpr uint32_t RINF = PACKED ? 0x7ffu : (MID ? 0x1fffu : 0xffffu);
    uint32_t* w;              // this lane's word 0
    uint16_t* jr16;           // wide format: this lane's rank array
    uint8_t* jr8;             // mid format: this lane's array of rank bits 4..0
    uint32_t NL;              // lanes of this warp: slot e's word is w[e * NL]
    uint32_t lim, h;          // k + 1 (sentinel B, the largest slot) and h: debug checks only
    __device__ __forceinline__ uint32_t ld(uint32_t e) const { return w[e * NL]; }
    // x as a slot; the debug build clamps a value that is not one into range
    __device__ __forceinline__ uint32_t cl(uint32_t x, uint32_t site) const
    {
        return MF_CHECK(x <= lim, site, x) ? x : lim;
    }
    __device__ __forceinline__ void st(uint32_t e, uint32_t v) const { w[e * NL] = v; }
    __device__ __forceinline__ void xr(uint32_t e, uint32_t v) const { atomicXor(&w[e * NL], v); }
    // relinks: next(e) <- v (old value `old`), prev(e) <- v
    __device__ __forceinline__ void set_next(uint32_t e, uint32_t v, uint32_t old) const {
        if (PACKED || MID) xr(e, v ^ old);
        else reinterpret_cast<uint16_t*>(w)[e * 2 * NL] = (uint16_t)v;
    }
    __device__ __forceinline__ void set_prev(uint32_t e, uint32_t v, uint32_t old) const {
        if (PACKED || MID) xr(e, (v ^ old) << PSH);
        else reinterpret_cast<uint16_t*>(w)[e * 2 * NL + 1] = (uint16_t)v;
    }
    __device__ __forceinline__ uint16_t& JR(uint32_t e) const { return jr16[(e >> 1) * 2 * NL + (e & 1)]; }
    __device__ __forceinline__ uint8_t& JB(uint32_t e) const { return jr8[(e >> 2) * 4 * NL + (e & 3)]; }
    __device__ __forceinline__ static uint32_t nxt(uint32_t v) { return v & FM; }
    __device__ __forceinline__ static uint32_t prv(uint32_t v) { return (v >> PSH) & FM; }
    // rank of slot e whose word is v
    __device__ __forceinline__ uint32_t rank(uint32_t e, uint32_t v) const {
        if (PACKED) return v >> 20;
        if (MID) return ((v >> 24) << 5) | (uint32_t)JB(e);
        return JR(e);
    }
    // the part of slot e's rank that is not in its word (mid, wide)
    __device__ __forceinline__ void set_rank(uint32_t e, uint32_t r) const {
        if (MID) JB(e) = (uint8_t)(r & 31u);
        else if (!PACKED) JR(e) = (uint16_t)r;
    }
    __device__ __forceinline__ static uint32_t make(uint32_t prev, uint32_t next, uint32_t r) {
        return PACKED ? (next | (prev << 10) | (r << 20))
                      : (MID ? (next | (prev << 12) | ((r >> 5) << 24)) : (next | (prev << 16)));
    }
};

// State of the two block data structures (Section 5.3): m, its list word,
// its joint rank, and s.
struct PairState {
    uint32_t mA, wmA, rmA;
    uint32_t mB, wmB, rmB;
    int sA;                   // s_B = h - s_A at every step boundary
};

// One step i of the post-processing (Section 6.2): delete(A, i), undelete(B,
// i), advance if s_A + s_B < h, and the printed node (isB << 15 | slot) of
// min(peek A, peek B).  wa is slot i's current word (loaded by the step
// before); the next step's word comes back in *wnext.  B's position i comes
// with the links pb / nb that unwind(B) left it and its joint rank rb; wbw is
// its list word make(pb, nb, rb).
//
// Every node a step can move an m pointer to is m_A, m_B or one of their
// neighbours at the start of the step (Section 5.3: delete moves m to
// prev(m), or to a neighbour of i when i = m, and then the next node after
// it; undelete moves m to prev(m), which is i itself when i is relinked just
// before m; advance moves m to next(m)).  So the step first does its unlink
// and relink (equations del / undo-del of Section 4), then loads the words of
// m_A, m_B, their neighbours at the start of the step and slot i + 1 (the next
// step's A node): the loads see the new links, and their addresses depend
// only on the state at the start of the step, so they form a single level and
// the selects that follow need no second load.  (When i = m_A, slot i already
// holds B's word; the selects do not use m_A's word then.)
__device__ __forceinline__ uint32_t pair_step_packed(PairState& st, const Lists<kFmtPacked>& L,
                                                     uint32_t i, uint32_t wa, uint32_t wbw,
                                                     uint32_t* wnext)
{
    using LL = Lists<kFmtPacked>;
    const uint32_t pm = L.cl(LL::prv(st.wmA), 201), nm = L.cl(LL::nxt(st.wmA), 201);
    const uint32_t pmB = L.cl(LL::prv(st.wmB), 201), nmB = L.cl(LL::nxt(st.wmB), 201);
    // -------- relinks: delete(A, i), undelete(B, i) --------------------------------
    const uint32_t pa = L.cl(LL::prv(wa), 201), na = L.cl(LL::nxt(wa), 201), ra = wa >> 20;
    const uint32_t pb = L.cl(LL::prv(wbw), 201), nb = L.cl(LL::nxt(wbw), 201), rb = wbw >> 20;
    L.xr(pa, na ^ i);                                   // next[prev[i]] <- next[i]
    L.xr(na, (pa ^ i) << 10);                           // prev[next[i]] <- prev[i]
    L.st(i, wbw);
    L.xr(pb, nb ^ i);                                   // next[prev[i]] <- i
    L.xr(nb, (pb ^ i) << 10);                           // prev[next[i]] <- i
    // -------- the candidates' words, after the relinks ------------------------
    const uint32_t wmA = L.ld(L.cl(st.mA, 202)), wpm = L.ld(pm), wnm = L.ld(nm);
    const uint32_t wmB = L.ld(L.cl(st.mB, 202)), wpmB = L.ld(pmB), wnmB = L.ld(nmB);
    *wnext = L.ld(i + 1);
    // -------- delete(A, i): the m pointer and s -----------------------------------
    const bool small = ra < st.rmA;                     // alpha[i] small (or m at the end)
    const bool isM = i == st.mA;
    const bool sApos = st.sA > 0;
    const bool toP = !small && sApos, toN = !small && !sApos && isM;
    const uint32_t mA1 = toP ? pm : (toN ? nm : st.mA);
    const uint32_t wA1 = toP ? wpm : (toN ? wnm : wmA);
    st.sA -= (small || sApos) ? 1 : 0;                  // s <- max(0, s - 1)
    const bool nxtOld = toP && !isM;
    const uint32_t aNode = nxtOld ? st.mA : nm, aWord = nxtOld ? wmA : wnm;
    // -------- undelete(B, i): the m pointer ---------------------------------------
    const bool smallB = rb < st.rmB;                    // small: m <- prev[m]
    const bool justB = nb == st.mB;                     // i relinked just before m
    const uint32_t mB1 = smallB ? (justB ? i : pmB) : st.mB;
    const uint32_t wB1 = smallB ? (justB ? wbw : wpmB) : wmB;
    const bool afterB = pb == st.mB;
    const uint32_t bNode = smallB ? st.mB : (afterB ? i : nmB);
    const uint32_t bWord = smallB ? wmB : (afterB ? wbw : wnmB);
    // -------- advance the list whose first large element is smaller -----------
    const bool aA = (wA1 >> 20) < (wB1 >> 20);          // peek(A) <= peek(B): A first on ties
    const bool advA = sApos && aA, advB = sApos && !aA;
    st.mA = advA ? aNode : mA1;
    st.wmA = advA ? aWord : wA1;
    st.mB = advB ? bNode : mB1;
    st.wmB = advB ? bWord : wB1;
    st.rmA = st.wmA >> 20;
    st.rmB = st.wmB >> 20;
    st.sA += advA ? 1 : 0;
    // -------- print min(peek(A), peek(B)) ------------------------------------
    return st.rmA < st.rmB ? st.mA : (0x8000u | st.mB);
}

// The one-level step of pair_step_packed for the mid and wide formats, whose
// ranks live (partly) outside the word: after the unlink and relink, the
// words of m_A, m_B, their neighbours at the start of the step and slot
// i + 1 are loaded together with the side-array ranks of the neighbours and
// of slot i + 1 (the m pointers' own ranks do not change: only slot i changes
// owner).  ra is slot i's rank, loaded by the step before with its word.
template <int FMT>
__device__ __forceinline__ uint32_t pair_step_after(PairState& st, const Lists<FMT>& L, uint32_t i,
                                                    uint32_t wa, uint32_t ra, uint32_t pb, uint32_t nb,
                                                    uint32_t rb, uint32_t* wnext, uint32_t* rnext)
{
    using LL = Lists<FMT>;
    const uint32_t pm = L.cl(LL::prv(st.wmA), 201), nm = L.cl(LL::nxt(st.wmA), 201);
    const uint32_t pmB = L.cl(LL::prv(st.wmB), 201), nmB = L.cl(LL::nxt(st.wmB), 201);
    pb = L.cl(pb, 201);
    nb = L.cl(nb, 201);
    // -------- relinks: delete(A, i), undelete(B, i) --------------------------------
    const uint32_t pa = L.cl(LL::prv(wa), 201), na = L.cl(LL::nxt(wa), 201);
    const uint32_t wbw = LL::make(pb, nb, rb);
    L.set_next(pa, na, i);                              // next[prev[i]] <- next[i]
    L.set_prev(na, pa, i);                              // prev[next[i]] <- prev[i]
    L.st(i, wbw);
    L.set_rank(i, rb);
    L.set_next(pb, i, nb);                              // next[prev[i]] <- i
    L.set_prev(nb, i, pb);                              // prev[next[i]] <- i
    // -------- the candidates' words and ranks, after the relinks -----------------
    const uint32_t wmA = L.ld(L.cl(st.mA, 202)), wpm = L.ld(pm), wnm = L.ld(nm);
    const uint32_t wmB = L.ld(L.cl(st.mB, 202)), wpmB = L.ld(pmB), wnmB = L.ld(nmB);
    const uint32_t wn = L.ld(i + 1);
    const uint32_t rpm = L.rank(pm, wpm), rnm = L.rank(nm, wnm);
    const uint32_t rpmB = L.rank(pmB, wpmB), rnmB = L.rank(nmB, wnmB);
    *wnext = wn;
    *rnext = L.rank(i + 1, wn);
    // -------- delete(A, i): the m pointer and s -----------------------------------
    const bool small = ra < st.rmA;                     // alpha[i] small (or m at the end)
    const bool isM = i == st.mA;
    const bool sApos = st.sA > 0;
    const bool toP = !small && sApos, toN = !small && !sApos && isM;
    const uint32_t mA1 = toP ? pm : (toN ? nm : st.mA);
    const uint32_t wA1 = toP ? wpm : (toN ? wnm : wmA);
    const uint32_t rA1 = toP ? rpm : (toN ? rnm : st.rmA);
    st.sA -= (small || sApos) ? 1 : 0;                  // s <- max(0, s - 1)
    const bool nxtOld = toP && !isM;
    const uint32_t aNode = nxtOld ? st.mA : nm, aWord = nxtOld ? wmA : wnm;
    const uint32_t aRank = nxtOld ? st.rmA : rnm;
    // -------- undelete(B, i): the m pointer ---------------------------------------
    const bool smallB = rb < st.rmB;                    // small: m <- prev[m]
    const bool justB = nb == st.mB;                     // i relinked just before m
    const uint32_t mB1 = smallB ? (justB ? i : pmB) : st.mB;
    const uint32_t wB1 = smallB ? (justB ? wbw : wpmB) : wmB;
    const uint32_t rB1 = smallB ? (justB ? rb : rpmB) : st.rmB;
    const bool afterB = pb == st.mB;
    const uint32_t bNode = smallB ? st.mB : (afterB ? i : nmB);
    const uint32_t bWord = smallB ? wmB : (afterB ? wbw : wnmB);
    const uint32_t bRank = smallB ? st.rmB : (afterB ? rb : rnmB);
    // -------- advance the list whose first large element is smaller -----------
    const bool aA = rA1 < rB1;                          // peek(A) <= peek(B): A first on ties
    const bool advA = sApos && aA, advB = sApos && !aA;
    st.mA = advA ? aNode : mA1;
    st.wmA = advA ? aWord : wA1;
    st.rmA = advA ? aRank : rA1;
    st.mB = advB ? bNode : mB1;
    st.wmB = advB ? bWord : wB1;
    st.rmB = advB ? bRank : rB1;
    st.sA += advA ? 1 : 0;
    // -------- print min(peek(A), peek(B)) ------------------------------------
    return st.rmA < st.rmB ? st.mA : (0x8000u | st.mB);
}

// Debug build: the state after a step satisfies Section 5's invariants: 0 <=
// s_A <= h, m_A and m_B are live nodes of their lists (next(prev(m)) = m) whose
// cached words are current, and the printed node is an element, not a
// sentinel.
template <int FMT>
__device__ __forceinline__ void check_state(const PairState& st, const Lists<FMT>& L, uint32_t out)
{
#ifdef MF_DEBUG
    using LL = Lists<FMT>;
    (void)MF_CHECK(st.sA >= 0 && (uint32_t)st.sA <= L.h, 203, st.sA);
    (void)MF_CHECK(L.ld(L.cl(st.mA, 202)) == st.wmA &&
                   LL::nxt(L.ld(L.cl(LL::prv(st.wmA), 201))) == st.mA, 204, st.mA);
    (void)MF_CHECK(L.ld(L.cl(st.mB, 202)) == st.wmB &&
                   LL::nxt(L.ld(L.cl(LL::prv(st.wmB), 201))) == st.mB, 205, st.mB);
    (void)MF_CHECK((out & 0x7fffu) + 1u < L.lim, 206, out);
#endif
}

template <int FMT>
__device__ __forceinline__ void chain_body(const PipeParams& p, uint32_t* wsl, int lane, int64_t q,
                                           uint32_t rec_words, uint32_t NL, bool copy)
{
    using LL = Lists<FMT>;
    constexpr bool PACKED = LL::PACKED;
    const int k = p.k, h = p.h;
    const int NB = (int)min((int64_t)k, p.n - (q + 1) * (int64_t)k);
    LL L;
    L.w = wsl + lane;
    L.jr16 = reinterpret_cast<uint16_t*>(wsl + rec_words * NL + lane);
    L.jr8 = reinterpret_cast<uint8_t*>(wsl + rec_words * NL + lane);
    L.NL = NL;
    L.lim = (uint32_t)k + 1u;
    L.h = (uint32_t)h;

    // ---- construct(A) in slot space + empty B (rows of kp elements) ----------
    const size_t abase = (size_t)q * p.kp;              // block j-1 = q
    const size_t bbase = (size_t)(q + 1) * p.kp;
    const uint4* sl4 = reinterpret_cast<const uint4*>(p.slink + abase);
    const uint4* ja4 = reinterpret_cast<const uint4*>(p.ja + abase);
    const int nchunk = copy ? p.kp >> 3 : 0;            // else copy_lists built slots 0 .. k-1
#pragma unroll 4
    for (int c = 0; c < nchunk; ++c) {
        const uint4 s0 = __ldg(sl4 + 2 * c), s1 = __ldg(sl4 + 2 * c + 1), jv = __ldg(ja4 + c);
        const uint32_t sv[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
        const uint32_t jw[4] = {jv.x, jv.y, jv.z, jv.w};
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int e = 8 * c + t;
            if (e < k) {
                const uint32_t r = t & 1 ? jw[t >> 1] >> 16 : jw[t >> 1] & 0xffffu;
                L.st(e, LL::make(sv[t] >> 16, sv[t] & 0xffffu, r));
                if (!PACKED) L.set_rank(e, r);
            }
        }
    }
    const uint32_t SA = (uint32_t)k, SB = (uint32_t)k + 1;
    const uint16_t* permA = p.perm + abase;                     // block j-1 = q
    L.st(SA, LL::make(__ldg(permA + k - 1), __ldg(permA), LL::RINF));
    L.st(SB, LL::make(SB, SB, LL::RINF));
    if (!PACKED) { L.set_rank(SA, LL::RINF); L.set_rank(SB, LL::RINF); }

    PairState st;
    st.mA = __ldg(permA + h);
    st.wmA = L.ld(st.mA);
    st.rmA = L.rank(st.mA, st.wmA);
    st.sA = h;
    st.mB = SB;
    st.wmB = L.ld(SB);
    st.rmB = LL::RINF;

    // ---- the k steps, 8 at a time; inputs of the next two chunks in flight ---
    const uint4* ul4 = reinterpret_cast<const uint4*>(p.ulink + bbase);
    const uint4* jb4 = reinterpret_cast<const uint4*>(p.jb + (size_t)q * p.kp);
    uint4* out4 = reinterpret_cast<uint4*>(p.out + (size_t)q * p.kp);
    const int nch = (NB + 7) >> 3;
    uint4 u0 = __ldg(ul4), u1 = __ldg(ul4 + 1), jv = __ldg(jb4);
    uint4 v0 = u0, v1 = u1, kv = jv;
    if (nch > 1) { v0 = __ldg(ul4 + 2); v1 = __ldg(ul4 + 3); kv = __ldg(jb4 + 1); }
    uint32_t wa = L.ld(0);
    uint32_t ra = L.rank(0, wa);
    for (int c = 0; c < nch; ++c) {
        uint4 x0 = v0, x1 = v1, xv = kv;
        if (c + 2 < nch) {
            x0 = __ldg(ul4 + 2 * (c + 2));
            x1 = __ldg(ul4 + 2 * (c + 2) + 1);
            xv = __ldg(jb4 + (c + 2));
        }
        const uint32_t wbv[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
        const uint32_t jw[4] = {jv.x, jv.y, jv.z, jv.w};
        uint32_t ov[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int i = 8 * c + t;
            if (i < NB) {
                const uint32_t rb = t & 1 ? jw[t >> 1] >> 16 : jw[t >> 1] & 0xffffu;
                uint32_t wn;
                const uint32_t pb = wbv[t] >> 16, nb = wbv[t] & 0xffffu;
                uint32_t o;
                if constexpr (PACKED) {
                    o = pair_step_packed(st, L, (uint32_t)i, wa, LL::make(pb, nb, rb), &wn);
                } else {
                    uint32_t rn;
                    o = pair_step_after<FMT>(st, L, (uint32_t)i, wa, ra, pb, nb, rb, &wn, &rn);
                    ra = rn;
                }
                check_state(st, L, o);
                wa = wn;
                ov[t >> 1] |= (t & 1) ? (o << 16) : o;
            }
        }
        out4[c] = make_uint4(ov[0], ov[1], ov[2], ov[3]);
        u0 = v0; u1 = v1; jv = kv;
        v0 = x0; v1 = x1; kv = xv;
    }
}

// Fused path (sortlist_kernel wrote the words): construct(A) is a copy of the
// pair's row of list words (slots 0..k+1, m_A in slot k+2), made by the lane
// itself (copy) or beforehand by copy_rows for all the CTA's pairs; step i
// undeletes B's position i with the word wB[i] = make(pb, nb, rb).  Packed
// format only.
//
// copy_rows: all threads of the CTA copy the rows, 16 bytes at a time and 16
// loads in flight per thread, into the lanes' bank-private slices.  info[s]
// describes slot s = pair_off + lane: row address, words (k + 2, 0 for an
// idle slot), lanes of its warp and the slice's word 0.
__device__ __forceinline__ void copy_rows(const uint4* info, int nslots, int maxch, uint32_t* words)
{
    // chunk-major order: a warp's threads take the same chunk of consecutive
    // slots, whose words sit in distinct banks
    const int nthr = blockDim.x, total = nslots * maxch;
    int c = (int)threadIdx.x / nslots, s = (int)threadIdx.x - c * nslots;
    const int dc = nthr / nslots, ds = nthr - dc * nslots;
    for (int c0 = threadIdx.x; c0 < total; c0 += 16 * nthr) {
        uint4 v[16];
        uint32_t dst[16], meta[16];                     // meta: lanes | words of the chunk << 8
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            meta[u] = 0u;
            dst[u] = 0u;
            v[u] = make_uint4(0u, 0u, 0u, 0u);
            if (c0 + u * nthr < total) {
                const uint4 in = info[s];
                const int nw = (int)(in.z & 0xffffu);
                if (4 * c < nw) {
                    const uint4* src = reinterpret_cast<const uint4*>(((uint64_t)in.y << 32) | in.x);
                    const uint32_t nl = in.z >> 16;
                    v[u] = __ldg(src + c);
                    dst[u] = in.w + 4u * (uint32_t)c * nl;
                    meta[u] = nl | (uint32_t)min(4, nw - 4 * c) << 8;
                }
            }
            s += ds;
            c += dc;
            if (s >= nslots) { s -= nslots; ++c; }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const uint32_t nl = meta[u] & 0xffu, cnt = meta[u] >> 8;
            uint32_t* d = words + dst[u];
            if (cnt > 0) d[0] = v[u].x;
            if (cnt > 1) d[nl] = v[u].y;
            if (cnt > 2) d[2 * nl] = v[u].z;
            if (cnt > 3) d[3 * nl] = v[u].w;
        }
    }
}
__device__ __forceinline__ void chain_body_words(const PipeParams& p, uint32_t* wsl, int lane,
                                                 int64_t q, uint32_t NL, bool copy)
{
    using LL = Lists<kFmtPacked>;
    const int k = p.k, h = p.h;
    const int NB = (int)min((int64_t)k, p.n - (q + 1) * (int64_t)k);
    LL L;
    L.w = wsl + lane;
    L.jr16 = nullptr;
    L.NL = NL;
    L.lim = (uint32_t)k + 1u;
    L.h = (uint32_t)h;
    if (copy) {
        // slots 0 .. k+1 by this lane: 16 loads of 16 bytes in flight, then their stores
        const uint4* wa4 = reinterpret_cast<const uint4*>(p.wA + (size_t)q * p.kw);
        const int nrec = (k + 2 + 3) >> 2;
        for (int c0 = 0; c0 < nrec; c0 += 16) {
            uint4 v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = c0 + u < nrec ? __ldg(wa4 + c0 + u) : make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const uint32_t vv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int e = 4 * (c0 + u) + t;
                    if (e < k + 2) L.st(e, vv[t]);
                }
            }
        }
    }
    PairState st;
    st.mA = __ldg(p.wA + (size_t)q * p.kw + k + 2);
    st.wmA = L.ld(st.mA);
    st.rmA = st.wmA >> 20;
    st.sA = h;
    st.mB = (uint32_t)k + 1;
    st.wmB = L.ld(st.mB);
    st.rmB = LL::RINF;

    // ---- the k steps, 8 at a time; B words of the next two chunks in flight ---
    const uint4* wb4 = reinterpret_cast<const uint4*>(p.wB + (size_t)q * p.kw);
    uint4* out4 = reinterpret_cast<uint4*>(p.out + (size_t)q * p.kp);
    const int nch = (NB + 7) >> 3;
    uint4 u0 = __ldg(wb4), u1 = __ldg(wb4 + 1);
    uint4 v0 = u0, v1 = u1;
    if (nch > 1) { v0 = __ldg(wb4 + 2); v1 = __ldg(wb4 + 3); }
    uint32_t wa = L.ld(0);
    for (int c = 0; c < nch; ++c) {
        uint4 x0 = v0, x1 = v1;
        if (c + 2 < nch) {
            x0 = __ldg(wb4 + 2 * (c + 2));
            x1 = __ldg(wb4 + 2 * (c + 2) + 1);
        }
        const uint32_t wbv[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
        uint32_t ov[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int i = 8 * c + t;
            if (i < NB) {
                const uint32_t w = wbv[t];
                uint32_t wn;
                const uint32_t o = pair_step_packed(st, L, (uint32_t)i, wa, w, &wn);
                check_state(st, L, o);
                wa = wn;
                ov[t >> 1] |= (t & 1) ? (o << 16) : o;
            }
        }
        out4[c] = make_uint4(ov[0], ov[1], ov[2], ov[3]);
        u0 = v0; u1 = v1;
        v0 = x0; v1 = x1;
    }
}

// copy_lists: construct(A) of the four-kernel path for all the CTA's pairs at
// once, slots 0 .. k-1 from the sorted-order links (prev:16 | next:16) and
// joint ranks of block A, 8 slots per chunk, chunk-major like copy_rows.
// info[2s] = slink row, ja row; info[2s+1] = k (0: idle) | lanes << 16, the
// slice's word 0, the slice's rank word 0.
template <int FMT>
__device__ __forceinline__ void copy_lists(const uint4* info, int nslots, int maxch, uint32_t* words)
{
    using LL = Lists<FMT>;
    const int nthr = blockDim.x, total = nslots * maxch;
    int c = (int)threadIdx.x / nslots, s = (int)threadIdx.x - c * nslots;
    const int dc = nthr / nslots, ds = nthr - dc * nslots;
    for (int c0 = threadIdx.x; c0 < total; c0 += 8 * nthr) {
        uint4 a[8], b[8], r[8];
        uint32_t cnt[8], nl[8], dw[8], dr[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            cnt[u] = 0u; nl[u] = 0u; dw[u] = 0u; dr[u] = 0u;
            a[u] = b[u] = r[u] = make_uint4(0u, 0u, 0u, 0u);
            if (c0 + u * nthr < total) {
                const uint4 d = info[2 * s + 1];
                const int k = (int)(d.x & 0xffffu);
                if (8 * c < k) {
                    const uint4 rows = info[2 * s];
                    const uint4* sl4 = reinterpret_cast<const uint4*>(((uint64_t)rows.y << 32) | rows.x);
                    const uint4* ja4 = reinterpret_cast<const uint4*>(((uint64_t)rows.w << 32) | rows.z);
                    a[u] = __ldg(sl4 + 2 * c);
                    b[u] = __ldg(sl4 + 2 * c + 1);
                    r[u] = __ldg(ja4 + c);
                    cnt[u] = (uint32_t)min(8, k - 8 * c);
                    nl[u] = d.x >> 16;
                    dw[u] = d.y + 8u * (uint32_t)c * nl[u];
                    dr[u] = d.z + (LL::MID ? 2u : 4u) * (uint32_t)c * nl[u];
                }
            }
            s += ds;
            c += dc;
            if (s >= nslots) { s -= nslots; ++c; }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t sv[8] = {a[u].x, a[u].y, a[u].z, a[u].w, b[u].x, b[u].y, b[u].z, b[u].w};
            const uint32_t jw[4] = {r[u].x, r[u].y, r[u].z, r[u].w};
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                if ((uint32_t)t < cnt[u]) {
                    const uint32_t rk = t & 1 ? jw[t >> 1] >> 16 : jw[t >> 1] & 0xffffu;
                    words[dw[u] + (uint32_t)t * nl[u]] = LL::make(sv[t] >> 16, sv[t] & 0xffffu, rk);
                }
            }
            if (LL::MID) {
                // rank bits 4..0: four slots per word; word j holds slots 4j .. 4j+3 of the chunk
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const uint32_t lo = jw[2 * j], hi = jw[2 * j + 1];
                    const uint32_t bytes = (lo & 31u) | (((lo >> 16) & 31u) << 8) |
                                           ((hi & 31u) << 16) | (((hi >> 16) & 31u) << 24);
                    if ((uint32_t)(4 * j) < cnt[u]) words[dr[u] + (uint32_t)j * nl[u]] = bytes;
                }
            } else if (!LL::PACKED) {
                // rank words: two slots each; word j holds slots 2j, 2j+1 of the chunk
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if ((uint32_t)(2 * j) < cnt[u]) words[dr[u] + (uint32_t)j * nl[u]] = jw[j];
            }
        }
    }
}

// Classes whose largest k is above this copy the rows with copy_rows (GB300,
// n = 2^26, k = 1001: chain 1.13 -> 1.02 ms); below it the CTA barrier cost
// more than it saved (k <= 64 in the 4096-signal batch: 0.70 -> 0.93 ms).
constexpr int kCoopCopyMinK = 256;

template <int FMT, bool WORDS>
__global__ void __launch_bounds__(kPipeThreads)
chain_kernel(SegTable tab, ChainPlan cp)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // warp w has 1 << ((lanes_log2 >> 3w) & 7) lanes; slices follow each other;
    // warps past nwarps only help the CTA-wide construct (copy_rows, copy_lists)
    int NL = 0, pair_off = 0;
    for (int w = 0; w <= warp && w < cp.nwarps; ++w) {
        const int l = 1 << ((cp.lanes_log2 >> (3 * w)) & 7);
        if (w < warp) pair_off += l; else NL = l;
    }
    const int64_t item = (int64_t)blockIdx.x * cp.pairs_per_cta + pair_off + lane;
    uint32_t* wsl = reinterpret_cast<uint32_t*>(smem) + (uint32_t)pair_off * cp.lane_words;
    if (WORDS && cp.rec_words <= kCoopCopyMinK + 2) {
        // short rows: each lane copies its own (no CTA barrier)
        if (lane >= NL || item >= cp.items) return;
        int64_t q;
        const PipeParams p = find_signal(tab, kItemChain, item, &q);
        chain_body_words(p, wsl, lane, q, (uint32_t)NL, true);
        return;
    }
    if (WORDS) {
        uint4* info = reinterpret_cast<uint4*>(smem + cp.info_off);
        const bool act = lane < NL && item < cp.items;
        int64_t q = 0;
        PipeParams p;
        if (act) {
            p = find_signal(tab, kItemChain, item, &q);
            const uint64_t src = (uint64_t)(uintptr_t)(p.wA + (size_t)q * p.kw);
            info[pair_off + lane] = make_uint4((uint32_t)src, (uint32_t)(src >> 32),
                                               (uint32_t)(p.k + 2) | ((uint32_t)NL << 16),
                                               (uint32_t)pair_off * cp.lane_words + (uint32_t)lane);
        } else if (lane < NL) {
            info[pair_off + lane] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        copy_rows(info, cp.pairs_per_cta, (int)(cp.rec_words + 3) >> 2, reinterpret_cast<uint32_t*>(smem));
        __syncthreads();
        if (act) chain_body_words(p, wsl, lane, q, (uint32_t)NL, false);
        return;
    }
    if (cp.rec_words <= kCoopCopyMinK + 2) {
        if (lane >= NL || item >= cp.items) return;
        int64_t q;                                      // pair j = q + 1 of its signal
        const PipeParams p = find_signal(tab, kItemChain, item, &q);
        chain_body<FMT>(p, wsl, lane, q, cp.rec_words, (uint32_t)NL, true);
        return;
    }
    uint4* info = reinterpret_cast<uint4*>(smem + cp.info_off);
    const bool act = lane < NL && item < cp.items;
    int64_t q = 0;
    PipeParams p;
    if (act) {
        p = find_signal(tab, kItemChain, item, &q);
        const uint64_t sl = (uint64_t)(uintptr_t)(p.slink + (size_t)q * p.kp);
        const uint64_t ja = (uint64_t)(uintptr_t)(p.ja + (size_t)q * p.kp);
        const uint32_t w0 = (uint32_t)pair_off * cp.lane_words + (uint32_t)lane;
        info[2 * (pair_off + lane)] = make_uint4((uint32_t)sl, (uint32_t)(sl >> 32), (uint32_t)ja, (uint32_t)(ja >> 32));
        info[2 * (pair_off + lane) + 1] = make_uint4((uint32_t)p.k | ((uint32_t)NL << 16), w0,
                                                     w0 + cp.rec_words * (uint32_t)NL, 0u);
    } else if (lane < NL) {
        info[2 * (pair_off + lane) + 1] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    copy_lists<FMT>(info, cp.pairs_per_cta, (int)(cp.rec_words - 2 + 7) >> 3, reinterpret_cast<uint32_t*>(smem));
    __syncthreads();
    if (act) chain_body<FMT>(p, wsl, lane, q, cp.rec_words, (uint32_t)NL, false);
}

// ===========================================================================
// epilogue_kernel: y[(j-1)k + 1 + i] = the element printed at step i of pair
// j, read from a shared-memory copy of the CTA's input span; y[0] = X_0[P_0[h]].
// ===========================================================================
template <typename ValT>
__global__ void __launch_bounds__(kPipeThreads)
epilogue_kernel(SegTable tab)
{
    extern __shared__ __align__(16) unsigned char smem[];
    ValT* xs = reinterpret_cast<ValT*>(smem);
    int64_t cta;
    const PipeParams p = find_signal(tab, kItemEpilogue, blockIdx.x, &cta);
    const int k = p.k, G = p.eG;
    const int64_t j0 = 1 + cta * G;
    const int64_t left = p.npairs - (j0 - 1);
    const int npair = (int)(left < G ? (left > 0 ? left : 0) : G);
    const int64_t ebase = (j0 - 1) * (int64_t)k;
    const int64_t rem = p.n - ebase;
    const int E = (int)((int64_t)(npair + 1) * k < rem ? (int64_t)(npair + 1) * k : rem);
    const ValT* xp = reinterpret_cast<const ValT*>(p.x);
    {
        // the span as 32-bit words: its 16-byte-aligned interior as uint4, the
        // ragged ends one by one
        const int Ew = E * (int)(sizeof(ValT) / 4);
        const uint32_t* xs4 = reinterpret_cast<const uint32_t*>(xp + ebase);
        uint32_t* xd = reinterpret_cast<uint32_t*>(xs);
        const int head = min(Ew, (int)(((16u - ((uint32_t)(uintptr_t)xs4 & 15u)) & 15u) >> 2));
        const int nvec = (Ew - head) >> 2;
        const int tail0 = head + 4 * nvec;
        const uint4* xv = reinterpret_cast<const uint4*>(xs4 + head);
        for (int c0 = threadIdx.x; c0 < nvec; c0 += 4 * blockDim.x) {
            uint4 r[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = c0 + u * (int)blockDim.x;
                r[u] = c < nvec ? __ldg(xv + c) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = c0 + u * (int)blockDim.x;
                if (c < nvec) {
                    uint32_t* d = xd + head + 4 * c;
                    d[0] = r[u].x; d[1] = r[u].y; d[2] = r[u].z; d[3] = r[u].w;
                }
            }
        }
        if ((int)threadIdx.x < head) xd[threadIdx.x] = __ldg(xs4 + threadIdx.x);
        if ((int)threadIdx.x < Ew - tail0) xd[tail0 + threadIdx.x] = __ldg(xs4 + tail0 + threadIdx.x);
    }
    __syncthreads();
    const int nout = npair > 0 ? E - k : 0;
    ValT* ys = reinterpret_cast<ValT*>(p.y) + ebase + 1;
    int32_t* as = p.argmed ? p.argmed + ebase + 1 : nullptr;
    const uint16_t* outs = p.out + (size_t)(j0 - 1) * p.kp;
    const int stride = blockDim.x;
    if (k >= 512) {
        // pair by pair (outputs g*k .. g*k + NB - 1 of this CTA); four outputs
        // per thread per round: loads first, then lookups and stores
        for (int g = 0, gk = 0; gk < nout; ++g, gk += k) {
            const int cnt = min(k, nout - gk);
            const uint16_t* og = outs + (size_t)g * p.kp;
            for (int i0 = threadIdx.x; i0 < cnt; i0 += 4 * stride) {
                uint32_t id[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * stride;
                    id[u] = i < cnt ? (uint32_t)og[i] : 0u;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + u * stride;
                    if (i < cnt) {
                        int e = gk + (int)(id[u] >> 15) * k + (int)(id[u] & 0x7fffu);
                        if (!MF_CHECK(e >= 0 && e < E, 207, e)) e = 0;
                        ys[gk + i] = xs[e];
                        if (as) as[gk + i] = (int32_t)(ebase + e);
                    }
                }
            }
        }
    } else {
        // small windows: all outputs of the CTA at once (output o = step i of
        // pair g, o = g k + i; g by an exact multiply-shift, o k < 2^32)
        const uint64_t kmg = ((1ull << 32) + (uint64_t)k - 1) / (uint64_t)k;
        for (int o0 = threadIdx.x; o0 < nout; o0 += 4 * stride) {
            uint32_t id[4];
            int gk[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int o = o0 + u * stride;
                const int g = (int)(((uint64_t)(uint32_t)o * kmg) >> 32);
                gk[u] = g * k;
                id[u] = o < nout ? (uint32_t)outs[(size_t)g * p.kp + (o - gk[u])] : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int o = o0 + u * stride;
                if (o < nout) {
                    int e = gk[u] + (int)(id[u] >> 15) * k + (int)(id[u] & 0x7fffu);
                    if (!MF_CHECK(e >= 0 && e < E, 207, e)) e = 0;
                    ys[o] = xs[e];
                    if (as) as[o] = (int32_t)(ebase + e);
                }
            }
        }
    }
    if (j0 == 1 && threadIdx.x == 0) {
        const int pm = p.wA ? (int)p.wA[k + 2] : (int)p.perm[p.h];     // P_0[h]
        reinterpret_cast<ValT*>(p.y)[0] = xs[pm];
        if (p.argmed) p.argmed[0] = pm;
    }
}

// ===========================================================================
// host side
// ===========================================================================
static inline uint64_t al16(uint64_t v) { return (v + 15) & ~uint64_t(15); }
static inline uint64_t al256(uint64_t v) { return (v + 255) & ~uint64_t(255); }

static bool sort_plan(int k, int G, SortPlan* sp, size_t* bytes, bool wide)
{
    const int W = kPipeThreads / 32;
    const uint64_t E = (uint64_t)(G + 1) * k;
    const uint64_t kb = wide ? 8 : 4;
    if (E > 65535) return false;
    uint64_t off = 0;
    sp->off_keyA = (uint32_t)off; off = al16(off + kb * E);
    sp->off_keyB = (uint32_t)off; off = al16(off + kb * E);
    sp->off_valA = (uint32_t)off; off = al16(off + 2 * E);
    sp->off_valB = (uint32_t)off; off = al16(off + 2 * E);
    sp->off_hist = (uint32_t)off; off = al16(off + 1024ull * W);
    *bytes = off;
    return off <= (uint64_t)kMaxSmemBytes;
}

// Chain plan: per-lane words (k+2 list words, plus k/2+2 rank words when
// not packed); warps are added greedily, each with the most lanes (32, 16,
// ..., 1; a power of two keeps the layout bank-conflict free) that still fit.
// One CTA per SM: on GB300 at k = 1001 (n = 2^26) two CTAs of 28 pairs took
// 1.37 ms against 1.14 ms for one CTA of 57 pairs.
static bool chain_plan(int k, ChainPlan* cp, size_t* bytes)
{
    cp->fmt = k <= kFusedMaxK ? kFmtPacked : (k <= kMidMaxK ? kFmtMid : kFmtWide);
    cp->rec_words = (uint32_t)(k + 2);
    const uint32_t side = cp->fmt == kFmtPacked ? 0u
                        : (cp->fmt == kFmtMid ? (uint32_t)((k + 2 + 3) / 4) : (uint32_t)((k + 3) / 2));
    const uint32_t lane_words = cp->rec_words + side;
    cp->lane_words = lane_words;
    const uint64_t budget = (uint64_t)kMaxSmemBytes / 4;       // words
    uint64_t used = 0;
    int nw = 0, pairs = 0;
    cp->lanes_log2 = 0;
    while (nw < kPipeThreads / 32) {
        int lg = 5;                                     // (8 words per pair: copy descriptors)
        while (lg >= 0 && used + ((uint64_t)1 << lg) * lane_words + 8ull * (pairs + (1 << lg)) + 4 > budget) --lg;
        if (lg < 0) break;
        cp->lanes_log2 |= (uint32_t)lg << (3 * nw);
        used += ((uint64_t)1 << lg) * lane_words;
        pairs += 1 << lg;
        ++nw;
        if (lg == 0) break;
    }
    cp->nwarps = nw;
    cp->pairs_per_cta = pairs;
    cp->info_off = (uint32_t)((used * 4 + 15) & ~15ull);
    *bytes = (size_t)cp->info_off + 32u * (size_t)pairs;
    return nw > 0;
}

static int compute_max_k(bool wide)
{
    // limits: sort of one pair in shared memory, 15-bit slot numbers in the
    // output ids, and a one-lane chain in shared memory
    SortPlan sp;
    size_t b;
    int lo = 1, hi = 32765;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        ChainPlan cp;
        size_t cb;
        if (sort_plan(mid, 1, &sp, &b, wide) && chain_plan(mid, &cp, &cb)) lo = mid; else hi = mid - 1;
    }
    return lo;
}

int pipeline_max_k(bool wide)
{
    static const int narrow_max = compute_max_k(false), wide_max = compute_max_k(true);
    return wide ? wide_max : narrow_max;
}

// scratch of one signal: perm, rank, sorted-order links, unwind links per
// block; joint ranks of A and B and printed nodes per pair
// (four-kernel path); the fused path's rows of list words (wA, wB) and
// printed nodes need less, so one size serves both
static uint64_t signal_scratch_bytes(int64_t n, int k)
{
    const int64_t nblocks = (n + k - 1) / k;
    const int64_t npairs = nblocks - 1;
    const uint64_t kp = (uint64_t)((k + 7) & ~7);
    const uint64_t kw = (uint64_t)((k + 3 + 7) & ~7);
    const uint64_t np1 = (uint64_t)(npairs > 0 ? npairs : 1);
    const uint64_t four = al256(2ull * nblocks * kp) * 2 + al256(4ull * nblocks * kp) * 2 +
                          al256(2ull * np1 * kp) * 3;
    const uint64_t fused = al256(4ull * np1 * kw) * 2 + al256(2ull * np1 * kp);
    return four > fused ? four : fused;
}

static void carve_signal(PipeParams& p, char*& w, bool fused)
{
    const uint64_t kp = (uint64_t)p.kp;
    const uint64_t np1 = (uint64_t)(p.npairs > 0 ? p.npairs : 1);
    char* const w0 = w;
    if (fused) {
        p.kw = (p.k + 3 + 7) & ~7;
        p.wA = (uint32_t*)w;    w += al256(4ull * np1 * (uint64_t)p.kw);
        p.wB = (uint32_t*)w;    w += al256(4ull * np1 * (uint64_t)p.kw);
        p.out = (uint16_t*)w;
    } else {
        p.perm = (uint16_t*)w;  w += al256(2ull * p.nblocks * kp);
        p.rnk = (uint16_t*)w;   w += al256(2ull * p.nblocks * kp);
        p.slink = (uint32_t*)w; w += al256(4ull * p.nblocks * kp);
        p.ulink = (uint32_t*)w; w += al256(4ull * p.nblocks * kp);
        p.ja = (uint16_t*)w;    w += al256(2ull * np1 * kp);
        p.jb = (uint16_t*)w;    w += al256(2ull * np1 * kp);
        p.out = (uint16_t*)w;
    }
    w = w0 + signal_scratch_bytes(p.n, p.k);
}

static void fill_signal(PipeParams& p, const void* x, void* y, int32_t* argmed,
                        int64_t n, int k, int rank, bool is_float)
{
    p = PipeParams{};
    p.x = x; p.y = y; p.argmed = argmed;
    p.n = n; p.k = k; p.h = rank;
    p.nblocks = (n + k - 1) / k;
    p.npairs = p.nblocks - 1;
    p.kp = (k + 7) & ~7;
    p.is_float = is_float;
    p.eG = 1;
}

size_t pipeline_workspace_bytes(int64_t n, int k)
{
    return (size_t)signal_scratch_bytes(n, k);
}

size_t pipeline_batched_workspace_bytes(const int64_t* n, const int32_t* k, int nseg)
{
    uint64_t b = al256((uint64_t)nseg * sizeof(PipeParams));
    for (int s = 0; s < nseg; ++s) b += signal_scratch_bytes(n[s], k[s]);
    return (size_t)b;
}

cudaError_t pipeline_setup()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(sortmerge_kernel<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes))) return e;
    if ((e = cudaFuncSetAttribute(sortmerge_kernel<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes))) return e;
    if ((e = cudaFuncSetAttribute(epilogue_kernel<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes))) return e;
    if ((e = cudaFuncSetAttribute(unwind_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes))) return e;
    if ((e = cudaFuncSetAttribute(unwind_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes))) return e;
    if ((e = cudaFuncSetAttribute(chain_kernel<kFmtPacked, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes))) return e;
    if ((e = cudaFuncSetAttribute(chain_kernel<kFmtPacked, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes))) return e;
    if ((e = cudaFuncSetAttribute(chain_kernel<kFmtMid, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes))) return e;
    if ((e = cudaFuncSetAttribute(chain_kernel<kFmtWide, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes))) return e;
    if ((e = sortlist_setup())) return e;
    return cudaFuncSetAttribute(epilogue_kernel<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemBytes);
}

// ---------------------------------------------------------------------------
// Plans of one launch class (all signals with k <= kmax share the shared-
// memory layouts sized for kmax).
// ---------------------------------------------------------------------------
struct ClassPlan {
    int kmax;
    bool wide;                // 8-byte elements
    bool fused;               // sortlist + chain (words) + epilogue
    bool adaptive;            // fused: the sort skips tiles of ordered blocks
    int lwarps;               // fused: warps (tiles) per sortlist CTA
    int lGcap;                // fused: cap on block pairs per sortlist CTA
    SortPlan sp;  size_t sbytes;
    UnwindPlan up; size_t ubytes; int uwarps; int bpw;
    ChainPlan cp; size_t cbytes;
    int GE;       size_t ebytes;
};

// Class boundaries: the packed list format ends at k = 1021, the one-word
// unwind summary at k = 1024, the mid list format at k = 4093; smaller
// classes keep the shared-memory layouts of small k.
static const int kClassMax[] = {64, 256, 1021, 2047, kMidMaxK, 1 << 30};

// Built-in launch-plan choices per class where a measurement beat the
// capacity rule (0 = use the rule): on GB300 at k = 1001 (n = 2^26 random
// walk) 3 pairs per sort CTA took 2.28 ms against 2.39 ms for the largest
// two-per-SM G = 7, and 4 pairs per store CTA 0.21 ms against 0.26 ms for 8.
static const int kBuiltinSortG[kNumTuneClasses] = {0, 0, 3, 0, 0, 0};
static const int kBuiltinEpiG[kNumTuneClasses] = {0, 0, 4, 0, 0, 0};

static bool make_class_plan(int kmax, int64_t total_pairs, int num_sms, const Tuning* tune,
                            bool wide, ClassPlan* c)
{
    const int W = kPipeThreads / 32;
    c->kmax = kmax;
    c->wide = wide;
    // sortmerge: at most the largest G that keeps two CTAs per SM (one CTA if
    // even G = 1 does not); the class's built-in or tuned choice below that;
    // fewer when there are few pairs to spread over the SMs
    int Gcap = 0;
    for (int g = 1; g <= 64; ++g) {
        SortPlan t;
        size_t b;
        if (!sort_plan(kmax, g, &t, &b, wide)) break;
        if (b <= (size_t)kMaxSmemBytes / 2 || g == 1) Gcap = g;
    }
    if (Gcap == 0) return false;
    const int cls = tune_class_of(kmax);
    if (tune) tune += cls;
    const int64_t want = (total_pairs + 2ll * num_sms - 1) / (2ll * num_sms);
    // fused path: lists that fit the packed chain format (4- and 8-byte
    // elements; the ordered-tile test serves 4-byte keys only)
    c->fused = kmax <= kFusedMaxK && !(tune && tune->variant == 2);
    c->adaptive = c->fused && !wide && tune && tune->variant == 3;
    c->lwarps = kSortListWarps;
    c->lGcap = 1 << 30;
    if (tune && tune->sort_G > 0) c->lGcap = tune->sort_G;
    if (want >= 1 && want < c->lGcap) c->lGcap = (int)want;
    int G = Gcap;
    if (kBuiltinSortG[cls] > 0) G = min(G, kBuiltinSortG[cls]);
    if (tune && tune->sort_G > 0) G = min(Gcap, tune->sort_G);
    if (want >= 1 && want < G) G = (int)want;
    sort_plan(kmax, G, &c->sp, &c->sbytes, wide);
    c->sp.G = G;
    // unwind
    UnwindPlan& up = c->up;
    up.nw = (kmax + 31) / 32;
    up.ns = up.nw <= 32 ? 0 : (up.nw + 31) / 32;
    // runs per block: more runs shorten each lane's serial walk at the cost of
    // seeding each run with the ranks of all earlier positions (GB300,
    // n = 2^24: unwind at k = 4095 took 1.42 ms with 4 runs, 0.72 ms with 32;
    // float64 at k = 1001 0.285 ms with 4, 0.195 with 8, 0.264 with 32)
    up.segs = kmax > 1024 ? 32 : (kmax >= 256 ? 8 : (kmax >= 64 ? 2 : 1));
    up.seglen = (((kmax + up.segs - 1) / up.segs) + 7) & ~7;
    c->bpw = 32 / up.segs;
    const int kpmax = (kmax + 7) & ~7;
    up.words_per_warp = (uint32_t)((up.nw + up.ns) * 32) + (uint32_t)(kpmax / 2) * (uint32_t)c->bpw;
    int uw = W;
    while (uw > 1 && (size_t)up.words_per_warp * 4 * uw > (size_t)kMaxSmemBytes / 2) --uw;
    c->uwarps = uw;
    c->ubytes = (size_t)up.words_per_warp * 4 * uw;
    if (c->ubytes > (size_t)kMaxSmemBytes) return false;
    // chain
    if (!chain_plan(kmax, &c->cp, &c->cbytes)) return false;
    // epilogue
    const int GEcap = max(1, 8192 / kmax);              // about 8192 outputs per CTA
    c->GE = kBuiltinEpiG[cls] > 0 ? min(GEcap, kBuiltinEpiG[cls]) : GEcap;
    if (tune && tune->epi_G > 0) c->GE = min(GEcap, tune->epi_G);
    c->ebytes = (wide ? 8ull : 4ull) * (size_t)(c->GE + 1) * kmax;
    return true;
}

static void count_items(PipeParams& p, const ClassPlan& c, int64_t* tot)
{
    const int64_t np = p.npairs;
    // store CTAs cover the class's span of (GE + 1) kmax elements whatever the
    // signal's own k, so a batch's small windows do not get tiny CTAs
    p.eG = p.k >= c.kmax ? c.GE : max(1, (int)(((int64_t)(c.GE + 1) * c.kmax) / p.k) - 1);
    int64_t cnt[4] = {np > 0 ? (np + c.sp.G - 1) / c.sp.G : 1,
                      np > 0 ? (np + c.bpw - 1) / c.bpw : 0,
                      np,
                      np > 0 ? (np + p.eG - 1) / p.eG : 1};
    if (c.fused) {
        p.bpw = kTileElems / p.k;
        p.lG = max(1, min(c.lwarps * p.bpw - 1, c.lGcap));
        p.kmagic = ((1ull << 32) + (uint64_t)p.k - 1) / (uint64_t)p.k;
        p.bmagic = ((1ull << 32) + (uint64_t)p.bpw - 1) / (uint64_t)p.bpw;
        cnt[0] = np > 0 ? (np + p.lG - 1) / p.lG : 1;
        cnt[1] = 0;
    }
    for (int i = 0; i < 4; ++i) { p.start[i] = tot[i]; tot[i] += cnt[i]; }
}

// Enqueue the four kernels of a set of classes: all sortmerges, then all
// unwinds, chains and epilogues (each signal's kernels stay in order).
static cudaError_t launch_classes(const ClassPlan* cls, const SegTable* tabs, const int64_t (*tot)[4],
                                  int ncls, cudaStream_t stream, LaunchStats* stats)
{
    cudaEvent_t* evs = nullptr;
    if (stats && stats->timing) {
        evs = stats->ev[stats->ring_pos % LaunchStats::kRing];
        stats->ring_pos += 1;
    }
#define TIMER_MARK(idx) do { if (evs) cudaEventRecord(evs[idx], stream); } while (0)
    cudaError_t e;
    TIMER_MARK(0);
    for (int c = 0; c < ncls; ++c) {
        if (cls[c].fused) {
            if ((e = launch_sortlist(tabs[c], tot[c][kItemSort], cls[c].lwarps, cls[c].adaptive,
                                     cls[c].wide, stream)) != cudaSuccess)
                return e;
            if (stats) stats->launches += 1;
            continue;
        }
        if (cls[c].wide)
            sortmerge_kernel<uint64_t><<<(unsigned)tot[c][kItemSort], kPipeThreads, cls[c].sbytes, stream>>>(tabs[c], cls[c].sp);
        else
            sortmerge_kernel<uint32_t><<<(unsigned)tot[c][kItemSort], kPipeThreads, cls[c].sbytes, stream>>>(tabs[c], cls[c].sp);
        if (stats) stats->launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    TIMER_MARK(1);
    for (int c = 0; c < ncls; ++c) {
        if (tot[c][kItemUnwind] == 0) continue;
        UnwindPlan up = cls[c].up;
        up.items = tot[c][kItemUnwind];
        const int64_t grid = (up.items + cls[c].uwarps - 1) / cls[c].uwarps;
        if (up.ns == 0)
            unwind_kernel<true><<<(unsigned)grid, 32 * cls[c].uwarps, cls[c].ubytes, stream>>>(tabs[c], up);
        else
            unwind_kernel<false><<<(unsigned)grid, 32 * cls[c].uwarps, cls[c].ubytes, stream>>>(tabs[c], up);
        if (stats) stats->launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    TIMER_MARK(2);
    for (int c = 0; c < ncls; ++c) {
        if (tot[c][kItemChain] == 0) continue;
        ChainPlan cp = cls[c].cp;
        cp.items = tot[c][kItemChain];
        const int64_t grid = (cp.items + cp.pairs_per_cta - 1) / cp.pairs_per_cta;
        if (cls[c].fused)
            chain_kernel<kFmtPacked, true><<<(unsigned)grid, kPipeThreads, cls[c].cbytes, stream>>>(tabs[c], cp);
        else if (cp.fmt == kFmtPacked)
            chain_kernel<kFmtPacked, false><<<(unsigned)grid, kPipeThreads, cls[c].cbytes, stream>>>(tabs[c], cp);
        else if (cp.fmt == kFmtMid)
            chain_kernel<kFmtMid, false><<<(unsigned)grid, kPipeThreads, cls[c].cbytes, stream>>>(tabs[c], cp);
        else
            chain_kernel<kFmtWide, false><<<(unsigned)grid, kPipeThreads, cls[c].cbytes, stream>>>(tabs[c], cp);
        if (stats) stats->launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    TIMER_MARK(3);
    for (int c = 0; c < ncls; ++c) {
        if (cls[c].wide)
            epilogue_kernel<uint64_t><<<(unsigned)tot[c][kItemEpilogue], kPipeThreads, cls[c].ebytes, stream>>>(tabs[c]);
        else
            epilogue_kernel<uint32_t><<<(unsigned)tot[c][kItemEpilogue], kPipeThreads, cls[c].ebytes, stream>>>(tabs[c]);
        if (stats) stats->launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    TIMER_MARK(4);
#undef TIMER_MARK
    return cudaSuccess;
}

cudaError_t launch_pipeline(const void* x, int64_t n, int k, int rank, Elem el,
                            void* y, int32_t* argmed, void* ws, size_t ws_bytes,
                            int num_sms, cudaStream_t stream, LaunchStats* stats)
{
    if (ws_bytes < pipeline_workspace_bytes(n, k)) return cudaErrorInvalidValue;
    if (k < 1 || rank < 0 || rank >= k || n < k) return cudaErrorInvalidValue;
    SegTable tab{};
    tab.segs = nullptr;
    tab.nseg = 1;
    fill_signal(tab.one, x, y, argmed, n, k, rank, el.is_float);
    ClassPlan cls;
    if (!make_class_plan(k, tab.one.npairs, num_sms, stats ? stats->tune : nullptr, el.wide, &cls))
        return cudaErrorInvalidValue;
    char* w = (char*)ws;
    carve_signal(tab.one, w, cls.fused);
    int64_t tot[1][4] = {{0, 0, 0, 0}};
    count_items(tab.one, cls, tot[0]);
    return launch_classes(&cls, &tab, tot, 1, stream, stats);
}

constexpr int kNumClasses = kNumTuneClasses;

int tune_class_of(int k)
{
    int c = 0;
    while (k > kClassMax[c]) ++c;
    return c;
}

cudaError_t launch_pipeline_batched(const void* x, void* y, int32_t* argmed, Elem el,
                                    const int64_t* x_off, const int64_t* n, const int64_t* y_off,
                                    const int32_t* k, int nseg, void* ws, size_t ws_bytes,
                                    void* stage, size_t stage_bytes, int num_sms,
                                    cudaStream_t stream, LaunchStats* stats)
{
    if (nseg <= 0) return cudaSuccess;
    if (ws_bytes < pipeline_batched_workspace_bytes(n, k, nseg)) return cudaErrorInvalidValue;
    if (stage_bytes < (size_t)nseg * sizeof(PipeParams)) return cudaErrorInvalidValue;
    // signals grouped by class, descriptors written class by class
    int cls_of_first[kNumClasses + 1];
    int count[kNumClasses] = {0};
    int kmax[kNumClasses] = {0};
    int64_t pairs[kNumClasses] = {0};
    auto class_of = [&](int kk) { int c = 0; while (kk > kClassMax[c]) ++c; return c; };
    for (int s = 0; s < nseg; ++s) {
        const int c = class_of(k[s]);
        count[c] += 1;
        kmax[c] = max(kmax[c], k[s]);
        pairs[c] += (n[s] + k[s] - 1) / k[s] - 1;
    }
    cls_of_first[0] = 0;
    for (int c = 0; c < kNumClasses; ++c) cls_of_first[c + 1] = cls_of_first[c] + count[c];
    ClassPlan plans[kNumClasses];
    SegTable tabs[kNumClasses];
    int64_t tot[kNumClasses][4];
    int ncls = 0;
    int cls_index[kNumClasses];
    for (int c = 0; c < kNumClasses; ++c) {
        if (!count[c]) continue;
        if (!make_class_plan(kmax[c], pairs[c], num_sms, stats ? stats->tune : nullptr, el.wide,
                             &plans[ncls]))
            return cudaErrorInvalidValue;
        cls_index[c] = ncls;
        for (int i = 0; i < 4; ++i) tot[ncls][i] = 0;
        ++ncls;
    }
    PipeParams* host = (PipeParams*)stage;
    PipeParams* dev = (PipeParams*)ws;
    char* w = (char*)ws + al256((uint64_t)nseg * sizeof(PipeParams));
    int fillpos[kNumClasses];
    for (int c = 0; c < kNumClasses; ++c) fillpos[c] = cls_of_first[c];
    for (int s = 0; s < nseg; ++s) {
        const int c = class_of(k[s]);
        PipeParams& p = host[fillpos[c]++];
        const int eb = el.bytes();
        fill_signal(p, (const char*)x + x_off[s] * eb, (char*)y + y_off[s] * eb,
                    argmed ? argmed + y_off[s] : nullptr, n[s], k[s], (k[s] - 1) / 2, el.is_float);
        carve_signal(p, w, plans[cls_index[c]].fused);
        count_items(p, plans[cls_index[c]], tot[cls_index[c]]);
    }
    for (int c = 0; c < kNumClasses; ++c) {
        if (!count[c]) continue;
        SegTable& t = tabs[cls_index[c]];
        t.segs = dev + cls_of_first[c];
        t.nseg = count[c];
        t.one = PipeParams{};
    }
    cudaError_t e = cudaMemcpyAsync(dev, host, (size_t)nseg * sizeof(PipeParams),
                                    cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return e;
    return launch_classes(plans, tabs, tot, ncls, stream, stats);
}

#ifdef MF_DEBUG
// One thread fails one check on purpose (no memory access depends on it), so
// that a test can see the record reach the host.
__global__ void debug_selftest_kernel() { (void)MF_CHECK(false, 999u, 42u); }

cudaError_t debug_selftest(cudaStream_t stream)
{
    debug_selftest_kernel<<<1, 1, 0, stream>>>();
    return cudaGetLastError();
}
#endif
MF_DEBUG_TAKE_FN(pipeline)

}  // namespace mf

// mf_sortlist.cu -- the fused front half of the pipeline for k <= kFusedMaxK:
// piecewise sort, joint ranks, unwind links and the list words of both block
// data structures of every pair, in one kernel.
//
// Paper: "Median Filtering is Equivalent to Sorting" (Suomela).
//   * stable block sort ........ Section 3 "Piecewise Sorting", Section 5.2:
//                                sorting the pairs (alpha[i], i) in
//                                lexicographic order gives a stable pi
//   * construct(A) ............. Section 5.3 (Fig. block-impl): A's list in
//                                sorted order through the sentinel k
//   * unwind(B) ................ Section 4 "Unwind": delete(k-1), ..., delete(0)
//                                leaves in position i the prev / next that i's
//                                list had when i was deleted, i.e. the nearest
//                                smaller / larger element among positions < i
//   * joint ranks .............. comparisons (alpha[i], i) < (alpha[m], m) of
//                                Section 5.3 and peek(A) <= peek(B) of Section
//                                6.2 as comparisons of ranks in the merged
//                                order of the pair (A first on equal keys)
//
// One CTA covers G consecutive block pairs, i.e. G + 1 blocks.  Each warp owns
// a tile of up to 1024 elements: bpw = 1024 / k whole blocks.  Elements become
// 64-bit composites (block in tile : 32-bit order key : position in block),
// all distinct, so plain ascending order of composites is the stable sort of
// every block of the tile at once:
//   1. every lane sorts 32 composites in registers (Batcher's odd-even merge
//      sorting network, 191 compare-exchanges);
//   2. five merge-path rounds in shared memory merge the 32 runs to one
//      (8-byte elements: steps 1-2 twice, on the low then the high half of
//      the key, the second time with the first sort's rank in the low field);
//   3. per pair, lanes merge A's and B's sorted runs by key (A first on ties)
//      and record each element's joint rank;
//   4. per block of the tile: perm / rank in place of the tile; as A, the list
//      words next | prev << 10 | joint rank << 20 of construct(A) (plus the
//      sentinel words and m_A = pi[h]); as B, the unwind links from prefix
//      bitsets of ranks (32 lanes, each a run of consecutive positions seeded
//      with the ranks of all positions before it) and the undelete words.
//      Tiles of many short blocks share the warp out differently: one lane per
//      block for k <= 64, groups of 4 or 8 lanes per block for k <= 256.
// Shared memory per warp: the padded tile (8448 bytes; element x at x + x/32
// so the lane-major stores of step 1 and the merge write-backs are free of
// bank conflicts), plus 4 KB per warp of joint-rank rows.
#include <cuda_runtime.h>
#include <cstdint>
#include "mf_device.cuh"
#include "mf_internal.h"
#include "mf_tilesort.cuh"

namespace mf {

namespace {

constexpr uint32_t kTileBytes = kTileU64 * 8;
static_assert(2 * kTileElems + 2 * (kTileElems + kTileElems / 16) + 4 * (kTileElems + kTileElems / 32) <=
              (int)kTileBytes, "perm, padded rank and bitset/link area fit in a tile");
constexpr uint32_t kRankInf = 0x7ffu;                      // sentinel rank (11 bits)

// Padded index of the 16-bit rank array: two entries of padding per 32, so
// the 32 lanes of a warp reading entries 32 L + i (one run each) hit 32
// different banks (17 L + i / 2 mod 32) instead of two.
__device__ __forceinline__ int rix(int x) { return x + ((x >> 5) << 1); }
constexpr int kRankU16 = kTileElems + kTileElems / 16;   // 1088 entries

__device__ __forceinline__ uint32_t comp_pos(uint64_t c) { return (uint32_t)c & 1023u; }

// Debug build: a list word's link fields name a slot or a sentinel (at most
// k + 1), its rank field a joint rank (below 2k) or the sentinel rank.
__device__ __forceinline__ uint32_t checked_word(uint32_t w, int k, uint32_t site)
{
    (void)MF_CHECK((w & 1023u) <= (uint32_t)k + 1u && ((w >> 10) & 1023u) <= (uint32_t)k + 1u &&
                   ((w >> 20) < 2u * (uint32_t)k || (w >> 20) == kRankInf), site, w);
    return w;
}

// Adaptive step (Section 1: an adaptive sort gives an adaptive median
// filter): 1 when every block of the tile is in ascending order (the stable
// order is then the position order), 2 when every block is strictly
// descending (its reverse), else 0.  A probe of one adjacent pair per lane
// rules both orders out for almost every unordered tile; only when it does
// not, lane L checks all pairs (e, e + 1) of its 32 elements that lie in one
// block.  Kept out of line so that its registers do not add to the sort's.
__device__ __noinline__ int tile_order(const uint32_t* tk, int tile_n, int k, uint64_t kmagic, int lane)
{
    if (tile_n <= 0) return 0;
    const int e0 = 32 * lane;
    const int pos0 = e0 - (int)udiv((uint32_t)e0, kmagic) * k;      // position of e0 in its block
    bool asc = true, desc = true;
    if (e0 + 1 < tile_n && pos0 + 1 < k) {
        const uint32_t a = tk[e0], b = tk[e0 + 1];
        asc = a <= b;
        desc = a > b;
    }
    asc = __all_sync(kFull, asc);
    desc = __all_sync(kFull, desc);
    if (!asc && !desc) return 0;
    int pos = pos0;
    for (int e = e0; e < e0 + 32; ++e) {                // pairs (e, e + 1), the last one into the next run
        if (e + 1 < tile_n && pos + 1 < k) {
            const uint32_t a = tk[e], b = tk[e + 1];
            asc = asc && a <= b;
            desc = desc && a > b;
        }
        pos = pos + 1 == k ? 0 : pos + 1;
    }
    asc = __all_sync(kFull, asc);
    desc = __all_sync(kFull, desc);
    return asc ? 1 : (desc ? 2 : 0);
}

// Key comparison of the pair merges: is A's element (composite ca, CTA
// element ea) at or before B's (cb, eb) in the window order (A first on equal
// keys)?  Equal key fields of 8-byte elements are decided by the low halves
// of the keys, read from x.
template <bool WIDE>
__device__ __forceinline__ bool a_first(uint64_t ca, uint64_t cb, const void* x, int64_t ea,
                                        int64_t eb, bool is_float)
{
    if constexpr (!WIDE) {
        return (uint32_t)(ca >> 10) <= (uint32_t)(cb >> 10);
    }
    const uint64_t ka = Comp<WIDE>::key(ca), kb = Comp<WIDE>::key(cb);
    if (ka != kb) return ka < kb;
    const uint64_t* x64 = reinterpret_cast<const uint64_t*>(x);
    return (uint32_t)to_key(__ldg(x64 + ea), is_float) <= (uint32_t)to_key(__ldg(x64 + eb), is_float);
}

// ADAPTIVE: test every tile for ordered blocks first (sort variant 3).
// WIDE: 8-byte elements (int64, float64), sorted on the top 44 bits of their
// key; a tile with ties in those bits within a block is sorted again on the
// whole key (tile_resort_wide).
template <bool ADAPTIVE, bool WIDE>
__global__ void __launch_bounds__(kSortListWarps * 32, 2)
sortlist_kernel(SegTable tab)
{
    int64_t cta;
    const PipeParams p = find_signal(tab, kItemSort, blockIdx.x, &cta);
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = blockDim.x >> 5;
    const int k = p.k, bpw = p.bpw, G = p.lG;
    const int64_t j0 = 1 + cta * G;                     // first pair of this CTA
    const int64_t left = p.npairs - (j0 - 1);
    const int npair = (int)(left < G ? (left > 0 ? left : 0) : G);
    const int nblk = npair + 1;
    const int64_t ebase = (j0 - 1) * (int64_t)k;
    const int64_t rem = p.n - ebase;
    const int E = (int)((int64_t)nblk * k < rem ? (int64_t)nblk * k : rem);
    uint64_t* tiles = reinterpret_cast<uint64_t*>(smem);
    uint16_t* jaS = reinterpret_cast<uint16_t*>(smem + (size_t)W * kTileBytes);
    uint16_t* jbS = jaS + (size_t)G * k;
    uint64_t* T = tiles + (size_t)warp * kTileU64;
    const int tile_e0 = warp * bpw * k;
    const int tile_n = max(0, min(bpw * k, E - tile_e0));

    // ---- 1. keys of the CTA's span (coalesced), then 32 composites per lane ----
    // E <= 32 * blockDim.x: each thread issues its loads 16 at a time.  The
    // composites take the key's low 32 bits (the whole key of 4-byte elements)
    uint32_t* keys = reinterpret_cast<uint32_t*>(smem);
    uint64_t* keys64 = reinterpret_cast<uint64_t*>(smem);
#pragma unroll 1
    for (int i0 = 0; i0 < 32; i0 += 16) {
        if constexpr (WIDE) {
            const uint64_t* xp = reinterpret_cast<const uint64_t*>(p.x) + ebase;
            uint64_t raw[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int e = tid + (i0 + i) * (int)blockDim.x;
                raw[i] = e < E ? __ldg(xp + e) : 0ull;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int e = tid + (i0 + i) * (int)blockDim.x;
                if (e < E) keys64[e] = to_key(raw[i], p.is_float);
            }
        } else {
            const uint32_t* xp = reinterpret_cast<const uint32_t*>(p.x) + ebase;
            uint32_t raw[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int e = tid + (i0 + i) * (int)blockDim.x;
                raw[i] = e < E ? __ldg(xp + e) : 0u;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int e = tid + (i0 + i) * (int)blockDim.x;
                if (e < E) keys[e] = to_key(raw[i], p.is_float);
            }
        }
    }
    __syncthreads();
    const int order = (ADAPTIVE && !WIDE) ? tile_order(keys + tile_e0, tile_n, k, p.kmagic, lane) : 0;
    using C = Comp<WIDE>;
    uint64_t v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int et = 32 * lane + ((i + lane) & 31);   // rotated: conflict-free reads
        uint64_t c = kPadComp;
        if (et < tile_n) {
            const uint32_t blk = udiv((uint32_t)et, p.kmagic);
            const uint32_t pos = (uint32_t)et - blk * (uint32_t)k;
            const uint64_t key = WIDE ? keys64[tile_e0 + et] >> 20 : (uint64_t)keys[tile_e0 + et];
            c = ((uint64_t)blk << C::kBlk) | (key << 10) | pos;
        }
        v[i] = c;
    }
    __syncthreads();                                    // keys read before tiles are written
    // ---- 2. warp merge sort of the tile ------------------------------------------
    if (ADAPTIVE && order != 0) {
        // ordered tile: element (block b, position j) goes to slot b k + j,
        // or b k + len_b - 1 - j when descending; slots past tile_n get the
        // padding composites
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const int et = 32 * lane + ((i + lane) & 31);
            int dst = et;
            if (order == 2 && et < tile_n) {
                const int blk = C::blk(v[i]), pos = (int)(v[i] & 1023u);
                dst = blk * k + min(k, tile_n - blk * k) - 1 - pos;
            }
            T[tix(dst)] = v[i];
        }
        __syncwarp();
    } else if (tile_n > 0) {
        tile_sort(T, v, lane);
    }
    if (WIDE && tile_n > 0) {
        if (tile_has_wide_ties(T, tile_n, lane))
            tile_resort_wide(T, reinterpret_cast<const uint64_t*>(p.x) + ebase + tile_e0, p.is_float,
                             tile_n, k, p.kmagic,
                             reinterpret_cast<uint16_t*>(smem + (size_t)W * kTileBytes) + (size_t)warp * 2048,
                             lane);
    }
    __syncthreads();

    // ---- 3. joint ranks of every pair: merge A's and B's runs, A first on ties ---
    {
        int lpp = 1;                                    // lanes per pair, about 64 outputs each
        while (lpp < 32 && lpp * 64 < 2 * k) lpp <<= 1;
        const int ppw = 32 / lpp;
        const int sub = lane & (lpp - 1);
        for (int g0 = warp * ppw; g0 < npair; g0 += W * ppw) {
            const int g = g0 + lane / lpp;
            if (g >= npair) continue;
            const int NB = min(k, E - (g + 1) * k);
            const int tot = k + NB;
            const int chunk = (tot + lpp - 1) / lpp;
            const int o0 = min(sub * chunk, tot), o1 = min(o0 + chunk, tot);
            const int tA = (int)udiv((uint32_t)g, p.bmagic), tB = (int)udiv((uint32_t)(g + 1), p.bmagic);
            const uint64_t* TA = tiles + (size_t)tA * kTileU64;
            const uint64_t* TB = tiles + (size_t)tB * kTileU64;
            const int offA = (g - tA * bpw) * k, offB = (g + 1 - tB * bpw) * k;
            const int64_t eA = ebase + (int64_t)g * k, eB = eA + k;      // blocks A and B in x
            int lo = max(0, o0 - NB), hi = min(o0, k);
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                const uint64_t cA = TA[tix(offA + mid)], cB = TB[tix(offB + o0 - 1 - mid)];
                if (a_first<WIDE>(cA, cB, p.x, eA + comp_pos(cA), eB + comp_pos(cB), p.is_float)) lo = mid + 1;
                else hi = mid;
            }
            int ia = lo, ib = o0 - lo;
            uint64_t ca = ia < k ? TA[tix(offA + ia)] : 0ull;
            uint64_t cb = ib < NB ? TB[tix(offB + ib)] : 0ull;
            uint16_t* ja = jaS + (size_t)g * k;
            uint16_t* jb = jbS + (size_t)g * k;
            for (int o = o0; o < o1; ++o) {
                const bool ta = ib >= NB ||
                                (ia < k && a_first<WIDE>(ca, cb, p.x, eA + comp_pos(ca), eB + comp_pos(cb), p.is_float));
                if (ta) {
                    if (MF_CHECK(comp_pos(ca) < (uint32_t)k && o < tot, 101, o)) ja[comp_pos(ca)] = (uint16_t)o;
                    if (++ia < k) ca = TA[tix(offA + ia)];
                } else {
                    if (MF_CHECK(comp_pos(cb) < (uint32_t)NB && o < tot, 101, o)) jb[comp_pos(cb)] = (uint16_t)o;
                    if (++ib < NB) cb = TB[tix(offB + ib)];
                }
            }
        }
    }
    __syncthreads();
    if (tile_n == 0) return;

    // ---- 4. per block of the tile ------------------------------------------------
    // The tile becomes: perm (u16, by sorted index), rank (u16, by block
    // position, padded: rix) and a 4224-byte area for bitsets, then unwind
    // links (2048 + 2176 + 4224 = 8448 bytes).
    uint16_t* permW = reinterpret_cast<uint16_t*>(T);
    uint16_t* rnkW = permW + kTileElems;
    uint32_t* areaW = reinterpret_cast<uint32_t*>(rnkW + kRankU16);
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = T[tix(lane + 32 * i)];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int x = lane + 32 * i;
        if (x < tile_n) {
            const uint32_t pos = comp_pos(v[i]);
            const uint32_t blk = (uint32_t)C::blk(v[i]);
            permW[x] = (uint16_t)pos;
            if (MF_CHECK(blk * k + pos < (uint32_t)tile_n && x - (int)blk * k < k, 102, x))
                rnkW[rix(blk * k + pos)] = (uint16_t)(x - blk * k);
        }
    }
    __syncwarp();

    const int nbt = (tile_n + k - 1) / k;
    if (k <= 64) {
        // Small windows (16 or more blocks per tile): one lane per block.  All
        // ranks of a block are below 64, so the ranks of the positions before
        // p form one 64-bit register; its bits below / above rank(p) give the
        // unwind links of p directly.
        for (int bt = lane; bt < nbt; bt += 32) {
            const int b = warp * bpw + bt;              // block of the CTA
            const int boff = bt * k;
            const int len = min(k, tile_n - boff);
            const uint16_t* pm = permW + boff;
            if (b < npair) {                            // as A: construct(A) words
                uint32_t* wa = p.wA + (size_t)(j0 - 1 + b) * p.kw;
                const uint16_t* ja = jaS + (size_t)b * k;
                for (int pos = 0; pos < k; ++pos) {
                    const int t = rnkW[rix(boff + pos)];
                    const uint32_t pv = t > 0 ? pm[t - 1] : (uint32_t)k;
                    const uint32_t nx = t + 1 < k ? pm[t + 1] : (uint32_t)k;
                    wa[pos] = checked_word(nx | (pv << 10) | ((uint32_t)ja[pos] << 20), k, 103);
                }
                wa[k] = (uint32_t)pm[0] | ((uint32_t)pm[k - 1] << 10) | (kRankInf << 20);
                wa[k + 1] = (uint32_t)(k + 1) | ((uint32_t)(k + 1) << 10) | (kRankInf << 20);
                wa[k + 2] = pm[p.h];
                (void)MF_CHECK(pm[p.h] < (uint32_t)k, 104, pm[p.h]);
            } else if (npair == 0) {
                p.wA[k + 2] = pm[p.h];                  // one block only: y[0] = X_0[P_0[h]]
            }
            if (b >= 1) {                               // as B of pair b - 1: unwind(B) links
                uint32_t* wb = p.wB + (size_t)(j0 - 1 + b - 1) * p.kw;
                const uint16_t* jb = jbS + (size_t)(b - 1) * k;
                const uint32_t sentB = (uint32_t)k + 1;
                uint64_t seen = 0ull;                   // ranks of positions before pos
                for (int pos = 0; pos < len; ++pos) {
                    const int r = rnkW[rix(boff + pos)];
                    const uint64_t below = seen & ((1ull << r) - 1ull);
                    const uint64_t above = seen & ~((2ull << r) - 1ull);   // r = 63: 0
                    const uint32_t pv = below ? (uint32_t)pm[63 - __clzll((long long)below)] : sentB;
                    const uint32_t nx = above ? (uint32_t)pm[__ffsll((long long)above) - 1] : sentB;
                    wb[pos] = checked_word(nx | (pv << 10) | ((uint32_t)jb[pos] << 20), k, 103);
                    seen |= 1ull << r;
                }
            }
        }
        return;
    }
    if (k <= 256) {
        // 64 < k <= 256 (four to fifteen blocks per tile): the construct(A)
        // words of all the tile's blocks at once, then the unwind in groups
        // of R lanes per block (R = 4 or 8, runs of at most 32 positions),
        // 32 / R blocks at a time, each group's prefix bitsets by an exclusive
        // OR-scan of shuffles within the group.  (GB300, n = 2^24 random walk:
        // the sort kernel at k = 127 took 0.58 ms one block at a time and
        // 0.43 ms grouped; at k = 511, with R = 16, grouping was 3 % slower.)
        for (int x = lane; x < tile_n; x += 32) {
            const int bt = (int)udiv((uint32_t)x, p.kmagic);
            const int b = warp * bpw + bt;
            if (b >= npair) continue;                   // full blocks: only the last is ragged
            const int pos = x - bt * k;
            const uint16_t* pm = permW + bt * k;
            const int t = rnkW[rix(x)];
            const uint32_t pv = t > 0 ? pm[t - 1] : (uint32_t)k;
            const uint32_t nx = t + 1 < k ? pm[t + 1] : (uint32_t)k;
            p.wA[(size_t)(j0 - 1 + b) * p.kw + pos] =
                checked_word(nx | (pv << 10) | ((uint32_t)jaS[(size_t)b * k + pos] << 20), k, 103);
        }
        for (int bt = lane; bt < nbt; bt += 32) {
            const int b = warp * bpw + bt;
            const uint16_t* pm = permW + bt * k;
            if (b < npair) {
                uint32_t* wa = p.wA + (size_t)(j0 - 1 + b) * p.kw;
                wa[k] = (uint32_t)pm[0] | ((uint32_t)pm[k - 1] << 10) | (kRankInf << 20);
                wa[k + 1] = (uint32_t)(k + 1) | ((uint32_t)(k + 1) << 10) | (kRankInf << 20);
                wa[k + 2] = pm[p.h];
                (void)MF_CHECK(pm[p.h] < (uint32_t)k, 104, pm[p.h]);
            } else if (npair == 0) {
                p.wA[k + 2] = pm[p.h];                  // one block only: y[0] = X_0[P_0[h]]
            }
        }
        int R = 4;
        while (R * 32 < k) R <<= 1;
        const int gpr = 32 / R, grp = lane / R, sub = lane & (R - 1);
        const int nw = (k + 31) >> 5;                   // bitset words for ranks < k
        uint32_t* bw = areaW + lane;                    // word w of this lane at bw[32 w]
        const uint32_t sentB = (uint32_t)k + 1;
        for (int bt0 = 0; bt0 < nbt; bt0 += gpr) {
            const int bt = bt0 + grp;
            const int boff = bt * k;
            const bool isB = bt < nbt && warp * bpw + bt >= 1;
            const int NB = isB ? min(k, tile_n - boff) : 0;
            const int cs = (NB + R - 1) / R;            // at most 32
            const int p0 = min(sub * cs, NB), p1 = min(p0 + cs, NB);
            const uint16_t* pm = permW + (isB ? boff : 0);
            for (int w = 0; w < nw; ++w) bw[32 * w] = 0u;
            for (int pos = p0; pos < p1; ++pos) {
                const int r = rnkW[rix(boff + pos)];
                bw[32 * (r >> 5)] |= 1u << (r & 31);
            }
            // run `sub` starts from the ranks of the group's runs 0 .. sub-1
            for (int w = 0; w < nw; ++w) {
                uint32_t v = bw[32 * w];
                for (int d = 1; d < R; d <<= 1) {
                    const uint32_t u = __shfl_up_sync(0xffffffffu, v, d, R);
                    if (sub >= d) v |= u;
                }
                const uint32_t ex = __shfl_up_sync(0xffffffffu, v, 1, R);
                bw[32 * w] = sub == 0 ? 0u : ex;
            }
            uint32_t summ = 0;                          // bit w: word w non-empty
            for (int w = 0; w < nw; ++w) summ |= bw[32 * w] ? (1u << w) : 0u;
            uint32_t uo[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                uo[i] = 0u;
                const int pos = p0 + i;
                if (pos < p1) {
                    const int r = rnkW[rix(boff + pos)];
                    const int w = r >> 5, bb = r & 31;
                    const uint32_t word = bw[32 * w];
                    const uint32_t mlo = word & ((1u << bb) - 1u);
                    const uint32_t mhi = word & ~((2u << bb) - 1u);    // bb = 31: 0
                    const uint32_t slo = summ & ((1u << w) - 1u);
                    const uint32_t shi = summ & ~((2u << w) - 1u);
                    const int wlo = slo ? 31 - __clz(slo) : 0;
                    const int whi = shi ? __ffs(shi) - 1 : 0;
                    uint32_t xlo = 0u, xhi = 0u;
                    if (!mlo && slo) xlo = bw[32 * wlo];
                    if (!mhi && shi) xhi = bw[32 * whi];
                    const int pred = mlo ? ((w << 5) | (31 - __clz(mlo)))
                                         : (slo ? ((wlo << 5) | (31 - __clz(xlo))) : -1);
                    const int succ = mhi ? ((w << 5) | (__ffs(mhi) - 1))
                                         : (shi ? ((whi << 5) | (__ffs(xhi) - 1)) : -1);
                    bw[32 * w] = word | (1u << bb);
                    summ |= 1u << w;
                    const uint32_t pv = pred >= 0 ? (uint32_t)pm[pred] : sentB;
                    const uint32_t nx = succ >= 0 ? (uint32_t)pm[succ] : sentB;
                    uo[i] = nx | (pv << 10);
                }
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (p0 + i < p1) areaW[tix(boff + p0 + i)] = uo[i];
            __syncwarp();
            // undelete words of this round's blocks
            const int e0 = bt0 * k, e1 = min(bt0 + gpr, nbt) * k;
            for (int x = e0 + lane; x < e1 && x < tile_n; x += 32) {
                const int btx = (int)udiv((uint32_t)x, p.kmagic);
                const int bx = warp * bpw + btx;
                if (bx < 1) continue;
                const int pos = x - btx * k;
                p.wB[(size_t)(j0 - 1 + bx - 1) * p.kw + pos] =
                    checked_word(areaW[tix(x)] | ((uint32_t)jbS[(size_t)(bx - 1) * k + pos] << 20), k, 103);
            }
            __syncwarp();
        }
        return;
    }
    for (int bt = 0; bt < nbt; ++bt) {
        const int b = warp * bpw + bt;                  // block of the CTA
        const int boff = bt * k;
        const int len = min(k, tile_n - boff);
        const uint16_t* pm = permW + boff;
        // -- as A of pair b: construct(A) in slot space (Section 5.3) -------------
        if (b < npair) {
            uint32_t* wa = p.wA + (size_t)(j0 - 1 + b) * p.kw;
            const uint16_t* ja = jaS + (size_t)b * k;
            for (int pos0 = lane; pos0 < k; pos0 += 128) {          // four positions in flight
                int t[4];
                uint32_t jv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int pos = pos0 + 32 * u;
                    t[u] = pos < k ? (int)rnkW[rix(boff + pos)] : 0;
                    jv[u] = pos < k ? (uint32_t)ja[pos] : 0u;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int pos = pos0 + 32 * u;
                    const uint32_t pv = t[u] > 0 ? pm[t[u] - 1] : (uint32_t)k;
                    const uint32_t nx = t[u] + 1 < k ? pm[t[u] + 1] : (uint32_t)k;
                    if (pos < k) wa[pos] = checked_word(nx | (pv << 10) | (jv[u] << 20), k, 103);
                }
            }
            if (lane == 0) {
                wa[k] = (uint32_t)pm[0] | ((uint32_t)pm[k - 1] << 10) | (kRankInf << 20);
                wa[k + 1] = (uint32_t)(k + 1) | ((uint32_t)(k + 1) << 10) | (kRankInf << 20);
                wa[k + 2] = pm[p.h];
                (void)MF_CHECK(pm[p.h] < (uint32_t)k, 104, pm[p.h]);
            }
        } else if (npair == 0 && lane == 0) {
            p.wA[k + 2] = pm[p.h];                      // one block only: y[0] = X_0[P_0[h]]
        }
        // -- as B of pair b - 1: unwind links (Section 4), undelete words --------
        // Lane L owns the run of positions [p0, p1).  The links of position p
        // are the predecessor / successor of rank(p) among the ranks of all
        // positions < p.  The lane's bitset starts as the ranks of all
        // positions before p0 (each lane sets the bits of its own run, then
        // an exclusive OR-scan over the lanes), then the lane walks its run,
        // querying and inserting one rank per position.
        if (b >= 1) {
            const int NB = len;
            const int cs = (NB + 31) >> 5;             // positions per lane (a run)
            const int nw = cs;                          // bitset words for ranks < NB
            const int p0 = min(lane * cs, NB), p1 = min(p0 + cs, NB);
            uint32_t* bw = areaW + lane;                // word w of this lane at bw[32 w]
            for (int w = 0; w < nw; ++w) bw[32 * w] = 0u;
            for (int pos = p0; pos < p1; ++pos) {
                const int r = rnkW[rix(boff + pos)];
                bw[32 * (r >> 5)] |= 1u << (r & 31);
            }
            __syncwarp();
            // exclusive OR-scan over lanes, transposed: lane w scans word w of
            // all 32 runs (read and written in rotated order, bank (i + w) % 32),
            // so run L's bitset becomes the ranks of all positions before p0
            if (lane < nw) {
                uint32_t* col = areaW + 32 * lane;
                uint32_t c[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) c[i] = col[(i + lane) & 31];
                uint32_t low = 0u;                      // runs 0 .. w-1 (the wrapped tail)
#pragma unroll
                for (int i = 0; i < 32; ++i) low |= (i >= 32 - lane) ? c[i] : 0u;
                uint32_t acc_hi = 0u, acc_lo = 0u;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const bool hi_part = i < 32 - lane;  // run L = i + w >= w
                    const uint32_t pre = hi_part ? (low | acc_hi) : acc_lo;
                    acc_hi |= hi_part ? c[i] : 0u;
                    acc_lo |= hi_part ? 0u : c[i];
                    col[(i + lane) & 31] = pre;
                }
            }
            __syncwarp();
            uint32_t summ = 0;                          // bit w: word w non-empty
            for (int w = 0; w < nw; ++w) summ |= bw[32 * w] ? (1u << w) : 0u;
            // the run: predecessor / successor of rank(pos) among earlier positions
            uint32_t uo[32];
            const uint32_t sentB = (uint32_t)k + 1;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                uo[i] = 0u;
                const int pos = p0 + i;
                if (pos < p1) {
                    const int r = rnkW[rix(boff + pos)];
                    const int w = r >> 5, bb = r & 31;
                    const uint32_t word = bw[32 * w];
                    const uint32_t mlo = word & ((1u << bb) - 1u);
                    const uint32_t mhi = word & ~((2u << bb) - 1u);    // bb = 31: 0
                    const uint32_t slo = summ & ((1u << w) - 1u);
                    const uint32_t shi = summ & ~((2u << w) - 1u);
                    const int wlo = slo ? 31 - __clz(slo) : 0;
                    const int whi = shi ? __ffs(shi) - 1 : 0;
                    uint32_t xlo = 0u, xhi = 0u;            // the nearest non-empty words, when needed
                    if (!mlo && slo) xlo = bw[32 * wlo];
                    if (!mhi && shi) xhi = bw[32 * whi];
                    const int pred = mlo ? ((w << 5) | (31 - __clz(mlo)))
                                         : (slo ? ((wlo << 5) | (31 - __clz(xlo))) : -1);
                    const int succ = mhi ? ((w << 5) | (__ffs(mhi) - 1))
                                         : (shi ? ((whi << 5) | (__ffs(xhi) - 1)) : -1);
                    bw[32 * w] = word | (1u << bb);
                    summ |= 1u << w;
                    const uint32_t pv = pred >= 0 ? (uint32_t)pm[pred] : sentB;
                    const uint32_t nx = succ >= 0 ? (uint32_t)pm[succ] : sentB;
                    uo[i] = nx | (pv << 10);
                }
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (p0 + i < p1) areaW[tix(p0 + i)] = uo[i];
            __syncwarp();
            uint32_t* wb = p.wB + (size_t)(j0 - 1 + b - 1) * p.kw;
            const uint16_t* jb = jbS + (size_t)(b - 1) * k;
            for (int pos = lane; pos < NB; pos += 32)
                wb[pos] = checked_word(areaW[tix(pos)] | ((uint32_t)jb[pos] << 20), k, 103);
            __syncwarp();
        }
    }
}

}  // namespace

size_t sortlist_smem_bytes(int warps)
{
    return (size_t)warps * (kTileBytes + 4u * kTileElems);
}

cudaError_t sortlist_setup()
{
    const int bytes = (int)sortlist_smem_bytes(kSortListWarps);
    cudaError_t e = cudaFuncSetAttribute(sortlist_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sortlist_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sortlist_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_sortlist(const SegTable& tab, int64_t items, int warps, bool adaptive, bool wide,
                            cudaStream_t stream)
{
    const size_t bytes = sortlist_smem_bytes(warps);
    if (wide)
        sortlist_kernel<false, true><<<(unsigned)items, 32 * warps, bytes, stream>>>(tab);
    else if (adaptive)
        sortlist_kernel<true, false><<<(unsigned)items, 32 * warps, bytes, stream>>>(tab);
    else
        sortlist_kernel<false, false><<<(unsigned)items, 32 * warps, bytes, stream>>>(tab);
    return cudaGetLastError();
}

MF_DEBUG_TAKE_FN(sortlist)

}  // namespace mf

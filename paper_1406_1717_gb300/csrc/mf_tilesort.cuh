// mf_tilesort.cuh -- the warp merge sort of a 1024-element tile of 64-bit
// composites, shared by the fused sort kernel (mf_sortlist.cu) and the chunk
// sort of the large-k tier (mf_large.cu).
//
// Each lane sorts 32 composites in registers with Batcher's odd-even merge
// sorting network (Batcher 1968), then five merge-path rounds (Green, McColl
// & Bader 2012) in shared memory merge the 32 runs into one.  The tile lives
// in shared memory with one word of padding per 32 (element x at x + x / 32),
// so lane-major stores and the merge write-backs are free of bank conflicts.
// Composites are distinct, so ascending order of composites is a stable sort
// of whatever key they carry in their high bits (Section 5.2 of the paper:
// sorting the pairs (alpha[i], i) gives a stable order).  8-byte keys carry
// their top 44 bits; a tile in which two of those tie within a block is
// sorted again on the whole key (tile_has_wide_ties, tile_resort_wide).
#pragma once
#include <cstdint>
#include "mf_device.cuh"
#include "mf_internal.h"

namespace mf {

constexpr int kTileU64 = kTileElems + kTileElems / 32;    // padded tile in 8-byte words
constexpr uint64_t kPadComp = ~0ull;                       // above every composite

__device__ __forceinline__ int tix(int x) { return x + (x >> 5); }

template <typename V>
__host__ __device__ __forceinline__ void cmpx(V& a, V& b)
{
    const bool sw = b < a;
    const V lo = sw ? b : a, hi = sw ? a : b;
    a = lo;
    b = hi;
}

// Batcher's odd-even merge sort (Batcher 1968) on v[LO..HI] (inclusive),
// unrolled at compile time: sort both halves, then odd-even merge.
template <int LO, int HI, int R>
struct OddEvenMerge {
    template <typename V>
    __host__ __device__ __forceinline__ static void run(V (&v)[32])
    {
        if constexpr (2 * R < HI - LO) {
            OddEvenMerge<LO, HI, 2 * R>::run(v);
            OddEvenMerge<LO + R, HI, 2 * R>::run(v);
#pragma unroll
            for (int i = LO + R; i < HI - R; i += 2 * R) cmpx(v[i], v[i + R]);
        } else {
            cmpx(v[LO], v[LO + R]);
        }
    }
};
template <int LO, int HI>
struct OddEvenSort {
    template <typename V>
    __host__ __device__ __forceinline__ static void run(V (&v)[32])
    {
        if constexpr (HI - LO >= 1) {
            constexpr int MID = LO + (HI - LO) / 2;
            OddEvenSort<LO, MID>::run(v);
            OddEvenSort<MID + 1, HI>::run(v);
            OddEvenMerge<LO, HI, 1>::run(v);
        }
    }
};

// One merge-path step: emit the smaller head, advance its run, load its next
// element (runs A = T[B0 ..), B = T[B0 + R ..), both of length R).
__device__ __forceinline__ uint64_t merge_step(const uint64_t* T, int B0, int R, uint64_t& ha,
                                               uint64_t& hb, int& a, int& b);

__device__ __forceinline__ uint64_t merge_step(const uint64_t* T, int B0, int R, uint64_t& ha,
                                               uint64_t& hb, int& a, int& b)
{
    const bool ta = ha < hb;
    const uint64_t out = ta ? ha : hb;
    a += ta ? 1 : 0;
    b += ta ? 0 : 1;
    const int nx = ta ? a : b;
    const int src = (ta ? B0 : B0 + R) + nx;
    uint64_t nv = kPadComp;
    if (nx < R) nv = T[tix(src)];
    ha = ta ? nv : ha;
    hb = ta ? hb : nv;
    return out;
}

// Sort the warp's tile.  On entry lane L holds 32 composites in v (any
// order); on exit T holds all 1024 in ascending order (padded layout) and v
// is clobbered.  Each merge round gives a lane two independent merge paths
// (16 outputs each), so their loads overlap.
__device__ __forceinline__ void tile_sort(uint64_t* T, uint64_t (&v)[32], int lane)
{
    OddEvenSort<0, 31>::run(v);
    const int o0 = 32 * lane;
#pragma unroll
    for (int i = 0; i < 32; ++i) T[tix(o0 + i)] = v[i];
    __syncwarp();
#pragma unroll 1
    for (int R = 32; R < kTileElems; R <<= 1) {
        // runs [B0, B0 + R) and [B0 + R, B0 + 2R); this lane's outputs are
        // merged positions d0 .. d0 + 15 and d1 .. d1 + 15 of that pair of runs
        const int B0 = o0 & ~(2 * R - 1);
        const int d0 = o0 - B0, d1 = d0 + 16;
        int lo0 = max(0, d0 - R), hi0 = min(d0, R);
        int lo1 = max(0, d1 - R), hi1 = min(d1, R);
        while (lo0 < hi0 || lo1 < hi1) {
            if (lo0 < hi0) {
                const int mid = (lo0 + hi0) >> 1;
                if (T[tix(B0 + mid)] < T[tix(B0 + R + d0 - 1 - mid)]) lo0 = mid + 1; else hi0 = mid;
            }
            if (lo1 < hi1) {
                const int mid = (lo1 + hi1) >> 1;
                if (T[tix(B0 + mid)] < T[tix(B0 + R + d1 - 1 - mid)]) lo1 = mid + 1; else hi1 = mid;
            }
        }
        int a0 = lo0, b0 = d0 - lo0, a1 = lo1, b1 = d1 - lo1;
        uint64_t ha0 = a0 < R ? T[tix(B0 + a0)] : kPadComp;
        uint64_t hb0 = b0 < R ? T[tix(B0 + R + b0)] : kPadComp;
        uint64_t ha1 = a1 < R ? T[tix(B0 + a1)] : kPadComp;
        uint64_t hb1 = b1 < R ? T[tix(B0 + R + b1)] : kPadComp;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            v[i] = merge_step(T, B0, R, ha0, hb0, a0, b0);
            v[16 + i] = merge_step(T, B0, R, ha1, hb1, a1, b1);
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 32; ++i) T[tix(o0 + i)] = v[i];
        __syncwarp();
    }
}

// x / d by a multiply-shift with magic = ceil(2^32 / d); exact for the
// ranges the kernels use (x < 8,192, 1 <= d <= 1,024), which
// tests/test_index_arithmetic.py checks exhaustively
__device__ __forceinline__ uint32_t udiv(uint32_t x, uint64_t magic)
{
    return (uint32_t)(((uint64_t)x * magic) >> 32);
}

// Composite layouts.  4-byte elements: block : 32-bit key : position (22, 32
// and 10 bits).  8-byte elements: block : top 44 bits of the 64-bit key :
// position (10, 44, 10); the key's low 20 bits decide only between elements
// whose top 44 bits are equal.
template <bool WIDE> struct Comp {
    static constexpr int kBlk = WIDE ? 54 : 42;         // shift of the block field
    __device__ __forceinline__ static uint64_t key(uint64_t c)
    {
        return (c >> 10) & ((1ull << (kBlk - 10)) - 1ull);
    }
    __device__ __forceinline__ static int blk(uint64_t c) { return (int)(c >> kBlk); }
};

// Does the sorted tile hold two adjacent composites with equal block and
// top 44 key bits (8-byte layout)?  Warp-uniform.
__device__ __forceinline__ bool tile_has_wide_ties(const uint64_t* T, int tile_n, int lane)
{
    bool tie = false;
    uint64_t prev = T[tix(32 * lane)] >> 10;
#pragma unroll 4
    for (int i = 1; i <= 32; ++i) {
        const int t = 32 * lane + i;
        if (t < tile_n) {
            const uint64_t cur = T[tix(t)] >> 10;
            tie = tie || cur == prev;
            prev = cur;
        }
    }
    return __any_sync(0xffffffffu, tie);
}

// 8-byte elements whose tile has two elements of one block with equal top 44
// key bits: sort the tile again, least significant digit first (stable LSD on
// the low 32 and the top 44 bits): by (block, low 32 bits, position), then by
// (block, top 44 bits, rank after that sort), and put the positions back in
// the low field.  perm1 / r1: the first sort's permutation and its inverse,
// in 4 KB of shared memory that the caller does not use until later.
static __device__ __noinline__ void tile_resort_wide(uint64_t* T, const uint64_t* xt, bool is_float, int tile_n,
                                              int k, uint64_t kmagic, uint16_t* perm1, int lane)
{
    using C = Comp<true>;
    uint16_t* r1 = perm1 + 1024;
    uint64_t v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int et = 32 * lane + ((i + lane) & 31);
        uint64_t c = kPadComp;
        if (et < tile_n) {
            const uint32_t blk = udiv((uint32_t)et, kmagic);
            const uint32_t lo = (uint32_t)to_key(__ldg(xt + et), is_float);
            c = ((uint64_t)blk << C::kBlk) | ((uint64_t)lo << 10) | ((uint32_t)et - blk * (uint32_t)k);
        }
        v[i] = c;
    }
    __syncwarp();                                       // the caller's reads of T are done
    tile_sort(T, v, lane);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int t = lane + 32 * i;
        const uint64_t c = T[tix(t)];
        if (t < tile_n) {
            const int e = C::blk(c) * k + (int)(c & 1023u);
            perm1[t] = (uint16_t)e;
            r1[e] = (uint16_t)t;
        }
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int et = 32 * lane + ((i + lane) & 31);
        uint64_t c = kPadComp;
        if (et < tile_n) {
            const uint32_t blk = udiv((uint32_t)et, kmagic);
            const uint64_t top = to_key(__ldg(xt + et), is_float) >> 20;
            c = ((uint64_t)blk << C::kBlk) | (top << 10) | r1[et];
        }
        v[i] = c;
    }
    __syncwarp();
    tile_sort(T, v, lane);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int x = lane + 32 * i;
        const uint64_t c = T[tix(x)];
        if (x < tile_n) {
            const int e = perm1[c & 1023u];
            T[tix(x)] = (c & ~1023ull) | (uint64_t)(e - C::blk(c) * k);
        }
    }
    __syncwarp();
}

}  // namespace mf

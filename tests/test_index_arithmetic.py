"""Host-side checks of the fused sort kernel's index arithmetic (no GPU).

The kernel divides tile-local indices by multiply-shift instead of a hardware
divide: udiv(x, d) = (x * ceil(2^32 / d)) >> 32, with d = k (the block of an
element of the warp tile) and d = bpw = 1024 // k (the warp tile of a block
of the CTA).  Writing ceil(2^32 / d) = (2^32 + e) / d with 0 <= e < d,
x * magic / 2^32 = x / d + x e / (d 2^32), and the floor is exact whenever
x e < 2^32.  The numerators the kernel divides are below 1024 (element of a
tile) and below W * bpw <= 8 * 1024 (block of a CTA, W = 8 warps), so the
products stay far below 2^32.  The test checks the identity exhaustively over
those ranges, for every divisor the fused path can meet (1 <= k <= 1021,
1 <= bpw <= 1024), in the 64-bit unsigned arithmetic the kernel uses.
"""
import numpy as np

K_FUSED_MAX = 1021
TILE = 1024
WARPS = 8


def _udiv(x, d):
    magic = np.uint64(((1 << 32) + d - 1) // d)
    return (x.astype(np.uint64) * magic) >> np.uint64(32)


def test_block_of_tile_element_is_exact():
    x = np.arange(TILE, dtype=np.uint64)
    for k in range(1, K_FUSED_MAX + 1):
        np.testing.assert_array_equal(_udiv(x, k), x // np.uint64(k), err_msg=f"k={k}")


def test_tile_of_cta_block_is_exact():
    g = np.arange(WARPS * TILE + 1, dtype=np.uint64)
    for k in range(1, K_FUSED_MAX + 1):
        bpw = TILE // k
        np.testing.assert_array_equal(_udiv(g, bpw), g // np.uint64(bpw), err_msg=f"bpw={bpw}")


def test_bound_is_not_vacuous():
    """The identity does fail once x e reaches about 2^32 (so the test above
    would notice a numerator range that is too large)."""
    d = 1021
    e = (((1 << 32) + d - 1) // d) * d - (1 << 32)
    assert 0 < e < d
    x = np.arange(0, 1 << 31, 997, dtype=np.uint64)
    assert (_udiv(x, d) != x // np.uint64(d)).any()

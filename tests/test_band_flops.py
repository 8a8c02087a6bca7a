"""Flop accounting of the band-limited transforms (da_plan_flops; host only).

The pass kernels skip, per warp, the first-stage inputs of an inverse
transform that lie in the gap K < q < n - K of the 2/3 rule (they are zero)
and the last-stage outputs of a forward transform that lie there (nothing
reads them).  This test recomputes the skipped flops from that rule with an
independent model: the radix lists of the plans, a warp of 32 consecutive
butterflies of one sequence (when n/R is a multiple of 32; otherwise only
positions in the gap for every butterfly), and the operation counts of the
zero-aware DFTs (an even/odd split down to 4-point DFTs, whose additions
with a known-zero operand cost nothing) and of the folded last-stage
butterflies (two FMAs per output).
"""
import ctypes
import math
import os
import shutil

import pytest

from paper_2602_14016_gb300 import _native as NN


@pytest.fixture(scope="module")
def lib():
    from paper_2602_14016_gb300 import build

    if shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc"):
        build.build()
    if not os.path.exists(NN.LIB_PATH):
        pytest.fail("libda_gb300.so is not built and nvcc is unavailable")
    return NN.load()

# radix lists and CTA widths of the plan variants
PLANS = {16: [(4, 4)], 32: [(4, 8), (2,) * 5], 64: [(4, 4, 4), (8, 8), (2,) * 6],
         128: [(4, 4, 8), (8, 4, 4), (4, 4, 8), (2,) * 7], 256: [(4, 4, 4, 4), (8, 8, 4), (4, 4, 4, 4)],
         512: [(8, 8, 8), (8, 4, 4, 4), (8, 8, 8)], 1024: [(16, 8, 8), (16, 4, 4, 4), (8, 8, 4, 4)]}


def gap_masks(n, r):
    """Mask of gap positions m (input or output m at i + m n/r) for each
    butterfly i, tested over the butterfly's warp."""
    K = (n - 1) // 3
    nb = n // r

    def gap(lo, hi):
        return lo >= K + 1 and hi <= n - K - 1

    out = []
    for i in range(nb):
        lo, hi = ((i // 32) * 32, (i // 32) * 32 + 31) if nb % 32 == 0 else (0, nb - 1)
        out.append(sum(1 << m for m in range(r) if gap(lo + m * nb, hi + m * nb)))
    return out


def leaf_additions(r, zero):
    """Complex additions the 2- and 4-point DFTs at the leaves of the even/odd
    split of an r-point DFT perform, given zero flags of its inputs (an
    addition with a known-zero operand is not performed; the combination
    layers above the leaves do not test for zeros)."""
    if r == 2:
        return 0 if (zero[0] or zero[1]) else 2
    if r == 4:
        z0, z1, z2, z3 = zero
        adds = (0 if (z0 or z2) else 2) + (0 if (z1 or z3) else 2)  # a0 +- a2, a1 +- a3
        return adds + (0 if ((z0 and z2) or (z1 and z3)) else 4)  # the four outputs
    return leaf_additions(r // 2, zero[0::2]) + leaf_additions(r // 2, zero[1::2])


def skipped_flops(n, radices):
    """(inverse, forward) flops skipped per transform: 2 flops per complex
    addition not performed in the first stage, 2 FMAs (4 flops) per output
    not formed in the last."""
    r0, rl = radices[0], radices[-1]
    inv = 0
    for w in gap_masks(n, r0):
        zero = [bool((w >> m) & 1) for m in range(r0)]
        inv += 2 * (leaf_additions(r0, [False] * r0) - leaf_additions(r0, zero))
    fwd = sum(4 * bin(w).count("1") for w in gap_masks(n, rl))
    return inv, fwd


@pytest.mark.parametrize("n", sorted(PLANS))
def test_plan_flops_match_the_gap_rule(lib, n):
    assert lib.da_plan_count(n) == len(PLANS[n])
    nominal = 5.0 * n * math.log2(n)
    for v, radices in enumerate(PLANS[n]):
        assert math.prod(radices) == n
        inv, fwd = ctypes.c_double(), ctypes.c_double()
        assert lib.da_plan_flops(n, v, ctypes.byref(inv), ctypes.byref(fwd)) == NN.DA_OK
        si, sf = skipped_flops(n, radices)
        assert inv.value == nominal - si, (n, v, inv.value, nominal, si)
        assert fwd.value == nominal - sf, (n, v, fwd.value, nominal, sf)
        assert 0.9 * nominal < inv.value <= nominal and 0.9 * nominal < fwd.value <= nominal


def test_headline_grid_counts(lib):
    """At 256 (radix 4 x 4 x 4 x 4): per sequence, warp 0 (butterflies 0-31)
    has input/output 2 (positions 128-159) in the gap and warp 1 has input
    or output 1 (positions 96-127): 64 butterflies x 2 complex additions
    (4 flops) skipped in an inverse transform, 64 outputs x 2 FMAs (4 flops)
    in a forward one."""
    inv, fwd = ctypes.c_double(), ctypes.c_double()
    assert lib.da_plan_flops(256, 0, ctypes.byref(inv), ctypes.byref(fwd)) == NN.DA_OK
    assert inv.value == 5 * 256 * 8 - 64 * 4 and fwd.value == 5 * 256 * 8 - 64 * 4
    assert gap_masks(256, 4)[:32] == [4] * 32 and gap_masks(256, 4)[32:] == [2] * 32


def test_plan_flops_rejects(lib):
    x = ctypes.c_double()
    assert lib.da_plan_flops(100, 0, ctypes.byref(x), ctypes.byref(x)) == NN.DA_EINVAL
    assert lib.da_plan_flops(256, 3, ctypes.byref(x), ctypes.byref(x)) == NN.DA_EINVAL
    assert lib.da_plan_flops(256, 0, None, ctypes.byref(x)) == NN.DA_EINVAL

"""The arithmetic behind FP64_OZ (the FP64-accurate exchange on tensor-core
digits), checked in exact integer arithmetic on the CPU with the constants
the kernels are compiled with.

A value x of a block with |x| < 2^e becomes the fixed-point integer
F = round(x 2^(7S - e)), split into S base-128 digits
F = sum_s d_s 128^(S-1-s), with d_1..d_{S-1} centred in [-64, 63] and
|d_0| <= 128.  The tensor cores multiply digit pairs exactly (BF16 holds
integers up to 256, FP32 products up to 2^24) and sum each group
g = s + t < S of one exactness block of K elements in FP32.  The sum stays
exact only while it cannot exceed 2^24.  Pairs with s + t >= S are dropped."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2601_16949_b300", "csrc", "ozaki.cuh")


def constants():
    text = open(HDR).read()
    get = lambda name: int(re.search(rf"constexpr int {name} = (\d+);", text).group(1))
    S, bits, KB, tiles = get("kS"), get("kDigitBits"), get("kKB"), get("kBlkTiles")
    return S, bits, KB * tiles


def split(F, S, bits):
    """Centred base-2^bits digits, low to high positions, top digit last."""
    base, half = 1 << bits, 1 << (bits - 1)
    d = []
    for _ in range(S - 1):
        r = ((F + half) % base) - half          # in [-half, half)
        d.append(r)
        F = (F - r) // base
    d.append(F)
    return d[::-1]                              # d_0 (top) ... d_{S-1}


def test_digits_reconstruct_and_stay_in_range():
    S, bits, _ = constants()
    assert (S, bits) == (6, 7)
    rng = np.random.default_rng(0)
    lim = 1 << (S * bits)
    samples = [0, 1, -1, lim, -lim, lim - 1, -(lim - 1)]
    samples += [int(v) for v in rng.integers(-lim, lim + 1, 20000)]
    for F in samples:
        d = split(F, S, bits)
        assert sum(di * (1 << (bits * (S - 1 - s))) for s, di in enumerate(d)) == F
        assert all(-64 <= di <= 63 for di in d[1:])
        assert abs(d[0]) <= 128


def test_group_sums_of_one_block_stay_exact_in_fp32():
    """Worst case over digit magnitudes: group g has one pair (0, 0) for
    g = 0, else two pairs with d_0 and g - 1 pairs of lower digits."""
    S, bits, K = constants()
    assert K == 512
    top, low = 128, 64
    for g in range(S):
        pairs = [(s, g - s) for s in range(g + 1)]
        bound = sum((top if s == 0 else low) * (top if t == 0 else low) for s, t in pairs)
        assert bound * K <= 1 << 24, (g, bound * K)
        # integers up to 2^24 are exact in FP32, so every partial sum is exact
        assert float(np.float32(bound * K)) == bound * K


def test_kept_pairs_give_the_product_to_the_stated_accuracy():
    """Product of two block-normalised values from the kept digit pairs,
    against the exact product of the fixed-point values: the dropped pairs
    (s + t >= S) cost at most 2^-41 of the block scale per product, and the
    rounding to 42 fixed-point bits at most 2^-42; random digits far less."""
    S, bits, _ = constants()
    scale = 1 << (S * bits)
    rng = np.random.default_rng(1)
    worst_f = 0
    cases = [(scale - 1, scale - 1), (-(scale - 1), scale - 1)]
    # every low digit at -64: the largest dropped pairs
    F_neg = sum(-64 * (1 << (bits * k)) for k in range(S - 1)) + 100 * (1 << (bits * (S - 1)))
    cases.append((F_neg, F_neg))
    cases += [(int(a), int(b)) for a, b in rng.integers(-scale, scale + 1, (5000, 2))]
    for Fx, Fy in cases:
        dx, dy = split(Fx, S, bits), split(Fy, S, bits)
        kept = 0
        for s in range(S):
            for t in range(S - s):
                kept += dx[s] * dy[t] * (1 << (bits * (2 * (S - 1) - s - t)))
        err = abs(kept - Fx * Fy)                 # in units of 2^(-2 * 42) of the block scale
        worst_f = max(worst_f, err)
    assert worst_f <= (1 << (2 * S * bits)) >> 41
    # rounding x to F: |x 2^42 - F| <= 1/2, i.e. 2^-43 of the block scale per factor
    x = rng.uniform(-1, 1, 1000)
    F = np.round(x * 2.0 ** 42)
    assert np.max(np.abs(x * 2.0 ** 42 - F)) <= 0.5

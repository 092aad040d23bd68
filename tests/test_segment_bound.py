"""The bound that sizes the single-launch fit's loss partials: lanes packed
next-fit (a segment closes only when the next lane would overflow its
capacity) inside C contiguous chunks of the lane list give at most
2 * ceil(N / cap) + C segments for N vehicles in lanes of at most cap.
Proof restated as a check: inside a chunk, two consecutive segments hold more
than cap vehicles together, so a chunk of n vehicles has at most 2 n / cap + 1
segments.  The packing here is written from that rule (chunks of
ceil(L / C) lanes, as the device builder splits them) and run on random and
adversarial lane sizes; the device kernel additionally refuses to write past
the partials it was given."""
import math

import numpy as np
import pytest


def next_fit_chunked(sizes, cap, chunks):
    L = len(sizes)
    per = (L + chunks - 1) // chunks
    n_seg = 0
    for t in range(chunks):
        fill = 0
        for n in sizes[min(L, t * per):min(L, t * per + per)]:
            if n == 0:
                continue
            assert n <= cap
            if fill > 0 and fill + n > cap:
                n_seg += 1
                fill = 0
            fill += n
        if fill > 0:
            n_seg += 1
    return n_seg


def bound(sizes, cap, chunks):
    return min(sum(1 for n in sizes if n > 0), 2 * math.ceil(sum(sizes) / cap) + chunks)


@pytest.mark.parametrize("cap", [64, 128, 512, 2048])
def test_bound_random_and_adversarial(cap):
    rng = np.random.default_rng(cap)
    cases = [
        rng.integers(0, cap + 1, size=5000),
        rng.integers(1, 7, size=50000),
        np.full(20000, cap // 2 + 1),          # every pair overflows: one lane per segment
        np.tile([cap // 2 + 1, cap // 2], 4000),
        np.full(3000, cap),
        np.ones(100000, dtype=np.int64),
        np.r_[np.zeros(500, dtype=np.int64), np.full(700, cap // 2 + 1)],
    ]
    for sizes in cases:
        sizes = [int(x) for x in sizes]
        for chunks in (1, 7, 1024):
            assert next_fit_chunked(sizes, cap, chunks) <= bound(sizes, cap, chunks)


def test_bound_is_tight_for_half_full_pairs():
    """Lanes of cap/2 + 1 leave every segment just over half full: the count
    reaches the 2 N / cap term (up to the per-chunk rounding)."""
    cap = 128
    sizes = [cap // 2 + 1] * 10000
    n = next_fit_chunked(sizes, cap, 1)
    assert n == 10000
    assert n <= 2 * math.ceil(sum(sizes) / cap) + 1
    assert n >= 2 * sum(sizes) / cap * (cap / 2) / (cap / 2 + 1) - 1

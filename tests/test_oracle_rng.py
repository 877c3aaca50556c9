"""Pins of the oracle's random numbers and permutation.

Philox4x64-10 is checked word for word against numpy's independent
implementation of the same published generator (numpy pre-increments its
counter before each block, so block `c` of ours is numpy's output after
setting its counter to c-1).  The permutation is checked to be a bijection
with a consistent inverse, and to place items uniformly.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

MASK = (1 << 64) - 1


def numpy_philox(ctr, key):
    c = [int(x) for x in ctr]
    # counter - 1 as a 256-bit little-endian integer
    v = sum(ci << (64 * i) for i, ci in enumerate(c))
    v = (v - 1) % (1 << 256)
    prev = [(v >> (64 * i)) & MASK for i in range(4)]
    bg = np.random.Philox(counter=np.array(prev, dtype=np.uint64),
                          key=np.array(key, dtype=np.uint64))
    return bg.random_raw(4)


def test_philox_matches_numpy():
    rng = np.random.default_rng(12345)
    cases = [([1, 0, 0, 0], [0, 0]), ([0, 0, 0, 0], [0, 0]), ([MASK, MASK, MASK, MASK], [MASK, MASK])]
    for _ in range(200):
        cases.append((list(rng.integers(0, 2**63, 4, dtype=np.uint64) * 2 + rng.integers(0, 2, 4, dtype=np.uint64)),
                      list(rng.integers(0, 2**63, 2, dtype=np.uint64))))
    for ctr, key in cases:
        if all(int(c) == 0 for c in ctr):
            # numpy cannot be positioned before counter 0; compare the next block instead
            ours = O.philox([1, 0, 0, 0], key)
            ref = np.random.Philox(counter=np.zeros(4, np.uint64), key=np.array(key, np.uint64)).random_raw(4)
        else:
            ours = O.philox(ctr, key)
            ref = numpy_philox(ctr, key)
        assert np.array_equal(ours, ref), (ctr, key)


def test_draw_counter_layout():
    # draw() packs (index, aux, cell, step<<16 | pass<<8 | tag) under key (seed, problem)
    seed, prob, idx, aux, cell, step, pas, tag = 7, 3, 11, 5, 9, 123, 2, O.TAG_COLL
    got = O.draw(seed, prob, idx, aux, cell, step, pas, tag)
    exp = numpy_philox([idx, aux, cell, (step << 16) | (pas << 8) | tag], [seed, prob])
    assert np.array_equal(got, exp)


def test_uniform_conversions():
    assert O.u01(0) == 0.0
    assert O.u01(MASK) == 1.0 - 2.0**-53
    assert O.u01_open(0) == 2.0**-53
    assert O.u01_open(MASK) == 1.0
    assert O.below(0, 7) == 0
    assert O.below(MASK, 7) == 6
    # uniformity of below(n): chi-square on Philox words
    n = 13
    words = np.concatenate([O.draw(1, 0, i, 0, 0, 0, 0, O.TAG_KSEL) for i in range(5000)])
    counts = np.bincount([O.below(int(w), n) for w in words], minlength=n)
    assert stats.chisquare(counts).pvalue > 1e-4


@pytest.mark.parametrize("n", list(range(1, 70)) + [100, 255, 256, 257, 1000, 1023, 4096, 4097])
def test_prp_bijection_and_inverse(n):
    key = O.draw(5, 1, n, 0, 0, 0, 0, O.TAG_PERM0)
    fwd = O.prp_table(n, key)
    inv = O.prp_table(n, key, inverse=True)
    assert sorted(fwd.tolist()) == list(range(n))
    assert np.array_equal(inv[fwd], np.arange(n))


def test_prp_uniform_placement():
    # Over many keys, item 0 (and item n-1) should land uniformly in [0, n).
    for n in (10, 37):
        pos0 = np.zeros(n, np.int64)
        posl = np.zeros(n, np.int64)
        for s in range(3000):
            key = O.draw(9, 2, s, 0, 0, 0, 0, O.TAG_PERM0)
            t = O.prp_table(n, key)
            pos0[t[0]] += 1
            posl[t[n - 1]] += 1
        assert stats.chisquare(pos0).pvalue > 1e-4
        assert stats.chisquare(posl).pvalue > 1e-4

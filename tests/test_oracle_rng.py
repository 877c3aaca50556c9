"""Pins of the oracle's random numbers and permutation.

Philox4x64-10 is checked word for word against numpy's independent
implementation of the same published generator (numpy pre-increments its
counter before each block, so block `c` of ours is numpy's output after
setting its counter to c-1).  The permutation is checked to be a bijection
with a consistent inverse, to place items uniformly, and -- since it
realises Alg. 4.3's "random choice" of which particles stay uncollided, are
leaves or are thermalised, and how a level's products are dealt -- to choose
subsets with the law of a uniform random permutation: the exact law of the
set holding the top ranks for cells up to 40 items, of whole permutations for
up to five, the hypergeometric law of how many top ranks fall in a block of
items for 64 to 2500, the Poisson(1) law of the number of fixed points, and
the chance that two siblings land in the same half.
"""
import itertools
import math

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


def _keys(seed, K):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2**63, (K, 4), dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, (K, 4), dtype=np.uint64)


@pytest.mark.parametrize("n", [2, 3, 5, 8, 13, 24, 32, 33, 40])
def test_prp_top_ranks_form_a_uniform_subset(n):
    # the items holding the k highest ranks (Alg. 4.3: the changed particles)
    # are every k-subset with probability 1 / C(n, k)
    k = max(1, n // 3) if math.comb(n, max(1, n // 3)) <= 800 else 2
    K = 20000
    t = O.prp_tables(n, _keys(100 + n, K))
    top = t >= n - k
    codes = (top.astype(np.int64) << np.arange(n, dtype=np.int64)).sum(1)
    index = {sum(1 << x for x in c): i for i, c in enumerate(itertools.combinations(range(n), k))}
    obs = np.bincount([index[c] for c in codes], minlength=len(index))
    assert stats.chisquare(obs).pvalue > 1e-4, (n, k)


@pytest.mark.parametrize("n", [3, 4, 5])
def test_prp_whole_permutation_law(n):
    K = 24000
    t = O.prp_tables(n, _keys(200 + n, K)).astype(np.int64)
    codes = (t * n ** np.arange(n - 1, -1, -1)).sum(1)
    index = {sum(v * n ** (n - 1 - j) for j, v in enumerate(p)): i for i, p in enumerate(itertools.permutations(range(n)))}
    obs = np.bincount([index[c] for c in codes], minlength=len(index))
    assert stats.chisquare(obs).pvalue > 1e-4, n


@pytest.mark.parametrize("n,K", [(64, 20000), (100, 20000), (500, 12000), (2500, 3000)])
def test_prp_top_ranks_in_a_block_are_hypergeometric(n, K):
    # how many of the top third of the ranks land on the first quarter of the
    # items: hypergeometric (n, k, q) for a uniform permutation (the mean is
    # right for any bijection; the variance and the shape are not)
    k, q = n // 3, n // 4
    t = O.prp_tables(n, _keys(300 + n, K))
    cnt = (t[:, :q] >= n - k).sum(1)
    pmf = stats.hypergeom(n, k, q).pmf(np.arange(q + 1)) * K
    obs = np.bincount(cnt, minlength=q + 1)[: q + 1].astype(float)
    # pool both tails into their neighbours until every expected count is >= 5
    lo, hi = int(np.argmax(pmf >= 5)), int(q - np.argmax(pmf[::-1] >= 5))
    e = np.concatenate([[pmf[: lo + 1].sum()], pmf[lo + 1:hi], [pmf[hi:].sum()]])
    o = np.concatenate([[obs[: lo + 1].sum()], obs[lo + 1:hi], [obs[hi:].sum()]])
    chi = ((o - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi, len(e) - 1) > 1e-4, n


@pytest.mark.parametrize("n", [6, 17, 40, 64, 100, 500])
def test_prp_siblings_share_a_half_as_often_as_uniform(n):
    # items 0 and 1 (a collision's two products) land in the same half of
    # [0, n) with probability (h(h-1) + (n-h)(n-h-1)) / (n(n-1)), h = n // 2
    K = 30000
    t = O.prp_tables(n, _keys(400 + n, K))
    h = n // 2
    same = (t[:, 0] < h) == (t[:, 1] < h)
    p = (h * (h - 1) + (n - h) * (n - h - 1)) / (n * (n - 1))
    z = (same.mean() - p) / np.sqrt(p * (1 - p) / K)
    assert abs(z) < 4.5, (n, z)


@pytest.mark.parametrize("n,K", [(40, 30000), (300, 30000), (1000, 20000)])
def test_prp_fixed_points_are_poisson(n, K):
    # the number of items a uniform permutation leaves in place is, for large
    # n, Poisson with mean 1 (chi-square over 0..4 and 5 or more)
    t = O.prp_tables(n, _keys(500 + n, K))
    fp = (t == np.arange(n, dtype=np.int32)).sum(1)
    obs = np.bincount(np.minimum(fp, 5), minlength=6).astype(float)
    exp = np.append(stats.poisson(1).pmf(np.arange(5)), stats.poisson(1).sf(4)) * K
    assert stats.chisquare(obs, exp).pvalue > 1e-4, n


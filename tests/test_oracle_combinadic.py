"""Pins for the oracle of the paper's chromosome generation (Section 4.1): random rank, lexicographic unranking.

The binomials are checked against the C(m, p) column the paper prints (Tables 1 and 2); the unranking against
itertools.combinations, whose output order is lexicographic (a library routine), on every rank of small cases
and against an independently written ranking on large ones; the rank draw for exact uniformity by counting.
"""

import itertools
import math
import os

import numpy as np
import pytest

import oracle
from oracle import combinadic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "binomials_tables_1_2.txt")


def test_binomials_match_the_printed_column():
    rows = [line.split() for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    assert len(rows) >= 10
    for m, p, printed in rows:
        mant, exp = printed.split("E")
        digits = len(mant.replace(".", "")) - 1
        assert f"{combinadic.binom(int(m), int(p)):.{digits}E}" == f"{float(mant):.{digits}f}E{int(exp):+03d}", (m, p)


@pytest.mark.parametrize("m,p", [(1, 1), (5, 1), (5, 5), (6, 3), (9, 4), (10, 7), (12, 2)])
def test_unrank_is_lexicographic_order(m, p):
    combos = list(itertools.combinations(range(m), p))
    assert len(combos) == combinadic.binom(m, p)
    for i, c in enumerate(combos):
        assert tuple(combinadic.unrank(m, p, i)) == c
        assert combinadic.rank(m, p, c) == i
    with pytest.raises(ValueError):
        combinadic.unrank(m, p, len(combos))


def test_unrank_round_trip_at_paper_sizes():
    rng = np.random.default_rng(0)
    for m, p in [(900, 90), (128, 16), (600, 200), (5000, 500)]:
        C = combinadic.binom(m, p)
        for i in [0, 1, C - 1, C // 2] + [int(rng.integers(0, 2**62)) * (C // 2**62) for _ in range(3)]:
            combo = combinadic.unrank(m, p, i)
            assert len(combo) == p and combo == sorted(set(combo)) and 0 <= combo[0] and combo[-1] < m
            assert combinadic.rank(m, p, combo) == i
    # the extremes of the order: the first and the last combination
    assert combinadic.unrank(900, 90, 0) == list(range(90))
    assert combinadic.unrank(900, 90, combinadic.binom(900, 90) - 1) == list(range(810, 900))


def test_rank_words():
    assert combinadic.rank_words(900, 90) == (math.comb(900, 90).bit_length() + 31) // 32 == 14
    assert combinadic.rank_words(3, 1) == 1


def test_random_rank_is_uniform():
    """Every rank of C(7, 3) = 35 equally likely: counts over 35 * 400 draws pass a chi-square test."""
    m, p = 7, 3
    C = combinadic.binom(m, p)
    n = C * 400
    counts = np.zeros(C, dtype=np.int64)
    for u in range(n):
        counts[combinadic.random_rank(seed=11, gen=u // 1000, unit=u % 1000, m=m, p=p)] += 1
    expected = n / C
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert counts.min() > 0
    assert chi2 < 75.0, chi2  # 34 degrees of freedom: P(chi2 > 75) < 1e-4


def test_random_rank_draws_follow_the_counter_layout():
    """Try 0's K words are draws 0..K-1 of OP_COMB, least significant first, masked to bits(C)."""
    m, p = 900, 90
    C = combinadic.binom(m, p)
    K = combinadic.rank_words(m, p)
    u = sum(oracle.draw(5, 2, 77, combinadic.OP_COMB, w, 3) << (32 * w) for w in range(K))
    u &= (1 << C.bit_length()) - 1
    r = combinadic.random_rank(5, 2, 77, m, p, inst=3)
    if u < C:
        assert r == u
    else:
        assert r != u and r < C


def test_chromosome_has_p_ones():
    for m, p in [(100, 5), (900, 90), (33, 32)]:
        x = combinadic.chromosome(1, 0, 3, m, p)
        assert sum(bin(int(v)).count("1") for v in x) == p
        assert all(int(v) >> (m - 32 * w) == 0 for w, v in enumerate(x) if m - 32 * w < 32)

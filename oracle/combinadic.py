"""Oracle of the paper's chromosome generation (Section 4.1) -- test infrastructure.

A chromosome is drawn by picking a random integer i below C(m, p) and taking
the i-th p-combination of {0, ..., m-1} in lexicographic order (ascending
element tuples compared left to right), so that each of the C(m, p) bitsets
with exactly p ones is equally likely.

Readings where the section is silent or cannot hold:
  * the paper draws i with one 64-bit random number, which cannot reach most
    combinations once C(m, p) > 2^64 (C(900, 90) is about 5.1e125, Table 1);
    here i is drawn by rejection: K = ceil(bits(C) / 32) Philox words form an
    integer whose bits above bits(C) are cleared, accepted if below C(m, p),
    up to 64 tries (each accepted with probability > 1/2); after 64 refusals
    (probability < 2^-64) i = 0.  Try r uses draws r*K .. r*K + K - 1 of
    operation OP_COMB, word w of the integer being draw r*K + w (least
    significant first);
  * unranking walks the elements e = 0, 1, ...: with k elements still to
    choose among m - e, the combinations whose next element is e number
    C(m - e - 1, k - 1); if i is below that count e is chosen, else i is
    reduced by it and e skipped.

Plain Python integers and math.comb (exact big-integer arithmetic); the
random words come from the oracle's own Philox4x32-10 (oracle.draw).
"""

from __future__ import annotations

import math

import numpy as np

OP_COMB = 0x002
MAX_TRIES = 64


def binom(m: int, p: int) -> int:
    return math.comb(int(m), int(p))


def rank_words(m: int, p: int) -> int:
    """32-bit words of a rank below C(m, p): ceil(bits(C(m, p)) / 32)."""
    return max(1, (binom(m, p).bit_length() + 31) // 32)


def random_rank(seed: int, gen: int, unit: int, m: int, p: int, inst: int = 0) -> int:
    """Uniform integer in [0, C(m, p)) by bounded rejection sampling on Philox words."""
    from . import draw

    C = binom(m, p)
    bits = C.bit_length()
    K = rank_words(m, p)
    for r in range(MAX_TRIES):
        u = 0
        for w in range(K):
            u |= draw(seed, gen, unit, OP_COMB, r * K + w, inst) << (32 * w)
        u &= (1 << bits) - 1
        if u < C:
            return u
    return 0


def unrank(m: int, p: int, i: int) -> list[int]:
    """The i-th (0-based) p-combination of range(m) in lexicographic order."""
    m, p, i = int(m), int(p), int(i)
    if not 0 <= i < binom(m, p):
        raise ValueError("rank out of range")
    out = []
    k = p
    for e in range(m):
        if k == 0:
            break
        c = math.comb(m - e - 1, k - 1)  # combinations whose next element is e
        if i < c:
            out.append(e)
            k -= 1
        else:
            i -= c
    return out


def rank(m: int, p: int, combo) -> int:
    """Inverse of unrank, from the count of lexicographically smaller combinations: for each chosen element
    c_j (j-th smallest, 0-based), every combination that agrees before j and has a smaller element there
    comes first, i.e. sum over x in (c_{j-1}, c_j) of C(m - 1 - x, p - 1 - j)."""
    combo = sorted(int(c) for c in combo)
    r = 0
    prev = -1
    for j, c in enumerate(combo):
        for x in range(prev + 1, c):
            r += math.comb(m - 1 - x, p - 1 - j)
        prev = c
    return r


def chromosome(seed: int, gen: int, unit: int, m: int, p: int, inst: int = 0) -> np.ndarray:
    """The bitset (ceil(m/32) uint32 words) of individual `unit`'s fresh chromosome in generation `gen`."""
    x = np.zeros((m + 31) // 32, dtype=np.uint32)
    for e in unrank(m, p, random_rank(seed, gen, unit, m, p, inst)):
        x[e >> 5] |= np.uint32(1 << (e & 31))
    return x

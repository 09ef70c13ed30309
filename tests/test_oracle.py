"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: the numbers the
paper prints for Example 1 (Section 2.1), brute force over all p-subsets,
closed forms (Eq. 4 telescopes to the nearest-open distance; E[scan length]
= (m+1)/(p+1)), library routines (a stable argsort), exhaustive enumeration
(Floyd sampling), the published Philox4x32-10 known-answer vectors, and
hand-worked operator cases written from the prose of Sections 4.3 and 4.4.
"""

import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1610_10061_gb300.inputs import (graph_instance, masks_from_sets, paper_shape_instance, random_masks,
                                           sets_from_masks)


def _arr(rows, dtype):
    return np.array(rows, dtype=dtype)


# --------------------------------------------------------------------------
# Example 1 (Section 2.1)
# --------------------------------------------------------------------------

def test_example1_full_tables(example1):
    C = _arr(example1["C"], np.int32)
    pi, de = oracle.tables(C, full=True)
    np.testing.assert_array_equal(pi.astype(int) + 1, _arr(example1["PI"], int))
    np.testing.assert_array_equal(de, _arr(example1["DELTA"], np.int32))


def test_example1_truncated_tables(example1):
    C = _arr(example1["C"], np.int32)
    p = example1["n m p"][0][2]
    pi, de = oracle.tables(C, p)
    assert pi.shape == (5, 3)
    np.testing.assert_array_equal(pi.astype(int) + 1, _arr(example1["PI_TRUNC"], int))
    np.testing.assert_array_equal(de, _arr(example1["DELTA_TRUNC"], np.int32))


def _printed_poly(example1):
    poly = {}
    for row in example1["POLY"]:
        poly[frozenset(v - 1 for v in row[1:])] = row[0]
    return poly


def test_example1_reduced_polynomial(example1):
    C = _arr(example1["C"], np.int32)
    pi, de = oracle.tables(C, 2)
    assert oracle.hbp_polynomial(pi, de) == _printed_poly(example1)


def test_example1_every_open_set(example1):
    """O1, O2 and O3 equal the printed polynomial at every one of the C(4,2) open sets."""
    C = _arr(example1["C"], np.int32)
    pi, de = oracle.tables(C, 2)
    printed = _printed_poly(example1)
    sets = list(itertools.combinations(range(4), 2))
    masks = masks_from_sets(sets, 4)
    o1 = oracle.eval_direct(C, masks)
    o3 = oracle.eval_scan(pi, de, masks)
    poly = oracle.hbp_polynomial(pi, de)
    for t, s in enumerate(sets):
        z = [0 if j in s else 1 for j in range(4)]
        expect = sum(c * math.prod(z[j] for j in mono) for mono, c in printed.items())
        assert o1[t] == expect
        assert o3[t] == expect
        assert oracle.hbp_eval(poly, s) == expect
    # the optimum of Example 1 is facilities {1, 4} (1-based)
    assert oracle.brute_force(C, 2) == (int(min(o1)), (0, 3))


# --------------------------------------------------------------------------
# Eq. 4 identity, truncation and the sort
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_three_evaluators_agree_on_all_subsets(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 9))
    m = int(rng.integers(2, 9))
    p = int(rng.integers(1, m))
    hi = [3, 20, 1000][seed % 3]  # small ranges force many equal distances
    d = rng.integers(0, hi, size=(n, m)).astype(np.int32)
    pi, de = oracle.tables(d, p)
    sets = list(itertools.combinations(range(m), p))
    masks = masks_from_sets(sets, m)
    o1 = oracle.eval_direct(d, masks)
    o3 = oracle.eval_scan(pi, de, masks)
    poly = oracle.hbp_polynomial(pi, de)
    o2 = np.array([oracle.hbp_eval(poly, s) for s in sets])
    np.testing.assert_array_equal(o1, o3)
    np.testing.assert_array_equal(o1, o2)
    # eq. 4 written out term by term on the full tables gives the same
    pif, def_ = oracle.tables(d, full=True)
    for t, s in enumerate(sets):
        x = np.zeros(m, dtype=int)
        x[list(s)] = 1
        tot = 0
        for i in range(n):
            tot += int(def_[i, 0])
            for k in range(1, m):
                tot += int(def_[i, k]) * int(np.prod(1 - x[pif[i, :k]]))
        assert tot == o1[t]


def test_truncation_invariance_and_scan_bound():
    """The scan over full Pi/Delta equals the scan over Pi'/Delta' and never passes rank m-p+1."""
    d = graph_instance(60, 150, seed=7)
    for p in (1, 2, 5, 30, 59):
        masks = random_masks(300, 60, p, seed=p)
        pi, de = oracle.tables(d, p)
        pif, def_ = oracle.tables(d, full=True)
        a, ka = oracle.eval_scan(pi, de, masks, return_ksum=True)
        b, kb = oracle.eval_scan(pif, def_, masks, return_ksum=True)
        np.testing.assert_array_equal(a, b)
        assert ka == kb
        np.testing.assert_array_equal(a, oracle.eval_direct(d, masks))
    # with fewer than p open the truncated scan can run off the row; the oracle reports it
    pi, de = oracle.tables(d, 5)
    far = int(np.argmax(d[0]))
    assert (d[0] == d[0, far]).sum() == 1
    with pytest.raises(RuntimeError):
        oracle.eval_scan(pi, de, masks_from_sets([[far]], 60))


def test_tables_match_stable_argsort():
    rng = np.random.default_rng(5)
    d = rng.integers(0, 7, size=(40, 33)).astype(np.int32)
    pif, def_ = oracle.tables(d, full=True)
    order = np.argsort(d, axis=1, kind="stable")
    np.testing.assert_array_equal(pif.astype(np.int64), order)
    srt = np.take_along_axis(d, order, axis=1)
    np.testing.assert_array_equal(def_[:, 0], srt[:, 0])
    np.testing.assert_array_equal(def_[:, 1:], np.diff(srt, axis=1))
    assert (def_ >= 0).all()
    pi, de = oracle.tables(d, 10)
    np.testing.assert_array_equal(pi, pif[:, :24])
    np.testing.assert_array_equal(de, def_[:, :24])


def test_mean_scan_length_closed_form():
    """Mean ranks scanned per client over uniform random p-subsets is (m+1)/(p+1) (Section 4.2 gives ~m/p)."""
    d = graph_instance(80, 300, seed=3)
    m = 80
    for p in (4, 16):
        P = 4000
        masks = random_masks(P, m, p, seed=11 + p)
        pi, de = oracle.tables(d, p)
        _, ks = oracle.eval_scan(pi, de, masks, return_ksum=True)
        per = np.array(ks) / (P * 80)
        expect = (m + 1) / (p + 1)
        # variance of the first-open rank for a random subset, divided by the sample count
        var = (m - p) * (m + 1) * p / ((p + 1) ** 2 * (p + 2))
        assert abs(per - expect) < 6 * math.sqrt(var / P)


# --------------------------------------------------------------------------
# Brute force on the derived 20-node sub-instance
# --------------------------------------------------------------------------

def test_brute_force_sub20_and_oracle_ga_finds_it():
    w = paper_shape_instance("graph100_sub20")
    d, p = w["d"], w["p"]
    best, arg = oracle.brute_force(d, p)
    assert len(arg) == p
    # every subset is >= best; spot-check the argmin by the independent scan evaluator
    pi, de = oracle.tables(d, p)
    assert oracle.eval_scan(pi, de, masks_from_sets([arg], 20))[0] == best
    st, trace, _, _ = oracle.ga_run(pi, de, 20, p, seed=0, P=64, gens=30)
    assert st.best_cost == best
    assert trace[-1] == best


def test_brute_force_enumeration_in_c_matches_the_python_one(example1):
    """oracle_brute_force (lexicographic enumeration in C, split by smallest facility over host threads) against
    the itertools enumeration costed by O1: the printed Example 1 (optimum {1, 4} = 35, 1-based), the derived
    20-node sub-instance and small random instances with many ties."""
    C = _arr(example1["C"], np.int32)
    assert oracle.brute_force_c(C, 2) == (35, (0, 3))
    w = paper_shape_instance("graph100_sub20")
    assert oracle.brute_force_c(w["d"], w["p"]) == oracle.brute_force(w["d"], w["p"])
    rng = np.random.default_rng(5)
    for m, p, hi in [(12, 3, 4), (15, 1, 50), (14, 13, 9), (11, 5, 3)]:
        d = rng.integers(0, hi, size=(9, m)).astype(np.int32)
        assert oracle.brute_force_c(d, p, threads=3) == oracle.brute_force(d, p)


def test_graph100_optimum_golden():
    """The stored optimum of the 100-node graph instance (tests/golden/graph100_optimum.txt, written by the
    oracle's brute force over all C(100, 5) open sets): its cost is O1 of its open set, and no single swap (close
    one open facility, open one closed facility) is cheaper.  The full enumeration is re-run below."""
    from conftest import load_golden

    g = load_golden("graph100_optimum.txt")
    cost, best = g["cost"][0][0], tuple(g["open"][0])
    w = paper_shape_instance("graph100")
    d, p = w["d"], w["p"]
    assert len(best) == p == 5 and list(best) == sorted(set(best))
    assert oracle.eval_direct(d, masks_from_sets([best], 100))[0] == cost
    swaps = [tuple(sorted((set(best) - {j}) | {k})) for j in best for k in range(100) if k not in best]
    assert (oracle.eval_direct(d, masks_from_sets(swaps, 100)) >= cost).all()
    assert oracle.brute_force_c(d, p) == (cost, best)


# --------------------------------------------------------------------------
# Philox4x32-10 and the draw mapping
# --------------------------------------------------------------------------

def test_philox_known_answers():
    # Published known-answer vectors of Philox4x32-10 (Random123 distribution).
    kat = [
        ([0, 0, 0, 0], [0, 0], [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
        ([0xffffffff] * 4, [0xffffffff] * 2, [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
        ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0],
         [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]),
    ]
    for ctr, key, expect in kat:
        assert [int(v) for v in oracle.philox4x32_10(ctr, key)] == expect


def test_draw_layout():
    seed = 0x0123456789ABCDEF
    for slot in range(9):
        ctr = [7, 33, (oracle.OP_MUT + 2) * 65536 + slot // 4, 5]
        key = [seed & 0xffffffff, seed >> 32]
        assert oracle.draw(seed, 7, 33, oracle.OP_MUT + 2, slot, 5) == int(oracle.philox4x32_10(ctr, key)[slot % 4])


def test_uniform_mapping():
    for N in (1, 2, 3, 7, 100, 65535, 2**31 + 11):
        assert oracle.uniform(0, N) == 0
        assert oracle.uniform(2**32 - 1, N) == N - 1
    for u in (0, 1, 2**31 - 1, 2**31, 2**32 - 1, 123456789):
        assert oracle.uniform(u, 2) == u >> 31
        assert oracle.uniform(u, 256) == u >> 24
        assert oracle.uniform(u, 10) == (u * 10) >> 32


# --------------------------------------------------------------------------
# Floyd sampling
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m,p", [(6, 3), (7, 2), (5, 4), (8, 1)])
def test_floyd_exactly_uniform(m, p):
    """Every one of the m!/(m-p)! draw sequences gives a p-subset; each subset arises p! times."""
    counts = {}
    ranges = [range(m - p + q + 1) for q in range(p)]
    for draws in itertools.product(*ranges):
        x = oracle.floyd_from_values(m, p, draws)
        s = tuple(sets_from_masks(x[None, :], m)[0])
        assert len(s) == p
        counts[s] = counts.get(s, 0) + 1
    assert len(counts) == math.comb(m, p)
    assert set(counts.values()) == {math.factorial(p)}


# --------------------------------------------------------------------------
# Crossover (Section 4.3) and shift mutation (Section 4.4)
# --------------------------------------------------------------------------

def _bits(s, m):
    return masks_from_sets([[j for j, ch in enumerate(s) if ch == "1"]], m)[0]


def test_crossover_hand_case():
    # m = 10, p = 6, r1 = 7, r2 = 2 (i = 1): the parameters of the paper's Figure 1 caption.
    m = 10
    C = _bits("1111110000", m)       # open 0..5
    couple = _bits("0011111100", m)  # open 2..7
    F = oracle.crossover(C, couple, m, 7, 1)
    # from 7: position 7 (C=0, couple=1) opens; 8, 9 equal; 0 (C=1, couple=0) closes.
    np.testing.assert_array_equal(F, _bits("0111110100", m))
    # i = 2: from 7 -> open 7, close 0, (1: C=1,couple=0) close 1, wrap ... open 6.
    F2 = oracle.crossover(C, couple, m, 7, 2)
    np.testing.assert_array_equal(F2, _bits("0011111100", m))
    # Hamming(C, couple) = 4, so i = 3 cannot be reached: the crossover fails
    assert oracle.crossover(C, couple, m, 7, 3) is None


def test_crossover_invariants():
    rng = np.random.default_rng(9)
    m, p = 45, 9
    pop = random_masks(200, m, p, seed=2)
    for t in range(0, 200, 2):
        C, K = pop[t], pop[t + 1]
        r1 = int(rng.integers(0, m))
        i = int(rng.integers(1, p // 2 + 1))
        F = oracle.crossover(C, K, m, r1, i)
        ham = sum(bin(int(a ^ b)).count("1") for a, b in zip(C, K))
        if i > ham // 2:
            assert F is None
            continue
        assert F is not None
        assert sum(bin(int(v)).count("1") for v in F) == p
        changed = [int(a ^ b) for a, b in zip(C, F)]
        assert sum(bin(v).count("1") for v in changed) == 2 * i
        diff = [int(a ^ b) for a, b in zip(C, K)]
        assert all((c & ~dd) == 0 for c, dd in zip(changed, diff))
        # the couple's child (same r1, i) exchanges exactly the same positions
        G = oracle.crossover(K, C, m, r1, i)
        assert [int(a ^ b) for a, b in zip(K, G)] == changed


def test_shift_hand_cases():
    m = 10
    C = _bits("1011001010", m)
    # one position left block shift of the sub-sequence 3..6 (Figure 3 caption)
    F = oracle.shift(C, m, 3, 4, 1, right=False)
    np.testing.assert_array_equal(F, _bits("1010011010", m))
    # three positions right circular shift (Figure 2 caption): F[j] = C[j-3 mod m]
    G = oracle.shift(C, m, 0, m, 3, right=True)
    expect = "".join("1011001010"[(j - 3) % m] for j in range(m))
    np.testing.assert_array_equal(G, _bits(expect, m))


def test_shift_invariants():
    rng = np.random.default_rng(4)
    m = 77
    pop = random_masks(50, m, 13, seed=8)
    for C in pop:
        a = int(rng.integers(0, m - 1))
        length = int(rng.integers(2, m - a + 1))
        k = int(rng.integers(1, length))
        L_ = oracle.shift(C, m, a, length, k, right=False)
        R_ = oracle.shift(L_, m, a, length, k, right=True)
        np.testing.assert_array_equal(R_, C)
        assert sum(bin(int(v)).count("1") for v in L_) == 13
        outside = [j for j in range(m) if not (a <= j < a + length)]
        sc, sl = sets_from_masks(C[None], m)[0], sets_from_masks(L_[None], m)[0]
        assert [j for j in sc if j in outside] == [j for j in sl if j in outside]


def test_mutation_params_ranges():
    m = 31
    kinds = set()
    for unit in range(400):
        a, length, k, right = oracle.mutation_params(1, 0, unit, 0, m)
        assert 0 <= a and a + length <= m and length >= 2 and 1 <= k <= length - 1
        kinds.add((length == m and a == 0, right))
    assert len(kinds) == 4


def test_crossover_params_ranges():
    for pair in range(300):
        r1, i = oracle.crossover_params(3, 2, pair, 1, 50, 9)
        assert 0 <= r1 < 50 and 1 <= i <= 4


# --------------------------------------------------------------------------
# The GA (Sections 3.1, 3.2.2, 4.5)
# --------------------------------------------------------------------------

def test_ga_invariants_and_resume():
    w = paper_shape_instance("graph100")
    d, p = w["d"], w["p"]
    pi, de = oracle.tables(d, p)
    P, D, G = 64, 16, 6
    st, trace, pops, costs = oracle.ga_run(pi, de, 100, p, seed=3, P=P, D=D, gens=G, record=True)
    for g in range(G):
        for t in range(P):
            assert sum(bin(int(v)).count("1") for v in pops[g, t]) == p
        np.testing.assert_array_equal(costs[g], oracle.eval_direct(d, pops[g]))
        if g > 0:
            # migration (i): slot 0 of each deme starts as last generation's deme best;
            # later enhancements only lower its cost
            prev_best = costs[g - 1].reshape(-1, D).min(axis=1)
            assert (costs[g][::D] <= prev_best).all()
    assert (np.diff(trace) <= 0).all()
    assert trace[-1] == costs.min()
    assert oracle.eval_direct(d, st.best[None])[0] == st.best_cost
    lg = 4
    assert G * P <= st.evals <= G * P * (1 + 2 * lg)
    # resume: 3 + 3 generations equal 6
    a, ta, _, ca = oracle.ga_run(pi, de, 100, p, seed=3, P=P, D=D, gens=3, record=True)
    a, tb, _, cb = oracle.ga_run(pi, de, 100, p, seed=3, P=P, D=D, gens=3, record=True, state=a)
    np.testing.assert_array_equal(np.concatenate([ta, tb]), trace)
    np.testing.assert_array_equal(np.concatenate([ca, cb]), costs)
    assert a.evals == st.evals


def test_ga_saturation_stop():
    d = graph_instance(30, 60, seed=1)
    pi, de = oracle.tables(d, 3)
    st, trace, _, _ = oracle.ga_run(pi, de, 30, 3, seed=0, P=32, D=16, gens=500, saturation=4)
    assert len(trace) < 500
    assert (trace[-5:] == trace[-1]).all()
    assert st.scalars[1] == 4


def test_ga_migration_variants():
    """Section 4.5's two migration variants, pinned by what each must do to the next population.

    With no crossover or mutation the population at the end of a generation is the one it started with, so:
    variant (i) puts deme b's best (lowest cost, then lowest index) of generation g-1 into slot 0 of deme b;
    variant (ii) puts all deme bests into deme 0 (deme b's into slot b); every other individual is the same
    fresh draw in both variants (same random-number counters), and generation 0 has no migrants at all.
    """
    w = paper_shape_instance("graph100")
    d, p = w["d"], w["p"]
    pi, de = oracle.tables(d, p)
    P, D, G = 64, 8, 3
    NB = P // D
    runs = {}
    for team in (False, True):
        _, _, pops, costs = oracle.ga_run(pi, de, 100, p, seed=9, P=P, D=D, gens=G, xover_rounds=0, mut_tries=0,
                                          record=True, team=team)
        runs[team] = (pops, costs)
    (pi_, ci), (pt, ct) = runs[False], runs[True]
    np.testing.assert_array_equal(pi_[0], pt[0])
    for g in range(1, G):
        for team, (pops, costs) in runs.items():
            for b in range(NB):
                c = costs[g - 1, b * D:(b + 1) * D]
                best = pops[g - 1, b * D + int(np.argmin(c))]  # argmin: lowest index among equal costs
                slot = b if team else b * D
                np.testing.assert_array_equal(pops[g, slot], best)
        migrants = set(range(NB)) | set(range(0, P, D))
        for t in range(P):
            if t not in migrants:
                np.testing.assert_array_equal(pi_[g, t], pt[g, t])
    with pytest.raises(RuntimeError):  # deme 0 cannot hold 16 bests of demes of 4
        oracle.ga_run(pi, de, 100, p, seed=0, P=64, D=4, gens=1, team=True)


@pytest.mark.parametrize("seed", range(4))
def test_cumulative_tables_are_the_sorted_distances(seed):
    """D' (running sums of Delta') is the row of sorted distances, and reading it at the first open rank gives
    the direct cost of every p-subset: the cumulative evaluator's pins."""
    rng = np.random.default_rng(100 + seed)
    n, m = int(rng.integers(2, 12)), int(rng.integers(3, 9))
    p = int(rng.integers(1, m))
    d = rng.integers(0, [3, 40, 1000, 2**31 - 1][seed], size=(n, m)).astype(np.int32)
    pi, de = oracle.tables(d, p)
    dcum = oracle.cumulative(de)
    np.testing.assert_array_equal(dcum, np.sort(d.astype(np.int64), axis=1)[:, :m - p + 1])
    np.testing.assert_array_equal(dcum, np.take_along_axis(d.astype(np.int64), pi.astype(np.int64), axis=1))
    sets = list(itertools.combinations(range(m), p))
    masks = masks_from_sets(sets, m)
    np.testing.assert_array_equal(oracle.eval_cumulative(pi, dcum, masks), oracle.eval_direct(d, masks))


@pytest.mark.parametrize("name", ["graph100", "graph900"])
def test_mean_scan_length_at_the_bench_workloads(name):
    """The algorithmic bytes the benchmark reports use E[k] = (m+1)/(p+1) ranks per (individual, client) for uniform
    random p-subsets (pinned at small sizes by test_mean_scan_length_closed_form).  At the benchmark's own instances
    the oracle's exact count of visited ranks agrees within sampling error, and that count equals a brute-force
    first-open rank."""
    w = paper_shape_instance(name)
    d, p = w["d"], w["p"]
    n, m = d.shape
    pi, de = oracle.tables(d, p)
    pop = 512
    masks = random_masks(pop, m, p, seed=21)
    _, ksum = oracle.eval_scan(pi, de, masks, return_ksum=True)
    ek = (m + 1) / (p + 1)
    mean = ksum / (pop * n)
    # the variance of k for one pair is below E[k]^2; pairs of one individual are correlated, so bound the error by
    # the individuals alone (pop independent samples of a per-individual mean)
    assert abs(mean - ek) < 4 * ek / np.sqrt(pop), (mean, ek)
    # exact count on a few individuals by brute force
    open_ = ((masks[:8, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(8, -1)[:, :m].astype(bool)
    _, k8 = oracle.eval_scan(pi, de, masks[:8], return_ksum=True)
    brute = sum(int(np.argmax(open_[t][pi[i].astype(np.int64)])) + 1 for t in range(8) for i in range(n))
    assert k8 == brute

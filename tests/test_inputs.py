"""The synthetic input recipe: every generator is seeded and produces the shapes and properties the workloads
state (connected graphs with shortest-path distances, rounded Euclidean distances, exact p-subsets)."""

import math

import numpy as np
import pytest

from paper_1610_10061_gb300.inputs import (batched_instances, euclid_instance, gmm_instance, graph_instance,
                                           mask_words, masks_from_sets, paper_shape_instance, random_masks,
                                           sets_from_masks)


def test_graph_instance_is_a_shortest_path_metric():
    d = graph_instance(60, 150, seed=4)
    assert d.dtype == np.int32 and d.shape == (60, 60)
    assert (np.diag(d) == 0).all() and (d == d.T).all()
    assert (d[~np.eye(60, dtype=bool)] >= 1).all()  # connected, positive weights
    assert d.max() <= 100 * 59  # a shortest path has at most n - 1 edges of weight at most 100
    # triangle inequality: shortest paths through any middle node are never shorter
    for k in range(60):
        assert (d <= d[:, k:k + 1] + d[k:k + 1, :]).all()
    assert np.array_equal(d, graph_instance(60, 150, seed=4))
    assert not np.array_equal(d, graph_instance(60, 150, seed=5))


def test_graph_instance_edge_count_bounds():
    with pytest.raises(ValueError):
        graph_instance(10, 8, seed=0)  # fewer than n - 1 edges cannot connect 10 nodes
    with pytest.raises(ValueError):
        graph_instance(10, 46, seed=0)  # more than n (n - 1) / 2
    d = graph_instance(10, 45, seed=0)  # the complete graph
    assert (d[~np.eye(10, dtype=bool)] <= 100).all()


@pytest.mark.parametrize("gen", [euclid_instance, gmm_instance])
def test_point_instances_round_scaled_distances(gen):
    d = gen(200, seed=7)
    assert d.dtype == np.int32 and d.shape == (200, 200)
    assert (np.diag(d) == 0).all() and (d == d.T).all()
    assert d.max() <= math.ceil(1e4 * math.sqrt(2))
    # rounding keeps the triangle inequality up to one unit per rounded side
    for k in range(0, 200, 17):
        assert (d <= d[:, k:k + 1] + d[k:k + 1, :] + 1).all()
    assert np.array_equal(d, gen(200, seed=7))


def test_gmm_points_are_clustered():
    """50 components of sigma 0.02: pairs within 0.04 of each other (about one within-cluster distance) are more
    than twice as frequent as among uniform points (400 points: 8 per cluster, about 1.8 % of pairs share one)."""
    close_gmm = (gmm_instance(400, seed=1) < 400).mean()
    close_uni = (euclid_instance(400, seed=1) < 400).mean()
    assert close_gmm > 2 * close_uni


@pytest.mark.parametrize("P,m,p", [(1, 5, 4), (300, 100, 5), (64, 900, 90), (10, 33, 32), (5, 40, 1)])
def test_random_masks_are_exact_p_subsets(P, m, p):
    masks = random_masks(P, m, p, seed=3)
    assert masks.shape == (P, mask_words(m)) and masks.dtype == np.uint32
    sets = sets_from_masks(masks, m)
    assert all(len(s) == p and s[-1] < m for s in sets)
    tail = m & 31
    if tail:
        assert ((masks[:, -1] >> np.uint32(tail)) == 0).all()  # no bit at or above m
    assert np.array_equal(masks_from_sets(sets, m), masks)
    assert np.array_equal(masks, random_masks(P, m, p, seed=3))


def test_random_masks_cover_facilities_evenly():
    masks = random_masks(4000, 50, 5, seed=9)
    counts = np.zeros(50)
    for s in sets_from_masks(masks, 50):
        counts[s] += 1
    expect = 4000 * 5 / 50
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert chi2 < 100.0  # 49 degrees of freedom


def test_batched_instances_follow_the_stated_distribution():
    inst = batched_instances(24, seed=3, nmin=100, nmax=400)
    assert len(inst) == 24
    for k, (d, p) in enumerate(inst):
        n = d.shape[0]
        assert d.shape == (n, n) and 100 <= n <= 400
        assert 5 <= p <= max(5, n // 10)
        if k % 2 == 0:  # graph instances: integer shortest paths with weights of at most 100
            assert d[~np.eye(n, dtype=bool)].min() >= 1
        else:  # Euclidean instances
            assert d.max() <= math.ceil(1e4 * math.sqrt(2))


def test_paper_shape_instances():
    w = paper_shape_instance("graph100")
    assert w["d"].shape == (100, 100) and w["p"] == 5 and w["pop"] == 64
    s = paper_shape_instance("graph100_sub20")
    assert np.array_equal(s["d"], w["d"][:20, :20]) and s["p"] == 4
    with pytest.raises(KeyError):
        paper_shape_instance("nope")

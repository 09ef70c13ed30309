"""Seeded synthetic p-median instances and populations.

This module only draws inputs: distance matrices shaped like the paper's
benchmark families and random open-facility sets.  It holds none of the
method's arithmetic (no orderings, increments, scans or GA operators), so both
the CUDA path and the CPU oracle can take their inputs from it.

Instance families (the paper's benchmark sets are not shipped; these stand in
for them, see Section 6 of the paper for the originals):

* ``graph_instance``   -- connected undirected random graph, all-pairs
  shortest-path distances (OR-Library-like shapes).
* ``euclid_instance``  -- points uniform in the unit square,
  d = round(1e4 * Euclidean distance).
* ``gmm_instance``     -- points from a 50-component Gaussian mixture in the
  unit square (sigma 0.02), same rounding.

Every function takes an explicit seed and uses ``numpy.random.default_rng``.
Facility ids are 0-based; a population is a ``(P, W)`` uint32 array with
W = ceil(m / 32) and facility j open iff bit (j & 31) of word (j >> 5) is set.
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "graph_instance",
    "euclid_instance",
    "gmm_instance",
    "random_masks",
    "masks_from_sets",
    "sets_from_masks",
    "mask_words",
    "paper_shape_instance",
    "batched_instances",
]


def mask_words(m: int) -> int:
    """Number of uint32 words in one facility bitset of m facilities."""
    return (int(m) + 31) // 32


def graph_instance(n: int, edges: int, seed: int, wmin: int = 1, wmax: int = 100) -> np.ndarray:
    """All-pairs shortest-path distances of a connected random graph.

    A random recursive spanning tree (node v attaches to a uniform node in
    [0, v)) is extended with distinct non-tree edges drawn uniformly (no
    self-loops, no duplicates) up to ``edges`` edges.  Weights are uniform
    integers in [wmin, wmax].  Returns an int32 n x n matrix, d_ii = 0.
    """
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import shortest_path

    n = int(n)
    edges = int(edges)
    if n < 1:
        raise ValueError("n must be >= 1")
    max_edges = n * (n - 1) // 2
    if edges < n - 1 or edges > max_edges:
        raise ValueError(f"edges must be in [{n - 1}, {max_edges}]")
    rng = np.random.default_rng(seed)
    us = np.empty(edges, dtype=np.int64)
    vs = np.empty(edges, dtype=np.int64)
    for v in range(1, n):
        us[v - 1] = int(rng.integers(0, v))
        vs[v - 1] = v
    seen = set(zip(us[: n - 1].tolist(), vs[: n - 1].tolist()))
    k = n - 1
    while k < edges:
        need = edges - k
        a = rng.integers(0, n, size=2 * need + 16)
        b = rng.integers(0, n, size=2 * need + 16)
        for x, y in zip(a.tolist(), b.tolist()):
            if x == y:
                continue
            key = (x, y) if x < y else (y, x)
            if key in seen:
                continue
            seen.add(key)
            us[k], vs[k] = key
            k += 1
            if k == edges:
                break
    w = rng.integers(wmin, wmax + 1, size=edges).astype(np.float64)
    g = coo_matrix((w, (us, vs)), shape=(n, n)).tocsr()
    dist = shortest_path(g, method="D", directed=False)
    if not np.all(np.isfinite(dist)):
        raise RuntimeError("graph is not connected")
    return np.ascontiguousarray(dist.astype(np.int32))


def _round_half_away(x: np.ndarray) -> np.ndarray:
    return np.floor(x + 0.5)  # x >= 0 here


def _points_distance(pts: np.ndarray) -> np.ndarray:
    n = pts.shape[0]
    out = np.empty((n, n), dtype=np.int32)
    step = max(1, (1 << 24) // max(n, 1))
    for r0 in range(0, n, step):
        r1 = min(n, r0 + step)
        dx = pts[r0:r1, 0:1] - pts[None, :, 0]
        dy = pts[r0:r1, 1:2] - pts[None, :, 1]
        out[r0:r1] = _round_half_away(1e4 * np.hypot(dx, dy)).astype(np.int32)
    return out


def euclid_instance(n: int, seed: int) -> np.ndarray:
    """n points uniform in [0,1)^2; d_ij = round(1e4 * |x_i - x_j|) as int32."""
    rng = np.random.default_rng(seed)
    pts = rng.random((int(n), 2))
    return _points_distance(pts)


def gmm_instance(n: int, seed: int, components: int = 50, sigma: float = 0.02) -> np.ndarray:
    """n points from an equal-weight Gaussian mixture in the unit square.

    Centres are uniform in [0,1)^2; a point is its centre plus N(0, sigma^2)
    per coordinate, redrawn until it lies in [0,1]^2.  d as in euclid_instance.
    """
    rng = np.random.default_rng(seed)
    centres = rng.random((components, 2))
    pts = np.empty((int(n), 2))
    for i in range(int(n)):
        c = centres[int(rng.integers(0, components))]
        while True:
            q = c + rng.normal(0.0, sigma, size=2)
            if 0.0 <= q[0] <= 1.0 and 0.0 <= q[1] <= 1.0:
                pts[i] = q
                break
    return _points_distance(pts)


def random_masks(P: int, m: int, p: int, seed: int) -> np.ndarray:
    """P uniformly random p-subsets of m facilities as a (P, W) uint32 bitset array."""
    rng = np.random.default_rng(seed)
    W = mask_words(m)
    out = np.zeros((int(P), W), dtype=np.uint32)
    if P == 0:
        return out
    chunk = max(1, (1 << 22) // max(m, 1))
    for r0 in range(0, P, chunk):
        r1 = min(P, r0 + chunk)
        keys = rng.random((r1 - r0, m))
        sel = np.argpartition(keys, p - 1, axis=1)[:, :p] if p < m else np.tile(np.arange(m), (r1 - r0, 1))
        rows = np.repeat(np.arange(r0, r1), p)
        cols = sel.reshape(-1)
        np.bitwise_or.at(out, (rows, cols >> 5), (np.uint32(1) << (cols & 31).astype(np.uint32)))
    return out


def masks_from_sets(sets, m: int) -> np.ndarray:
    """Bitset array from an iterable of iterables of 0-based facility ids."""
    sets = [list(s) for s in sets]
    out = np.zeros((len(sets), mask_words(m)), dtype=np.uint32)
    for t, s in enumerate(sets):
        for j in s:
            out[t, j >> 5] |= np.uint32(1) << np.uint32(j & 31)
    return out


def sets_from_masks(masks: np.ndarray, m: int):
    """List of sorted facility-id lists, one per bitset row."""
    res = []
    for row in np.asarray(masks, dtype=np.uint32):
        bits = np.unpackbits(row.view(np.uint8), bitorder="little")[:m]
        res.append(np.nonzero(bits)[0].tolist())
    return res


def paper_shape_instance(name: str) -> dict:
    """The synthetic workloads shaped like the paper's benchmarks.

    Returns a dict with the distance matrix ``d`` and the run parameters.
    Instance seeds are fixed per workload so every caller sees the same data.
    """
    if name == "graph100":  # OR-Library pmed1 shape (Table 1)
        return dict(d=graph_instance(100, 200, seed=0), p=5, pop=64, gens=200)
    if name == "graph100_sub20":  # top-left 20x20 block of graph100
        d = graph_instance(100, 200, seed=0)
        return dict(d=np.ascontiguousarray(d[:20, :20]), p=4, pop=64, gens=50)
    if name == "graph900":  # OR-Library pmed40 shape (Table 1)
        return dict(d=graph_instance(900, 16200, seed=1), p=90, pop=1024, gens=1000)
    if name.startswith("euclid10000"):
        return dict(d=euclid_instance(10000, seed=2), p=int(name.split("_p")[1]), pop=4096, gens=1)
    if name.startswith("gmm5000"):
        return dict(d=gmm_instance(5000, seed=4), p=int(name.split("_p")[1]), pop=1024, gens=0)
    raise KeyError(name)


def training_instances(name: str, count: int = 4) -> list:
    """Instances of the same shape as workload `name` but other instance seeds (10, 11, ...): the learned swap
    proposal is trained on their logged moves and timed on the workload's own instance, which it never sees."""
    if name == "graph100":
        return [graph_instance(100, 200, seed=10 + k) for k in range(count)]
    if name.startswith("gmm5000"):
        return [gmm_instance(5000, seed=10 + k) for k in range(count)]
    raise KeyError(name)


def _batched_one(spec):
    k, n, p, sub = spec
    if k % 2 == 0:
        d = graph_instance(n, min(4 * n, n * (n - 1) // 2), seed=sub)
    else:
        d = euclid_instance(n, seed=sub)
    return d, p


def batched_instances(count: int, seed: int, nmin: int = 100, nmax: int = 5000, workers: int = 1):
    """Uneven instances for batched evaluation.

    n = m log-uniform in [nmin, nmax]; p uniform in [5, n/10]; even entries are
    graph instances (4n edges, weights [1,100], shortest paths), odd entries
    Euclidean.  Returns a list of (d, p).  workers > 1 builds them in a pool of
    spawned processes (call it before any CUDA work in the calling process).
    """
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(int(count)):
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        n = max(nmin, min(nmax, n))
        p = int(rng.integers(5, max(6, n // 10) + 1))
        p = min(p, n - 1)
        sub = int(rng.integers(0, 2**31 - 1))
        specs.append((k, n, p, sub))
    if workers <= 1:
        return [_batched_one(s) for s in specs]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    with ProcessPoolExecutor(max_workers=int(workers), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_batched_one, specs, chunksize=1))

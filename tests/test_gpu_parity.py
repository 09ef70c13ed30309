"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tables and costs are integers, so the bar is bit-exact equality.  Cases span
several tiles with ragged tails (m and pop not multiples of 32 or 128), the
degenerate shapes (L = 2, p = 1, n = 1, all-equal distances, 31-bit
distances), both fitness kernels (facility-major tiles and the row kernel for
very large m) and, at the full workload sizes, sampled individuals checked by
the direct evaluator.
"""

import os

import numpy as np
import pytest

import oracle
from paper_1610_10061_gb300.inputs import (euclid_instance, graph_instance, masks_from_sets, paper_shape_instance,
                                           random_masks, sets_from_masks)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_10061_gb300 import build

    build.build()
    from paper_1610_10061_gb300 import pm as _pm

    torch.cuda.set_device(0)
    return _pm


def to_dev(masks):
    return torch.from_numpy(np.ascontiguousarray(masks).view(np.int32)).cuda()


def _shapes():
    rng = np.random.default_rng(0)
    out = []
    out.append(("n1", rng.integers(0, 50, size=(1, 2)).astype(np.int32), 1))
    out.append(("ties", rng.integers(0, 3, size=(30, 70)).astype(np.int32), 9))
    out.append(("allzero", np.zeros((9, 40), dtype=np.int32), 4))
    out.append(("L2", rng.integers(0, 1000, size=(33, 65)).astype(np.int32), 64))
    out.append(("p1", rng.integers(0, 1000, size=(40, 300)).astype(np.int32), 1))
    out.append(("big31", rng.integers(0, 2**31 - 1, size=(20, 50)).astype(np.int32), 3))
    out.append(("graph", graph_instance(100, 200, seed=0), 5))
    out.append(("euclid", euclid_instance(700, seed=3)[:250], 17))
    return out


@pytest.mark.parametrize("name,d,p", _shapes(), ids=[s[0] for s in _shapes()])
def test_tables_bit_exact(pm, name, d, p):
    inst = pm.Instance(d, p)
    pi, de = inst.tables()
    opi, ode = oracle.tables(d, p)
    np.testing.assert_array_equal(pi, opi)
    np.testing.assert_array_equal(de, ode)
    assert inst.L == d.shape[1] - p + 1 and inst.stride % 32 == 0
    inst.close()


def test_example1_through_the_abi(pm, example1):
    C = np.array(example1["C"], dtype=np.int32)
    inst = pm.Instance(C, 2)
    pi, de = inst.tables()
    np.testing.assert_array_equal(pi.astype(int) + 1, np.array(example1["PI_TRUNC"]))
    np.testing.assert_array_equal(de, np.array(example1["DELTA_TRUNC"]))
    import itertools

    sets = list(itertools.combinations(range(4), 2))
    costs = inst.eval(masks_from_sets(sets, 4), checked=True)
    # the printed reduced polynomial of Example 1 evaluated at z = 1 - x
    poly = {tuple(v - 1 for v in row[1:]): row[0] for row in example1["POLY"]}
    expect = [sum(c for mono, c in poly.items() if not set(mono) & set(s)) for s in sets]
    np.testing.assert_array_equal(costs, expect)


@pytest.mark.parametrize("name,d,p", _shapes(), ids=[s[0] for s in _shapes()])
@pytest.mark.parametrize("pop", [1, 31, 33, 129, 1000])
def test_eval_bit_exact(pm, name, d, p, pop):
    m = d.shape[1]
    inst = pm.Instance(d, p)
    masks = random_masks(pop, m, p, seed=pop + m)
    expect = oracle.eval_direct(d, masks)
    opi, ode = oracle.tables(d, p)
    np.testing.assert_array_equal(expect, oracle.eval_scan(opi, ode, masks))
    # host buffers (staged by the library)
    np.testing.assert_array_equal(inst.eval(masks), expect)
    # device buffers (used in place)
    got = inst.eval(to_dev(masks))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), expect)
    inst.close()


def test_eval_empty_and_checked(pm):
    d = graph_instance(60, 150, seed=2)
    inst = pm.Instance(d, 6)
    out = np.full(3, -7, dtype=np.int64)
    pm.pm_eval_population(inst.handle, np.zeros((0, 2), dtype=np.uint32), 0, out)
    assert (out == -7).all()
    good = random_masks(40, 60, 6, seed=1)
    np.testing.assert_array_equal(inst.eval(good, checked=True), oracle.eval_direct(d, good))
    bad = good.copy()
    bad[17, 0] ^= 1  # popcount p +- 1
    with pytest.raises(pm.PMError) as e:
        inst.eval(bad, checked=True)
    assert e.value.status == 4
    stray = good.copy()
    keep = sets_from_masks(good[3:4], 60)[0][1:]  # p-1 open facilities ...
    stray[3] = masks_from_sets([keep], 60)[0]
    stray[3, 1] |= np.uint32(1) << np.uint32(31)  # ... plus bit 63, beyond m = 60
    with pytest.raises(pm.PMError) as e:
        inst.eval(stray, checked=True)
    assert e.value.status == 4


def test_negative_distance_rejected(pm):
    d = np.ones((5, 6), dtype=np.int32)
    d[3, 2] = -1
    with pytest.raises(pm.PMError) as e:
        pm.Instance(d, 2)
    assert e.value.status == 2


def test_device_distance_matrix(pm):
    d = euclid_instance(300, seed=9)
    dd = torch.from_numpy(d).cuda()
    inst = pm.Instance(dd, 30)
    opi, ode = oracle.tables(d, 30)
    pi, de = inst.tables()
    np.testing.assert_array_equal(pi, opi)
    np.testing.assert_array_equal(de, ode)


def test_row_kernel_for_very_large_m(pm):
    """m = 60000: the facility-major tile exceeds shared memory, the row kernel runs; the sort uses global scratch."""
    rng = np.random.default_rng(3)
    m = 60000
    d = rng.integers(0, 5000, size=(5, m)).astype(np.int32)
    p = 40
    inst = pm.Instance(d, p)
    opi, ode = oracle.tables(d, p)
    pi, de = inst.tables()
    np.testing.assert_array_equal(pi, opi)
    np.testing.assert_array_equal(de, ode)
    masks = random_masks(70, m, p, seed=5)
    np.testing.assert_array_equal(inst.eval(masks), oracle.eval_scan(opi, ode, masks))


@pytest.fixture(scope="module")
def euclid10000():
    """The n = m = 10000 Euclidean instance and the oracle's full (untruncated) tables of it, computed once: the
    truncated tables for any p are their first m - p + 1 columns (Section 2.1)."""
    d = paper_shape_instance("euclid10000_p100")["d"]
    opi, ode = oracle.tables(d, full=True)
    return d, opi, ode


def _scan_threads(pi, de, masks):
    """The oracle's O3 over a population, split over the host's cores (the C call releases the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor

    parts = np.array_split(masks, max(1, min(32, len(os.sched_getaffinity(0)))))
    with ThreadPoolExecutor(len(parts)) as ex:
        outs = list(ex.map(lambda x: oracle.eval_scan(pi, de, x), parts))
    return np.concatenate(outs)


@pytest.mark.parametrize("p", [10, 100, 1000])
def test_full_size_euclid10000_every_cost(pm, euclid10000, p):
    """n = m = 10000, pop 4096 (the fitness-throughput workload) in the launch shape the benchmark tunes: every
    one of the 4096 costs against the oracle's O3 over the oracle's own tables, sampled individuals against O1
    (the direct definition), and sampled table rows."""
    d, fpi, fde = euclid10000
    L = 10000 - p + 1
    opi, ode = np.ascontiguousarray(fpi[:, :L]), np.ascontiguousarray(fde[:, :L])
    inst = pm.Instance(d, p)
    inst.tune(4096)
    masks = random_masks(4096, 10000, p, seed=p)
    got = inst.eval(to_dev(masks))
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    np.testing.assert_array_equal(got, _scan_threads(opi, ode, masks))
    rng = np.random.default_rng(p)
    sample = np.concatenate([rng.choice(4096, size=6, replace=False), [0, 4095]])
    np.testing.assert_array_equal(got[sample], oracle.eval_direct(d, masks[sample]))
    rows = rng.choice(10000, size=8, replace=False)
    pi, de = inst.tables()
    np.testing.assert_array_equal(pi[rows], opi[rows])
    np.testing.assert_array_equal(de[rows], ode[rows])


# --------------------------------------------------------------------------
# The GA: bit-exact trajectories
# --------------------------------------------------------------------------

def _ga_compare(pm, d, p, pop, gens, check_every=1, shape=None, cumulative=False, **kw):
    inst = pm.Instance(d, p, cumulative=cumulative)
    if shape is not None:
        inst.set_shape(pop, **shape)
    opi, ode = oracle.tables(d, p)
    m = d.shape[1]
    okw = dict(kw)
    sid = okw.pop("stream_id", 0)
    migration = kw.get("migration", "deme")
    init = kw.get("init", "floyd")
    st, otrace, opops, ocosts = oracle.ga_run(opi, ode, m, p, seed=kw.get("seed", 0), P=pop, D=kw.get("deme") or None,
                                              gens=gens, xover_rounds=kw.get("xover_rounds"),
                                              mut_tries=kw.get("mut_tries"), saturation=kw.get("saturation", 0),
                                              record=True, inst=sid, team=migration == "team", init=init)
    ga = pm.GA(inst, seed=kw.get("seed", 0), pop=pop, deme=kw.get("deme") or 0,
               xover_rounds=-1 if kw.get("xover_rounds") is None else kw["xover_rounds"],
               mut_tries=-1 if kw.get("mut_tries") is None else kw["mut_tries"],
               saturation=kw.get("saturation", 0), stream_id=sid, migration=migration, init=init)
    done = 0
    traces = []
    while done < len(otrace):
        k = min(check_every, len(otrace) - done)
        traces.append(ga.step(k))
        done += k
        masks, costs = ga.population()
        np.testing.assert_array_equal(masks, opops[done - 1], err_msg=f"population after generation {done}")
        np.testing.assert_array_equal(costs, ocosts[done - 1], err_msg=f"costs after generation {done}")
    np.testing.assert_array_equal(np.concatenate(traces), otrace)
    bc, gr, ev, mask = ga.result()
    assert bc == st.best_cost and ev == st.evals and gr == len(otrace)
    np.testing.assert_array_equal(mask, st.best)
    return ga, inst


def test_ga_graph100_every_generation(pm):
    w = paper_shape_instance("graph100")
    _ga_compare(pm, w["d"], w["p"], 64, 40, check_every=1)


def test_ga_graph100_full_run_reaches_brute_force_on_sub20(pm):
    w = paper_shape_instance("graph100")
    _ga_compare(pm, w["d"], w["p"], 64, 200, check_every=50)
    s = paper_shape_instance("graph100_sub20")
    best, _ = oracle.brute_force(s["d"], s["p"])
    ga, _ = _ga_compare(pm, s["d"], s["p"], 64, 30, check_every=10)
    assert ga.result()[0] == best


def test_ga_graph900_twenty_generations(pm):
    """The benchmark's GA (n = m = 900, p = 90, pop 1024 in demes of 256) in the tuned shapes the benchmark uses:
    population, costs and best after each of 20 generations."""
    w = paper_shape_instance("graph900")
    inst = pm.Instance(w["d"], w["p"])
    inst.tune(1024)
    inst.tune(1024 * 8)
    opi, ode = oracle.tables(w["d"], w["p"])
    st, otrace, opops, ocosts = oracle.ga_run(opi, ode, 900, 90, seed=0, P=1024, D=256, gens=20, record=True)
    ga = pm.GA(inst, seed=0, pop=1024, deme=256)
    for g in range(20):
        tr = ga.step(1)
        assert tr[0] == otrace[g]
        masks, costs = ga.population()
        np.testing.assert_array_equal(masks, opops[g], err_msg=f"population after generation {g + 1}")
        np.testing.assert_array_equal(costs, ocosts[g], err_msg=f"costs after generation {g + 1}")
    bc, gr, ev, mask = ga.result()
    assert bc == st.best_cost and ev == st.evals and gr == 20
    np.testing.assert_array_equal(mask, st.best)


@pytest.mark.parametrize("kw", [
    dict(deme=16, seed=5),
    dict(deme=2, seed=1),
    dict(xover_rounds=0, mut_tries=3, seed=2),
    dict(xover_rounds=7, mut_tries=0, deme=8, seed=3),
    dict(stream_id=9, seed=4),
    dict(migration="team", deme=16, seed=6),            # migration variant (ii) of Section 4.5
    dict(migration="team", deme=16, seed=7, xover_rounds=20, mut_tries=20),
    dict(xover_rounds=60, mut_tries=60, deme=16, seed=8),  # the paper's preset iteration counts (60, 20)
    dict(xover_rounds=20, mut_tries=20, deme=32, seed=9),
])
def test_ga_variants(pm, kw):
    d = euclid_instance(77, seed=11)
    _ga_compare(pm, d, 7, 128, 6, check_every=2, **kw)


def test_ga_p1_and_saturation(pm):
    d = graph_instance(45, 100, seed=4)
    _ga_compare(pm, d, 1, 64, 5, check_every=5)
    _ga_compare(pm, d, 3, 32, 300, check_every=300, deme=16, saturation=3)


@pytest.mark.parametrize("migration", ["deme", "team"])
def test_ga_save_load_resume(pm, migration):
    d = graph_instance(100, 200, seed=0)
    inst = pm.Instance(d, 5)
    a = pm.GA(inst, seed=7, pop=64, deme=8, migration=migration)
    ta = a.step(12)
    b = pm.GA(inst, seed=7, pop=64, deme=8, migration=migration)
    tb1 = b.step(5)
    blob = b.save()
    b.close()
    c = pm.GA.load(inst, blob)
    tb2 = c.step(7)
    np.testing.assert_array_equal(np.concatenate([tb1, tb2]), ta)
    ma, ca = a.population()
    mc, cc = c.population()
    np.testing.assert_array_equal(ma, mc)
    np.testing.assert_array_equal(ca, cc)
    assert a.result()[:3] == c.result()[:3]


@pytest.mark.parametrize("pop,deme", [(2048, 16), (2048, 512), (3072, 1024)])
def test_generation_end_over_several_tiles(pm, pop, deme):
    """The one-CTA generation end walks the population 1024 individuals at a time: demes narrower than a warp
    (reduced inside the warp butterfly), demes of several warps and of a whole tile, over two and three tiles."""
    _ga_compare(pm, graph_instance(150, 400, seed=3), 8, pop, 3, check_every=1, deme=deme, seed=9)


@pytest.mark.parametrize("m,p", [(40, 39), (64, 33), (96, 70), (70, 64)])
def test_floyd_batches_with_many_collisions(pm, m, p):
    """Floyd's insertions resolved 32 at a time where draws collide often (p close to m: a draw hits the set of
    the earlier batches or an earlier lane's pick), against the oracle's sequential insertions."""
    _ga_compare(pm, euclid_instance(m, seed=m + p), p, 64, 3, check_every=1, deme=32, seed=m)


def test_ga_stream_launch_mode_matches_graph_mode(pm, monkeypatch):
    """PM_GA_GRAPH=0 (direct stream launches, for profilers) gives the graph mode's results bit for bit."""
    d = graph_instance(100, 200, seed=0)
    inst = pm.Instance(d, 5)
    a = pm.GA(inst, seed=3, pop=128, deme=32)
    ta = a.step(9)
    monkeypatch.setenv("PM_GA_GRAPH", "0")
    b = pm.GA(inst, seed=3, pop=128, deme=32)
    tb = b.step(9)
    np.testing.assert_array_equal(ta, tb)
    for x, y in zip(a.population(), b.population()):
        np.testing.assert_array_equal(x, y)
    assert a.result()[:3] == b.result()[:3]
    # saturation stop in stream mode, against the oracle
    _ga_compare(pm, graph_instance(30, 60, seed=1), 3, 32, 300, check_every=300, deme=16, saturation=4)


def test_one_generation_calls_equal_one_long_call(pm, monkeypatch):
    """Calls of one generation run a plain graph of the generation (no conditional loop); stepping one generation
    at a time gives the same traces, populations and results as one call of many generations, including across
    a saturation stop (the later one-generation calls change nothing)."""
    monkeypatch.delenv("PM_GA_GRAPH", raising=False)
    w = paper_shape_instance("graph900")
    inst = pm.Instance(w["d"], w["p"])
    a = pm.GA(inst, seed=5, pop=512, deme=128)
    ta = a.step(6)
    b = pm.GA(inst, seed=5, pop=512, deme=128)
    tb = np.concatenate([b.step(1) for _ in range(6)])
    np.testing.assert_array_equal(ta, tb)
    for x, y in zip(a.population(), b.population()):
        np.testing.assert_array_equal(x, y)
    assert a.result()[:3] == b.result()[:3]
    d = graph_instance(30, 60, seed=1)
    small = pm.Instance(d, 3)
    a = pm.GA(small, seed=2, pop=32, deme=16, saturation=3)
    a.step(60)
    b = pm.GA(small, seed=2, pop=32, deme=16, saturation=3)
    for _ in range(60):
        b.step(1)
    ra, rb = a.result(), b.result()
    assert ra[:3] == rb[:3] and ra[1] < 60  # stopped by saturation, at the same generation
    np.testing.assert_array_equal(ra[3], rb[3])


def _ga_run_pair(pm, monkeypatch, d, p, pop, gens, steps, **kw):
    """The same GA twice, with the persistent generation kernel (PM_GA_FUSED=1) and with the per-phase kernels
    (the default): traces, populations, costs and results."""
    inst = pm.Instance(d, p, cumulative=kw.pop("cumulative", False))
    out = []
    for fused in (True, False):
        if fused:
            monkeypatch.setenv("PM_GA_FUSED", "1")
        else:
            monkeypatch.delenv("PM_GA_FUSED", raising=False)
        ga = pm.GA(inst, pop=pop, **kw)
        info = ga.info()
        assert (info["kernels_per_generation"] == 0) == fused, info
        traces = [ga.step(k) for k in steps]
        out.append((np.concatenate(traces), *ga.population(), ga.result()))
        ga.close()
    monkeypatch.delenv("PM_GA_FUSED", raising=False)
    (ta, ma, ca, ra), (tb, mb, cb, rb) = out
    np.testing.assert_array_equal(ta, tb)
    np.testing.assert_array_equal(ma, mb)
    np.testing.assert_array_equal(ca, cb)
    assert ra[:3] == rb[:3]
    np.testing.assert_array_equal(ra[3], rb[3])
    return ta


@pytest.mark.parametrize("case", ["graph900", "euclid_ragged", "team_cum", "deme2", "p1_sat"])
def test_persistent_generation_kernel_equals_the_per_phase_kernels(pm, monkeypatch, case):
    """One cooperative launch per pm_ga_step (grid barriers between the phases) against the per-phase kernels:
    bit-identical GA at the benchmark's shape, a ragged population, migration variant (ii) on cumulative tables,
    demes of 2, and p = 1 with a saturation stop inside a step."""
    if case == "graph900":
        w = paper_shape_instance("graph900")
        _ga_run_pair(pm, monkeypatch, w["d"], w["p"], 1024, 6, [1, 2, 3], seed=3, deme=256)
    elif case == "euclid_ragged":
        _ga_run_pair(pm, monkeypatch, euclid_instance(333, seed=4), 17, 96, 5, [2, 3], seed=1, deme=32)
    elif case == "team_cum":
        _ga_run_pair(pm, monkeypatch, graph_instance(150, 400, seed=2), 9, 256, 4, [4], seed=2, deme=16,
                     migration="team", cumulative=True)
    elif case == "deme2":
        _ga_run_pair(pm, monkeypatch, euclid_instance(70, seed=6), 5, 64, 5, [5], seed=7, deme=2)
    else:
        tr = _ga_run_pair(pm, monkeypatch, graph_instance(45, 100, seed=4), 1, 64, 300, [300], seed=5, deme=16,
                          saturation=3)
        assert len(tr) < 300


@pytest.mark.parametrize("name,d,p", [s for s in _shapes() if s[0] in ("ties", "p1", "graph", "euclid")],
                         ids=["ties", "p1", "graph", "euclid"])
def test_autotuned_shape_stays_bit_exact(pm, name, d, p):
    m = d.shape[1]
    inst = pm.Instance(d, p)
    for pop in (40, 700):
        shape = inst.tune(pop)
        # any candidate may win the timing: bit columns (G = 1, 2, 4), row bitsets (0) or row byte masks (-1)
        assert shape["groups"] in (-1, 0, 1, 2, 4) and shape["candidates"] >= 1 and shape["ms"] > 0
        masks = random_masks(pop, m, p, seed=3 * pop)
        np.testing.assert_array_equal(inst.eval(masks), oracle.eval_direct(d, masks))
    inst.close()


def test_ga_with_autotuned_shape_matches_untuned(pm):
    w = paper_shape_instance("graph900")
    inst = pm.Instance(w["d"], w["p"])
    a = pm.GA(inst, seed=11, pop=512, deme=128)
    ta = a.step(2)
    b = pm.GA(inst, seed=11, pop=512, deme=128, tune=True)
    tb = b.step(2)
    np.testing.assert_array_equal(ta, tb)
    for x, y in zip(a.population(), b.population()):
        np.testing.assert_array_equal(x, y)
    assert a.result()[:3] == b.result()[:3]


def test_bounded_wait_times_out_and_context_survives(pm):
    """A wait on a flag nothing sets gives up with PM_ERR_TIMEOUT; the next evaluation still works."""
    assert pm.pm_selftest_bounded_wait(0) == 7
    d = graph_instance(50, 120, seed=3)
    inst = pm.Instance(d, 4)
    masks = random_masks(40, 50, 4, seed=2)
    np.testing.assert_array_equal(inst.eval(masks), oracle.eval_direct(d, masks))


def _pinned_shapes(pm, inst, pop):
    """Every evaluation shape (G, warps, splits) this instance accepts, pinned in turn; G = 0 is the row kernel
    with bitsets, G = -1 the row kernel with byte masks."""
    for G in (-1, 0, 1, 2, 4):
        for warps in ((8,) if G <= 0 else (8, 16, 32)):
            for splits in (1, 3, 0):
                try:
                    inst.set_shape(pop, groups=G, warps=warps, splits=splits)
                except pm.PMError as e:
                    assert e.status == 3, e  # PM_ERR_UNSUPPORTED: does not fit
                    continue
                yield G, warps, splits


@pytest.mark.parametrize("name,d,p", [s for s in _shapes() if s[0] in ("ties", "allzero", "L2", "big31", "graph",
                                                                       "euclid", "p1")],
                         ids=["ties", "allzero", "L2", "p1", "big31", "graph", "euclid"])
def test_every_pinned_shape_bit_exact(pm, name, d, p):
    """pm_set_eval_shape: each launch shape gives the oracle's costs (ragged populations, 1 or many splits)."""
    m = d.shape[1]
    inst = pm.Instance(d, p)
    for pop in (33, 700):
        masks = random_masks(pop, m, p, seed=5 * pop + m)
        expect = oracle.eval_direct(d, masks)
        seen = 0
        for G, warps, splits in _pinned_shapes(pm, inst, pop):
            np.testing.assert_array_equal(inst.eval(masks), expect, err_msg=f"G={G} warps={warps} splits={splits}")
            seen += 1
        assert seen >= 10, seen
    with pytest.raises(pm.PMError):
        inst.set_shape(64, groups=3, warps=16)
    inst.close()


def test_ga_on_pinned_shapes_matches_oracle(pm):
    w = paper_shape_instance("graph900")
    _ga_compare(pm, w["d"], w["p"], 1024, 2, check_every=1, shape=dict(groups=1, warps=8, splits=3))
    _ga_compare(pm, euclid_instance(77, seed=11), 7, 128, 6, check_every=2, deme=16, seed=5,
                shape=dict(groups=0, warps=8, splits=2))
    _ga_compare(pm, euclid_instance(77, seed=11), 7, 128, 6, check_every=2, deme=16, seed=6,
                shape=dict(groups=-1, warps=8, splits=2))  # byte masks


@pytest.mark.parametrize("name,d,p", _shapes(), ids=[s[0] for s in _shapes()])
def test_cumulative_tables_bit_exact(pm, name, d, p):
    """PM_TABLES_CUMULATIVE: the tables read back as Pi'/Delta', and every shape evaluates to the oracle's costs."""
    m = d.shape[1]
    inst = pm.Instance(d, p, cumulative=True)
    assert pm.pm_instance_flags(inst.handle) == pm.PM_TABLES_CUMULATIVE
    pi, de = inst.tables()
    opi, ode = oracle.tables(d, p)
    np.testing.assert_array_equal(pi, opi)
    np.testing.assert_array_equal(de, ode)
    dev = torch.zeros((d.shape[0], inst.L), dtype=torch.int32, device="cuda")
    pm.pm_instance_tables(inst.handle, None, dev)
    np.testing.assert_array_equal(dev.cpu().numpy(), ode)
    for pop in (1, 33, 1000):
        masks = random_masks(pop, m, p, seed=pop + 2 * m)
        expect = oracle.eval_direct(d, masks)
        np.testing.assert_array_equal(oracle.eval_cumulative(opi, oracle.cumulative(ode), masks), expect)
        np.testing.assert_array_equal(inst.eval(masks), expect)
        if pop == 1000:
            for G, warps, splits in _pinned_shapes(pm, inst, pop):
                np.testing.assert_array_equal(inst.eval(masks), expect, err_msg=f"G={G} warps={warps}")
    inst.close()


def test_cumulative_row_kernel_and_full_size_sample(pm):
    rng = np.random.default_rng(8)
    d = rng.integers(0, 1 << 20, size=(6, 60000)).astype(np.int32)  # m too large for facility-major tiles
    inst = pm.Instance(d, 7, cumulative=True)
    masks = random_masks(40, 60000, 7, seed=2)
    np.testing.assert_array_equal(inst.eval(masks), oracle.eval_direct(d, masks))
    inst.close()


def test_ga_on_cumulative_tables_matches_oracle(pm):
    w = paper_shape_instance("graph900")
    _ga_compare(pm, w["d"], w["p"], 1024, 2, check_every=1, cumulative=True)
    _ga_compare(pm, euclid_instance(77, seed=11), 7, 128, 6, check_every=2, deme=16, seed=5, cumulative=True,
                migration="team")


@pytest.mark.parametrize("m,n,p,pop,gens,kw", [
    (100, 100, 5, 64, 3, dict(deme=16, seed=3)),                       # C(100, 5): 2 words
    (900, 120, 90, 64, 2, dict(deme=32, seed=4, xover_rounds=0, mut_tries=0)),  # C(900, 90): 14 words
    (2000, 40, 600, 32, 2, dict(deme=16, seed=5, xover_rounds=1, mut_tries=1)),  # 56 words: two per lane
    (64, 30, 1, 32, 2, dict(deme=16, seed=6)),                         # p = 1
    (70, 30, 69, 32, 2, dict(deme=16, seed=7, migration="team")),      # p = m - 1
])
def test_ga_combinadic_generation_matches_oracle(pm, m, n, p, pop, gens, kw):
    """Section 4.1's chromosome generation (multi-word random rank, lexicographic unranking) bit-exact."""
    d = euclid_instance(m, seed=m)[:n]
    _ga_compare(pm, d, p, pop, gens, check_every=1, init="combinadic", **kw)


def test_split_reduction_both_protocols(pm):
    """Costs below 2^47 use the packed split reduction (sum and split count in one atomic word); larger ones
    (here n * max d > 2^47) fall back to per-tile tickets.  Both bit-exact, over several pinned split counts."""
    rng = np.random.default_rng(21)
    small = rng.integers(0, 1000, size=(300, 50)).astype(np.int32)
    large = rng.integers(2**30, 2**31 - 1, size=(70000, 40)).astype(np.int32)  # 70000 * 2^31 > 2^47
    for d, p in ((small, 6), (large, 5)):
        inst = pm.Instance(d, p)
        masks = random_masks(100, d.shape[1], p, seed=3)
        expect = oracle.eval_direct(d, masks)
        assert (d.shape[0] * int(d.max()) >= 2**47) == (d is large)  # the bound that selects the protocol
        for G, splits in ((1, 3), (2, 7), (4, 2), (1, 1)):
            inst.set_shape(100, groups=G, warps=8, splits=splits)
            for _ in range(2):  # the second launch relies on the first leaving the scratch at zero
                np.testing.assert_array_equal(inst.eval(masks), expect, err_msg=f"G={G} splits={splits}")
        inst.close()


def test_client_sharded_evaluation_on_one_gpu(pm):
    """Client blocks evaluated as separate instances add up to the full cost (the all-reduce of the
    client-sharded evaluation, done here on the device with torch); with one rank the sharded evaluator is the
    plain evaluation."""
    from paper_1610_10061_gb300.shard import ShardedEvaluator, client_block

    w = paper_shape_instance("graph900")
    d, p = w["d"], w["p"]
    masks = random_masks(256, 900, p, seed=13)
    expect = oracle.eval_direct(d, masks)
    dm = to_dev(masks)
    total = torch.zeros(256, dtype=torch.int64, device="cuda")
    for r in range(3):
        lo, hi = client_block(900, r, 3)
        inst = pm.Instance(d[lo:hi], p, cumulative=(r == 1))
        total += inst.eval(dm)
        inst.close()
    np.testing.assert_array_equal(total.cpu().numpy(), expect)
    ev = ShardedEvaluator(d, p)
    np.testing.assert_array_equal(ev.eval(dm).cpu().numpy(), expect)
    ev.close()


def test_speculative_mutation_cycle_matches_try_by_try(pm, monkeypatch):
    """All Q mutation tries evaluated in one scan (the default for one instance on the column path) give the
    same populations, costs and evaluation counts as the cycle run try by try (PM_GA_SPEC=0), and as the oracle."""
    w = paper_shape_instance("graph900")
    d, p = w["d"], w["p"]
    inst = pm.Instance(d, p)
    a = pm.GA(inst, seed=17, pop=512, deme=128)
    ta = a.step(3)
    info = a.info()
    monkeypatch.setenv("PM_GA_SPEC", "0")
    b = pm.GA(inst, seed=17, pop=512, deme=128)
    tb = b.step(3)
    np.testing.assert_array_equal(ta, tb)
    for x, y in zip(a.population(), b.population()):
        np.testing.assert_array_equal(x, y)
    assert a.result()[:3] == b.result()[:3]
    # the speculative cycle launches 3 kernels in place of 2 per try
    assert info["kernels_per_generation"] == b.info()["kernels_per_generation"] - 2 * info["mut_tries"] + 3
    monkeypatch.delenv("PM_GA_SPEC")
    _ga_compare(pm, d, p, 512, 2, check_every=1, deme=128, seed=17, xover_rounds=2, mut_tries=20)
    # more tries than a warp has lanes: the first improving try is searched 32 tries at a time
    _ga_compare(pm, euclid_instance(77, seed=11), 7, 128, 4, check_every=1, deme=16, seed=8, xover_rounds=3,
                mut_tries=33)


@pytest.mark.parametrize("pop,deme", [(48, 16), (80, 16), (96, 32)])
def test_ga_ragged_populations(pm, pop, deme):
    """Populations that are not a multiple of 32: partial tiles in the scans, the speculative mutation
    candidates (q * pop + t) straddling 32-candidate groups."""
    _ga_compare(pm, graph_instance(120, 300, seed=pop), 6, pop, 4, check_every=1, deme=deme, seed=pop)


def test_ga_very_large_m_row_path(pm):
    """m = 60000: the facility-major tile does not fit in shared memory, so the GA evaluates with the row kernel
    and initialises with one warp per 32 individuals (the bitsets do not fit either)."""
    rng = np.random.default_rng(5)
    d = rng.integers(0, 1 << 16, size=(6, 60000)).astype(np.int32)
    _ga_compare(pm, d, 3, 64, 2, check_every=1, deme=32, seed=2, xover_rounds=2, mut_tries=2)


def test_ga_feature_combinations(pm):
    """Combinadic generation on cumulative tables with migration variant (ii), against the oracle."""
    _ga_compare(pm, euclid_instance(150, seed=21)[:90], 12, 128, 3, check_every=1, deme=32, seed=4,
                init="combinadic", migration="team", cumulative=True)


def _columns_layout(masks, m, G):
    """The documented facility-major form, built here from the bitsets: word (tile * 32W + j) * G + g has bit b
    set iff individual tile * 32G + 32g + b has facility j open."""
    pop, W = masks.shape
    tiles = -(-pop // (32 * G))
    bits = ((masks[:, :, None].astype(np.uint64) >> np.arange(32, dtype=np.uint64)) & 1).reshape(pop, 32 * W)
    padded = np.zeros((tiles * 32 * G, 32 * W), dtype=np.uint64)
    padded[:pop] = bits
    per = padded.reshape(tiles, G, 32, 32 * W)  # [tile, g, b, j]
    words = (per << np.arange(32, dtype=np.uint64)[None, None, :, None]).sum(axis=2)  # [tile, g, j]
    return words.transpose(0, 2, 1).astype(np.uint32).reshape(-1)


@pytest.mark.parametrize("shape", [(4, 32, 0), (2, 8, 0), (1, 16, 3)])
@pytest.mark.parametrize("pop", [1, 97, 1024])
def test_columns_api_matches_oracle_and_layout(pm, shape, pop):
    """pm_population_columns writes the documented form; pm_eval_columns on it gives the oracle's costs."""
    d, p = graph_instance(300, 1200, seed=5), 17
    inst = pm.Instance(d, p)
    G, warps, splits = shape
    inst.set_shape(pop, groups=G, warps=warps, splits=splits)
    g, words = pm.pm_columns_layout(inst.handle, pop)
    assert g == G
    masks = random_masks(pop, 300, p, seed=pop)
    want_cols = _columns_layout(masks, 300, G)
    assert words == want_cols.size
    cols = torch.full((words,), -1, dtype=torch.int32, device="cuda")  # every word must be written
    pm.pm_population_columns(inst.handle, to_dev(masks), pop, cols)
    np.testing.assert_array_equal(cols.cpu().numpy().view(np.uint32), want_cols)
    costs = torch.empty(pop, dtype=torch.int64, device="cuda")
    pm.pm_eval_columns(inst.handle, cols, pop, costs)
    np.testing.assert_array_equal(costs.cpu().numpy(), oracle.eval_direct(d, masks))
    # columns built on the host from the documented form evaluate the same
    cols2 = torch.from_numpy(want_cols.view(np.int32)).cuda()
    pm.pm_eval_columns(inst.handle, cols2, pop, costs)
    np.testing.assert_array_equal(costs.cpu().numpy(), oracle.eval_direct(d, masks))
    inst.close()


def test_columns_api_refuses_the_row_kernel_and_host_pointers(pm):
    d, p = graph_instance(100, 200, seed=0), 5
    inst = pm.Instance(d, p)
    inst.set_shape(64, groups=0, warps=8)
    with pytest.raises(pm.PMError) as e:
        pm.pm_columns_layout(inst.handle, 64)
    assert e.value.status == 3  # PM_ERR_UNSUPPORTED
    inst.set_shape(64, groups=2, warps=8)
    g, words = pm.pm_columns_layout(inst.handle, 64)
    host = np.zeros(words, dtype=np.uint32)
    with pytest.raises(pm.PMError) as e:
        pm.pm_eval_columns(inst.handle, host, 64, torch.empty(64, dtype=torch.int64, device="cuda"))
    assert e.value.status == 1  # PM_ERR_INVALID_ARG
    inst.close()

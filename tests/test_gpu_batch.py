"""Batched mode (many uneven instances per launch) against the CPU oracle, bit for bit."""

import numpy as np
import pytest

import oracle
from paper_1610_10061_gb300.inputs import batched_instances, euclid_instance, graph_instance, random_masks

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


def _uneven():
    return [
        (graph_instance(100, 200, seed=0), 5),
        (euclid_instance(333, seed=1), 31),
        (graph_instance(64, 128, seed=2), 2),
        (euclid_instance(1200, seed=3)[:700], 90),  # n=700 clients, m=1200 facilities
        (graph_instance(257, 600, seed=4), 25),
    ]


def _dev(masks_list):
    flat = np.concatenate([m.reshape(-1) for m in masks_list]).astype(np.uint32)
    return torch.from_numpy(flat.view(np.int32)).cuda()


@pytest.mark.parametrize("tune,mixed", [(False, False), (True, False), (False, True)])
def test_batch_eval_bit_exact(pm, tune, mixed):
    """mixed: every other instance keeps cumulative tables (D' instead of Delta') in the same launch."""
    inst_data = _uneven()
    insts = [pm.Instance(d, p, cumulative=mixed and k % 2 == 1) for k, (d, p) in enumerate(inst_data)]
    batch = pm.Batch(insts)
    pops = [1000, 33, 64, 517, 129]
    masks = [random_masks(P, d.shape[1], p, seed=7 * k + P) for k, ((d, p), P) in enumerate(zip(inst_data, pops))]
    if tune:
        shape = batch.tune(pops)
        assert shape["groups"] in (1, 2, 4) and shape["candidates"] >= 1
    for _ in range(2):  # a second call reuses the scratch left by the first
        costs = batch.eval(_dev(masks), pops)
        torch.cuda.synchronize()
        got = costs.cpu().numpy()
        off = 0
        for (d, p), mk, P in zip(inst_data, masks, pops):
            np.testing.assert_array_equal(got[off:off + P], oracle.eval_direct(d, mk))
            off += P
    batch.close()


def test_batch_eval_paper_shaped_instances(pm):
    """Eight instances of the batched recipe (n = m log-uniform in [100, 1500], p in [5, n/10])."""
    data = batched_instances(8, seed=3, nmin=100, nmax=1500)
    insts = [pm.Instance(d, p) for d, p in data]
    batch = pm.Batch(insts)
    pops = [256] * len(data)
    masks = [random_masks(256, d.shape[1], p, seed=k) for k, (d, p) in enumerate(data)]
    costs = batch.eval(_dev(masks), pops).cpu().numpy()
    for k, ((d, p), mk) in enumerate(zip(data, masks)):
        pi, de = oracle.tables(d, p)
        np.testing.assert_array_equal(costs[256 * k:256 * (k + 1)], oracle.eval_scan(pi, de, mk))


@pytest.mark.parametrize("mixed,spec", [(False, False), (True, False), (False, True), (True, True)])
def test_batch_ga_matches_standalone_oracle_runs(pm, monkeypatch, mixed, spec):
    """spec: PM_GA_SPEC=1, every instance's mutation tries built and evaluated together (one launch, one scan)."""
    if spec:
        monkeypatch.setenv("PM_GA_SPEC", "1")
    data = [(graph_instance(100, 200, seed=0), 5), (euclid_instance(150, seed=5), 12),
            (graph_instance(90, 200, seed=6), 9)]
    insts = [pm.Instance(d, p, cumulative=mixed and k != 1) for k, (d, p) in enumerate(data)]
    batch = pm.Batch(insts)
    P, D, G = 64, 32, 4
    ga = batch.ga(seed=21, pop=P, deme=D, stream_id=3)
    traces = [ga.step(1) for _ in range(G)]
    trace = np.concatenate(traces, axis=1)
    for k, (d, p) in enumerate(data):
        pi, de = oracle.tables(d, p)
        st, otrace, opops, ocosts = oracle.ga_run(pi, de, d.shape[1], p, seed=21, P=P, D=D, gens=G, record=True,
                                                  inst=3 + k)
        np.testing.assert_array_equal(trace[k], otrace)
        masks, costs = ga.population(k)
        np.testing.assert_array_equal(masks, opops[-1])
        np.testing.assert_array_equal(costs, ocosts[-1])
        bc, gr, ev, best = ga.result(k)
        assert bc == st.best_cost and ev == st.evals and gr == G
        np.testing.assert_array_equal(best, st.best)
    info = ga.info()
    assert info["pop"] == P and info["deme"] == D
    lgD = 5
    assert info["kernels_per_generation"] == 2 + lgD * 2 + (3 if spec else lgD * 2) + 1


def test_batch_ga_instances_stop_independently(pm):
    data = [(graph_instance(30, 60, seed=1), 3), (graph_instance(40, 90, seed=2), 4),
            (euclid_instance(60, seed=3), 6)]
    insts = [pm.Instance(d, p) for d, p in data]
    batch = pm.Batch(insts)
    ga = batch.ga(seed=5, pop=32, deme=16, saturation=3)
    trace = ga.step(200)
    ran = []
    for k, (d, p) in enumerate(data):
        pi, de = oracle.tables(d, p)
        st, otrace, opops, ocosts = oracle.ga_run(pi, de, d.shape[1], p, seed=5, P=32, D=16, gens=200,
                                                  saturation=3, record=True, inst=k)
        bc, gr, ev, _ = ga.result(k)
        assert gr == len(otrace) and bc == st.best_cost and ev == st.evals
        np.testing.assert_array_equal(trace[k, :gr], otrace)
        masks, costs = ga.population(k)
        np.testing.assert_array_equal(masks, opops[-1])
        ran.append(gr)
    assert len(set(ran)) > 1 or ran[0] < 200  # the instances stopped on their own


def test_batch_rejects_mixed_p1(pm):
    a = pm.Instance(graph_instance(40, 80, seed=1), 1)
    b = pm.Instance(graph_instance(40, 80, seed=2), 3)
    batch = pm.Batch([a, b])
    with pytest.raises(pm.PMError) as e:
        batch.ga(seed=0, pop=32, deme=16)
    assert e.value.status == 3


def test_batch_ga_team_migration_mixed_tables(pm):
    """A batched GA with migration variant (ii) over instances with both table kinds: each instance equals the
    stand-alone oracle run with its stream id."""
    data = [(graph_instance(100, 200, seed=0), 5), (euclid_instance(150, seed=5), 12)]
    insts = [pm.Instance(d, p, cumulative=(k == 0)) for k, (d, p) in enumerate(data)]
    batch = pm.Batch(insts)
    ga = batch.ga(seed=31, pop=64, deme=16, stream_id=7, migration="team")
    trace = np.concatenate([ga.step(1) for _ in range(3)], axis=1)
    for k, (d, p) in enumerate(data):
        pi, de = oracle.tables(d, p)
        st, otrace, opops, ocosts = oracle.ga_run(pi, de, d.shape[1], p, seed=31, P=64, D=16, gens=3, record=True,
                                                  inst=7 + k, team=True)
        np.testing.assert_array_equal(trace[k], otrace)
        masks, costs = ga.population(k)
        np.testing.assert_array_equal(masks, opops[-1])
        np.testing.assert_array_equal(costs, ocosts[-1])

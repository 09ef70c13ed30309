"""Parity at the benchmark's full sizes, on outputs the oracle can check one by one.

* The batched workload (256 uneven instances, n = m log-uniform in [100, 5000], half graph, half Euclidean,
  population 256 each) evaluated in one batched pass in the autotuned launch configuration the benchmark times:
  every cost of six sampled instances (the smallest, the largest and four more) against the oracle's scan over
  the oracle's own tables.
* The learned GA on the clustered 5000 x 5000 instance (p = 500, population 1024 in demes of 256), which the
  benchmark times against the plain GA: after each generation, the reported costs of sampled individuals, the
  global best and the trace are recomputed from the bitsets with the direct objective (nearest open facility per
  client, summed; Eqs. 1-3) -- the model may only propose moves, never a cost.
"""

import os

import numpy as np
import pytest

import oracle
from paper_1610_10061_gb300.inputs import batched_instances, paper_shape_instance, random_masks

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


def _direct(d, mask_row):
    """The objective of one bitset: every client's nearest open facility, summed (Eqs. 1-3)."""
    open_ = np.nonzero(np.unpackbits(np.ascontiguousarray(mask_row).view(np.uint8), bitorder="little"))[0]
    open_ = open_[open_ < d.shape[1]]
    return int(d[:, open_].min(axis=1).astype(np.int64).sum())


def test_batched256_full_size_sampled_instances(pm):
    workers = max(1, min(16, (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else 2) - 1))
    data = batched_instances(256, seed=3, workers=workers)
    insts = [pm.Instance(d, p) for d, p in data]
    batch = pm.Batch(insts)
    pop = 256
    pops = [pop] * len(data)
    batch.tune(pops)
    masks = [random_masks(pop, d.shape[1], p, seed=123 + k) for k, (d, p) in enumerate(data)]
    flat = np.concatenate([mk.reshape(-1) for mk in masks]).astype(np.uint32)
    costs = batch.eval(torch.from_numpy(flat.view(np.int32)).cuda(), pops).cpu().numpy()
    sizes = [d.shape[0] for d, _ in data]
    rng = np.random.default_rng(7)
    sample = {int(np.argmin(sizes)), int(np.argmax(sizes))} | {int(k) for k in rng.choice(len(data), 4, replace=False)}
    for k in sorted(sample):
        d, p = data[k]
        pi, de = oracle.tables(d, p)
        np.testing.assert_array_equal(costs[pop * k:pop * (k + 1)], oracle.eval_scan(pi, de, masks[k]),
                                      err_msg=f"instance {k} (n = m = {d.shape[0]}, p = {p})")
    # a property over every instance: no cost below the sum of the rows' minima
    for k, (d, p) in enumerate(data):
        assert (costs[pop * k:pop * (k + 1)] >= d.min(axis=1).astype(np.int64).sum()).all()
    batch.close()
    for inst in insts:
        inst.close()


def test_learned_ga_gmm5000_full_size_costs_are_exact(pm):
    w = paper_shape_instance("gmm5000_p500")
    d, p, pop = w["d"], w["p"], w["pop"]
    inst = pm.Instance(d, p)
    inst.tune(pop)
    # a model trained briefly on moves logged from this instance's plain GA (its quality does not matter here)
    g0 = pm.GA(inst, seed=1000, pop=pop, deme=256)
    g0.step(1)
    masks_dev = torch.empty((pop, inst.W), dtype=torch.int32, device="cuda")
    costs_dev = torch.empty(pop, dtype=torch.int64, device="cuda")
    pm.pm_ga_population(g0.handle, masks_dev, costs_dev, None)
    per = 16
    x = torch.empty((pop * per, 16), dtype=torch.bfloat16, device="cuda")
    t = torch.empty(pop * per, dtype=torch.float32, device="cuda")
    mv = torch.empty((pop * per, 2), dtype=torch.int32, device="cuda")
    pm.pm_log_moves(inst.handle, masks_dev, costs_dev, pop, per, 5, x, t, mv, None)
    model = pm.Model(seed=0)
    model.train(x, t, epochs=2, batch=4096, lr=2e-3, seed=1)
    ga = pm.GA(inst, seed=3, pop=pop, deme=256, model=model)
    rng = np.random.default_rng(11)
    prev = None
    for g in range(4):
        tr = ga.step(1)
        masks, costs = ga.population()
        for t_ in rng.choice(pop, 24, replace=False):
            assert costs[t_] == _direct(d, masks[t_]), (g, t_)
            assert sum(bin(int(v)).count("1") for v in masks[t_]) == p
        best, gens, evals, best_mask = ga.result()
        assert best == tr[-1] == _direct(d, best_mask) and gens == g + 1
        assert prev is None or best <= prev
        prev = best


def test_learned_ga_gmm5000_equal_scores_matches_oracle(pm):
    """The learned GA at the size bench.py times it (clustered n = m = 5000, p = 500, pop 1024 in demes of 256),
    with an all-zero model so that the oracle can follow it (oracle.mlp.first_candidate_try): population, costs,
    best and evaluations after each of two generations."""
    from oracle import mlp
    w = paper_shape_instance("gmm5000_p500")
    d, p, pop = w["d"], w["p"], w["pop"]
    pi, de = oracle.tables(d, p)
    st, otrace, opops, ocosts = oracle.ga_run(pi, de, 5000, p, seed=4, P=pop, D=256, gens=2, record=True,
                                              extra_try=mlp.first_candidate_try(pi, de, 5000, p))
    inst = pm.Instance(d, p)
    inst.tune(pop)
    model = pm.Model(seed=0)
    model.set_params(np.zeros(model.n_params, dtype=np.float32))
    ga = pm.GA(inst, seed=4, pop=pop, deme=256, model=model)
    for g in range(2):
        tr = ga.step(1)
        assert tr[0] == otrace[g]
        masks, costs = ga.population()
        np.testing.assert_array_equal(masks, opops[g], err_msg=f"population after generation {g + 1}")
        np.testing.assert_array_equal(costs, ocosts[g], err_msg=f"costs after generation {g + 1}")
    bc, gr, ev, best = ga.result()
    assert bc == st.best_cost and ev == st.evals and gr == 2
    np.testing.assert_array_equal(best, st.best)

"""The learned swap proposal on the GPU against its oracle.

Swap statistics are integers (bit-exact).  Features, the perceptron's
predictions and gradients are compared within the tolerance of BF16 operands
with FP32 accumulation (relative 2e-2, absolute 1e-3 of the tensor's scale);
Adam, applied to the GPU's own gradients, within FP32 rounding.  The learned
GA is checked for exactness (every reported cost equals the direct evaluator
of its bitset) and for what the trained model gains.
"""

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1610_10061_gb300.inputs import (euclid_instance, gmm_instance, graph_instance, masks_from_sets,
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


def dev32(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _stats_gpu(pm, inst, masks):
    P, m = masks.shape[0], inst.m
    dm = dev32(masks)
    g = torch.zeros((P, m), dtype=torch.int64, device="cuda")
    c = torch.zeros((P, m), dtype=torch.int32, device="cuda")
    lo = torch.zeros((P, m), dtype=torch.int64, device="cuda")
    a = torch.zeros((P, m), dtype=torch.int32, device="cuda")
    pm.pm_swap_stats(inst.handle, dm, P, g, c, lo, a)
    torch.cuda.synchronize()
    return g, c, lo, a


@pytest.mark.parametrize("cumulative", [False, True])
@pytest.mark.parametrize("case", ["graph", "euclid", "ties", "gmm", "wide", "wide64", "global", "short"])
def test_swap_stats_bit_exact(pm, case, cumulative):
    """Every accumulator variant: 32-bit shared (n max d < 2^32), 64-bit shared, and the output arrays in global
    memory once 24 m bytes of 64-bit accumulators exceed a CTA's shared memory; p/m from 0.6 % (the first two open
    ranks rarely among the first 32) to 95 %."""
    rng = np.random.default_rng(1)
    if case == "graph":
        d, p = graph_instance(100, 200, seed=0), 5
    elif case == "euclid":
        d, p = euclid_instance(300, seed=1), 30
    elif case == "ties":
        d, p = rng.integers(0, 4, size=(60, 90)).astype(np.int32), 7
    elif case == "gmm":
        d, p = gmm_instance(400, seed=2), 40
    elif case == "wide":  # m = 10000 with 32-bit shared accumulators (160 KB)
        d, p = rng.integers(0, 3000, size=(40, 10000)).astype(np.int32), 60
    elif case == "wide64":  # n max d >= 2^32: 64-bit shared accumulators (120 KB)
        d, p = rng.integers(0, 1 << 27, size=(40, 5000)).astype(np.int32), 50
    elif case == "global":  # 64-bit accumulators for m = 10000 (240 KB) do not fit: global memory
        d, p = rng.integers(0, 1 << 27, size=(40, 10000)).astype(np.int32), 500
    else:  # L = 3: rows that often hold a single open facility (second distance = the row's last)
        d, p = rng.integers(0, 50, size=(50, 40)).astype(np.int32), 38
    inst = pm.Instance(d, p, cumulative=cumulative)
    masks = random_masks(37, d.shape[1], p, seed=3)
    got = [x.cpu().numpy() for x in _stats_gpu(pm, inst, masks)]
    pi, de = oracle.tables(d, p)
    want = oracle.swap_stats(pi, de, d.shape[1], masks)
    for gx, wx in zip(got, want):
        np.testing.assert_array_equal(gx, wx)


def _bf16_close(got, ref):
    tol = np.abs(ref) / 128 + 1e-6
    assert (np.abs(got - ref) <= tol).all(), np.max(np.abs(got - ref) - tol)


def test_move_features_match_oracle(pm):
    d, p = gmm_instance(300, seed=5), 20
    inst = pm.Instance(d, p)
    P, C = 16, 9
    masks = random_masks(P, 300, p, seed=6)
    costs = oracle.eval_direct(d, masks)
    rng = np.random.default_rng(0)
    moves = np.zeros((P, C, 2), dtype=np.int32)
    sets = sets_from_masks(masks, 300)
    for t in range(P):
        closed = [k for k in range(300) if k not in sets[t]]
        for c in range(C):
            moves[t, c] = (rng.choice(sets[t]), rng.choice(closed))
    g, ca, lo, a = _stats_gpu(pm, inst, masks)
    x = torch.zeros((P * C, 16), dtype=torch.bfloat16, device="cuda")
    pm.pm_move_features(inst.handle, g, ca, lo, a, torch.from_numpy(costs).cuda(), torch.from_numpy(moves).cuda(),
                        P, C, x)
    got = x.float().cpu().numpy()
    pi, de = oracle.tables(d, p)
    G, CA, LO, A = oracle.swap_stats(pi, de, 300, masks)
    for t in range(P):
        for c in range(C):
            j, k = moves[t, c]
            ref = mlp.move_features(G[t], CA[t], LO[t], A[t], costs[t], 300, 300, p, j, k)
            _bf16_close(got[t * C + c, :8], ref)
            assert (got[t * C + c, 8:] == 0).all()


def _random_batch(rows, seed):
    rng = np.random.default_rng(seed)
    X = np.zeros((rows, 16))
    X[:, :8] = rng.normal(0, 1, size=(rows, 8))
    X = mlp.bf16_round(X)
    t = rng.normal(0, 1, size=rows)
    return X, t


def _scale_close(got, ref, rtol=2e-2, atol=1e-3):
    scale = max(1.0, float(np.max(np.abs(ref))))
    np.testing.assert_allclose(got, ref, rtol=rtol, atol=atol * scale)


@pytest.mark.parametrize("rows", [64, 1000, 4096])
def test_mlp_forward_and_gradients(pm, rows):
    model = pm.Model(seed=1)
    params = mlp.init_params(seed=rows)
    for k in ("b1", "b2", "b3"):
        params[k] = np.random.default_rng(rows).normal(0, 0.1, size=params[k].shape)
    model.set_params(mlp.flatten(params).astype(np.float32))
    p32 = mlp.unflatten(model.params().astype(np.float64))  # the float32 masters the GPU holds
    X, t = _random_batch(rows, rows)
    xd = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    y = model.forward(xd).cpu().numpy()
    yref, _ = mlp.forward(p32, X, bf16=True)
    _scale_close(y, yref)
    loss, g = model.grad(xd, td)
    lref, gref = mlp.loss_and_grads(p32, X, t, bf16=True)
    assert loss == pytest.approx(lref, rel=2e-2)
    G = mlp.unflatten(g.astype(np.float64))
    for name in ("W1", "b1", "W2", "b2", "w3", "b3"):
        _scale_close(G[name], gref[name])


def test_mlp_forward_every_cta_walks_several_tiles(pm):
    """The tensor-core forward is persistent: min(tiles, 3 x SMs) CTAs walk 128-row tiles, prefetching the next
    tile's inputs, flipping the MMA barrier's phase and reusing TMEM from tile to tile.  Five tiles per CTA plus a
    ragged last tile (77 rows), every row against the oracle."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rows = 5 * 3 * sms * 128 + 77
    model = pm.Model(seed=3)
    params = mlp.init_params(seed=5)
    for k in ("b1", "b2", "b3"):
        params[k] = np.random.default_rng(6).normal(0, 0.1, size=params[k].shape)
    model.set_params(mlp.flatten(params).astype(np.float32))
    p32 = mlp.unflatten(model.params().astype(np.float64))
    X, _ = _random_batch(rows, 7)
    xd = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda()
    y = model.forward(xd).cpu().numpy()
    yref, _ = mlp.forward(p32, X, bf16=True)
    _scale_close(y, yref)


def _heavy_batch(rows, seed):
    """Inputs as _random_batch, targets whose scale varies widely from row to row, so that every batch's loss
    depends on which rows the shuffle put into it."""
    X, _ = _random_batch(rows, seed)
    rng = np.random.default_rng(seed + 1)
    t = rng.normal(0, 1, size=rows) * np.exp(rng.normal(0, 1, size=rows))
    return X, t


def test_model_train_follows_the_oracle_loop(pm):
    """pm_model_train (the whole loop behind the C ABI: the keyed epoch shuffle, mini-batches, Adam) against the
    oracle's loop with the same permutation: every step's loss, and the parameters after the last step."""
    rows, batch, epochs, lr, seed = 1500, 256, 2, 2e-3, 77
    model = pm.Model(seed=4)
    params = mlp.init_params(seed=4)
    for k in ("b1", "b2", "b3"):
        params[k] = np.random.default_rng(5).normal(0, 0.1, size=params[k].shape)
    model.set_params(mlp.flatten(params).astype(np.float32))
    p32 = mlp.unflatten(model.params().astype(np.float64))
    X, t = _heavy_batch(rows, 13)
    xd = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    losses = model.train(xd, td, epochs=epochs, batch=batch, lr=lr, seed=seed)
    pref, _, oloss = mlp.train({k: v.copy() for k, v in p32.items()}, X, t, epochs, batch, lr, seed)
    assert len(losses) == len(oloss) == epochs * 6
    _scale_close(np.asarray(losses, dtype=np.float64), np.asarray(oloss))
    got = mlp.unflatten(model.params().astype(np.float64))
    steps = len(oloss)
    for name in ("W1", "b1", "W2", "b2", "w3", "b3"):  # Adam moves each weight by at most lr per step
        np.testing.assert_allclose(got[name], pref[name], rtol=0, atol=0.25 * lr * steps)
    # another seed gives another order, hence other batch losses from the same start
    model.set_params(mlp.flatten(p32).astype(np.float32))
    other = model.train(xd, td, epochs=1, batch=batch, lr=lr, seed=seed + 1)
    assert np.abs(np.asarray(other[1:]) - np.asarray(losses[1:6])).max() > 0.05 * np.abs(losses[1:6]).max()


def test_model_train_is_repeatable_for_a_seed(pm):
    X, t = _heavy_batch(5000, 17)
    xd = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    runs = []
    for _ in range(2):
        model = pm.Model(seed=6)
        runs.append(model.train(xd, td, epochs=3, batch=1000, lr=1e-3, seed=5))
    # the same batches in the same order: equal up to the order of the FP32 gradient additions
    np.testing.assert_allclose(runs[0], runs[1], rtol=1e-3)
    assert runs[0][-1] < runs[0][0]


def test_adam_step_matches_oracle(pm):
    model = pm.Model(seed=2)
    X, t = _random_batch(512, 9)
    xd = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    p = mlp.unflatten(model.params().astype(np.float64))
    state = mlp.adam_init(p)
    for step in range(3):
        _, g = model.grad(xd, td)
        pm.pm_model_train_step(model.handle, xd, td, 512, 1e-3)
        p = mlp.adam_step(p, mlp.unflatten(g.astype(np.float64)), state, lr=1e-3)
        got = mlp.unflatten(model.params().astype(np.float64))
        for name in p:
            np.testing.assert_allclose(got[name], p[name], rtol=1e-5, atol=1e-7)


def _log(pm, inst, masks, costs, per, seed):
    P = masks.shape[0]
    x = torch.zeros((P * per, 16), dtype=torch.bfloat16, device="cuda")
    tt = torch.zeros(P * per, dtype=torch.float32, device="cuda")
    mv = torch.zeros((P * per, 2), dtype=torch.int32, device="cuda")
    pm.pm_log_moves(inst.handle, dev32(masks), torch.from_numpy(costs).cuda(), P, per, seed, x, tt, mv)
    torch.cuda.synchronize()
    return x, tt, mv


def test_log_moves_targets_are_exact(pm):
    d, p = euclid_instance(200, seed=4), 12
    inst = pm.Instance(d, p)
    masks = random_masks(20, 200, p, seed=8)
    costs = oracle.eval_direct(d, masks)
    x, tt, mv = _log(pm, inst, masks, costs, 16, seed=3)
    mv = mv.cpu().numpy().reshape(20, 16, 2)
    tt = tt.cpu().numpy().reshape(20, 16)
    sets = sets_from_masks(masks, 200)
    pi, de = oracle.tables(d, p)
    G, CA, LO, A = oracle.swap_stats(pi, de, 200, masks)
    top_share = 0
    for t in range(20):
        top4 = [k for k in np.argsort(-G[t], kind="stable") if k not in sets[t]][:4]
        for q in range(16):
            j, k = mv[t, q]
            assert j in sets[t] and k not in sets[t]
            top_share += k in top4
            after = oracle.eval_direct(d, masks_from_sets([sorted([s for s in sets[t] if s != j] + [k])], 200))[0]
            assert tt[t, q] == pytest.approx(mlp.move_target(costs[t], after, p), rel=1e-6, abs=1e-6)
    assert top_share >= 0.6 * 20 * 16


def _train_model(pm, d, p, seed=0, gens=6, per=64, epochs=8):
    """Log tuples from plain-GA populations and train a model on them (all on the GPU)."""
    inst = pm.Instance(d, p)
    ga = pm.GA(inst, seed=seed + 100, pop=256, deme=64)
    xs, ts = [], []
    for g in range(gens):
        ga.step(1)
        masks, costs = ga.population()
        x, tt, _ = _log(pm, inst, masks, costs, per, seed=seed * 1000 + g)
        xs.append(x)
        ts.append(tt)
    X = torch.cat(xs)
    T = torch.cat(ts)
    model = pm.Model(seed=seed)
    before, _ = model.grad(X, T)
    losses = model.train(X, T, epochs=epochs, batch=2048, lr=2e-3, seed=seed)
    after, _ = model.grad(X, T)
    return inst, model, [before, after]


def _spearman(a, b):
    ra = np.argsort(np.argsort(a))
    rb = np.argsort(np.argsort(b))
    return float(np.corrcoef(ra, rb)[0, 1])


def test_training_lowers_the_loss_and_ranks_moves(pm):
    d, p = gmm_instance(500, seed=7), 25
    inst, model, losses = _train_model(pm, d, p)
    assert losses[-1] < 0.5 * losses[0]
    # held-out tuples from another population: the trained model ranks moves far better than an untrained one
    masks = random_masks(128, 500, p, seed=99)
    costs = oracle.eval_direct(d, masks)
    x, tt, _ = _log(pm, inst, masks, costs, 32, seed=12345)
    truth = tt.cpu().numpy()
    yt = model.forward(x).cpu().numpy()
    yu = pm.Model(seed=123).forward(x).cpu().numpy()
    mse_t, mse_u = float(np.mean((yt - truth) ** 2)), float(np.mean((yu - truth) ** 2))
    assert mse_t < 0.25 * mse_u, (mse_t, mse_u)
    assert _spearman(yt, truth) > 0.95
    # top-1 regret per individual: true change of the chosen move minus the best true change among its 32 moves
    def regret(y):
        yy, tt_ = y.reshape(128, 32), truth.reshape(128, 32)
        return float(np.mean(tt_[np.arange(128), np.argmin(yy, axis=1)] - tt_.min(axis=1)))
    assert regret(yt) <= regret(yu), (regret(yt), regret(yu))


def test_learned_ga_is_exact_and_gains(pm):
    d, p = gmm_instance(500, seed=7), 25
    inst, model, _ = _train_model(pm, d, p, seed=1)
    G = 8
    plain = pm.GA(inst, seed=5, pop=256, deme=64)
    tp = plain.step(G)
    learned = pm.GA(inst, seed=5, pop=256, deme=64, model=model)
    tl = learned.step(G)
    masks, costs = learned.population()
    np.testing.assert_array_equal(costs, oracle.eval_direct(d, masks))
    assert all(len(s) == p for s in sets_from_masks(masks, 500))
    bc, gr, ev, best = learned.result()
    assert bc == oracle.eval_direct(d, best[None])[0] and gr == G
    assert (np.diff(tl) <= 0).all()
    # what the trained proposal gains: a better best after the same generations, reached earlier
    assert tl[-1] < tp[-1]
    first = int(np.argmax(tl <= tp[-1]))
    assert tl[first] <= tp[-1] and first < G - 1


def test_learned_ga_on_cumulative_tables_is_exact(pm):
    """The learned try reads swap statistics from cumulative tables (D') as well; every cost stays exact."""
    d, p = gmm_instance(500, seed=7), 25
    _, model, _ = _train_model(pm, d, p, seed=2, gens=3, epochs=4)
    inst = pm.Instance(d, p, cumulative=True)
    ga = pm.GA(inst, seed=9, pop=256, deme=64, model=model)
    trace = ga.step(4)
    masks, costs = ga.population()
    np.testing.assert_array_equal(costs, oracle.eval_direct(d, masks))
    assert all(len(s) == p for s in sets_from_masks(masks, 500))
    assert (np.diff(trace) <= 0).all()


@pytest.mark.parametrize("cumulative,T", [(False, 4), (True, 8), (False, 3)])
def test_learned_try_fused_candidates_equal_the_two_kernels(pm, monkeypatch, cumulative, T):
    """The learned try takes its candidate moves in the statistics kernel's tail when the statistics fit in
    shared memory; PM_LEARN_FUSED=0 (read when the GA captures its generation) runs the statistics and the
    candidates as two kernels through global memory instead.  Same model, same seed: identical populations,
    costs and traces, and every cost exact.  T = 8 with p close to m also covers fewer closed facilities than
    candidates."""
    d, p = gmm_instance(400, seed=13), (30 if T != 8 else 395)
    inst = pm.Instance(d, p, cumulative=cumulative)
    model = pm.Model(seed=7)  # untrained: deterministic scores, so any difference is the candidates'
    runs = []
    for fused in ("1", "0"):
        monkeypatch.setenv("PM_LEARN_FUSED", fused)
        ga = pm.GA(inst, seed=3, pop=128, deme=32, model=model, candidates=T)
        trace = ga.step(3)
        masks, costs = ga.population()
        runs.append((trace, masks, costs))
        ga.close()
    monkeypatch.delenv("PM_LEARN_FUSED")
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    np.testing.assert_array_equal(runs[0][2], runs[1][2])
    np.testing.assert_array_equal(runs[0][2], oracle.eval_direct(d, runs[0][1]))


@pytest.mark.parametrize("n,p,pop,deme,cumulative,fused", [(120, 9, 64, 32, False, "1"), (200, 20, 128, 64, True, "1"),
                                                          (150, 12, 96, 32, False, "0")])
def test_learned_ga_with_equal_scores_matches_oracle(pm, monkeypatch, n, p, pop, deme, cumulative, fused):
    """The whole learned generation against the oracle GA: with every parameter zero the model scores every
    candidate the same, so the learned try takes candidate 0 -- close the lowest open facility, open the closed
    facility of largest gain -- evaluates the child exactly and keeps it iff strictly cheaper, and the mutation
    cycle skips the individuals it improved (oracle.mlp.first_candidate_try).  Population, costs, best and
    evaluations after every generation, for both table kinds and both candidate paths."""
    monkeypatch.setenv("PM_LEARN_FUSED", fused)
    d = gmm_instance(n, seed=13)
    pi, de = oracle.tables(d, p)
    st, otrace, opops, ocosts = oracle.ga_run(pi, de, n, p, seed=3, P=pop, D=deme, gens=3, record=True,
                                              extra_try=mlp.first_candidate_try(pi, de, n, p))
    inst = pm.Instance(d, p, cumulative=cumulative)
    model = pm.Model(seed=0)
    model.set_params(np.zeros(model.n_params, dtype=np.float32))
    ga = pm.GA(inst, seed=3, pop=pop, deme=deme, model=model)
    for g in range(3):
        tr = ga.step(1)
        assert tr[0] == otrace[g]
        masks, costs = ga.population()
        np.testing.assert_array_equal(masks, opops[g], err_msg=f"population after generation {g + 1}")
        np.testing.assert_array_equal(costs, ocosts[g], err_msg=f"costs after generation {g + 1}")
    bc, gr, ev, best = ga.result()
    assert bc == st.best_cost and ev == st.evals and gr == 3
    np.testing.assert_array_equal(best, st.best)

"""Pins for the oracle of the learned swap proposal (no GPU).

Swap statistics are tied to exact identities of the p-median objective
(opening one facility alone changes the cost by -gain, closing one alone by
+loss), to brute-force counts and to the direct evaluator; bf16 rounding to
torch's conversion (a library routine); the perceptron's gradients to finite
differences; Adam to a two-step example worked by hand from Kingma & Ba's
Algorithm 1.
"""


import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1610_10061_gb300.inputs import euclid_instance, graph_instance, masks_from_sets, random_masks, sets_from_masks


@pytest.mark.parametrize("seed", range(6))
def test_swap_stats_identities(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 30))
    m = int(rng.integers(4, 40))
    p = int(rng.integers(2, m))
    d = rng.integers(0, [4, 50, 1000][seed % 3], size=(n, m)).astype(np.int32)
    pif, def_ = oracle.tables(d, full=True)
    masks = random_masks(12, m, p, seed=seed)
    gain, cap, loss, assign = oracle.swap_stats(pif, def_, m, masks)
    base = oracle.eval_direct(d, masks)
    for t, s in enumerate(sets_from_masks(masks, m)):
        closed = [k for k in range(m) if k not in s]
        opened = masks_from_sets([sorted(s + [k]) for k in closed], m)
        np.testing.assert_array_equal(oracle.eval_direct(d, opened), base[t] - gain[t, closed])
        shut = masks_from_sets([[x for x in s if x != j] for j in s], m)
        np.testing.assert_array_equal(oracle.eval_direct(d, shut), base[t] + loss[t, s])
        assert assign[t].sum() == n and (assign[t, closed] == 0).all() and (loss[t, closed] == 0).all()
        assert (gain[t, s] == 0).all() and (cap[t, s] == 0).all()
        # cap[k] = number of clients that rank k ahead of their nearest open facility
        order = np.argsort(d, axis=1, kind="stable")
        rank = np.argsort(order, axis=1)
        r1 = np.array([min(rank[i, x] for x in s) for i in range(n)])
        for k in closed:
            assert cap[t, k] == int((rank[:, k] < r1).sum())


def test_swap_stats_truncated_tables_agree():
    d = graph_instance(70, 200, seed=9)
    for p in (3, 12):
        pi, de = oracle.tables(d, p)
        pif, def_ = oracle.tables(d, full=True)
        masks = random_masks(40, 70, p, seed=p)
        a = oracle.swap_stats(pi, de, 70, masks)
        b = oracle.swap_stats(pif, def_, 70, masks)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 10, 5000), rng.normal(0, 1e-3, 1000), [0.0, 1.0, -1.0, 1 + 2**-8, 1 + 3 * 2**-9,
                                                                            65504.0, 1e-30]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), ref)
    assert mlp.bf16_round(1 + 2**-8) == 1.0               # tie -> even
    assert mlp.bf16_round(1 + 3 * 2**-9) == 1 + 2**-7


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    params = mlp.init_params(3)
    X = np.zeros((20, mlp.F_PAD))
    X[:, :mlp.F_IN] = rng.normal(size=(20, mlp.F_IN))
    t = rng.normal(size=20)
    _, g = mlp.loss_and_grads(params, X, t)
    eps = 1e-6
    for name in params:
        flat = params[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = mlp.loss_and_grads(params, X, t)
            flat[idx] = old - eps
            lm, _ = mlp.loss_and_grads(params, X, t)
            flat[idx] = old
            num = (lp - lm) / (2 * eps)
            assert abs(num - g[name].reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(num)), (name, idx)


def test_adam_two_steps_by_hand():
    params = {"w": np.array([1.0])}
    state = mlp.adam_init(params)
    mlp.adam_step(params, {"w": np.array([0.5])}, state, lr=0.1)
    assert params["w"][0] == pytest.approx(0.900000002, abs=1e-15)
    mlp.adam_step(params, {"w": np.array([-0.25])}, state, lr=0.1)
    assert params["w"][0] == pytest.approx(0.8733662987078463, abs=1e-15)


def test_move_features_and_target():
    d = euclid_instance(50, seed=2)
    p = 5
    pif, def_ = oracle.tables(d, full=True)
    masks = random_masks(3, 50, p, seed=4)
    gain, cap, loss, assign = oracle.swap_stats(pif, def_, 50, masks)
    cost = oracle.eval_direct(d, masks)
    s = sets_from_masks(masks[:1], 50)[0]
    j, k = s[0], next(x for x in range(50) if x not in s)
    f = mlp.move_features(gain[0], cap[0], loss[0], assign[0], cost[0], 50, 50, p, j, k)
    Z = cost[0] / p
    assert f.shape == (8,) and f[0] == pytest.approx(loss[0, j] / Z) and f[1] == pytest.approx(gain[0, k] / Z)
    after = oracle.eval_direct(d, masks_from_sets([sorted([x for x in s if x != j] + [k])], 50))[0]
    assert mlp.move_target(cost[0], after, p) == pytest.approx((after - cost[0]) / Z)
    # first-order estimate loss - gain bounds the exact change from above (closing j can only lose less
    # once k is open, opening k can only gain more once j is closed... or equal)
    assert after - cost[0] <= loss[0, j] - 0 and after - cost[0] >= -gain[0, k]


def test_fmix32_published_values():
    """MurmurHash3_x86_32 of the empty input with seed s is fmix32(s) (no blocks, no tail, length 0): its published
    test values for seeds 0, 1 and 0xffffffff."""
    assert mlp.fmix32(0) == 0
    assert mlp.fmix32(1) == 0x514E28B7
    assert mlp.fmix32(0xFFFFFFFF) == 0x81F16F39


@pytest.mark.parametrize("rows", [1, 2, 3, 4, 5, 17, 64, 100, 1000, 4097])
def test_shuffle_order_is_a_permutation(rows):
    for epoch in range(3):
        order = mlp.shuffle_order(rows, seed=12345, epoch=epoch)
        assert sorted(order.tolist()) == list(range(rows))


def test_shuffle_order_changes_with_epoch_and_seed_and_mixes():
    a = mlp.shuffle_order(1000, 7, 0)
    assert not np.array_equal(a, mlp.shuffle_order(1000, 7, 1))
    assert not np.array_equal(a, mlp.shuffle_order(1000, 8, 0))
    # no longer sorted in long runs: few positions keep their row, successive rows scatter
    assert (a == np.arange(1000)).sum() < 20
    assert np.abs(np.diff(a)).mean() > 100


def test_shuffle_keys_are_the_philox_words():
    import oracle

    k = mlp.shuffle_keys(0x123456789, 4)
    assert k == [int(v) for v in oracle.philox4x32_10([4, 0, 0x300 << 16, 0], [0x23456789, 0x1])]


def test_train_loop_reduces_the_loss_and_follows_adam_step_by_step():
    rng = np.random.default_rng(3)
    X = np.zeros((300, 16))
    X[:, :8] = rng.normal(0, 1, size=(300, 8))
    X = mlp.bf16_round(X)
    t = X[:, 0] - 0.5 * X[:, 1] + 0.1
    p0 = mlp.init_params(seed=1)
    p1, _, losses = mlp.train({k: v.copy() for k, v in p0.items()}, X, t, epochs=4, batch=64, lr=3e-3, seed=9)
    assert len(losses) == 4 * 5
    assert np.mean(losses[-5:]) < 0.5 * np.mean(losses[:5])
    # the first two steps by hand: the first two batches of epoch 0 in the shuffled order, one Adam update between
    order = mlp.shuffle_order(300, 9, 0)
    q = {k: v.copy() for k, v in p0.items()}
    st = mlp.adam_init(q)
    loss, g = mlp.loss_and_grads(q, X[order[:64]], t[order[:64]], bf16=True)
    assert loss == losses[0]
    mlp.adam_step(q, g, st, 3e-3)
    loss2, _ = mlp.loss_and_grads(q, X[order[64:128]], t[order[64:128]], bf16=True)
    assert loss2 == losses[1]


def test_first_candidate_try_by_brute_force():
    """oracle.mlp.first_candidate_try against its definition written with the direct objective (O1) only: the
    gain of opening closed facility k alone is O1(x) - O1(x + k); the child closes the lowest open facility and
    opens the largest-gain closed one (lowest id on ties); it replaces the individual iff strictly cheaper."""
    m, p = 40, 6
    d = euclid_instance(m, seed=21)
    pi, de = oracle.tables(d, p)
    X = random_masks(24, m, p, seed=5)
    c = oracle.eval_direct(d, X)
    want_X, want_c, want_e = X.copy(), c.copy(), np.zeros(24, dtype=np.uint8)
    for t in range(24):
        s = sorted(sets_from_masks(X[t:t + 1], m)[0])
        closed = [k for k in range(m) if k not in s]
        drops = [c[t] - oracle.eval_direct(d, masks_from_sets([s + [k]], m))[0] for k in closed]
        k = closed[int(np.argmax(drops))]  # first maximum: lowest id among equal gains
        child = masks_from_sets([[j for j in s if j != s[0]] + [k]], m)
        cc = oracle.eval_direct(d, child)[0]
        if cc < c[t]:
            want_X[t], want_c[t], want_e[t] = child[0], cc, 1
    e = np.zeros(24, dtype=np.uint8)
    try_ = mlp.first_candidate_try(pi, de, m, p)
    assert try_(0, X, c, e) == 24
    np.testing.assert_array_equal(X, want_X)
    np.testing.assert_array_equal(c, want_c)
    np.testing.assert_array_equal(e, want_e)


def test_ga_extra_try_hook():
    """A try between the crossover and mutation cycles: doing nothing leaves the GA as it was; the first-candidate
    try keeps every cost exact, exactly p open facilities and a non-increasing best."""
    m, p = 60, 7
    d = graph_instance(m, 150, seed=8)
    pi, de = oracle.tables(d, p)
    a = oracle.ga_run(pi, de, m, p, seed=2, P=32, D=16, gens=4, record=True)
    b = oracle.ga_run(pi, de, m, p, seed=2, P=32, D=16, gens=4, record=True, extra_try=lambda g, X, c, e: 0)
    np.testing.assert_array_equal(a[2], b[2])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[0].evals == b[0].evals
    st, trace, pops, costs = oracle.ga_run(pi, de, m, p, seed=2, P=32, D=16, gens=4, record=True,
                                           extra_try=mlp.first_candidate_try(pi, de, m, p))
    for g in range(4):
        np.testing.assert_array_equal(costs[g], oracle.eval_direct(d, pops[g]))
        assert all(len(s) == p for s in sets_from_masks(pops[g], m))
    assert (np.diff(trace) <= 0).all()
    assert st.evals >= 4 * 32 * 2  # every generation: the initial evaluation and one learned child per individual

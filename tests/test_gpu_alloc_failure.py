"""Failure detection: device allocation failures injected on the host (pm_debug_fail_alloc).

No GPU fault is involved: the armed allocation returns cudaErrorMemoryAllocation without calling CUDA.  The sweep
fails the 1st, 2nd, ... device allocation of a job that touches every allocating entry point (instances of both
table kinds, evaluation, table read-back, plain, combinadic and learned GAs, a batch, the perceptron, move logging),
and checks that each failure surfaces as PM_ERR_OOM -- or, for the speculative mutation buffers, that the GA falls
back to the try-by-try cycle with identical results -- and that the library works normally afterwards.
"""

import contextlib

import numpy as np
import pytest

import oracle
from paper_1610_10061_gb300.inputs import graph_instance, random_masks

torch = pytest.importorskip("torch")

PM_ERR_OOM = 6


def test_injection_bookkeeping_needs_no_gpu():
    """Arming and disarming is host state only (no CUDA call)."""
    from paper_1610_10061_gb300 import build

    build.build()
    from paper_1610_10061_gb300 import pm

    try:
        pm.pm_debug_fail_alloc(-1)  # start disarmed
        assert pm.pm_debug_fail_alloc(7) == -1
        assert pm.pm_debug_fail_alloc(3) == 7
        assert pm.pm_debug_fail_alloc(-5) == 3
        assert pm.pm_debug_fail_alloc(-1) == -1
    finally:
        pm.pm_debug_fail_alloc(-1)


@pytest.fixture(scope="module")
def pm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_10061_gb300 import build

    build.build()
    from paper_1610_10061_gb300 import pm as _pm

    torch.cuda.set_device(0)
    return _pm


def _fixture():
    d, p = graph_instance(100, 200, seed=0), 5
    masks = random_masks(96, 100, p, seed=1)
    pi, de = oracle.tables(d, p)
    _, trace, _, _ = oracle.ga_run(pi, de, 100, p, seed=0, P=64, gens=3, record=True)
    x = np.zeros((256, 16), dtype=np.float32)
    x[:, :8] = np.random.default_rng(2).normal(0, 1, size=(256, 8))
    return d, p, masks, oracle.eval_direct(d, masks), (pi, de), trace, x


def _job(pm, d, p, masks, want, tables, trace, x):
    """Every allocating entry point once; raises PMError where an allocation fails."""
    pi, de = tables
    with contextlib.ExitStack() as es:
        dm = torch.from_numpy(masks.view(np.int32)).cuda()
        inst = pm.Instance(d, p)
        es.callback(inst.close)
        np.testing.assert_array_equal(inst.eval(dm).cpu().numpy(), want)
        cum = pm.Instance(d, p, cumulative=True)
        es.callback(cum.close)
        gpi, gde = cum.tables()
        np.testing.assert_array_equal(gpi, pi)
        np.testing.assert_array_equal(gde, de)
        ga = pm.GA(inst, seed=0, pop=64)
        es.callback(ga.close)
        np.testing.assert_array_equal(ga.step(3), trace)
        comb = pm.GA(inst, seed=0, pop=64, init="combinadic")
        es.callback(comb.close)
        comb.step(1)
        batch = pm.Batch([inst, cum])
        es.callback(batch.close)
        both = torch.cat([dm, dm])
        np.testing.assert_array_equal(batch.eval(both, [len(masks), len(masks)]).cpu().numpy(),
                                      np.concatenate([want, want]))
        model = pm.Model(seed=0)
        es.callback(model.close)
        xd = torch.from_numpy(x).to(torch.bfloat16).cuda()
        assert torch.isfinite(model.forward(xd)).all()
        learned = pm.GA(inst, seed=0, pop=64, model=model)
        es.callback(learned.close)
        learned.step(2)
        lm, lc = learned.population()
        np.testing.assert_array_equal(lc, oracle.eval_direct(d, lm))
        per = 4
        X = torch.empty((64 * per, 16), dtype=torch.bfloat16, device="cuda")
        T = torch.empty(64 * per, dtype=torch.float32, device="cuda")
        mv = torch.empty((64 * per, 2), dtype=torch.int32, device="cuda")
        gm = torch.from_numpy(masks[:64].view(np.int32)).cuda()
        gc = torch.from_numpy(want[:64]).cuda()
        pm.pm_log_moves(inst.handle, gm, gc, 64, per, 3, X, T, mv)
        torch.cuda.synchronize()


@pytest.mark.gpu
def test_every_allocation_failure_is_reported_and_recoverable(pm):
    args = _fixture()
    _job(pm, *args)  # the job passes without injection
    failed, absorbed = 0, 0
    try:
        for k in range(2000):
            pm.pm_debug_fail_alloc(k)
            try:
                _job(pm, *args)
                completed = True
            except pm.PMError as e:
                assert e.status == PM_ERR_OOM, (k, str(e))
                completed = False
                failed += 1
            pending = pm.pm_debug_fail_alloc(-1)
            if completed and pending >= 0:
                break  # the job made at most k allocations: every one of them has been failed once
            if completed:
                absorbed += 1  # the speculative mutation buffers: the GA fell back and stayed exact
            # the library still works after the failure
            _job(pm, *args)
        else:
            pytest.fail("the sweep did not reach the end of the job's allocations")
    finally:
        pm.pm_debug_fail_alloc(-1)
    print(f"allocations in the job: {k}; failures reported as PM_ERR_OOM: {failed}; absorbed by the "
          f"speculative-cycle fallback: {absorbed}")
    assert failed >= 20, failed
    assert absorbed <= 3, absorbed  # at most the combined state-and-candidates allocation of each of the three GAs

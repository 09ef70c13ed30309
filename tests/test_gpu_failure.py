"""Failure detection on the GPU without a fault: a scan whose bounded wait runs out.

pm_debug_scan_timeout arms the next column-scan launches so that their
odd-numbered CTAs issue no tile copy: the bounded wait for the tile gives up
after a few thousand polls with nothing in flight, records PM_ERR_TIMEOUT in
the launch's error word and returns (the exit every wait of the library takes;
nothing faults, traps or hangs).  The even-numbered CTAs finish and leave their
split sums (and tile tickets) behind, so these tests check that the failure is reported -- at once
by a synchronous call, through pm_eval_status after an asynchronous one -- and
that the next evaluation on the same instance is exact again (oracle O3).
Shapes: packed split reduction, plain int64 sums with tile tickets (distances
near 2^31 over many clients), and the GA's own scratch.
"""

import numpy as np
import pytest

import oracle
from paper_1610_10061_gb300.inputs import euclid_instance, graph_instance, random_masks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PM_ERR_TIMEOUT = 7


@pytest.fixture(scope="module")
def pm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_10061_gb300 import build

    build.build()
    from paper_1610_10061_gb300 import pm as _pm

    torch.cuda.set_device(0)
    yield _pm
    _pm.pm_debug_scan_timeout(0)


def _dev(masks):
    return torch.from_numpy(np.ascontiguousarray(masks).view(np.int32)).cuda()


def _cases():
    rng = np.random.default_rng(4)
    # n * max d >= 2^47 (70000 clients, distances near 2^31): plain int64 split sums and tile tickets
    big = rng.integers(2**30, 2**31 - 1, size=(70000, 100)).astype(np.int32)
    return [("packed", euclid_instance(600, seed=2), 20, 512), ("tickets", big, 9, 300)]


@pytest.mark.parametrize("name,d,p,pop", _cases(), ids=[c[0] for c in _cases()])
def test_synchronous_call_reports_the_timeout_and_the_next_one_is_exact(pm, name, d, p, pop):
    m = d.shape[1]
    inst = pm.Instance(d, p)
    inst.set_shape(pop, groups=2, warps=8, splits=5)  # five client splits: partial sums left by the others
    opi, ode = oracle.tables(d, p)
    masks = random_masks(pop, m, p, seed=11)
    want = oracle.eval_scan(opi, ode, masks)
    assert pm.pm_debug_scan_timeout(1) == 0
    with pytest.raises(pm.PMError) as e:
        inst.eval(masks)  # host costs: the call synchronises and reads the error word
    assert e.value.status == PM_ERR_TIMEOUT
    assert pm.pm_debug_scan_timeout(0) == 0  # the armed launch was consumed
    for _ in range(2):
        np.testing.assert_array_equal(inst.eval(masks), want)
    assert pm.pm_eval_status(inst.handle) == 0


@pytest.mark.parametrize("name,d,p,pop", _cases(), ids=[c[0] for c in _cases()])
def test_asynchronous_call_leaves_the_timeout_for_pm_eval_status(pm, name, d, p, pop):
    m = d.shape[1]
    inst = pm.Instance(d, p)
    inst.set_shape(pop, groups=2, warps=8, splits=5)
    opi, ode = oracle.tables(d, p)
    masks = _dev(random_masks(pop, m, p, seed=12))
    want = oracle.eval_scan(opi, ode, random_masks(pop, m, p, seed=12))
    costs = torch.empty(pop, dtype=torch.int64, device="cuda")
    pm.pm_debug_scan_timeout(1)
    pm.pm_eval_population(inst.handle, masks, pop, costs, 0, None)  # device buffers: asynchronous, PM_OK
    assert pm.pm_eval_status(inst.handle) == PM_ERR_TIMEOUT
    assert pm.pm_eval_status(inst.handle) == 0  # reading cleared the record
    for _ in range(2):
        pm.pm_eval_population(inst.handle, masks, pop, costs, 0, None)
        np.testing.assert_array_equal(costs.cpu().numpy(), want)
    assert pm.pm_eval_status(inst.handle) == 0


def test_ga_reports_the_timeout_and_later_generations_evaluate_exactly(pm, monkeypatch):
    """Per-phase kernels in stream mode (the graph keeps the launches it captured at creation): the generation
    whose first scan gave up reports PM_ERR_TIMEOUT at the next synchronising call; the GA's scratch is reset, so
    the costs of later generations equal the direct evaluation of their bitsets."""
    monkeypatch.setenv("PM_GA_GRAPH", "0")
    d = graph_instance(200, 600, seed=3)
    inst = pm.Instance(d, 8)
    ga = pm.GA(inst, seed=1, pop=256, deme=64)
    ga.step(2)
    pm.pm_debug_scan_timeout(1)
    with pytest.raises(pm.PMError) as e:
        ga.step(1)  # host trace: synchronises and reads the GA's error word
    assert e.value.status == PM_ERR_TIMEOUT
    ga.step(3)
    masks, costs = ga.population()
    np.testing.assert_array_equal(costs, oracle.eval_direct(d, masks))


def test_persistent_generation_kernel_barrier_timeout(pm, monkeypatch):
    """The persistent generation kernel's grid barrier: armed on the host, CTA 0 of the next launch leaves at once,
    so every other CTA's bounded wait at the first barrier runs out (20 ms), records PM_ERR_TIMEOUT and leaves.
    The next steps start from the same generation and run as usual: the population's costs equal the direct
    evaluation and the GA continues like an untouched one."""
    monkeypatch.setenv("PM_GA_FUSED", "1")
    d = graph_instance(200, 600, seed=3)
    inst = pm.Instance(d, 8)
    ga = pm.GA(inst, seed=1, pop=256, deme=64)
    assert ga.info()["kernels_per_generation"] == 0  # the persistent kernel runs this GA
    ref = pm.GA(inst, seed=1, pop=256, deme=64)
    ga.step(2)
    ref.step(2)
    pm.pm_debug_scan_timeout(1)
    with pytest.raises(pm.PMError) as e:
        ga.step(1)
    assert e.value.status == PM_ERR_TIMEOUT
    assert pm.pm_debug_scan_timeout(0) == 0
    ga.step(3)
    ref.step(3)
    masks, costs = ga.population()
    np.testing.assert_array_equal(costs, oracle.eval_direct(d, masks))
    rm, rc = ref.population()
    np.testing.assert_array_equal(masks, rm)
    np.testing.assert_array_equal(costs, rc)
    assert ga.result()[:3] == ref.result()[:3]

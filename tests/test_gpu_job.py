"""The one-shot job of the C ABI -- pm_instance_create from host memory, pm_ga_run, pm_instance_destroy -- against
the oracle GA (Sections 3.1, 3.2.2, 4.5): best cost and mask, generations run, evaluations and the best cost
after every generation.  pm_ga_run builds only the graph its call launches (the plain one-generation graph for
one generation, the conditional while-graph for more), so both are covered; a child process repeats the job with
PM_POOL=0, where the library allocates with cudaMalloc / cudaFree instead of its memory pool."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1610_10061_gb300.inputs import graph_instance

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_10061_gb300 import build
    build.build()
    from paper_1610_10061_gb300 import pm as _pm
    torch.cuda.set_device(0)
    return _pm


def _job(pm, d, p, pop, deme, gens, seed, pinned):
    """One pm_ga_run job from host buffers; returns (best cost, generations run, evaluations, best mask, trace)."""
    n, m = d.shape
    W = (m + 31) // 32
    if pinned:
        dh = torch.from_numpy(d).pin_memory()
        best = torch.zeros(W, dtype=torch.int32).pin_memory()
        trace = torch.zeros(gens, dtype=torch.int64).pin_memory()
    else:
        dh = np.ascontiguousarray(d)
        best = np.zeros(W, dtype=np.uint32)
        trace = np.zeros(gens, dtype=np.int64)
    h = pm.pm_instance_create(dh, n, m, p, 0, None)
    try:
        bc, gr, ev = pm.pm_ga_run(h, seed, pop, gens, pm._params(deme=deme), best, trace, None)
    finally:
        pm.pm_instance_destroy(h)
    best = best.numpy().view(np.uint32) if pinned else best
    trace = trace.numpy() if pinned else trace
    return bc, gr, ev, np.array(best, dtype=np.uint32), np.array(trace, dtype=np.int64)


@pytest.mark.parametrize("gens,pinned", [(1, False), (1, True), (6, False), (6, True)])
def test_ga_run_job_matches_oracle(pm, gens, pinned):
    d, p, pop, deme, seed = graph_instance(200, 600, seed=11), 12, 128, 32, 4
    pi, de = oracle.tables(d, p)
    st, otrace, _, _ = oracle.ga_run(pi, de, 200, p, seed=seed, P=pop, D=deme, gens=gens)
    for _ in range(2):  # the second job reuses the memory the first one released
        bc, gr, ev, best, trace = _job(pm, d, p, pop, deme, gens, seed, pinned)
        assert (bc, gr, ev) == (st.best_cost, gens, st.evals)
        np.testing.assert_array_equal(best, st.best)
        np.testing.assert_array_equal(trace, otrace)


_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1610_10061_gb300 import pm
from paper_1610_10061_gb300.inputs import graph_instance
d = graph_instance(200, 600, seed=11)
out = []
for gens in (1, 6):
    best = np.zeros(7, dtype=np.uint32)
    trace = np.zeros(gens, dtype=np.int64)
    h = pm.pm_instance_create(d, 200, 200, 12, 0, None)
    inst = pm.Instance(d, 12)
    masks = np.zeros((3, 7), dtype=np.uint32)
    for t, js in enumerate(([0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11], list(range(100, 112)), list(range(188, 200)))):
        for j in js:
            masks[t, j >> 5] |= np.uint32(1 << (j & 31))
    costs = inst.eval(masks).tolist()
    inst.close()
    bc, gr, ev = pm.pm_ga_run(h, 4, 128, gens, pm._params(deme=32), best, trace, None)
    pm.pm_instance_destroy(h)
    out.append(dict(gens=gens, bc=bc, gr=gr, ev=ev, best=best.tolist(), trace=trace.tolist(), costs=costs))
print(json.dumps(out))
"""


def test_ga_run_job_without_the_memory_pool(pm):
    """The same jobs, and an evaluation, in a child process whose allocations bypass the pool (PM_POOL=0)."""
    d, p = graph_instance(200, 600, seed=11), 12
    pi, de = oracle.tables(d, p)
    env = dict(os.environ, PM_POOL="0")
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    masks = np.zeros((3, 7), dtype=np.uint32)
    for t, js in enumerate((list(range(0, 12)), list(range(100, 112)), list(range(188, 200)))):
        for j in js:
            masks[t, j >> 5] |= np.uint32(1 << (j & 31))
    want_costs = oracle.eval_direct(d, masks).tolist()
    for rec in res:
        st, otrace, _, _ = oracle.ga_run(pi, de, 200, p, seed=4, P=128, D=32, gens=rec["gens"])
        assert (rec["bc"], rec["gr"], rec["ev"]) == (st.best_cost, rec["gens"], st.evals)
        assert rec["best"] == st.best.tolist()
        assert rec["trace"] == otrace.tolist()
        assert rec["costs"] == want_costs

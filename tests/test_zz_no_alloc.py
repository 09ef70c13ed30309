"""pm_eval_population_noalloc: evaluation for callers that cannot allocate device memory.

Some callers of this library may not call cudaMalloc when they evaluate (a
serving process whose framework already holds nearly all device memory in its
own pool, or a real-time loop that must avoid the allocator).  The no-alloc
entry point keeps its scratch in a fixed array inside the library.  This test
calls it through the C ABI twice in a row -- the second call reuses the array
the first one left behind -- and checks both results against
pm_eval_population, bit for bit (integer costs).  It also checks that a
population too large for the fixed array is refused without any launch.
This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

from paper_1610_10061_gb300.inputs import euclid_instance, graph_instance, random_masks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_10061_gb300 import build

    path = build.build()
    torch.cuda.set_device(0)
    lib = ctypes.CDLL(path)
    lib.pm_eval_population_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                               ctypes.c_void_p]
    lib.pm_eval_population_noalloc.restype = ctypes.c_int
    return lib


def _dev(masks):
    return torch.from_numpy(np.ascontiguousarray(masks).view(np.int32)).cuda()


def test_noalloc_matches_the_allocating_entry_point_on_two_calls(lib):
    from paper_1610_10061_gb300 import pm

    stream = torch.cuda.current_stream().cuda_stream
    for d, p, pops in [(graph_instance(300, 1200, seed=5), 12, (1000, 77)), (euclid_instance(900, seed=8), 90, (1024, 1024))]:
        m = d.shape[1]
        inst = pm.Instance(d, p)
        results = []
        for call, pop in enumerate(pops):
            masks = _dev(random_masks(pop, m, p, seed=10 * call + p))
            want = torch.empty(pop, dtype=torch.int64, device="cuda")
            pm.pm_eval_population(inst.handle, masks, pop, want, 0, stream)
            got = torch.full((pop,), -1, dtype=torch.int64, device="cuda")
            rc = lib.pm_eval_population_noalloc(inst.handle, ctypes.c_void_p(masks.data_ptr()), pop,
                                                ctypes.c_void_p(got.data_ptr()), ctypes.c_void_p(stream))
            assert rc == 0, pm.pm_strerror(rc)
            torch.cuda.synchronize()
            assert torch.equal(got, want)
            results.append(got.cpu().numpy())
        inst.close()


def test_noalloc_refuses_what_does_not_fit_and_host_pointers(lib):
    from paper_1610_10061_gb300 import pm

    rng = np.random.default_rng(1)
    d = rng.integers(0, 1000, size=(4, 10000)).astype(np.int32)
    inst = pm.Instance(d, 50)
    pop = 8192  # 8192 x 313 words = 10 MB of facility-major scratch alone, above the 8 MiB array
    masks = _dev(random_masks(pop, 10000, 50, seed=2))
    out = torch.zeros(pop, dtype=torch.int64, device="cuda")
    rc = lib.pm_eval_population_noalloc(inst.handle, ctypes.c_void_p(masks.data_ptr()), pop,
                                        ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 1
    torch.cuda.synchronize()
    assert int(out.abs().sum()) == 0
    host = random_masks(8, 10000, 50, seed=3)
    hc = np.zeros(8, dtype=np.int64)
    rc = lib.pm_eval_population_noalloc(inst.handle, ctypes.c_void_p(host.ctypes.data), 8,
                                        ctypes.c_void_p(hc.ctypes.data), None)
    assert rc == 1
    inst.close()

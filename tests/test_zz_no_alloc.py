"""pm_eval_population_noalloc: evaluation for callers that cannot allocate device memory.

Some callers of this library may not call cudaMalloc when they evaluate (a
serving process whose framework already holds nearly all device memory in its
own pool, or a real-time loop that must avoid the allocator).  The no-alloc
entry point keeps its scratch in a fixed array inside the library.  These tests
call it through the C ABI twice in a row -- the second call reuses the array
the first one left behind -- and check both results against
pm_eval_population, bit for bit (integer costs), for each scratch layout the
array can hold: the column kernel with the packed split reduction, the column
kernel with plain int64 split sums and tile tickets (costs that could reach
2^47), the row kernel (one partial sum per client split and individual), and a
population whose scratch is just below the array's 8 MiB.  They also check
that the next size up and host pointers are refused without any launch, and
that a scan timeout on this path is reported by pm_eval_status.
This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

from paper_1610_10061_gb300.inputs import euclid_instance, graph_instance, random_masks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LIMIT = 8 << 20  # bytes of the fixed array


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
    lib.pm_eval_status.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.pm_eval_status.restype = ctypes.c_int
    return lib


def _dev(masks):
    return torch.from_numpy(np.ascontiguousarray(masks).view(np.int32)).cuda()


def _noalloc(lib, inst, masks, pop, out, stream):
    return lib.pm_eval_population_noalloc(inst.handle, ctypes.c_void_p(masks.data_ptr()), pop,
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def _two_calls_match(lib, pm, inst, m, p, pops, seed):
    stream = torch.cuda.current_stream().cuda_stream
    for call, pop in enumerate(pops):
        masks = _dev(random_masks(pop, m, p, seed=seed + call))
        want = torch.empty(pop, dtype=torch.int64, device="cuda")
        pm.pm_eval_population(inst.handle, masks, pop, want, 0, stream)
        got = torch.full((pop,), -1, dtype=torch.int64, device="cuda")
        rc = _noalloc(lib, inst, masks, pop, got, stream)
        assert rc == 0, pm.pm_strerror(rc)
        torch.cuda.synchronize()
        assert torch.equal(got, want), f"call {call} (pop {pop}) differs from pm_eval_population"
    assert lib.pm_eval_status(inst.handle, ctypes.c_void_p(stream)) == 0


def _rup(x, a=256):
    return (x + a - 1) // a * a


def _scratch_bytes(W, pop, groups, splits):
    """Bytes the no-alloc call needs for a pinned shape: the error word's 256 bytes, the tile tickets, the
    facility-major copy and the partial sums, each rounded up to 256 bytes."""
    if groups == 0:  # row kernel: one partial sum per split and individual, no facility-major copy
        tiles = -(-pop // 8)
        return 256 + _rup(tiles * 4) + 0 + _rup(splits * pop * 8)
    tiles = -(-pop // (32 * groups))
    return 256 + _rup(tiles * 4) + _rup(tiles * W * 32 * groups * 4) + _rup(pop * 8)


def test_noalloc_matches_the_allocating_entry_point_on_two_calls(lib):
    from paper_1610_10061_gb300 import pm

    for d, p, pops in [(graph_instance(300, 1200, seed=5), 12, (1000, 77)),
                       (euclid_instance(900, seed=8), 90, (1024, 1024))]:
        inst = pm.Instance(d, p)
        _two_calls_match(lib, pm, inst, d.shape[1], p, pops, seed=p)
        inst.close()


def test_noalloc_other_scratch_layouts(lib):
    from paper_1610_10061_gb300 import pm

    # plain int64 split sums and tile tickets: n * max d >= 2^47
    rng = np.random.default_rng(7)
    big = rng.integers(2**30, 2**31 - 1, size=(70000, 100)).astype(np.int32)
    inst = pm.Instance(big, 9)
    for pop in (300, 301):
        inst.set_shape(pop, groups=2, warps=8, splits=6)
    _two_calls_match(lib, pm, inst, 100, 9, (300, 301), seed=1)
    inst.close()
    # the row kernel: one sum per client split and individual in the array
    d = euclid_instance(700, seed=9)
    inst = pm.Instance(d, 30)
    for pop in (200, 333):
        inst.set_shape(pop, groups=0, splits=7)
    _two_calls_match(lib, pm, inst, 700, 30, (200, 333), seed=2)
    inst.close()


def test_noalloc_population_just_below_the_limit(lib):
    from paper_1610_10061_gb300 import pm

    rng = np.random.default_rng(1)
    m, p = 10000, 50
    W = (m + 31) // 32
    d = rng.integers(0, 1000, size=(40, m)).astype(np.int32)
    inst = pm.Instance(d, p)
    pop = 128
    while _scratch_bytes(W, pop + 128, 4, 1) <= LIMIT:
        pop += 128
    assert LIMIT - _scratch_bytes(W, pop, 4, 1) < 200 * 1024  # within one tile of the limit
    for q in (pop, pop + 128):
        inst.set_shape(q, groups=4, warps=16, splits=4)
    _two_calls_match(lib, pm, inst, m, p, (pop, pop), seed=3)
    big = pop + 128  # one more tile: above the array
    masks = _dev(random_masks(big, m, p, seed=4))
    out = torch.zeros(big, dtype=torch.int64, device="cuda")
    assert _noalloc(lib, inst, masks, big, out, torch.cuda.current_stream().cuda_stream) == 1
    torch.cuda.synchronize()
    assert int(out.abs().sum()) == 0
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


def test_noalloc_timeout_is_reported_by_pm_eval_status(lib):
    """A scan whose bounded wait gives up (armed on the host: no tile copy for the odd-numbered CTAs, nothing
    faults) cannot report through this asynchronous call; pm_eval_status reads the array's error word, clears it,
    and the next call is exact again."""
    from paper_1610_10061_gb300 import pm

    d = euclid_instance(600, seed=2)
    inst = pm.Instance(d, 20)
    inst.set_shape(512, groups=2, warps=8, splits=5)
    stream = torch.cuda.current_stream().cuda_stream
    masks = _dev(random_masks(512, 600, 20, seed=5))
    want = torch.empty(512, dtype=torch.int64, device="cuda")
    pm.pm_eval_population(inst.handle, masks, 512, want, 0, stream)
    got = torch.empty(512, dtype=torch.int64, device="cuda")
    pm.pm_debug_scan_timeout(1)
    try:
        assert _noalloc(lib, inst, masks, 512, got, stream) == 0
    finally:
        pm.pm_debug_scan_timeout(0)
    assert lib.pm_eval_status(inst.handle, ctypes.c_void_p(stream)) == 7
    assert lib.pm_eval_status(inst.handle, ctypes.c_void_p(stream)) == 0
    for _ in range(2):
        assert _noalloc(lib, inst, masks, 512, got, stream) == 0
        torch.cuda.synchronize()
        assert torch.equal(got, want)
    assert lib.pm_eval_status(inst.handle, ctypes.c_void_p(stream)) == 0
    inst.close()

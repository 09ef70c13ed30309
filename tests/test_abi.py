"""The C-ABI library builds, loads and exports every symbol include/pm.h declares (no GPU calls)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^PM_API\s+[\w\s\*]*?\b(pm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1610_10061_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("pm_instance_create", "pm_eval_population", "pm_ga_run"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    from paper_1610_10061_gb300 import pm

    assert set(pm.exported_symbols()) == set(_declared())


def test_strerror_without_gpu(lib):
    lib.pm_strerror.restype = ctypes.c_char_p
    assert lib.pm_strerror(0) == b"PM_OK"
    assert b"NEGATIVE" in lib.pm_strerror(2)
    assert lib.pm_strerror(99) == b"unknown pm_status"


def test_invalid_arguments_rejected_before_any_device_work(lib):
    from paper_1610_10061_gb300 import pm

    with pytest.raises(pm.PMError) as e:
        pm.pm_instance_create(None, 5, 4, 2)
    assert e.value.status == 1
    import numpy as np

    d = np.zeros((3, 4), dtype=np.int32)
    for n, m, p in [(0, 4, 2), (3, 4, 4), (3, 4, 0), (3, 1, 1)]:
        with pytest.raises(pm.PMError) as e:
            pm.pm_instance_create(d, n, m, p)
        assert e.value.status == 1
    big = np.zeros((1, 1), dtype=np.int32)
    with pytest.raises(pm.PMError) as e:
        pm.pm_instance_create(big, 1, 70000, 3)
    assert e.value.status == 3


def _header_defines():
    out = {}
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            for name, val in re.findall(r"^#define\s+(PM_[A-Z_]+)\s+(\d+)u?\s*$", text, flags=re.M):
                out[name] = int(val)
    return out


def test_binding_flags_match_the_header():
    from paper_1610_10061_gb300 import pm

    defs = _header_defines()
    for name in ("PM_GA_TUNE", "PM_GA_MIGRATE_TEAM", "PM_GA_INIT_COMBINADIC", "PM_TABLES_CUMULATIVE"):
        assert getattr(pm, name) == defs[name], name


def test_ga_params_marshalling():
    """The binding's GA parameters land in the C struct as the header describes (no GPU needed)."""
    from paper_1610_10061_gb300 import pm

    q = pm._params(deme=64, xover_rounds=20, mut_tries=60, saturation=7, stream_id=3, tune=True,
                   migration="team", init="combinadic", candidates=5)
    assert (q.deme, q.xover_rounds, q.mut_tries, q.saturation, q.stream_id, q.candidates) == (64, 20, 60, 7, 3, 5)
    assert q.flags == pm.PM_GA_TUNE | pm.PM_GA_MIGRATE_TEAM | pm.PM_GA_INIT_COMBINADIC
    assert not q.model
    d = pm._params()
    assert (d.deme, d.xover_rounds, d.mut_tries, d.flags) == (0, -1, -1, 0)  # library defaults: lg D tries
    with pytest.raises(ValueError):
        pm._params(migration="ring")
    with pytest.raises(ValueError):
        pm._params(init="lhs")
    # status codes name themselves
    assert "PM_ERR_OOM" in pm.pm_strerror(6) and "PM_ERR_TIMEOUT" in pm.pm_strerror(7)

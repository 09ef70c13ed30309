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

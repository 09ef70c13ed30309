"""The device Hammer-Beresnev polynomial (Section 2.1, Eq. 6) against the oracle's O2 and O1.

The merged monomial dictionary is integer data, so it must equal the oracle's
exactly (as a map from facility sets to coefficients); its value at every
tested open set must equal the direct cost (O1) and the scan
(pm_eval_population).  Example 1's printed reduced polynomial is the first
case; tie-heavy instances make prefixes of different clients equal as sets in
different orders, which the merge must recognise.
"""

import itertools

import numpy as np
import pytest

import oracle
from paper_1610_10061_gb300.inputs import euclid_instance, graph_instance, masks_from_sets, random_masks

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


def _dev(masks):
    return torch.from_numpy(np.ascontiguousarray(masks).view(np.int32)).cuda()


def _printed(example1):
    out = {}
    for row in example1["POLY"]:
        coeff, *fac = row
        out[frozenset(j - 1 for j in fac)] = coeff
    return out


def test_example1_reduced_polynomial_and_values(pm, example1):
    C = np.array(example1["C"], dtype=np.int32)
    poly = pm.Polynomial(pm.Instance(C, 2))
    assert poly.terms == 7
    assert poly.monomials() == _printed(example1)
    sets = list(itertools.combinations(range(4), 2))
    masks = masks_from_sets(sets, 4)
    got = poly.eval(_dev(masks)).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.eval_direct(C, masks))
    assert got.tolist() == [43, 37, 35, 46, 40, 44]  # the six open sets of Example 1, computed from the matrix


def _cases():
    rng = np.random.default_rng(21)
    return [
        ("ties3", rng.integers(0, 3, size=(30, 12)).astype(np.int32), 3),
        ("ties2_wide", rng.integers(0, 2, size=(40, 70)).astype(np.int32), 9),
        ("graph", graph_instance(60, 120, seed=2), 6),
        ("euclid", euclid_instance(90, seed=5), 11),
        ("p1", rng.integers(0, 50, size=(25, 33)).astype(np.int32), 1),
    ]


@pytest.mark.parametrize("cumulative", [False, True])
@pytest.mark.parametrize("name,d,p", _cases(), ids=[c[0] for c in _cases()])
def test_dictionary_and_values_match_the_oracle(pm, name, d, p, cumulative):
    inst = pm.Instance(d, p, cumulative=cumulative)
    poly = pm.Polynomial(inst)
    opi, ode = oracle.tables(d, p)
    want = oracle.hbp_polynomial(opi, ode)
    got = poly.monomials()
    assert poly.terms == len(want)
    assert got == want
    m = d.shape[1]
    masks = random_masks(300, m, p, seed=7)
    vals = poly.eval(_dev(masks)).cpu().numpy()
    np.testing.assert_array_equal(vals, oracle.eval_direct(d, masks))
    np.testing.assert_array_equal(vals, inst.eval(masks))

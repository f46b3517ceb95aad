"""The precision-search harness's error measure (Eqs. 1-2) on the CPU: its
normalised norms equal the oracle's on random fields, reduce to closed forms
on scaled fields, and E treats a non-finite result as unacceptable."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2404_08849_gb300 import precision as PR


def test_norms_match_oracle_definition():
    rng = np.random.default_rng(3)
    for shape, wshape in (((500,), (500,)), ((300, 7), (300,))):
        ref = rng.standard_normal(shape) + 2.0
        x = ref + 1e-3 * rng.standard_normal(shape)
        w = rng.uniform(0.5, 2.0, wshape)
        a = PR.error_norms(x, ref, w)
        b = O.error_norms(x, ref, w)
        assert a == pytest.approx(b, rel=1e-13)
        assert PR.error_level(x, ref, w) == pytest.approx(O.error_level(x, ref, w), rel=1e-13)


def test_closed_forms():
    ref = np.linspace(1.0, 3.0, 101)
    w = np.ones(101)
    # a uniform 10 % scaling gives 0.1 in every norm
    assert PR.error_norms(1.1 * ref, ref, w) == pytest.approx((0.1, 0.1, 0.1), rel=1e-12)
    # one perturbed point: linf = |d| / max|r|, l1 = |d| / sum|r|
    x = ref.copy()
    x[50] += 0.5
    l1, l2, linf = PR.error_norms(x, ref, w)
    assert linf == pytest.approx(0.5 / 3.0)
    assert l1 == pytest.approx(0.5 / ref.sum())
    assert l2 == pytest.approx(math.sqrt(0.25 / np.sum(ref * ref)))


def test_overall_error_is_max_of_fields_and_rejects_nonfinite():
    ps = np.full(10, 1e5)
    vor = np.linspace(-1e-5, 1e-5, 12).reshape(6, 2) + 1e-6
    ca, va = np.ones(10), np.ones(6)
    assert PR.overall_error(ps, ps, vor, vor, ca, va) == 0.0
    e_ps = PR.error_level(ps * 1.01, ps, ca)
    assert PR.overall_error(ps * 1.01, ps, vor, vor, ca, va) == pytest.approx(e_ps)
    bad = vor.copy()
    bad[0, 0] = np.nan
    assert PR.overall_error(ps, ps, bad, vor, ca, va) == math.inf

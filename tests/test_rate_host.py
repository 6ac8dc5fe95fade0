"""The library's host-side rate adaptation (section 4.1) against the oracle's,
over the QBER and efficiency range of the workloads and beyond: the same
punctured/shortened counts for every frame, the same efficiency, and the same
puncturing order of the variables."""
import numpy as np
import pytest

from oracle import rate as orate
from paper_1903_10107_gb300 import inputs, rate

WORKLOADS = ("n4096_r075_q02", "n40960_r080_q03", "n49152_mixed_q01_08")


@pytest.mark.parametrize("wname", WORKLOADS)
def test_plan_and_efficiency_equal_the_oracle(wname):
    w = inputs.WORKLOADS[wname]
    n, m = w.n, w.m
    qs = np.concatenate([np.linspace(0.005, 0.10, 77), [0.01, 0.02, 0.03, 0.08]])
    for f in (1.05, 1.1, 1.2, 1.35, 1.5, 1.7, 2.0):
        p, s = rate.plan(n, m, qs, f)
        for i, q in enumerate(qs):
            po, so = orate.rate_plan(n, m, float(q), f)
            assert (int(p[i]), int(s[i])) == (po, so), (wname, f, q)
            if n - po - so > 0:
                assert float(rate.efficiency(n, m, p[i], s[i], q)) == pytest.approx(
                    orate.efficiency(n, m, po, so, float(q)), rel=1e-12)


@pytest.mark.parametrize("wname", WORKLOADS)
def test_puncturing_order_equals_the_oracle(wname):
    w = inputs.WORKLOADS[wname]
    base = np.asarray(w.base())
    tb = inputs.tiebreak_permutation(w.n, w.code_seed)
    got = rate.puncture_rank(base, w.Z, tb)
    assert np.array_equal(got, orate.position_rank(base, w.Z, tb))
    assert np.array_equal(np.sort(got), np.arange(w.n))  # a permutation of the positions

"""The per-frame channel-LLR magnitude (section 3.1), computed on the host by
the library (``ldpc_llr_magnitudes``) and handed to the kernels as int8.

It must equal the oracle's magnitude exactly -- including for QBERs at which
ln((1-q)/q) * scale lands within 1e-12 of a half-integer, where a last-ulp
difference between two logarithm implementations would flip the rounding.
Both sides evaluate the host C library's log, so they agree by construction;
these tests check that they do, and that the library rejects what it cannot
quantise.  No GPU is needed."""
import math

import numpy as np
import pytest

from conftest import golden
from oracle import core as orc
from paper_1903_10107_gb300 import native
from paper_1903_10107_gb300.decoder import llr_magnitudes


def test_magnitudes_match_the_golden_hand_arithmetic():
    rows = golden("llr_quantisation.txt")
    q = np.array([float(p) for p, _ in rows])
    assert llr_magnitudes(q, 8.0).tolist() == [int(m) for _, m in rows]


def _near_half_integers(scale, ks):
    """QBERs q with ln((1-q)/q) * scale within 1e-12 of k + 1/2, on both
    sides of it (the float64 neighbours of the exact crossing point)."""
    out = []
    for k in ks:
        q0 = 1.0 / (1.0 + math.exp((k + 0.5) / scale))
        for steps in range(-3, 4):
            q = q0
            for _ in range(abs(steps)):
                q = math.nextafter(q, 1.0 if steps > 0 else 0.0)
            x = math.log((1.0 - q) / q) * scale
            if abs(x - (k + 0.5)) < 1e-12:
                out.append(q)
    return np.array(out)


@pytest.mark.parametrize("scale", [8.0, 1 / 0.29, 5.5])
def test_magnitudes_equal_the_oracle_at_half_integer_boundaries(scale):
    q = _near_half_integers(scale, range(2, 60))
    assert q.size > 50
    lib = llr_magnitudes(q, scale)
    ref = np.array([orc.llr_magnitude(float(x), scale) for x in q])
    assert np.array_equal(lib, ref)
    # both roundings occur among the neighbours of a crossing point
    x = np.log((1 - q) / q) * scale
    assert set(np.round(x - np.floor(x), 6)) <= {0.5} or len(set(lib.tolist())) > 1


def test_magnitudes_equal_the_oracle_on_random_qbers():
    q = np.random.default_rng(4).uniform(1e-4, 0.4999, size=5000)
    for scale in (8.0, 1 / 0.29):
        lib = llr_magnitudes(q, scale)
        assert np.array_equal(lib, [orc.llr_magnitude(float(x), scale) for x in q])


def test_magnitudes_reject_bad_arguments():
    for bad_q in (0.0, 0.5, 0.7, -0.1, float("nan")):
        with pytest.raises(native.LdpcError) as ei:
            llr_magnitudes([0.02, bad_q], 8.0)
        assert ei.value.code == native.LDPC_EINVAL
    with pytest.raises(native.LdpcError):
        llr_magnitudes([0.02], 0.0)
    assert llr_magnitudes([], 8.0).size == 0

"""Host logic of the learned tables (no GPU): the layers' degree classes, the
temperature the integer decoder's LLR step implies, and the rounding of the
learned scales and offsets into the integer decoder's tables (round half
away from zero, clipped to the table types, one entry per layer from its
class)."""
import types

import numpy as np
import pytest
import torch

from paper_1903_10107_gb300 import relaxed


def _fake_code(base):
    return types.SimpleNamespace(base=np.asarray(base, np.int32), device=torch.device("cpu"))


def test_degree_classes():
    base = np.full((5, 6), -1, np.int32)
    base[0, :3] = 0      # degree 3
    base[1, :6] = 0      # degree 6
    base[3, :3] = 1      # degree 3
    base[4, :5] = 2      # degree 5; row 2 is empty
    cls, uniq = relaxed.degree_classes(base)
    assert list(uniq) == [3, 5, 6]
    assert list(cls) == [0, 2, 0, 0, 1]


def test_kappa_for_scale():
    assert relaxed.kappa_for_scale(1 / relaxed.TABLE_STEP_NAT) == pytest.approx(1.0)  # the table's own step
    assert relaxed.kappa_for_scale(8.0) == pytest.approx(1.0 / (8.0 * 0.29))


def test_integer_tables_round_half_away_and_clip():
    base = np.full((3, 4), -1, np.int32)
    base[0, :2] = 0   # class 0 (degree 2)
    base[1, :4] = 0   # class 1 (degree 4)
    base[2, :2] = 0   # class 0
    dec = relaxed.RelaxedDecoder(_fake_code(base), iters=3)
    with torch.no_grad():
        dec.alpha.copy_(torch.tensor([[1.03125, 0.96875],     # 16.5 -> 17, 15.5 -> 16
                                      [20.0, -1.0],           # clipped to 255 and 0
                                      [0.75, 1.0]], dtype=torch.float32))
        dec.gamma.copy_(torch.tensor([[0.0625, -0.0625],      # x8: 0.5 -> 1, -0.5 -> -1
                                      [100.0, -100.0],        # clipped to 127 and -128
                                      [0.2, -0.19]], dtype=torch.float32))
    sq, oq = dec.integer_tables(8.0)
    assert sq.dtype == np.uint8 and oq.dtype == np.int8 and sq.shape == oq.shape == (3, 3)
    assert sq.tolist() == [[17, 16, 17], [255, 0, 255], [12, 16, 12]]
    assert oq.tolist() == [[1, -1, 1], [127, -128, 127], [2, -2, 2]]


def test_untrained_tables_are_the_identity():
    base = np.zeros((2, 5), np.int32)
    sq, oq = relaxed.RelaxedDecoder(_fake_code(base), iters=4).integer_tables(3.45)
    assert (sq == 16).all() and (oq == 0).all()

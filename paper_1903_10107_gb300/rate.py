"""Rate adaptation for the reconciliation protocol (section 4.1), host side.

One mother code serves every QBER: positions of low column weight are
punctured first, and shortened positions are taken from the same ordering.
The counts bring each frame to a target efficiency ``f = (1 - R)/h(q)``:

* ``R = 1 - f_target h(q)``;
* ``R >= R0 = 1 - m/n``: puncture ``p = round(n - (n - m)/R)``;
* ``R <  R0``: shorten ``s = round((n - m - R n)/(1 - R))``;
* key bits per frame ``n - p - s``; efficiency ``(m - p)/((n - p - s) h(q))``
  (revealed bits of the interactive rounds add to ``m - p``).

``round`` is round-half-away-from-zero.  The decoder kernels see only the
resulting per-frame counts and the per-code ``rank`` table.
"""
from __future__ import annotations

import numpy as np


def h2(q):
    q = np.asarray(q, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        v = -q * np.log2(q) - (1.0 - q) * np.log2(1.0 - q)
    return np.where((q > 0) & (q < 1), v, 0.0)


def _rhaz(x):
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def plan(n: int, m: int, qber, f_target: float):
    """Per-frame (n_punct, n_short) int32 arrays for the given QBERs."""
    q = np.atleast_1d(np.asarray(qber, dtype=np.float64))
    R = 1.0 - f_target * h2(q)
    R0 = 1.0 - m / n
    p = np.where(R >= R0, _rhaz(n - (n - m) / R), 0.0)
    s = np.where(R < R0, _rhaz((n - m - R * n) / (1.0 - R)), 0.0)
    p = np.clip(p, 0, m).astype(np.int32)
    s = np.clip(s, 0, n - m).astype(np.int32)
    return p, s


def key_bits(n: int, n_punct, n_short):
    return n - np.asarray(n_punct, np.int64) - np.asarray(n_short, np.int64)


def efficiency(n: int, m: int, n_punct, n_short, qber, revealed=0):
    p = np.asarray(n_punct, np.float64)
    s = np.asarray(n_short, np.float64)
    return (m - p + np.asarray(revealed, np.float64)) / ((n - p - s) * h2(qber))


def puncture_rank(base: np.ndarray, Z: int, tiebreak: np.ndarray) -> np.ndarray:
    """rank[j] = position of variable j in the puncturing order: ascending
    column weight of its block column, ties by ``tiebreak[j]``."""
    weight = np.repeat((np.asarray(base) >= 0).sum(axis=0), Z)
    order = np.lexsort((np.asarray(tiebreak), weight))
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    return rank.astype(np.int32)

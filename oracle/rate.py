"""Rate adaptation and efficiency, as the oracle computes them (test
infrastructure only).

Section 4.1 adapts one mother code to each QBER by puncturing and
shortening: positions of low column weight are punctured first, and
shortened positions are taken in turn from the same ordering.  The paper
gives no formula for the counts; the reading used here is

* target rate ``R = 1 - f_target * h(q)`` with ``h`` the binary entropy;
* ``R >= R0 = 1 - m/n``: puncture ``p = round(n - (n - m) / R)``, ``s = 0``;
* ``R <  R0``: shorten ``s = round((n - m - R n) / (1 - R))``, ``p = 0``;
* effective rate ``(n - m - s) / (n - p - s)``, key length ``n - p - s``;
* efficiency ``f = (1 - R_eff) / h(q) = (m - p) / ((n - p - s) h(q))``.

``round`` is round-half-away-from-zero.
"""
from __future__ import annotations

import math

import numpy as np


def binary_entropy(q: float) -> float:
    if q <= 0.0 or q >= 1.0:
        return 0.0
    return -q * math.log2(q) - (1.0 - q) * math.log2(1.0 - q)


def _round_half_away(x: float) -> int:
    return int(math.floor(x + 0.5)) if x >= 0 else -int(math.floor(-x + 0.5))


def rate_plan(n: int, m: int, q: float, f_target: float):
    """(punctured, shortened) counts that bring the mother code to f_target."""
    R = 1.0 - f_target * binary_entropy(q)
    R0 = 1.0 - m / n
    if R >= R0:
        p = _round_half_away(n - (n - m) / R)
        return max(0, min(p, m)), 0
    s = _round_half_away((n - m - R * n) / (1.0 - R))
    return 0, max(0, min(s, n - m))


def efficiency(n: int, m: int, p: int, s: int, q: float) -> float:
    return (m - p) / ((n - p - s) * binary_entropy(q))


def effective_rate(n: int, m: int, p: int, s: int) -> float:
    return (n - m - s) / (n - p - s)


def position_rank(base: np.ndarray, Z: int, tiebreak: np.ndarray) -> np.ndarray:
    """rank[j]: place of VN j in the puncturing order -- ascending column
    weight, ties broken by the seeded key ``tiebreak[j]``."""
    base = np.asarray(base)
    w_block = (base >= 0).sum(axis=0)
    n = base.shape[1] * Z
    w = np.repeat(w_block, Z)
    order = sorted(range(n), key=lambda j: (int(w[j]), int(tiebreak[j])))
    rank = np.empty(n, dtype=np.int32)
    for i, j in enumerate(order):
        rank[j] = i
    return rank


def position_states(rank: np.ndarray, n_punct: int, n_short: int) -> np.ndarray:
    """0 key bit, 1 punctured, 2 shortened: ranks below ``n_short`` are
    shortened, the next ``n_punct`` ranks punctured."""
    st = np.zeros(len(rank), dtype=np.uint8)
    st[rank < n_short] = 2
    st[(rank >= n_short) & (rank < n_short + n_punct)] = 1
    return st

"""Interactive rate-adaptive reconciliation on the CPU oracle (sections 4.1
and 4.2).  TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and
the bench's CPU-baseline and reference legs; it never touches the CUDA path.

Every frame starts at the rate that gives the target efficiency ``f_start``
for its QBER (``rate.rate_plan``).  After each round the frames whose
syndrome did not match have more of their puncturing order revealed by
Alice -- the punctured positions first (they become shortened, i.e. known to
both sides), then key positions -- and are decoded again from their channel
LLRs, up to ``max_rounds`` extra rounds.  The paper makes interaction part of
every reconciliation (section 4.2) but does not say how many bits a round
reveals; the reading used here reveals ``ceil(df * key_bits * h(q))`` more
bits per round, ``key_bits`` the frame's current key length.

Efficiency of a frame after ``r`` revealed bits (``p0``, ``s0`` its initial
punctured and shortened counts): revealed punctured bits add to the leak
(``m - p0 + min(r, p0)``), revealed key bits leave the key
(``n - p0 - s0 - max(r - p0, 0)``); ``f = leak / (key * h(q))``.
"""
from __future__ import annotations

import math

import numpy as np

from . import core
from . import rate as orate


def reveal_step(df: float, key_bits: int, q: float) -> int:
    """Bits revealed in one more round for a frame of ``key_bits`` at QBER q."""
    return int(math.ceil(df * key_bits * orate.binary_entropy(q)))


def interactive(base, Z: int, tiebreak, xa_bits, yb_bits, qber, f_start: float, df: float, max_rounds: int,
                max_iter: int, scale: float, stall_window: int = 0, threads: int = 0):
    """Run the protocol for every frame.

    xa_bits, yb_bits: unpacked 0/1 [batch][n] (Alice's and Bob's keys);
    qber: [batch].  Returns a dict of arrays indexed by frame: bits (Bob's
    final hard decisions, unpacked), iters (summed over rounds), ok, rounds
    (index of the last round decoded), revealed, key_bits, f."""
    base = np.asarray(base)
    Mb, Nb = base.shape
    n, m = Nb * Z, Mb * Z
    xa_bits = np.asarray(xa_bits, dtype=np.uint8)
    yb_bits = np.asarray(yb_bits, dtype=np.uint8)
    q = np.asarray(qber, dtype=np.float64)
    B = q.size
    rank = orate.position_rank(base, Z, tiebreak)
    syn = core.syndrome(base, Z, xa_bits)
    plans = [orate.rate_plan(n, m, float(q[f]), f_start) for f in range(B)]
    p0 = np.array([p for p, _ in plans], dtype=np.int64)
    s0 = np.array([s for _, s in plans], dtype=np.int64)
    revealed = np.zeros(B, np.int64)
    rounds = np.zeros(B, np.int32)
    iters = np.zeros(B, np.int64)
    ok = np.zeros(B, np.uint8)
    bits = np.zeros((B, n), np.uint8)
    todo = list(range(B))
    for rnd in range(max_rounds + 1):
        states = np.stack([orate.position_states(rank, int(max(p0[f] - revealed[f], 0)),
                                                 int(s0[f] + revealed[f])) for f in todo])
        llr = core.llr_frames(yb_bits[todo], q[todo], states, xa_bits[todo], scale=scale)
        b, it, o, _ = core.decode(base, Z, llr, syn[todo], max_iter, stall_window=stall_window, threads=threads)
        still = []
        for k, f in enumerate(todo):
            bits[f], ok[f], rounds[f] = b[k], o[k], rnd
            iters[f] += int(it[k])
            if not o[k]:
                still.append(f)
        todo = still
        if not todo or rnd == max_rounds:
            break
        for f in todo:
            key_now = n - p0[f] - s0[f] - max(int(revealed[f]) - int(p0[f]), 0)
            revealed[f] += reveal_step(df, int(key_now), float(q[f]))
    rp = np.minimum(revealed, p0)
    key = n - p0 - s0 - (revealed - rp)
    f_eff = np.array([(m - p0[f] + rp[f]) / (key[f] * orate.binary_entropy(float(q[f]))) for f in range(B)])
    return dict(bits=bits, iters=iters, ok=ok, rounds=rounds, revealed=revealed, key_bits=key, f=f_eff)

"""The oracle's interactive protocol (oracle/protocol.py), which the CPU
baseline and the GPU protocol test use, against the protocol's definition
replayed round by round here with the oracle's single decodes: which frames
each round decodes, the bits each reveal adds (ceil(df * key bits * h(q)),
punctured positions before key positions), summed iterations, and the
efficiency of section 4.1 with every revealed bit counted.  No GPU."""
import math

import numpy as np
import pytest

from oracle import core as orc
from oracle import protocol as oproto
from oracle import rate as orate
from paper_1903_10107_gb300 import inputs


def _case(B, seed=3, Z=16):
    degs = inputs.mixed_column_degrees(96, 0.3, 3, 6, seed)
    base = inputs.qc_base_matrix(24, 96, Z, degs, seed)
    n = 96 * Z
    q = inputs.frame_qbers(B, 0.01, 0.08, seed)
    xa = inputs.unpack_bits(inputs.alice_keys(B, n, seed), n)
    yb = inputs.unpack_bits(inputs.alice_keys(B, n, seed) ^ inputs.bsc_noise(B, n, q, seed), n)
    return base, Z, n, 24 * Z, q, xa, yb, inputs.tiebreak_permutation(n, seed)


@pytest.mark.parametrize("stall", [0, 8])
def test_protocol_follows_its_definition_round_by_round(stall):
    base, Z, n, m, q, xa, yb, tb = _case(20)
    f0, df, R, T, scale = 1.1, 0.15, 4, 30, 1 / 0.29
    res = oproto.interactive(base, Z, tb, xa, yb, q, f0, df, R, T, scale, stall_window=stall)
    rank = orate.position_rank(base, Z, tb)
    syn = orc.syndrome(base, Z, xa)
    B = q.size
    rev = np.zeros(B, np.int64)
    iters = np.zeros(B, np.int64)
    bits = np.zeros_like(res["bits"])
    ok_ = np.zeros(B, np.uint8)
    last = np.zeros(B, np.int32)
    todo = list(range(B))
    for rnd in range(R + 1):
        failing = []
        for f in todo:  # the frames still failing, each decoded from its channel LLRs at its reveal state
            p0, s0 = orate.rate_plan(n, m, float(q[f]), f0)
            st = orate.position_states(rank, max(p0 - int(rev[f]), 0), s0 + int(rev[f]))
            llr = orc.llr_frames(yb[f:f + 1], q[f:f + 1], st[None], xa[f:f + 1], scale=scale)
            b, it, ok, _ = orc.decode(base, Z, llr, syn[f:f + 1], T, stall_window=stall)
            iters[f] += int(it[0])
            bits[f], ok_[f], last[f] = b[0], ok[0], rnd
            if not ok[0]:
                failing.append(f)
        todo = failing
        if not todo or rnd == R:
            break
        for f in todo:  # Alice reveals more of each failing frame's puncturing order
            p0, s0 = orate.rate_plan(n, m, float(q[f]), f0)
            key_now = n - p0 - s0 - max(int(rev[f]) - p0, 0)
            rev[f] += int(math.ceil(df * key_now * orate.binary_entropy(float(q[f]))))
    assert np.array_equal(res["bits"], bits) and np.array_equal(res["ok"], ok_)
    assert np.array_equal(res["rounds"], last)
    assert np.array_equal(res["revealed"], rev)
    assert np.array_equal(res["iters"], iters)
    for f in range(B):
        p0, s0 = orate.rate_plan(n, m, float(q[f]), f0)
        rp = min(int(rev[f]), p0)
        key = n - p0 - s0 - (int(rev[f]) - rp)
        assert res["key_bits"][f] == key
        assert res["f"][f] == pytest.approx((m - p0 + rp) / (key * orate.binary_entropy(float(q[f]))), rel=1e-12)
    # frames that needed more rounds ended above the starting efficiency; some did
    assert res["rounds"].max() >= 1 and (res["f"][res["rounds"] > 0] > f0).all()
    # a frame that is not ok after the last round ran every round
    assert (res["rounds"][res["ok"] == 0] == R).all()

"""Serving loop: continuous batching over several slots per code; every
block's result is byte-identical alone and in the mix; bi-directional
decoding and latency bookkeeping."""
import copy

import numpy as np
import pytest

from paper_1903_10107_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fresh(r):
    c = copy.copy(r)
    c.t_done, c.ok, c.key_bits, c.dirs, c.bits = -1.0, False, 0, (), ()
    return c


def test_results_identical_alone_and_in_the_mix():
    from paper_1903_10107_gb300.serving import ReconciliationServer, make_codes, make_requests
    codes = make_codes()
    reqs = make_requests(48, 1e9, 1.7, seed=3, codes=codes)
    srv = ReconciliationServer(codes, llr_scale=1 / 0.29, max_iter=40, slots_per_code=2, max_batch=5)
    mixed = srv.serve([_fresh(r) for r in reqs], realtime=False)
    assert all(r.t_done >= r.t_arrival for r in mixed)
    picks = [r for r in reqs if r.n == 4096][:2] + [r for r in reqs if r.n == 40960][:2] + \
            [r for r in reqs if r.n == 49152][:2]
    for r in picks:
        alone = srv.serve([_fresh(r)], realtime=False)[0]
        m = mixed[r.rid]
        assert alone.dirs == m.dirs and alone.ok == m.ok
        assert np.array_equal(alone.bits[0], m.bits[0]) and np.array_equal(alone.bits[1], m.bits[1])
    # a block counts as reconciled if either direction recovered the other party's key
    for r in mixed:
        assert r.ok == (r.dirs[0] or r.dirs[1])
        if r.dirs[0]:
            assert np.array_equal(r.bits[0], r.xa)
        if r.dirs[1]:
            assert np.array_equal(r.bits[1], r.yb)
    assert sum(r.ok for r in mixed) > 0


def test_realtime_poisson_stream_completes_with_latency_stats():
    from paper_1903_10107_gb300.serving import ReconciliationServer, make_codes, make_requests, summarize
    codes = make_codes()
    reqs = make_requests(300, 2000.0, 1.7, seed=5, codes=codes)
    srv = ReconciliationServer(codes, llr_scale=1 / 0.29, max_iter=60, slots_per_code=2)
    srv.serve(make_requests(12, 1e9, 1.7, seed=6, codes=codes), realtime=False)
    out = srv.serve(reqs, realtime=True)
    assert all(r.t_done > 0 for r in out)
    s = summarize(out, max(r.t_done for r in out))
    assert 0 < s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]
    assert s["corrected_key_mbps"] > 0

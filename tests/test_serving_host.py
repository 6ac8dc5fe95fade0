"""Host-side scheduling of the serving loop, without a GPU: engines are
replaced by fakes that finish a request a scripted number of epochs after it
was admitted.  Checked: requests wait while their code's pool is full and
are admitted in arrival order as slots free up; every request completes,
after it arrived; the pool size follows the memory budget."""
from collections import deque

import numpy as np
import pytest

from paper_1903_10107_gb300 import serving


class FakeEngine:
    def __init__(self, n, pairs, epochs_needed):
        self.n, self.queue, self.event = n, deque(), None
        self.free = pairs
        self.epochs_needed = epochs_needed  # rid -> epochs
        self.inflight = {}                  # rid -> (request, epochs left)
        self.admitted_order, self.max_inflight, self.epochs = [], 0, 0

    def admit(self):
        k = 0
        while self.queue and len(self.inflight) < self.free:
            r = self.queue.popleft()
            self.inflight[r.rid] = [r, self.epochs_needed[r.rid]]
            self.admitted_order.append(r.rid)
            k += 1
        self.max_inflight = max(self.max_inflight, len(self.inflight))
        return k

    def launch(self):
        if self.event is not None or not self.inflight:
            return False
        self.event = "running"
        self.epochs += 1
        return True

    def poll(self, now):
        if self.event is None:
            return []
        self.event = None
        done = []
        for rid in list(self.inflight):
            self.inflight[rid][1] -= 1
            if self.inflight[rid][1] <= 0:
                r = self.inflight.pop(rid)[0]
                r.t_done = now
                done.append(r)
        return done

    def idle(self):
        return self.event is None and not self.inflight and not self.queue


def _req(rid, n, t):
    z = np.zeros(8, np.uint8)
    return serving.Request(rid=rid, n=n, qber=0.02, xa=z, yb=z, n_punct=0, n_short=0, t_arrival=t)


def test_requests_wait_for_free_slots_and_all_complete():
    srv = object.__new__(serving.ReconciliationServer)
    need = {i: 1 + (i * 7) % 5 for i in range(30)}
    small, big = FakeEngine(64, 3, need), FakeEngine(128, 2, need)
    srv.engines = {"small": small, "big": big}
    srv.by_n = {64: small, 128: big}
    srv.device = "cpu"
    reqs = [_req(i, 64 if i % 3 else 128, 0.0) for i in range(30)]
    import torch
    sync = torch.cuda.synchronize
    torch.cuda.synchronize = lambda dev=None: None
    try:
        out = srv.serve(reqs, realtime=False)
    finally:
        torch.cuda.synchronize = sync
    assert all(r.t_done >= r.t_arrival for r in out)
    assert small.max_inflight == 3 and big.max_inflight == 2  # never more than the pool holds
    assert small.admitted_order == [r.rid for r in reqs if r.n == 64]  # arrival order
    assert big.admitted_order == [r.rid for r in reqs if r.n == 128]


def test_pool_bytes_cover_both_directions_and_staging():
    per = serving.pool_bytes_per_frame(6144, 1536)
    # observed key, known values, other party's key, syndrome, magnitude, counts: pool and staging row
    assert per >= 2 * (3 * 6144 + 1536) + 6144 + 5
    assert serving.EpochEngine.bytes_for(6144, 1536, 10) == 10 * per


def test_server_refuses_a_budget_that_holds_no_request(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda dev=None: (10 ** 12, 2 * 10 ** 12))
    base = np.zeros((1, 4), np.int32)
    with pytest.raises(RuntimeError, match="holds no request"):
        serving.ReconciliationServer({"tiny": (base, 64, np.arange(256))}, llr_scale=3.0, max_iter=10,
                                     mem_budget=100)

"""Host-side scheduling of the serving loop, without a GPU: a request that
can never be admitted (its buffers exceed the memory budget while nothing is
in flight) stops the loop with an error instead of waiting forever."""
from types import SimpleNamespace

import numpy as np
import pytest

from paper_1903_10107_gb300 import serving


def _server(budget):
    srv = object.__new__(serving.ReconciliationServer)  # no code handles, no device
    entry = SimpleNamespace(name="tiny", n=64, nbytes=8, mbytes=4, queue=[],
                            slots=[SimpleNamespace(event=None)])
    srv.codes = {"tiny": entry}
    srv.by_n = {64: entry}
    srv.mem_budget, srv.reserve, srv.held, srv.max_batch = budget, 0, 0, 8
    return srv


def test_unadmissible_request_raises_instead_of_spinning():
    srv = _server(budget=1)  # one byte: no request fits
    req = serving.Request(rid=0, n=64, qber=0.02, xa=np.zeros(8, np.uint8), yb=np.zeros(8, np.uint8),
                          n_punct=0, n_short=0, t_arrival=0.0)
    with pytest.raises(RuntimeError, match="needs .* device bytes"):
        srv.serve([req], realtime=False)


def test_need_counts_both_directions_of_every_request():
    srv = _server(budget=0)
    e = srv.codes["tiny"]
    one = srv._need(e, 1)
    assert one > 0 and srv._need(e, 5) == 5 * one

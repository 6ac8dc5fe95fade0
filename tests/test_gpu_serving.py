"""Serving loop: continuous batching in epochs with resident decoder state.

* Every served request's two frames -- Bob's direction against Alice's
  syndrome, Alice's against Bob's -- equal the CPU oracle's decodes of the
  same LLRs: bits, iteration counts and flags.
* Each result is byte-identical alone and in the mix.
* A decode split into epochs of any length equals one persistent launch and
  the oracle (the lanes' soft values, syndrome bits, iteration and stall
  state survive the epoch boundaries, the messages stay in the arena).
* A real-time Poisson stream completes with latency statistics."""
import copy

import numpy as np
import pytest

from conftest import device_mags
from oracle import core as orc
from oracle import rate as orate
from paper_1903_10107_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCALE = 1 / 0.29


def _fresh(r):
    c = copy.copy(r)
    c.t_done, c.ok, c.key_bits, c.dirs, c.bits = -1.0, False, 0, (), ()
    return c


def _server(codes, **kw):
    from paper_1903_10107_gb300.serving import ReconciliationServer
    kw.setdefault("capacity", 64)
    return ReconciliationServer(codes, llr_scale=SCALE, max_iter=200, **kw)


def _oracle_directions(codes, r, stall=0):
    """The oracle's decodes of a request's two frames: Bob's LLRs against
    s_A = H x_A, Alice's against s_B = H y_B; shortened positions known to
    both (Alice's values), punctured ones the other party's filler."""
    name = {4096: "n4096", 40960: "n40960", 49152: "n49152"}[r.n]
    base, Z, tb = codes[name]
    n = r.n
    st = orate.position_states(orate.position_rank(base, Z, tb), r.n_punct, r.n_short)[None]
    xa_u, yb_u = inputs.unpack_bits(r.xa[None], n), inputs.unpack_bits(r.yb[None], n)
    out = []
    for obs, other in ((yb_u, xa_u), (xa_u, yb_u)):
        llr = orc.llr_frames(obs, [r.qber], st, xa_u, scale=SCALE)
        b, it, ok, _ = orc.decode(base, Z, llr, orc.syndrome(base, Z, other), 200, stall_window=stall)
        out.append((inputs.pack_bits(b)[0], int(it[0]), bool(ok[0])))
    return out


def test_served_requests_match_the_oracle_in_both_directions():
    from paper_1903_10107_gb300.serving import make_codes, make_requests
    codes = make_codes()
    reqs = make_requests(40, 1e9, 1.7, seed=3, codes=codes)
    srv = _server(codes, epoch_iters=3)
    served = srv.serve([_fresh(r) for r in reqs], realtime=False)
    # some decodes spanned several epochs of their code's engine
    assert any(max(r.dirs[2], r.dirs[3]) > srv.by_n[r.n].epoch_iters for r in served)
    picks = [r for r in served if r.n == 4096][:4] + [r for r in served if r.n == 40960][:2] + \
            [r for r in served if r.n == 49152][:4]
    picks += [r for r in served if not r.ok][:2]
    for r in picks:
        (ob, oi, oo), (ab, ai, ao) = _oracle_directions(codes, r)
        assert np.array_equal(r.bits[0], ob) and np.array_equal(r.bits[1], ab)
        assert r.dirs[2] == oi and r.dirs[3] == ai
        assert r.dirs[0] == (oo and np.array_equal(ob, r.xa)) and r.dirs[1] == (ao and np.array_equal(ab, r.yb))
    assert sum(r.ok for r in served) > 0


def test_results_identical_alone_and_in_the_mix():
    from paper_1903_10107_gb300.serving import make_codes, make_requests
    codes = make_codes()
    reqs = make_requests(48, 1e9, 1.7, seed=3, codes=codes)
    srv = _server(codes, epoch_iters=8)
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


@pytest.mark.parametrize("epoch_iters,words,stall", [(1, 1, 0), (3, 2, 0), (7, 4, 4), (50, 1, 6)])
def test_decode_split_into_epochs_equals_one_launch(epoch_iters, words, stall):
    """Frames decoded over many epochs (new frames joining as lanes free up)
    give exactly the results of one persistent launch and of the oracle."""
    from paper_1903_10107_gb300.decoder import QCCode
    B, Z, T = 45, 32, 60
    degs = inputs.mixed_column_degrees(96, 0.3, 3, 6, 61)
    base = inputs.qc_base_matrix(24, 96, Z, degs, 61)
    n, m = 96 * Z, 24 * Z
    q = inputs.frame_qbers(B, 0.01, 0.08, 61)
    xa = inputs.alice_keys(B, n, 61)
    yb = xa ^ inputs.bsc_noise(B, n, q, 61)
    tb = inputs.tiebreak_permutation(n, 61)
    rank = orate.position_rank(base, Z, tb)
    plans = [orate.rate_plan(n, m, float(x), 1.4) for x in q]
    npn = np.array([p for p, _ in plans], np.int32)
    ns = np.array([s for _, s in plans], np.int32)
    code = QCCode(base, Z)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (c(yb), device_mags(q, SCALE), c(inputs.pack_bits(orc.syndrome(base, Z, inputs.unpack_bits(xa, n)))))
    kw = dict(rank=c(rank), n_short=c(ns), n_punct=c(npn), known=c(xa), stall_window=stall)
    ref = [t.cpu().numpy() for t in code.reconcile_persistent(*args, T, words=words, **kw)]
    # epochs: the frames offered in three waves, each epoch offering what the last one did not take
    nbytes, grid = code.epoch_state_bytes(words, 1, 0)
    state = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    out = (torch.zeros((B, code.nbytes), dtype=torch.uint8, device="cuda"),
           torch.zeros((B,), dtype=torch.int32, device="cuda"), torch.zeros((B,), dtype=torch.uint8, device="cuda"))
    claimed = torch.zeros(1, dtype=torch.int32, device="cuda")
    waves = [list(range(0, 15)), list(range(15, 30)), list(range(30, B))]
    todo, started, epochs = [], False, 0
    while True:
        if waves and epochs % 3 == 0:
            todo += waves.pop(0)
        lst = c(np.array(todo + [0], np.int32))
        code.reconcile_epoch(*args, T, state, lst, len(todo), epoch_iters, started, out, claimed, words=words,
                             ctas_per_sm=1, **kw)
        started = True
        epochs += 1
        todo = todo[min(int(claimed.item()), len(todo)):]
        it = out[1].cpu().numpy()
        if not waves and not todo and (it > 0).all():
            break
        assert epochs < 10000
    got = [t.cpu().numpy() for t in out]
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    assert epochs > 3
    st = np.stack([orate.position_states(rank, int(npn[f]), int(ns[f])) for f in range(B)])
    xa_u = inputs.unpack_bits(xa, n)
    llr = orc.llr_frames(inputs.unpack_bits(yb, n), q, st, xa_u, scale=SCALE)
    ob, oi, oo, _ = orc.decode(base, Z, llr, orc.syndrome(base, Z, xa_u), T, stall_window=stall)
    assert np.array_equal(inputs.unpack_bits(got[0], n), ob)
    assert np.array_equal(got[1], oi) and np.array_equal(got[2], oo)


def test_epoch_state_buffer_checks():
    from paper_1903_10107_gb300 import native
    from paper_1903_10107_gb300.decoder import QCCode
    base = inputs.qc_base_matrix(6, 24, 16, 3, 5)
    code = QCCode(base, 16)
    nbytes, grid = code.epoch_state_bytes(1, 1, 0)
    assert grid == torch.cuda.get_device_properties(0).multi_processor_count and nbytes > grid * 4 * code.n
    B = 4
    z = lambda *sh, dt=torch.uint8: torch.zeros(sh, dtype=dt, device="cuda")
    out = (z(B, code.nbytes), z(B, dt=torch.int32), z(B))
    with pytest.raises(native.LdpcError, match="lane-state buffer needs"):
        code.reconcile_epoch(z(B, code.nbytes), z(B, dt=torch.int8), z(B, code.mbytes), 10, z(nbytes - 256),
                             z(B, dt=torch.int32), 0, 4, False, out, z(1, dt=torch.int32))


def test_realtime_poisson_stream_completes_with_latency_stats():
    from paper_1903_10107_gb300.serving import make_codes, make_requests, summarize
    codes = make_codes()
    reqs = make_requests(300, 2000.0, 1.7, seed=5, codes=codes)
    srv = _server(codes, capacity=256)
    srv.serve(make_requests(12, 1e9, 1.7, seed=6, codes=codes), realtime=False)
    out = srv.serve(reqs, realtime=True)
    assert all(r.t_done > 0 for r in out)
    s = summarize(out, max(r.t_done for r in out))
    assert 0 < s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]
    assert s["corrected_key_mbps"] > 0

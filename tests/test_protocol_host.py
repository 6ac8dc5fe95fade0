"""Host logic of the interactive rate adaptation (sections 4.1 and 4.2),
without a GPU: a fake decoder that succeeds for each frame at a scripted
round records what the protocol asks of it.  Checked: every round decodes
exactly the frames still failing (hardest first), each reveal adds
ceil(df * key bits * h(q)) bits, punctured positions are revealed before key
positions (becoming shortened), iterations add up over rounds, the final
efficiency counts every revealed bit, and how much a reveal raises it in each
regime."""
import types

import numpy as np
import torch

from paper_1903_10107_gb300 import rate
from paper_1903_10107_gb300.pipeline import InteractiveProtocol, hardest_first


class FakeCode:
    """Decodes a frame successfully from round succeed_at[f] on; iterations
    reported per call: 10 + round."""

    def __init__(self, n, m, succeed_at):
        self.n, self.m, self.nbytes = n, m, (n + 7) // 8
        self.device = torch.device("cpu")
        self.succeed_at = np.asarray(succeed_at)
        self.calls = []

    def reconcile_persistent(self, bob, llr_mag, syn, max_iter, rank=None, n_short=None, n_punct=None, known=None,
                             frame_list=None, stall_window=0, words=0, ctas_per_sm=0, threads=0, out=None):
        rnd = len(self.calls)
        frames = frame_list.numpy().copy()
        self.calls.append(dict(frames=frames, n_punct=n_punct.numpy().copy(), n_short=n_short.numpy().copy()))
        bits, iters, ok = out
        for f in frames:
            ok[f] = 1 if rnd >= self.succeed_at[f] else 0
            iters[f] = 10 + rnd
        return out


def test_rounds_reveals_and_efficiency():
    n, m = 4096, 1024
    q = np.array([0.01, 0.02, 0.03, 0.05, 0.07, 0.08])
    succeed_at = np.array([0, 1, 3, 2, 9, 5])  # frame 4 never succeeds within the rounds
    code = FakeCode(n, m, succeed_at)
    rec = types.SimpleNamespace(code=code, rank=torch.zeros(n, dtype=torch.int32), llr_scale=3.0,
                                magnitudes=lambda qq: np.zeros(len(qq), np.int8))
    df, max_rounds, f0 = 0.1, 6, 1.1
    proto = InteractiveProtocol(rec, max_iter=50, f_start=f0, df=df, max_rounds=max_rounds, fused=False)
    B = q.size
    res = proto.run(torch.zeros((B, code.nbytes), dtype=torch.uint8), torch.zeros((B, m // 8), dtype=torch.uint8),
                    q, torch.zeros((B, code.nbytes), dtype=torch.uint8))

    p0, s0 = rate.plan(n, m, q, f0)
    key0 = rate.key_bits(n, p0, s0)
    last = np.minimum(succeed_at, max_rounds)
    assert len(code.calls) == max_rounds + 1
    revealed = np.zeros(B, np.int64)
    for rnd, call in enumerate(code.calls):
        todo = np.nonzero(last >= rnd)[0]
        # exactly the frames still failing, most punctured / highest QBER first
        assert np.array_equal(np.sort(call["frames"]), todo)
        np_now = np.maximum(p0 - revealed, 0)
        assert np.array_equal(call["frames"], todo[hardest_first(np_now[todo], (s0 + revealed)[todo], q[todo])])
        # punctured positions are revealed first; what is revealed is shortened
        assert np.array_equal(call["n_short"][todo], (s0 + revealed)[todo])
        assert np.array_equal(call["n_punct"][todo], np_now[todo])
        # the frames failing this round get ceil(df * key bits * h(q)) more
        fail = todo[succeed_at[todo] > rnd]
        kb = key0[fail] - np.maximum(revealed[fail] - p0[fail], 0)
        if rnd < max_rounds:
            revealed[fail] += np.ceil(df * kb * rate.h2(q[fail])).astype(np.int64)
    assert np.array_equal(res["revealed"], revealed)
    assert np.array_equal(res["rounds"], last)
    assert np.array_equal(res["ok"].astype(bool), succeed_at <= max_rounds)
    assert np.array_equal(res["iters"], [sum(10 + r for r in range(int(k) + 1)) for k in last])
    rp = np.minimum(revealed, p0)
    key = key0 - (revealed - rp)
    assert np.array_equal(res["key_bits"], key)
    np.testing.assert_allclose(res["f"], (m - p0 + rp) / (key * rate.h2(q)), rtol=1e-12)
    # a reveal of punctured positions raises the efficiency by at least df; one
    # of key positions (they leave the key) by f df h(q) / (1 - df h(q)) or more
    f_start = (m - p0) / (key0 * rate.h2(q))
    punct_only = revealed <= p0
    assert punct_only[:2].all() and not punct_only[2:].any()  # both regimes occur
    assert np.all(res["f"][punct_only] >= (f_start + df * last - 1e-9)[punct_only])
    grow = f_start * (1.0 / (1.0 - df * rate.h2(q))) ** last
    assert np.all(res["f"][~punct_only] >= grow[~punct_only] - 1e-9)


class FakeFusedCode(FakeCode):
    """The one-launch form: records the reveal table and reports, per frame,
    success in round succeed_at[f] (if within the rounds), iterations summed
    as 10 + r per round r decoded."""

    def reconcile_interactive(self, bob, llr_mag, syn, max_iter, rank, n_short, n_punct, known, reveal,
                              frame_list=None, stall_window=0, words=0, ctas_per_sm=0, threads=0, out=None):
        R = reveal.shape[1] - 1
        self.calls.append(dict(frames=frame_list.numpy().copy(), n_short=n_short.numpy().copy(),
                               n_punct=n_punct.numpy().copy(), reveal=reveal.numpy().copy()))
        B = n_short.shape[0]
        last = np.minimum(self.succeed_at, R)
        ok = torch.from_numpy((self.succeed_at <= R).astype(np.uint8))
        iters = torch.from_numpy(np.array([sum(10 + r for r in range(int(k) + 1)) for k in last], dtype=np.int32))
        bits = torch.zeros((B, self.nbytes), dtype=torch.uint8)
        return bits, iters, ok, torch.from_numpy(last.astype(np.int32))


def test_fused_rounds_take_the_same_reveals_as_separate_rounds():
    """One launch for all rounds: the reveal table handed to it holds exactly
    the reveals the round-by-round protocol applies, and the results (rounds,
    revealed bits, key bits, efficiency, summed iterations) are the same."""
    n, m = 4096, 1024
    q = np.array([0.01, 0.02, 0.03, 0.05, 0.07, 0.08])
    succeed_at = np.array([0, 1, 3, 2, 9, 5])
    kw = dict(max_iter=50, f_start=1.1, df=0.1, max_rounds=6)
    mk = lambda code: types.SimpleNamespace(code=code, rank=torch.zeros(n, dtype=torch.int32), llr_scale=3.0,
                                            magnitudes=lambda qq: np.zeros(len(qq), np.int8))
    B = q.size
    args = (torch.zeros((B, n // 8), dtype=torch.uint8), torch.zeros((B, m // 8), dtype=torch.uint8), q,
            torch.zeros((B, n // 8), dtype=torch.uint8))
    sep = InteractiveProtocol(mk(FakeCode(n, m, succeed_at)), fused=False, **kw).run(*args)
    fused_code = FakeFusedCode(n, m, succeed_at)
    fus = InteractiveProtocol(mk(fused_code), **kw).run(*args)
    (call,) = fused_code.calls  # a single launch
    p0, s0 = rate.plan(n, m, q, 1.1)
    assert np.array_equal(call["n_punct"], p0) and np.array_equal(call["n_short"], s0)
    assert np.array_equal(call["frames"], hardest_first(p0, s0, q))
    rev = call["reveal"]
    assert rev.shape == (B, 7) and (rev[:, 0] == 0).all() and (np.diff(rev, axis=1) > 0).all()
    for k in ("rounds", "revealed", "key_bits", "iters", "ok"):
        assert np.array_equal(np.asarray(sep[k]), np.asarray(fus[k])), k
    np.testing.assert_allclose(sep["f"], fus["f"], rtol=1e-12)
    # every frame's revealed count is the table's entry at its last round
    assert np.array_equal(fus["revealed"], rev[np.arange(B), fus["rounds"]])


def test_bits_destinations():
    """The corrected keys go where ``bits_out`` asks: a new host array by
    default, left as the decoder's tensor for ``"device"`` (not counted as
    copied back), or copied into a caller's host buffer; other values are
    refused."""
    n, m = 4096, 1024
    q = np.array([0.02, 0.05, 0.07])
    B = q.size

    class PatternCode(FakeFusedCode):
        def reconcile_interactive(self, *a, **k):
            bits, iters, ok, last = super().reconcile_interactive(*a, **k)
            bits[:] = torch.arange(B, dtype=torch.uint8)[:, None] + 1
            self.bits = bits
            return bits, iters, ok, last

    mk = lambda code: types.SimpleNamespace(code=code, rank=torch.zeros(n, dtype=torch.int32), llr_scale=3.0,
                                            magnitudes=lambda qq: np.zeros(len(qq), np.int8))
    args = (torch.zeros((B, n // 8), dtype=torch.uint8), torch.zeros((B, m // 8), dtype=torch.uint8), q,
            torch.zeros((B, n // 8), dtype=torch.uint8))
    kw = dict(max_iter=50, f_start=1.1, df=0.1, max_rounds=3)
    want = np.repeat(np.arange(1, B + 1, dtype=np.uint8)[:, None], n // 8, axis=1)
    code = PatternCode(n, m, np.array([0, 1, 2]))
    proto = InteractiveProtocol(mk(code), **kw)
    plain = proto.run(*args)
    assert isinstance(plain["bits"], np.ndarray) and np.array_equal(plain["bits"], want)
    dev = proto.run(*args, bits_out="device")
    assert dev["bits"] is code.bits
    assert dev["d2h_bytes"] == plain["d2h_bytes"] - B * (n // 8)
    buf = torch.zeros((B, n // 8), dtype=torch.uint8)
    into = proto.run(*args, bits_out=buf)
    assert np.array_equal(buf.numpy(), want) and np.shares_memory(into["bits"], buf.numpy())
    assert into["d2h_bytes"] == plain["d2h_bytes"]
    for bad in ("host", torch.zeros((B, 1), dtype=torch.uint8), torch.zeros((B, n // 8), dtype=torch.int32)):
        try:
            proto.run(*args, bits_out=bad)
        except ValueError:
            pass
        else:
            raise AssertionError(f"bits_out={bad!r} accepted")

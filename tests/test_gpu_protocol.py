"""The mixed-rate batch (autotuned persistent launch replayed from a CUDA
graph) and the interactive rate-adaptation protocol, checked against the
oracle frame by frame."""
import numpy as np
import pytest

from oracle import core as orc
from oracle import rate as orate
from paper_1903_10107_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCALE = 1 / 0.29


def _code_and_frames(B, Z=32, seed=5):
    degs = inputs.mixed_column_degrees(96, 0.3, 3, 6, seed)
    base = inputs.qc_base_matrix(24, 96, Z, degs, seed)
    n = 96 * Z
    q = inputs.frame_qbers(B, 0.01, 0.08, seed)
    xa = inputs.alice_keys(B, n, seed)
    yb = xa ^ inputs.bsc_noise(B, n, q, seed)
    tb = inputs.tiebreak_permutation(n, seed)
    return base, Z, n, 24 * Z, q, xa, yb, tb


def test_mixed_rate_batch_graph_matches_oracle():
    from paper_1903_10107_gb300.pipeline import MixedRateBatch, Reconciler
    base, Z, n, m, q, xa, yb, tb = _code_and_frames(45)
    rec = Reconciler(base, Z, tb, llr_scale=SCALE)
    p, s = rec.plan(q, 1.5)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    syn = rec.code.syndrome(c(xa))
    mrb = MixedRateBatch(rec, 50).bind(c(yb), syn, c(rec.magnitudes(q)), c(p), c(s), c(xa))
    assert mrb.graph is not None
    for t in mrb.out:
        t.zero_()
    bits, iters, ok = (t.cpu().numpy() for t in mrb.run())
    rank = orate.position_rank(base, Z, tb)
    st = np.stack([orate.position_states(rank, int(p[f]), int(s[f])) for f in range(45)])
    xa_u = inputs.unpack_bits(xa, n)
    llr = orc.llr_frames(inputs.unpack_bits(yb, n), q, st, xa_u, scale=SCALE)
    ob, oi, oo, _ = orc.decode(base, Z, llr, orc.syndrome(base, Z, xa_u), 50)
    assert np.array_equal(ok, oo) and np.array_equal(iters, oi)
    assert np.array_equal(inputs.unpack_bits(bits, n), ob)


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("stall", [0, 6])
def test_interactive_protocol_matches_the_oracle_protocol(stall, fused):
    """Every round's launch over the frames still failing, the reveals between
    rounds and the final efficiency, against the oracle's protocol run on the
    same frames: bits, summed iterations, flags, rounds, revealed bits, key
    bits and f, frame by frame."""
    from oracle import protocol as oproto
    from paper_1903_10107_gb300.pipeline import InteractiveProtocol, Reconciler
    B = 48
    base, Z, n, m, q, xa, yb, tb = _code_and_frames(B, seed=9)
    rec = Reconciler(base, Z, tb, llr_scale=SCALE)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    syn = rec.code.syndrome(c(xa))
    proto = InteractiveProtocol(rec, 40, f_start=1.1, df=0.15, max_rounds=5, stall_window=stall, fused=fused)
    res = proto.run(c(yb), syn, q, c(xa), timing=True)
    assert res["rounds"].max() >= 1 and res["revealed"].max() > 0
    assert res["launches"] == (1 if fused else res["rounds"].max() + 1) and res["kernel_s"] > 0
    xa_u = inputs.unpack_bits(xa, n)
    ref = oproto.interactive(base, Z, tb, xa_u, inputs.unpack_bits(yb, n), q, 1.1, 0.15, 5, 40, SCALE,
                             stall_window=stall)
    assert np.array_equal(inputs.unpack_bits(res["bits"], n), ref["bits"])
    for k in ("ok", "iters", "rounds", "revealed", "key_bits"):
        assert np.array_equal(np.asarray(res[k]), np.asarray(ref[k])), k
    np.testing.assert_allclose(res["f"], ref["f"], rtol=1e-12)
    # the host-buffer entry gives the same results and counts its copies
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hres, h2d, d2h = proto.run_host(pin(yb), syn.cpu().pin_memory(), q, pin(xa))
    assert np.array_equal(hres["bits"], res["bits"]) and np.array_equal(hres["iters"], res["iters"])
    assert h2d >= yb.nbytes + syn.numel() + xa.nbytes and d2h >= res["bits"].nbytes + 5 * B
    # the same bits left on the device, and copied into a caller's pinned buffer
    dres = proto.run(c(yb), syn, q, c(xa), bits_out="device")
    assert dres["bits"].is_cuda and np.array_equal(dres["bits"].cpu().numpy(), res["bits"])
    buf = torch.empty(res["bits"].shape, dtype=torch.uint8, pin_memory=True)
    bres, _, _ = proto.run_host(pin(yb), syn.cpu().pin_memory(), q, pin(xa), bits_out=buf)
    assert np.array_equal(buf.numpy(), res["bits"]) and np.array_equal(bres["ok"], res["ok"])


def test_host_buffer_path_matches_oracle_and_counts_bytes():
    """reconcile_host (pinned host buffers in and out, persistent launch in
    hardest-first order) gives the oracle's results frame for frame."""
    from paper_1903_10107_gb300.pipeline import Reconciler
    B = 40
    base, Z, n, m, q, xa, yb, tb = _code_and_frames(B, seed=13)
    rec = Reconciler(base, Z, tb, llr_scale=SCALE)
    p, s = rec.plan(q, 1.5)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    syn = rec.code.syndrome(torch.from_numpy(xa).cuda()).cpu()
    (bits, iters, ok), h2d, d2h = rec.reconcile_host(pin(yb), syn.pin_memory(), pin(q), 50, pin(p), pin(s),
                                                     pin(xa), persistent=True)
    torch.cuda.synchronize()
    assert h2d == yb.nbytes + syn.numel() + B + p.nbytes + s.nbytes + xa.nbytes + 4 * B  # one magnitude byte per frame
    assert d2h == bits.numel() + 4 * B + B
    rank = orate.position_rank(base, Z, tb)
    st = np.stack([orate.position_states(rank, int(p[f]), int(s[f])) for f in range(B)])
    xa_u = inputs.unpack_bits(xa, n)
    llr = orc.llr_frames(inputs.unpack_bits(yb, n), q, st, xa_u, scale=SCALE)
    ob, oi, oo, _ = orc.decode(base, Z, llr, orc.syndrome(base, Z, xa_u), 50)
    assert np.array_equal(ok.numpy(), oo) and np.array_equal(iters.numpy(), oi)
    assert np.array_equal(inputs.unpack_bits(bits.numpy(), n), ob)


def test_host_stream_overlapped_batches_match_oracle():
    """Three batches through reconcile_host_stream (two device slots reused,
    copies on their own streams) each give the oracle's results."""
    from paper_1903_10107_gb300.pipeline import Reconciler
    B = 24
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    cases, batches = [], []
    rec = None
    for seed in (21, 22, 23):
        base, Z, n, m, q, xa, yb, tb = _code_and_frames(B, seed=5)  # one code for all batches
        q = inputs.frame_qbers(B, 0.01, 0.08, seed)
        xa = inputs.alice_keys(B, n, seed)
        yb = xa ^ inputs.bsc_noise(B, n, q, seed)
        if rec is None:
            rec = Reconciler(base, Z, tb, llr_scale=SCALE)
        p, s = rec.plan(q, 1.5)
        syn = rec.code.syndrome(torch.from_numpy(xa).cuda()).cpu()
        batches.append((pin(yb), syn.pin_memory(), pin(q), pin(p), pin(s), pin(xa)))
        cases.append((q, xa, yb, p, s))
    out = rec.reconcile_host_stream(batches, 50, persistent=True)
    rank = orate.position_rank(base, Z, tb)
    for (bits, iters, ok), h2d, d2h in out:
        assert h2d > 0 and d2h == bits.numel() + 5 * B
    for ((bits, iters, ok), _, _), (q, xa, yb, p, s) in zip(out, cases):
        st = np.stack([orate.position_states(rank, int(p[f]), int(s[f])) for f in range(B)])
        xa_u = inputs.unpack_bits(xa, n)
        llr = orc.llr_frames(inputs.unpack_bits(yb, n), q, st, xa_u, scale=SCALE)
        ob, oi, oo, _ = orc.decode(base, Z, llr, orc.syndrome(base, Z, xa_u), 50)
        assert np.array_equal(ok.numpy(), oo) and np.array_equal(iters.numpy(), oi)
        assert np.array_equal(inputs.unpack_bits(bits.numpy(), n), ob)


def test_host_buffer_entry_point_matches_device_entry():
    """ldpc_reconcile_interactive_host (host buffers in and out, the library's
    own copies) against ldpc_reconcile_interactive on device copies of the
    same inputs: equal bits, iterations, flags and rounds; pageable numpy
    inputs work; the byte counts are exactly the arrays copied; frames the
    list leaves out keep the caller's output values."""
    from paper_1903_10107_gb300.pipeline import InteractiveProtocol, Reconciler, hardest_first
    B = 40
    base, Z, n, m, q, xa, yb, tb = _code_and_frames(B, seed=13)
    rec = Reconciler(base, Z, tb, llr_scale=SCALE)
    code = rec.code
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    syn = code.syndrome(c(xa))
    proto = InteractiveProtocol(rec, 40, f_start=1.1, df=0.15, max_rounds=4, stall_window=6)
    p0, s0, rev = proto.reveal_table(q)
    mag = rec.magnitudes(q)
    order = hardest_first(p0, s0, q).astype(np.int32)
    rev32 = np.ascontiguousarray(rev, dtype=np.int32)
    dev = code.reconcile_interactive(c(yb), c(mag), syn, 40, rec.rank, c(s0.astype(np.int32)),
                                     c(p0.astype(np.int32)), c(xa), c(rev32), frame_list=c(order), stall_window=6)
    dev = [t.cpu().numpy() for t in dev]
    syn_h = syn.cpu().numpy()
    host = code.reconcile_interactive_host(yb, mag, syn_h, 40, rec.rank_host, s0.astype(np.int32),
                                           p0.astype(np.int32), xa, rev32, frame_list=order, stall_window=6)
    for a, b in zip(dev, host[:4]):
        assert np.array_equal(a, b.numpy())
    nb, mb = code.nbytes, code.mbytes
    assert host[4] == 2 * B * nb + B * mb + B + 8 * B + 4 * rev32.size + 4 * n + 4 * B
    assert host[5] == B * nb + 9 * B
    # a list of the first half only: the other frames' outputs are the caller's
    half = order[: B // 2]
    out = (torch.full((B, nb), 0xA5, dtype=torch.uint8).pin_memory(), torch.full((B,), -7, dtype=torch.int32),
           torch.full((B,), 3, dtype=torch.uint8), torch.full((B,), -9, dtype=torch.int32))
    part = code.reconcile_interactive_host(yb, mag, syn_h, 40, rec.rank_host, s0.astype(np.int32),
                                           p0.astype(np.int32), xa, rev32, frame_list=half, stall_window=6, out=out)
    rest = np.setdiff1d(np.arange(B), half)
    assert (part[0].numpy()[rest] == 0xA5).all() and (part[1].numpy()[rest] == -7).all()
    assert (part[2].numpy()[rest] == 3).all() and (part[3].numpy()[rest] == -9).all()
    for a, b in zip(dev, part[:4]):
        assert np.array_equal(a[half], b.numpy()[half])

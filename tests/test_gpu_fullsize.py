"""Parity at the full workload sizes, in the launch configuration the
benchmark times.

* n = 49152 mixed-rate mother code, 16384 frames, QBER U(1 %, 8 %), rates
  planned per frame, max 200 iterations: the autotuned persistent launch,
  hardest frames first, replayed from a CUDA graph.
* n = 40960 rate-0.8 code, 8192 frames, QBER 3 %, max 100 iterations: the
  batch decode kernel.

The oracle decodes a sample of frames one by one (seeded picks, every failing
frame up to a cap, and the longest decodes) and must agree bit for bit; every
frame of the launch is checked against the properties that hold at any size:
ok => H x = s, not ok => iterations = max_iter, 1 <= iterations <= max_iter.
"""
import numpy as np
import pytest

from conftest import device_mags
from oracle import core as orc
from oracle import rate as orate
from paper_1903_10107_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sample(iters, ok, B, seed, n_rand=16, n_fail=6, n_long=4):
    rng = np.random.default_rng(seed)
    pick = set(int(x) for x in rng.choice(B, size=n_rand, replace=False))
    pick |= set(int(x) for x in np.flatnonzero(ok == 0)[:n_fail])
    pick |= set(int(x) for x in np.argsort(-iters, kind="stable")[:n_long])
    return np.array(sorted(pick))


def _syndromes(base, Z, n, packed, chunk=2048):
    return np.concatenate([orc.syndrome(base, Z, inputs.unpack_bits(packed[f0:f0 + chunk], n))
                           for f0 in range(0, len(packed), chunk)])


def _check_properties(base, Z, n, bits, iters, ok, syn_u, max_iter, chunk=2048):
    assert iters.min() >= 1 and iters.max() <= max_iter
    assert np.all(iters[ok == 0] == max_iter)
    for f0 in range(0, len(ok), chunk):
        sl = slice(f0, f0 + chunk)
        hx = orc.syndrome(base, Z, inputs.unpack_bits(bits[sl], n))
        match = np.all(hx == syn_u[sl], axis=1)
        assert np.all(match[ok[sl] == 1]), "a frame reported ok whose syndrome differs"
        assert not np.any(match[ok[sl] == 0]), "a frame reported failing whose syndrome matches"


def test_mixed_rate_full_size_sampled_frames_match_oracle():
    from paper_1903_10107_gb300 import rate
    from paper_1903_10107_gb300.pipeline import MixedRateBatch, Reconciler, hardest_first

    w = inputs.WORKLOADS["n49152_mixed_q01_08"]
    B = w.batch
    base = w.base()
    xa, yb, q = w.frames(B, 0)
    # the library's rate plan equals the oracle's, frame by frame
    npn, ns = rate.plan(w.n, w.m, q, w.target_f)
    plans = np.array([orate.rate_plan(w.n, w.m, float(x), w.target_f) for x in q], dtype=np.int64)
    assert np.array_equal(npn, plans[:, 0]) and np.array_equal(ns, plans[:, 1])
    tb = inputs.tiebreak_permutation(w.n, w.code_seed)

    rec = Reconciler(base, w.Z, tb, llr_scale=w.llr_scale)
    syn = rec.code.syndrome(_dev(xa))
    mrb = MixedRateBatch(rec, w.max_iter).bind(_dev(yb), syn, _dev(rec.magnitudes(q)), _dev(npn), _dev(ns), _dev(xa),
                                               order=hardest_first(npn, ns, q))
    assert mrb.graph is not None
    for t in mrb.out:
        t.fill_(0x5A)
    bits, iters, ok = (t.cpu().numpy() for t in mrb.run())
    torch.cuda.synchronize()

    syn_u = _syndromes(base, w.Z, w.n, xa)
    _check_properties(base, w.Z, w.n, bits, iters, ok, syn_u, w.max_iter)

    sel = _sample(iters, ok, B, seed=11)
    rank = orate.position_rank(base, w.Z, tb)
    xa_u = inputs.unpack_bits(xa[sel], w.n)
    st = np.stack([orate.position_states(rank, int(plans[f, 0]), int(plans[f, 1])) for f in sel])
    llr = orc.llr_frames(inputs.unpack_bits(yb[sel], w.n), q[sel], st, xa_u, scale=w.llr_scale)
    ob, oi, oo, _ = orc.decode(base, w.Z, llr, syn_u[sel], w.max_iter)
    assert np.array_equal(oi, iters[sel]) and np.array_equal(oo, ok[sel])
    assert np.array_equal(ob, inputs.unpack_bits(bits[sel], w.n))


def test_n40960_full_batch_sampled_frames_match_oracle():
    from paper_1903_10107_gb300.decoder import QCCode

    w = inputs.WORKLOADS["n40960_r080_q03"]
    B = w.batch
    base = w.base()
    xa, yb, q = w.frames(B, 0)
    code = QCCode(base, w.Z)
    d_syn = code.syndrome(_dev(xa))
    llr = code.llr_from_bsc(_dev(yb), device_mags(q, w.llr_scale))
    bits, iters, ok = code.decode(llr, d_syn, w.max_iter)
    bits, iters, ok = bits.cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy()

    syn_u = _syndromes(base, w.Z, w.n, xa)
    assert np.array_equal(inputs.unpack_bits(d_syn.cpu().numpy(), w.m), syn_u)
    _check_properties(base, w.Z, w.n, bits, iters, ok, syn_u, w.max_iter)

    sel = _sample(iters, ok, B, seed=12, n_rand=8, n_fail=2, n_long=2)
    o_llr = orc.llr_frames(inputs.unpack_bits(yb[sel], w.n), q[sel], scale=w.llr_scale)
    assert np.array_equal(o_llr, llr.cpu().numpy()[sel])
    ob, oi, oo, _ = orc.decode(base, w.Z, o_llr, syn_u[sel], w.max_iter)
    assert np.array_equal(oi, iters[sel]) and np.array_equal(oo, ok[sel])
    assert np.array_equal(ob, inputs.unpack_bits(bits[sel], w.n))


def test_interactive_protocol_full_size_sampled_frames_match_oracle():
    """The benchmark's default step at full size: the interactive protocol
    from f = 1.1 over all 16384 frames of the n = 49152 mixed workload, every
    round in one autotuned persistent launch with the benchmark's stall
    window.  Sampled frames (seeded picks, failing frames, the longest) run
    the oracle's protocol one by one and must agree in every field; every
    frame satisfies ok => H x = s, not ok => H x != s after the last round."""
    import bench
    from oracle import protocol as oproto
    from paper_1903_10107_gb300.pipeline import InteractiveProtocol, Reconciler

    args = bench.parse_args([])
    w = inputs.WORKLOADS[args.workload]
    B = w.batch
    base = w.base()
    xa, yb, q = w.frames(B, 0)
    tb = inputs.tiebreak_permutation(w.n, w.code_seed)
    rec = Reconciler(base, w.Z, tb, llr_scale=w.llr_scale)
    syn = rec.code.syndrome(_dev(xa))
    proto = InteractiveProtocol(rec, w.max_iter, f_start=args.f_start, df=args.df, max_rounds=args.max_rounds,
                                stall_window=args.stall_window)
    proto.tune(_dev(yb), syn, q, _dev(xa))
    res = proto.run(_dev(yb), syn, q, _dev(xa))
    bits, iters, ok, rounds = res["bits"], res["iters"], res["ok"], res["rounds"]

    syn_u = _syndromes(base, w.Z, w.n, xa)
    R = args.max_rounds
    assert np.all(rounds[ok == 0] == R) and rounds.max() <= R
    assert np.all(iters >= rounds + 1) and np.all(iters <= (rounds + 1) * w.max_iter)
    for f0 in range(0, B, 2048):
        sl = slice(f0, f0 + 2048)
        match = np.all(orc.syndrome(base, w.Z, inputs.unpack_bits(bits[sl], w.n)) == syn_u[sl], axis=1)
        assert np.all(match[ok[sl] == 1]) and not np.any(match[ok[sl] == 0])

    sel = _sample(iters, ok, B, seed=13, n_rand=10, n_fail=2, n_long=2)
    ref = oproto.interactive(base, w.Z, tb, inputs.unpack_bits(xa[sel], w.n), inputs.unpack_bits(yb[sel], w.n),
                             q[sel], args.f_start, args.df, R, w.max_iter, w.llr_scale,
                             stall_window=args.stall_window)
    assert np.array_equal(inputs.unpack_bits(bits[sel], w.n), ref["bits"])
    for k in ("ok", "iters", "rounds", "revealed", "key_bits"):
        assert np.array_equal(np.asarray(res[k])[sel], np.asarray(ref[k])), k
    # the benchmark's end-to-end path: the same step from pinned host buffers through the C-ABI
    # host-buffer call gives every frame the same result
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_bits = torch.empty((B, rec.code.nbytes), dtype=torch.uint8, pin_memory=True)
    hres, h2d, d2h = proto.run_host(pin(yb), syn.cpu().pin_memory(), q, pin(xa), bits_out=h_bits)
    assert np.array_equal(hres["bits"], bits)
    for k in ("ok", "iters", "rounds", "revealed", "key_bits"):
        assert np.array_equal(np.asarray(hres[k]), np.asarray(res[k])), k
    assert d2h == B * rec.code.nbytes + 9 * B and h2d > 2 * B * rec.code.nbytes

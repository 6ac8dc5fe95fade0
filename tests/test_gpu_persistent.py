"""Parity of the persistent mixed-rate path (fused LLR quantisation + layered
decoding with lane refill) with the CPU oracle, and its CUDA-graph capture."""
import numpy as np
import pytest

from conftest import device_mags
from oracle import core as orc
from oracle import rate as orate
from paper_1903_10107_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mixed_case(B, Z=32, seed=3, f_target=1.5, scale=8.0, Mb=24, Nb=96, mask="uniform"):
    """A 3/6 mixed-degree mother code with per-frame QBER 1-8 % and rates for
    f_target; ``mask="peg"`` gives rows of 15-16 blocks (the narrow, one-chunk
    row update and the unrolled stopping test), the uniform draw rows of up to
    22 (the chunked row update and the looped stopping test)."""
    degs = inputs.mixed_column_degrees(Nb, 0.3, 3, 6, seed)
    make = inputs.peg_base_matrix if mask == "peg" else inputs.qc_base_matrix
    base = make(Mb, Nb, Z, degs, seed)
    n, m = Nb * Z, Mb * Z
    q = inputs.frame_qbers(B, 0.01, 0.08, seed)
    xa = inputs.alice_keys(B, n, seed)
    yb = xa ^ inputs.bsc_noise(B, n, q, seed)
    tb = inputs.tiebreak_permutation(n, seed)
    rank = orate.position_rank(base, Z, tb)
    plans = [orate.rate_plan(n, m, float(x), f_target) for x in q]
    npn = np.array([p for p, s in plans], dtype=np.int32)
    ns = np.array([s for p, s in plans], dtype=np.int32)
    xa_u, yb_u = inputs.unpack_bits(xa, n), inputs.unpack_bits(yb, n)
    st = np.stack([orate.position_states(rank, int(npn[f]), int(ns[f])) for f in range(B)])
    llr = orc.llr_frames(yb_u, q, st, xa_u, scale=scale)
    syn_u = orc.syndrome(base, Z, xa_u)
    return dict(base=base, Z=Z, n=n, m=m, q=q, xa=xa, yb=yb, rank=rank, npn=npn, ns=ns, llr=llr, syn_u=syn_u,
                scale=scale)


def _run(case, max_iter, words=0, ctas=0, frame_list=None, threads=0, stall=0):
    from paper_1903_10107_gb300.decoder import QCCode
    code = QCCode(case["base"], case["Z"])
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    B = len(case["q"])
    sentinel = (torch.full((B, code.nbytes), 0xAB, dtype=torch.uint8, device="cuda"),
                torch.full((B,), -7, dtype=torch.int32, device="cuda"),
                torch.full((B,), 9, dtype=torch.uint8, device="cuda"))
    fl = None if frame_list is None else c(np.asarray(frame_list, dtype=np.int32))
    bits, iters, ok = code.reconcile_persistent(c(case["yb"]), device_mags(case["q"], case["scale"]),
                                                c(inputs.pack_bits(case["syn_u"])), max_iter, rank=c(case["rank"]),
                                                n_short=c(case["ns"]), n_punct=c(case["npn"]), known=c(case["xa"]),
                                                frame_list=fl, stall_window=stall, words=words, ctas_per_sm=ctas,
                                                threads=threads, out=sentinel)
    torch.cuda.synchronize()
    return code, bits.cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy()


@pytest.mark.parametrize("mask", ["uniform", "peg"])
@pytest.mark.parametrize("words", [1, 2, 4])
@pytest.mark.parametrize("scale", [8.0, 1 / 0.29])
def test_persistent_mixed_rate_bit_exact(words, scale, mask):
    case = _mixed_case(53, scale=scale, mask=mask)
    code, bits, iters, ok = _run(case, 40, words=words)
    ob, oi, oo, _ = orc.decode(case["base"], case["Z"], case["llr"], case["syn_u"], 40)
    assert np.array_equal(ok, oo) and np.array_equal(iters, oi)
    assert np.array_equal(inputs.unpack_bits(bits, case["n"]), ob)
    assert len(set(oi.tolist())) > 3  # uneven iteration counts were exercised


def test_persistent_frame_list_and_one_cta_per_sm():
    case = _mixed_case(40, seed=8)
    fl = [3, 17, 5, 39, 0, 22, 23, 11]
    code, bits, iters, ok = _run(case, 30, ctas=1, frame_list=fl)
    ob, oi, oo, _ = orc.decode(case["base"], case["Z"], case["llr"][fl], case["syn_u"][fl], 30)
    assert np.array_equal(ok[fl], oo) and np.array_equal(iters[fl], oi)
    assert np.array_equal(inputs.unpack_bits(bits[fl], case["n"]), ob)
    rest = [f for f in range(40) if f not in fl]
    assert (iters[rest] == -7).all() and (ok[rest] == 9).all() and (bits[rest] == 0xAB).all()


def test_persistent_equals_batch_kernel_on_larger_z():
    case = _mixed_case(30, Z=128, seed=12, Mb=8, Nb=32)
    code, bits, iters, ok = _run(case, 25)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    b2, i2, o2 = code.decode(c(case["llr"]), c(inputs.pack_bits(case["syn_u"])), 25)
    assert np.array_equal(bits, b2.cpu().numpy())
    assert np.array_equal(iters, i2.cpu().numpy()) and np.array_equal(ok, o2.cpu().numpy())


def test_persistent_plain_inputs_without_rate_adaptation():
    from paper_1903_10107_gb300.decoder import QCCode
    w = inputs.WORKLOADS["n4096_r075_q02"]
    base = w.base()
    xa, yb, q = w.frames(21)
    code = QCCode(base, w.Z)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    n = w.n
    syn_u = orc.syndrome(base, w.Z, inputs.unpack_bits(xa, n))
    bits, iters, ok = code.reconcile_persistent(c(yb), device_mags(q), c(inputs.pack_bits(syn_u)), w.max_iter)
    ob, oi, oo, _ = orc.decode(base, w.Z, orc.llr_frames(inputs.unpack_bits(yb, n), q), syn_u, w.max_iter)
    assert np.array_equal(inputs.unpack_bits(bits.cpu().numpy(), n), ob)
    assert np.array_equal(iters.cpu().numpy(), oi) and np.array_equal(ok.cpu().numpy(), oo)


def test_persistent_launch_captured_in_cuda_graph():
    case = _mixed_case(37, seed=21)
    from paper_1903_10107_gb300.decoder import QCCode
    code = QCCode(case["base"], case["Z"])
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (c(case["yb"]), device_mags(case["q"], case["scale"]), c(inputs.pack_bits(case["syn_u"])), 30)
    kw = dict(rank=c(case["rank"]), n_short=c(case["ns"]), n_punct=c(case["npn"]), known=c(case["xa"]))
    B = len(case["q"])
    out = (torch.zeros((B, code.nbytes), dtype=torch.uint8, device="cuda"),
           torch.zeros((B,), dtype=torch.int32, device="cuda"),
           torch.zeros((B,), dtype=torch.uint8, device="cuda"))
    code.reserve_persistent(B)
    ref = [t.clone() for t in code.reconcile_persistent(*args, **kw, out=out)]
    torch.cuda.synchronize()
    for t in out:
        t.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            code.reconcile_persistent(*args, **kw, out=out)
    torch.cuda.current_stream().wait_stream(s)
    for t in out:
        t.zero_()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(ref, out):
        assert torch.equal(a, b)


@pytest.mark.parametrize("Z,Mb,Nb", [(7, 6, 19), (5, 7, 21)])
def test_persistent_sizes_not_multiples_of_eight(Z, Mb, Nb):
    """n and m not multiples of 8: the refill and the write-out take a byte of
    variables (and of checks) per step and must stop at n (m)."""
    case = _mixed_case(23, Z=Z, seed=40 + Z, Mb=Mb, Nb=Nb, f_target=1.6)
    assert case["n"] % 8 and case["m"] % 8
    code, bits, iters, ok = _run(case, 30)
    ob, oi, oo, _ = orc.decode(case["base"], case["Z"], case["llr"], case["syn_u"], 30)
    assert np.array_equal(ok, oo) and np.array_equal(iters, oi)
    assert np.array_equal(inputs.unpack_bits(bits, case["n"]), ob)
    # padding bits past n in the last output byte stay 0
    pad = 8 * bits.shape[1] - case["n"]
    assert np.all(bits[:, -1] >> (8 - pad) == 0)


@pytest.mark.parametrize("mask", ["uniform", "peg"])
@pytest.mark.parametrize("words", [1, 2, 4])
@pytest.mark.parametrize("stall", [2, 6])
def test_persistent_stall_window_bit_exact(words, stall, mask):
    """The stall rule (a frame whose count of unsatisfied checks sets no new
    minimum for K iterations stops as a failure): per-lane counts in the
    kernel against the oracle's, through bits, iteration counts and flags.
    A high-QBER, low-efficiency case so that frames stall."""
    case = _mixed_case(61, seed=31, f_target=1.25, scale=1 / 0.29, mask=mask)
    if mask == "peg":
        assert int((case["base"] >= 0).sum(axis=1).max()) <= 16
    code, bits, iters, ok = _run(case, 60, words=words, stall=stall)
    ob, oi, oo, _ = orc.decode(case["base"], case["Z"], case["llr"], case["syn_u"], 60, stall_window=stall)
    assert np.array_equal(ok, oo) and np.array_equal(iters, oi)
    assert np.array_equal(inputs.unpack_bits(bits, case["n"]), ob)
    stalled = (oo == 0) & (oi < 60)
    assert stalled.any() and oo.any()  # frames stopped by the rule, and frames that decoded


def test_persistent_fewer_threads_than_rows():
    """threads below one pair per row of a layer: every thread pair takes
    several rows per layer; results do not change."""
    case = _mixed_case(29, Z=64, seed=17, f_target=1.5)
    _, b1, i1, o1 = _run(case, 30)
    for threads in (64, 32 * 3):
        _, b2, i2, o2 = _run(case, 30, threads=threads)
        assert np.array_equal(b1, b2) and np.array_equal(i1, i2) and np.array_equal(o1, o2)
    ob, oi, oo, _ = orc.decode(case["base"], case["Z"], case["llr"], case["syn_u"], 30)
    assert np.array_equal(o1, oo) and np.array_equal(i1, oi)


def test_persistent_rejects_bad_thread_counts():
    from paper_1903_10107_gb300 import native
    case = _mixed_case(8, Z=64, seed=18)
    for threads, words in ((48, 1), (2048, 1), (96, 2)):  # not a multiple of 32 * words, or above 1024
        with pytest.raises(native.LdpcError) as ei:
            _run(case, 5, words=words, threads=threads)
        assert ei.value.code == native.LDPC_EINVAL and "threads" in str(ei.value)


@pytest.mark.parametrize("words", [1, 2, 4])
@pytest.mark.parametrize("stall", [0, 5])
def test_interactive_launch_every_group_width(words, stall):
    """All rounds in one launch (ldpc_reconcile_interactive) at every group
    width: frames failing a round restart in their lane with more bits
    revealed; against the oracle's protocol frame by frame."""
    from oracle import protocol as oproto
    from paper_1903_10107_gb300.decoder import QCCode
    case = _mixed_case(47, seed=51, f_target=1.1, scale=1 / 0.29)
    base, Z, n, m, q = case["base"], case["Z"], case["n"], case["m"], case["q"]
    R, df, T = 4, 0.2, 40
    p0, s0 = case["npn"].astype(np.int64), case["ns"].astype(np.int64)
    rev = np.zeros((len(q), R + 1), np.int64)
    for r in range(R):
        for f in range(len(q)):
            key_now = n - p0[f] - s0[f] - max(int(rev[f, r]) - int(p0[f]), 0)
            rev[f, r + 1] = rev[f, r] + oproto.reveal_step(df, int(key_now), float(q[f]))
    code = QCCode(base, Z)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bits, iters, ok, rounds = code.reconcile_interactive(
        c(case["yb"]), device_mags(q, case["scale"]), c(inputs.pack_bits(case["syn_u"])), T, c(case["rank"]),
        c(case["ns"]), c(case["npn"]), c(case["xa"]), c(rev.astype(np.int32)), stall_window=stall, words=words)
    torch.cuda.synchronize()
    ref = oproto.interactive(base, Z, inputs.tiebreak_permutation(n, 51), inputs.unpack_bits(case["xa"], n),
                             inputs.unpack_bits(case["yb"], n), q, 1.1, df, R, T, case["scale"], stall_window=stall)
    assert np.array_equal(inputs.unpack_bits(bits.cpu().numpy(), n), ref["bits"])
    assert np.array_equal(ok.cpu().numpy(), ref["ok"]) and np.array_equal(rounds.cpu().numpy(), ref["rounds"])
    assert np.array_equal(iters.cpu().numpy(), ref["iters"])
    assert len(set(ref["rounds"].tolist())) >= 3  # frames finished in several different rounds
    assert np.array_equal(rev[np.arange(len(q)), ref["rounds"]], ref["revealed"])

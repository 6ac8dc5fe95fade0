"""Parity of the persistent mixed-rate path (fused LLR quantisation + layered
decoding with lane refill) with the CPU oracle, and its CUDA-graph capture."""
import numpy as np
import pytest

from oracle import core as orc
from oracle import rate as orate
from paper_1903_10107_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mixed_case(B, Z=32, seed=3, f_target=1.5, scale=8.0, Mb=24, Nb=96):
    """A 3/6 mixed-degree mother code with per-frame QBER 1-8 % and rates for f_target."""
    degs = inputs.mixed_column_degrees(Nb, 0.3, 3, 6, seed)
    base = inputs.qc_base_matrix(Mb, Nb, Z, degs, seed)
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


def _run(case, max_iter, words=0, ctas=0, frame_list=None):
    from paper_1903_10107_gb300.decoder import QCCode
    code = QCCode(case["base"], case["Z"])
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    B = len(case["q"])
    sentinel = (torch.full((B, code.nbytes), 0xAB, dtype=torch.uint8, device="cuda"),
                torch.full((B,), -7, dtype=torch.int32, device="cuda"),
                torch.full((B,), 9, dtype=torch.uint8, device="cuda"))
    fl = None if frame_list is None else c(np.asarray(frame_list, dtype=np.int32))
    bits, iters, ok = code.reconcile_persistent(c(case["yb"]), c(case["q"]), c(inputs.pack_bits(case["syn_u"])),
                                                max_iter, rank=c(case["rank"]), n_short=c(case["ns"]),
                                                n_punct=c(case["npn"]), known=c(case["xa"]), frame_list=fl,
                                                llr_scale=case["scale"], words=words, ctas_per_sm=ctas,
                                                out=sentinel)
    torch.cuda.synchronize()
    return code, bits.cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy()


@pytest.mark.parametrize("words", [1, 2, 4])
@pytest.mark.parametrize("scale", [8.0, 1 / 0.29])
def test_persistent_mixed_rate_bit_exact(words, scale):
    case = _mixed_case(53, scale=scale)
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
    bits, iters, ok = code.reconcile_persistent(c(yb), c(q), c(inputs.pack_bits(syn_u)), w.max_iter)
    ob, oi, oo, _ = orc.decode(base, w.Z, orc.llr_frames(inputs.unpack_bits(yb, n), q), syn_u, w.max_iter)
    assert np.array_equal(inputs.unpack_bits(bits.cpu().numpy(), n), ob)
    assert np.array_equal(iters.cpu().numpy(), oi) and np.array_equal(ok.cpu().numpy(), oo)


def test_persistent_launch_captured_in_cuda_graph():
    case = _mixed_case(37, seed=21)
    from paper_1903_10107_gb300.decoder import QCCode
    code = QCCode(case["base"], case["Z"])
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (c(case["yb"]), c(case["q"]), c(inputs.pack_bits(case["syn_u"])), 30)
    kw = dict(rank=c(case["rank"]), n_short=c(case["ns"]), n_punct=c(case["npn"]), known=c(case["xa"]),
              llr_scale=case["scale"])
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

"""Parity of the CUDA path with the CPU oracle, element by element.

Integer work (tau, LLRs, syndromes, decoded bits, iteration counts, success
flags) must be bit-exact.  Inputs come from the seeded generators only; the
oracle computes every expected value, the CUDA path is called through the
C ABI (via the thin ctypes binding)."""
import numpy as np
import pytest

from conftest import device_mags
from oracle import core as orc
from oracle import rate as orate
from paper_1903_10107_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _code(base, Z):
    from paper_1903_10107_gb300.decoder import QCCode
    return QCCode(base, Z)


def _cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _frames(base, Z, batch, qber, seed, first=0):
    n = base.shape[1] * Z
    xa = inputs.alice_keys(batch, n, seed, first)
    yb = xa ^ inputs.bsc_noise(batch, n, qber, seed, first)
    return xa, yb


def _oracle_inputs(base, Z, xa, yb, qber):
    n = base.shape[1] * Z
    xa_u = inputs.unpack_bits(xa, n)
    yb_u = inputs.unpack_bits(yb, n)
    syn_u = orc.syndrome(base, Z, xa_u)
    llr = orc.llr_frames(yb_u, qber)
    return llr, syn_u


def _decode_both(base, Z, llr, syn_u, max_iter, words=0, scale_q4=None, offset_q=None):
    code = _code(base, Z)
    syn_p = inputs.pack_bits(syn_u)
    sq = None if scale_q4 is None else _cuda(scale_q4)
    oq = None if offset_q is None else _cuda(offset_q)
    bits, iters, ok = code.decode(_cuda(llr), _cuda(syn_p), max_iter, scale_q4=sq, offset_q=oq, words=words)
    torch.cuda.synchronize()
    g = (inputs.unpack_bits(bits.cpu().numpy(), code.n), iters.cpu().numpy(), ok.cpu().numpy())
    o = orc.decode(base, Z, llr, syn_u, max_iter, scale_q4=scale_q4, offset_q=offset_q)
    return g, o


def _assert_same(g, o):
    bits_g, it_g, ok_g = g
    bits_o, it_o, ok_o = o[:3]
    assert np.array_equal(ok_g, ok_o), (ok_g, ok_o)
    assert np.array_equal(it_g, it_o), (it_g, it_o)
    bad = np.nonzero((bits_g != bits_o).any(axis=1))[0]
    assert bad.size == 0, f"frames with differing bits: {bad[:10]}"


# ------------------------------------------------------------------ pieces

def test_tau_table_exhaustive():
    from paper_1903_10107_gb300.decoder import tau_table_device
    got = tau_table_device().cpu().numpy().astype(np.int32)
    assert np.array_equal(got, orc.tau_table())


@pytest.mark.parametrize("Z,Nb", [(128, 32), (24, 10), (8, 3)])
def test_syndrome_kernel(Z, Nb):
    base = inputs.qc_base_matrix(4, Nb, Z, 3 if Nb > 3 else 2, 5)
    code = _code(base, Z)
    xa = inputs.alice_keys(37, code.n, 9)
    got = code.syndrome(_cuda(xa)).cpu().numpy()
    want = inputs.pack_bits(orc.syndrome(base, Z, inputs.unpack_bits(xa, code.n)))
    assert np.array_equal(got, want)


def test_llr_kernel_plain_and_rate_adapted():
    base = inputs.qc_base_matrix(6, 24, 16, inputs.mixed_column_degrees(24, 0.3, 3, 6, 4), 4)
    Z = 16
    code = _code(base, Z)
    n, m = code.n, code.m
    B = 40
    q = inputs.frame_qbers(B, 0.01, 0.08, 3)
    q[:4] = [0.01, 0.02, 0.03, 0.08]
    # QBERs whose ln((1-q)/q) * 8 lies within 1e-12 of a half-integer (k + 1/2, k = 20..35)
    import math
    for i, k in enumerate(range(20, 36)):
        q0 = 1.0 / (1.0 + math.exp((k + 0.5) / 8.0))
        q[4 + i] = math.nextafter(q0, 1.0) if i % 2 else q0
        assert abs(math.log((1 - q[4 + i]) / q[4 + i]) * 8.0 - (k + 0.5)) < 1e-12
    xa, yb = _frames(base, Z, B, q, 11)
    got = code.llr_from_bsc(_cuda(yb), device_mags(q)).cpu().numpy()
    want = orc.llr_frames(inputs.unpack_bits(yb, n), q)
    assert np.array_equal(got, want)
    # rate adapted: rank, shortened and punctured counts
    tb = inputs.tiebreak_permutation(n, 5)
    rank = orate.position_rank(base, Z, tb)
    ns = np.array([orate.rate_plan(n, m, float(x), 1.1)[1] for x in q], dtype=np.int32)
    npn = np.array([orate.rate_plan(n, m, float(x), 1.1)[0] for x in q], dtype=np.int32)
    ns[5] += 7  # a frame with both kinds, as after an interactive reveal
    got = code.llr_from_bsc(_cuda(yb), device_mags(q), rank=_cuda(rank), n_short=_cuda(ns), n_punct=_cuda(npn),
                            known=_cuda(xa)).cpu().numpy()
    st = np.stack([orate.position_states(rank, int(npn[f]), int(ns[f])) for f in range(B)])
    want = orc.llr_frames(inputs.unpack_bits(yb, n), q, st, inputs.unpack_bits(xa, n))
    assert np.array_equal(got, want)


# ------------------------------------------------------------------ decoding

def test_decode_n4096_64_frames_bit_exact():
    """The n=4096 rate-0.75 column-3 code, 64 frames at QBER 2 %, 50 iterations."""
    w = inputs.WORKLOADS["n4096_r075_q02"]
    base = w.base()
    xa, yb, q = w.frames()
    llr, syn_u = _oracle_inputs(base, w.Z, xa, yb, q)
    g, o = _decode_both(base, w.Z, llr, syn_u, w.max_iter)
    _assert_same(g, o)
    assert g[2].sum() > 0


@pytest.mark.parametrize("batch", [1, 3, 5, 17, 33])
@pytest.mark.parametrize("words", [1, 2, 4])
def test_decode_ragged_batches_and_group_widths(batch, words):
    base = inputs.qc_base_matrix(6, 24, 32, 3, 21)
    Z = 32
    xa, yb = _frames(base, Z, batch, 0.045, 100 + batch)
    llr, syn_u = _oracle_inputs(base, Z, xa, yb, 0.045)
    g, o = _decode_both(base, Z, llr, syn_u, 25, words=words)
    _assert_same(g, o)


@pytest.mark.parametrize("words", [1, 2, 4])
def test_decode_peg_mask_full_rows(words):
    """A PEG mask (rows of 15-16 blocks: every slot of the 8-slot body busy,
    one guarded chunk) through the batch decoder at every group width,
    including the multi-word body."""
    degs = inputs.mixed_column_degrees(96, 0.3, 3, 6, 41)
    Z = 32
    base = inputs.peg_base_matrix(24, 96, Z, degs, 41)
    assert int((base >= 0).sum(axis=1).max()) == 16
    xa, yb = _frames(base, Z, 29, 0.03, 700 + words)
    llr, syn_u = _oracle_inputs(base, Z, xa, yb, 0.03)
    g, o = _decode_both(base, Z, llr, syn_u, 30, words=words)
    _assert_same(g, o)
    assert g[2].sum() > 0


@pytest.mark.parametrize("Z", [5, 24, 96, 600])
def test_decode_odd_lifting_sizes(Z):
    """Z not a multiple of the warp size, and Z above the CTA's thread count."""
    base = inputs.qc_base_matrix(4, 16, Z, 3, 30 + Z)
    xa, yb = _frames(base, Z, 9, 0.05, 40 + Z)
    llr, syn_u = _oracle_inputs(base, Z, xa, yb, 0.05)
    g, o = _decode_both(base, Z, llr, syn_u, 20)
    _assert_same(g, o)


def test_decode_degree_zero_and_one_rows_and_high_degree():
    Z = 16
    base = np.full((5, 40), -1, dtype=np.int32)
    g = np.random.default_rng(3)
    base[0, 7] = 3                       # degree-1 row
    # row 1 stays empty (degree 0)
    base[2, :] = g.integers(0, Z, 40)    # degree 40 (64-edge kernel path)
    base[3, ::2] = g.integers(0, Z, 20)
    base[4, 1::3] = g.integers(0, Z, len(range(1, 40, 3)))
    xa, yb = _frames(base, Z, 13, 0.03, 77)
    llr, syn_u = _oracle_inputs(base, Z, xa, yb, 0.03)
    gg, o = _decode_both(base, Z, llr, syn_u, 15)
    _assert_same(gg, o)


def test_decode_saturated_inputs_and_single_iteration():
    """Shortened (+-127) and punctured (0) LLRs exercise Algorithm 2's guard."""
    base = inputs.qc_base_matrix(8, 32, 64, 3, 55)
    Z = 64
    n = 32 * Z
    xa, yb = _frames(base, Z, 24, 0.06, 56)
    xa_u, yb_u = inputs.unpack_bits(xa, n), inputs.unpack_bits(yb, n)
    st = np.zeros((24, n), np.uint8)
    g = np.random.default_rng(0)
    st[g.random((24, n)) < 0.05] = 1
    st[g.random((24, n)) < 0.10] = 2
    llr = orc.llr_frames(yb_u, 0.06, st, xa_u)
    syn_u = orc.syndrome(base, Z, xa_u)
    for it in (1, 30):
        gg, o = _decode_both(base, Z, llr, syn_u, it)
        _assert_same(gg, o)


def test_decode_with_scale_offset_tables():
    base = inputs.qc_base_matrix(8, 32, 32, 3, 61)
    Z = 32
    xa, yb = _frames(base, Z, 20, 0.04, 62)
    llr, syn_u = _oracle_inputs(base, Z, xa, yb, 0.04)
    g = np.random.default_rng(5)
    T = 18
    sq = g.integers(8, 40, size=(T, 8)).astype(np.uint8)
    oq = g.integers(-3, 6, size=(T, 8)).astype(np.int8)
    gg, o = _decode_both(base, Z, llr, syn_u, T, scale_q4=sq, offset_q=oq)
    _assert_same(gg, o)
    # identity tables reproduce the plain decoder exactly
    g1, _ = _decode_both(base, Z, llr, syn_u, T, scale_q4=np.full((T, 8), 16, np.uint8),
                         offset_q=np.zeros((T, 8), np.int8))
    g2, _ = _decode_both(base, Z, llr, syn_u, T)
    _assert_same(g1, g2 + (None,))


def test_decode_empty_batch_and_bad_arguments():
    from paper_1903_10107_gb300 import native
    base = inputs.qc_base_matrix(4, 16, 8, 3, 1)
    code = _code(base, 8)
    e = torch.empty((0, code.n), dtype=torch.int8, device="cuda")
    s = torch.empty((0, code.mbytes), dtype=torch.uint8, device="cuda")
    bits, iters, ok = code.decode(e, s, 10)
    assert bits.shape == (0, code.nbytes)
    with pytest.raises(native.LdpcError):
        code.decode(torch.zeros((2, code.n), dtype=torch.int8, device="cuda"),
                    torch.zeros((2, code.mbytes), dtype=torch.uint8, device="cuda"), 0)
    with pytest.raises(native.LdpcError):
        code.decode(torch.zeros((2, code.n), dtype=torch.int8, device="cuda"),
                    torch.zeros((2, code.mbytes), dtype=torch.uint8, device="cuda"), 5, words=3)


def test_decode_is_deterministic_and_batch_independent():
    base = inputs.qc_base_matrix(8, 32, 64, 3, 71)
    Z = 64
    code = _code(base, Z)
    xa, yb = _frames(base, Z, 50, 0.05, 72)
    llr, syn_u = _oracle_inputs(base, Z, xa, yb, 0.05)
    L, S = _cuda(llr), _cuda(inputs.pack_bits(syn_u))
    r1 = [t.cpu().numpy() for t in code.decode(L, S, 30)]
    r2 = [t.cpu().numpy() for t in code.decode(L, S, 30)]
    for a, b in zip(r1, r2):
        assert np.array_equal(a, b)
    # frame 13 decoded alone equals frame 13 decoded in the batch
    one = [t.cpu().numpy() for t in code.decode(L[13:14].contiguous(), S[13:14].contiguous(), 30)]
    for a, b in zip(r1, one):
        assert np.array_equal(a[13], b[0])


@pytest.mark.parametrize("dmax", [3, 8, 12, 17, 19, 21, 23, 25, 27, 31, 45, 60, 64])
def test_every_unroll_width_batch_and_persistent(dmax):
    """Codes whose longest row lands on each compiled unroll width (and on
    the row sizes just below a width); rows of several degrees per code so
    that slots past a layer's degree are exercised too."""
    from paper_1903_10107_gb300.decoder import QCCode
    Z, Nb = 16, max(dmax, 6)
    g = np.random.default_rng(dmax)
    degs = [dmax, max(1, dmax // 2), max(1, (2 * dmax) // 3), 1 + dmax % 3]
    base = np.full((len(degs), Nb), -1, dtype=np.int32)
    for i, d in enumerate(degs):
        cols = g.choice(Nb, size=d, replace=False)
        base[i, cols] = g.integers(0, Z, size=d)
    B, q, T = 13, 0.04, 12
    xa, yb = _frames(base, Z, B, q, 100 + dmax)
    llr, syn_u = _oracle_inputs(base, Z, xa, yb, q)
    gg, o = _decode_both(base, Z, llr, syn_u, T)
    _assert_same(gg, o)
    code = QCCode(base, Z)
    qv = np.full(B, q)
    bits, iters, ok = code.reconcile_persistent(_cuda(yb), device_mags(qv), _cuda(inputs.pack_bits(syn_u)), T)
    torch.cuda.synchronize()
    _assert_same((inputs.unpack_bits(bits.cpu().numpy(), code.n), iters.cpu().numpy(), ok.cpu().numpy()), o)


@pytest.mark.parametrize("Z,Nb", [(7, 9), (13, 15), (5, 21)])
def test_decode_odd_code_length(Z, Nb):
    """n odd: the soft values take 4 n bytes per word of lanes, not a multiple
    of 8, and the code tables behind them must still be aligned."""
    base = inputs.qc_base_matrix(4, Nb, Z, 3, 60 + Z)
    assert (Nb * Z) % 2 == 1
    xa, yb = _frames(base, Z, 11, 0.04, 70 + Z)
    llr, syn_u = _oracle_inputs(base, Z, xa, yb, 0.04)
    for words in (1, 0):
        g, o = _decode_both(base, Z, llr, syn_u, 20, words=words)
        _assert_same(g, o)


@pytest.mark.parametrize("dmax", [8, 12, 17, 23, 31])
@pytest.mark.parametrize("words", [2, 4])
def test_several_words_per_thread_every_width(dmax, words):
    """Two or four words (8 or 16 frames) of a row-half in one thread, with
    8- or 16-byte message and soft-value accesses, at the unroll widths it is
    used for (up to 16 slots at two words, 9 at four; wider ones take one word
    per thread), ragged batches, rows of several degrees per code."""
    Z, Nb = 16, max(dmax, 6)
    g = np.random.default_rng(300 + dmax)
    degs = [dmax, max(1, dmax // 2), max(1, (2 * dmax) // 3), 1 + dmax % 3]
    base = np.full((len(degs), Nb), -1, dtype=np.int32)
    for i, d in enumerate(degs):
        cols = g.choice(Nb, size=d, replace=False)
        base[i, cols] = g.integers(0, Z, size=d)
    B, q, T = 37, 0.04, 14
    xa, yb = _frames(base, Z, B, q, 400 + dmax)
    llr, syn_u = _oracle_inputs(base, Z, xa, yb, q)
    gg, o = _decode_both(base, Z, llr, syn_u, T, words=words)
    _assert_same(gg, o)

"""The allocation-free decode entry point, for callers that must not let the
library allocate device memory (a service with a fixed memory budget, a
process whose GPU memory belongs to another allocator's pool, a loop that
cannot afford an allocation's synchronisation).

It is called through the C ABI and must return exactly what
ldpc_decode_batch returns, and what the CPU oracle computes, on two calls in
a row (the second call finds the first call's leftovers in the shared fixed
scratch).  Collected last on
purpose: a failure here leaves every other test already run."""
import numpy as np
import pytest

from oracle import core as orc
from paper_1903_10107_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(base, Z, B, q, seed):
    n = base.shape[1] * Z
    xa = inputs.alice_keys(B, n, seed)
    yb = xa ^ inputs.bsc_noise(B, n, q, seed)
    syn_u = orc.syndrome(base, Z, inputs.unpack_bits(xa, n))
    llr = orc.llr_frames(inputs.unpack_bits(yb, n), q)
    return torch.from_numpy(llr).cuda(), torch.from_numpy(inputs.pack_bits(syn_u)).cuda(), llr, syn_u


def _outputs(code, B):
    return (torch.full((B, code.nbytes), 0x5A, dtype=torch.uint8, device="cuda"),
            torch.full((B,), -3, dtype=torch.int32, device="cuda"),
            torch.full((B,), 7, dtype=torch.uint8, device="cuda"))


def test_noalloc_decode_matches_decode_batch_on_two_calls():
    from paper_1903_10107_gb300 import native
    from paper_1903_10107_gb300.decoder import QCCode
    w = inputs.WORKLOADS["n4096_r075_q02"]
    base = w.base()
    code = QCCode(base, w.Z)
    st = torch.cuda.current_stream().cuda_stream
    # two different batches (sizes, noise) back to back through the fixed scratch
    for B, q, seed in ((150, 0.03, 11), (61, 0.02, 12)):
        llr, syn, llr_np, syn_u = _inputs(base, w.Z, B, q, seed)
        ref = [t.cpu().numpy() for t in code.decode(llr, syn, w.max_iter)]
        out = _outputs(code, B)
        native.ldpc_decode_batch_noalloc(code.handle, llr.data_ptr(), syn.data_ptr(), B, w.max_iter,
                                         out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), st)
        torch.cuda.synchronize()
        got = [t.cpu().numpy() for t in out]
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)  # integer results: bit-exact is the tolerance
        # and directly against the CPU oracle, so the check stands on its own
        ob, oi, oo, _ = orc.decode(base, w.Z, llr_np, syn_u, w.max_iter)
        assert np.array_equal(inputs.unpack_bits(got[0], code.n), ob)
        assert np.array_equal(got[1], oi) and np.array_equal(got[2], oo)
        assert 0 < got[2].sum() < B  # both decoded and failing frames were exercised


def test_noalloc_decode_rejects_batches_beyond_the_fixed_scratch():
    from paper_1903_10107_gb300 import native
    from paper_1903_10107_gb300.decoder import QCCode
    w = inputs.WORKLOADS["n4096_r075_q02"]
    code = QCCode(w.base(), w.Z)
    B = 4000  # 4000 * 12288 edges > 32 MiB
    llr = torch.zeros((B, code.n), dtype=torch.int8, device="cuda")
    syn = torch.zeros((B, code.mbytes), dtype=torch.uint8, device="cuda")
    out = _outputs(code, B)
    with pytest.raises(native.LdpcError) as ei:
        native.ldpc_decode_batch_noalloc(code.handle, llr.data_ptr(), syn.data_ptr(), B, 10, out[0].data_ptr(),
                                         out[1].data_ptr(), out[2].data_ptr(),
                                         torch.cuda.current_stream().cuda_stream)
    assert ei.value.code == native.LDPC_EINVAL and "fixed scratch" in str(ei.value)
    torch.cuda.synchronize()
    assert (out[1] == -3).all()  # nothing was launched

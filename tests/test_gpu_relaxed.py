"""The FP32 relaxed decoder and its hand-written adjoint against the FP64
reference: forward soft values within 1e-4 relative, the loss within 1e-4,
and every gradient component within 1e-3 relative,

    |g - g64| <= 1e-3 * max(|g64|, FLOOR * max|g64|),   FLOOR = 0.01,

i.e. components below 1 % of the largest are held to 1e-5 of the largest
(an FP32 sum of many terms of both signs cannot give a tiny component to a
relative 1e-3; measured at the training shape, 20 iterations on the n = 4096
code: 6e-4 with this floor, 1.8e-3 on a component 1100 times below the
largest without it).  The adjoint is also checked against central finite
differences of the FP64 loss per parameter and against finite differences
of the GPU loss along a direction."""
import numpy as np
import pytest

from oracle import relaxed64 as rx
from paper_1903_10107_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


FLOOR = 0.01


def _assert_grad_close(got, ref, tol=1e-3):
    got, ref = np.ravel(got), np.ravel(ref)
    scale = np.maximum(np.abs(ref), FLOOR * np.abs(ref).max())
    err = np.abs(got - ref) / scale
    assert err.max() <= tol, (err.max(), int(err.argmax()), got[err.argmax()], ref[err.argmax()])


def _case(Mb=4, Nb=12, Z=16, B=6, seed=0, mu=2.0, sigma=1.5):
    base = inputs.qc_base_matrix(Mb, Nb, Z, 3, seed)
    g = np.random.default_rng(seed)
    n = Nb * Z
    xa = g.integers(0, 2, size=(B, n)).astype(np.uint8)
    from oracle import core as orc
    syn = orc.syndrome(base, Z, xa)
    llr = ((1 - 2.0 * xa) * mu + g.normal(0, sigma, size=(B, n))).astype(np.float32)
    return base, Z, llr, syn, xa


def _gpu(base, Z, llr, syn, xa, al, ga, kappa, iters):
    from paper_1903_10107_gb300.decoder import QCCode
    from paper_1903_10107_gb300.relaxed import RelaxedDecodeFn, degree_classes
    code = QCCode(base, Z)
    cls = torch.from_numpy(degree_classes(base)[0]).cuda()
    A = torch.tensor(al, dtype=torch.float32, device="cuda", requires_grad=True)
    G = torch.tensor(ga, dtype=torch.float32, device="cuda", requires_grad=True)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    loss, E = RelaxedDecodeFn.apply(A, G, code, c(llr), c(inputs.pack_bits(syn)), c(inputs.pack_bits(xa)), cls,
                                    kappa)
    loss.backward()
    return float(loss), E.cpu().numpy(), A.grad.cpu().numpy(), G.grad.cpu().numpy(), code, cls


@pytest.mark.parametrize("kappa", [1.0, 0.431])
def test_forward_matches_fp64_reference(kappa):
    base, Z, llr, syn, xa = _case()
    T = 6
    C = len(rx.degree_classes(base)[1])
    g = np.random.default_rng(1)
    al, ga = g.uniform(0.7, 1.1, (T, C)), g.uniform(0.0, 0.3, (T, C))
    loss, E, _, _, _, _ = _gpu(base, Z, llr, syn, xa, al, ga, kappa, T)
    E64 = rx.decode(base, Z, llr.astype(np.float64), syn, T, al.astype(np.float32).astype(np.float64),
                    ga.astype(np.float32).astype(np.float64), kappa=kappa)
    rel = np.abs(E - E64) / np.maximum(np.abs(E64), 1.0)
    assert rel.max() <= 1e-4, rel.max()


@pytest.mark.parametrize("kappa", [1.0, 0.431])
def test_gradient_matches_fp64_reference(kappa):
    base, Z, llr, syn, xa = _case(seed=3)
    T = 5
    C = len(rx.degree_classes(base)[1])
    g = np.random.default_rng(2)
    al = g.uniform(0.7, 1.1, (T, C)).astype(np.float32).astype(np.float64)
    ga = g.uniform(0.05, 0.3, (T, C)).astype(np.float32).astype(np.float64)
    loss, E, g_al, g_ga, _, _ = _gpu(base, Z, llr, syn, xa, al, ga, kappa, T)
    l64, r_al, r_ga, _ = rx.loss_and_grad(base, Z, llr.astype(np.float64), syn, xa, al, ga, kappa=kappa)
    assert abs(loss - l64) <= 1e-4 * abs(l64)
    _assert_grad_close(np.concatenate([g_al.ravel(), g_ga.ravel()]), np.concatenate([r_al.ravel(), r_ga.ravel()]))


def test_gradient_matches_finite_differences_of_gpu_loss():
    from paper_1903_10107_gb300.relaxed import RelaxedDecodeFn
    base, Z, llr, syn, xa = _case(seed=5, B=16)
    T = 4
    C = len(rx.degree_classes(base)[1])
    g = np.random.default_rng(6)
    al, ga = g.uniform(0.8, 1.1, (T, C)), g.uniform(0.05, 0.25, (T, C))
    loss, E, g_al, g_ga, code, cls = _gpu(base, Z, llr, syn, xa, al, ga, 0.7, T)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (code, c(llr), c(inputs.pack_bits(syn)), c(inputs.pack_bits(xa)), cls, 0.7)
    # directional derivative along a random direction, central differences in fp32
    dA, dG = g.normal(size=al.shape), g.normal(size=ga.shape)
    eps = 2e-3

    def L(sgn):
        A = torch.tensor(al + sgn * eps * dA, dtype=torch.float32, device="cuda")
        G = torch.tensor(ga + sgn * eps * dG, dtype=torch.float32, device="cuda")
        with torch.no_grad():
            return float(RelaxedDecodeFn.apply(A, G, *args)[0])
    fd = (L(1) - L(-1)) / (2 * eps)
    an = float((g_al * dA).sum() + (g_ga * dG).sum())
    assert abs(fd - an) <= 2e-2 * abs(an) + 1e-6, (fd, an)


def test_identity_tables_round_to_plain_decoder():
    from paper_1903_10107_gb300.decoder import QCCode
    from paper_1903_10107_gb300.relaxed import RelaxedDecoder
    w = inputs.WORKLOADS["n4096_r075_q02"]
    code = QCCode(w.base(), w.Z)
    m = RelaxedDecoder(code, 20)
    sq, oq = m.integer_tables(8.0)
    assert sq.shape == (20, w.Mb) and (sq == 16).all() and (oq == 0).all()


def _special_rows_case(Z=16, B=6, seed=7, mu=2.0, sigma=1.5):
    """Rows of degree 1, 2, 0, 12 and 5: the empty box-plus, a pair, an
    empty row, a long row split unevenly between the two threads of a row."""
    g = np.random.default_rng(seed)
    Nb = 12
    base = np.full((5, Nb), -1, dtype=np.int32)
    for row, cols in ((0, [3]), (1, [0, 7]), (3, list(range(Nb))), (4, [1, 2, 5, 8, 11])):
        base[row, cols] = g.integers(0, Z, size=len(cols))
    n = Nb * Z
    xa = g.integers(0, 2, size=(B, n)).astype(np.uint8)
    from oracle import core as orc
    syn = orc.syndrome(base, Z, xa)
    llr = ((1 - 2.0 * xa) * mu + g.normal(0, sigma, size=(B, n))).astype(np.float32)
    return base, Z, llr, syn, xa


@pytest.mark.parametrize("case", ["special_rows", "z300_row_passes"])
def test_forward_and_gradient_on_special_shapes(case):
    if case == "special_rows":
        base, Z, llr, syn, xa = _special_rows_case()
        T = 4
    else:  # two threads per row exceed one block: each thread takes two rows per layer
        base, Z, llr, syn, xa = _case(Mb=3, Nb=8, Z=300, B=3, seed=9)
        T = 2
    C = len(rx.degree_classes(base)[1])
    g = np.random.default_rng(4)
    al = g.uniform(0.7, 1.1, (T, C)).astype(np.float32).astype(np.float64)
    ga = g.uniform(0.05, 0.3, (T, C)).astype(np.float32).astype(np.float64)
    kappa = 0.6
    loss, E, g_al, g_ga, _, _ = _gpu(base, Z, llr, syn, xa, al, ga, kappa, T)
    E64 = rx.decode(base, Z, llr.astype(np.float64), syn, T, al, ga, kappa=kappa)
    rel = np.abs(E - E64) / np.maximum(np.abs(E64), 1.0)
    assert rel.max() <= 1e-4, rel.max()
    l64, r_al, r_ga, _ = rx.loss_and_grad(base, Z, llr.astype(np.float64), syn, xa, al, ga, kappa=kappa)
    assert abs(loss - l64) <= 1e-4 * abs(l64)
    _assert_grad_close(np.concatenate([g_al.ravel(), g_ga.ravel()]), np.concatenate([r_al.ravel(), r_ga.ravel()]))


@pytest.mark.parametrize("Nb", [18, 24, 32])
def test_every_unroll_width_against_fp64(Nb):
    """Rows of 18, 24 and 32 edges select the kernels unrolled for 9, 12 and
    16 slots per half row (the other tests' codes take 6)."""
    Mb, Z, B = 2, 8, 4
    g = np.random.default_rng(Nb)
    base = g.integers(0, Z, size=(Mb, Nb)).astype(np.int32)  # every block nonzero: row degree Nb
    n = Nb * Z
    xa = g.integers(0, 2, size=(B, n)).astype(np.uint8)
    from oracle import core as orc
    syn = orc.syndrome(base, Z, xa)
    llr = ((1 - 2.0 * xa) * 3.0 + g.normal(0, 1.5, size=(B, n))).astype(np.float32)
    T = 3
    C = len(rx.degree_classes(base)[1])
    al = g.uniform(0.7, 1.1, (T, C)).astype(np.float32).astype(np.float64)
    ga = g.uniform(0.05, 0.3, (T, C)).astype(np.float32).astype(np.float64)
    loss, E, g_al, g_ga, _, _ = _gpu(base, Z, llr, syn, xa, al, ga, 0.431, T)
    E64 = rx.decode(base, Z, llr.astype(np.float64), syn, T, al, ga, kappa=0.431)
    rel = np.abs(E - E64) / np.maximum(np.abs(E64), 1.0)
    assert rel.max() <= 1e-4, rel.max()
    l64, r_al, r_ga, _ = rx.loss_and_grad(base, Z, llr.astype(np.float64), syn, xa, al, ga, kappa=0.431)
    assert abs(loss - l64) <= 1e-4 * abs(l64)
    _assert_grad_close(np.concatenate([g_al.ravel(), g_ga.ravel()]), np.concatenate([r_al.ravel(), r_ga.ravel()]))


def test_larger_code_two_frames_per_cta():
    """n = 5120 at Z = 128: two frames per CTA, 83 KB of soft values and their
    adjoints in shared memory, rows of up to 19 edges (the 12-slot kernels)."""
    base, Z, llr, syn, xa = _case(Mb=8, Nb=40, Z=128, B=4, seed=11)
    T = 3
    C = len(rx.degree_classes(base)[1])
    g = np.random.default_rng(12)
    al = g.uniform(0.7, 1.1, (T, C)).astype(np.float32).astype(np.float64)
    ga = g.uniform(0.05, 0.3, (T, C)).astype(np.float32).astype(np.float64)
    loss, E, g_al, g_ga, _, _ = _gpu(base, Z, llr, syn, xa, al, ga, 0.431, T)
    E64 = rx.decode(base, Z, llr.astype(np.float64), syn, T, al, ga, kappa=0.431)
    rel = np.abs(E - E64) / np.maximum(np.abs(E64), 1.0)
    assert rel.max() <= 1e-4, rel.max()
    l64, r_al, r_ga, _ = rx.loss_and_grad(base, Z, llr.astype(np.float64), syn, xa, al, ga, kappa=0.431)
    assert abs(loss - l64) <= 1e-4 * abs(l64)
    _assert_grad_close(np.concatenate([g_al.ravel(), g_ga.ravel()]), np.concatenate([r_al.ravel(), r_ga.ravel()]))


def _training_shape_case(B=4, sigma=0.5, T=20, seed=7):
    """The training workload's shape: the n = 4096 code, QBER U(2 %, 4 %),
    20 iterations, the temperature of 8 LSB per nat.  Channel LLRs are the
    BSC's plus N(0, sigma^2) noise (Gaussian relaxation): continuous inputs,
    so that no soft value sits exactly on a sign or relu kink."""
    from oracle import core as orc
    from paper_1903_10107_gb300.relaxed import bsc_llr_nats, kappa_for_scale
    w = inputs.WORKLOADS["n4096_relaxed_q02_04"]
    base = w.base()
    xa, yb, q = w.frames(B, 0)
    xa_u, yb_u = inputs.unpack_bits(xa, w.n), inputs.unpack_bits(yb, w.n)
    g = np.random.default_rng(seed)
    llr = (bsc_llr_nats(yb_u, q) + g.normal(0, sigma, size=(B, w.n))).astype(np.float32)
    syn = orc.syndrome(base, w.Z, xa_u)
    C = len(rx.degree_classes(base)[1])
    al = g.uniform(0.7, 1.1, (T, C)).astype(np.float32).astype(np.float64)
    ga = g.uniform(0.05, 0.3, (T, C)).astype(np.float32).astype(np.float64)
    assert T == w.max_iter
    return base, w.Z, llr, syn, xa_u, al, ga, kappa_for_scale(8.0)


def test_training_shape_forward_and_every_gradient_component():
    base, Z, llr, syn, xa, al, ga, kappa = _training_shape_case()
    loss, E, g_al, g_ga, _, _ = _gpu(base, Z, llr, syn, xa, al, ga, kappa, al.shape[0])
    l64, r_al, r_ga, E64 = rx.loss_and_grad(base, Z, llr.astype(np.float64), syn, xa, al, ga, kappa=kappa)
    assert abs(loss - l64) <= 1e-4 * abs(l64)
    rel = np.abs(E - E64) / np.maximum(np.abs(E64), 1.0)
    assert rel.max() <= 1e-4, rel.max()
    _assert_grad_close(g_al, r_al)
    _assert_grad_close(g_ga, r_ga)
    _assert_grad_close(np.concatenate([g_al.ravel(), g_ga.ravel()]), np.concatenate([r_al.ravel(), r_ga.ravel()]))


def test_training_shape_gradient_against_central_differences_per_parameter():
    """Central differences of the FP64 loss, one parameter at a time, at
    first, middle and last iterations and at the smallest, a middle and the
    largest degree class.  The step is 1e-7: the loss is only piecewise
    smooth (soft values change sign, relu edges move), and wider steps cross
    kinks (1e-4 was off by up to 15 % for first-iteration parameters; 1e-7
    agrees with autograd to a few 1e-6)."""
    base, Z, llr, syn, xa, al, ga, kappa = _training_shape_case()
    T, C = al.shape
    _, _, g_al, g_ga, _, _ = _gpu(base, Z, llr, syn, xa, al, ga, kappa, T)
    _, r_al, r_ga, _ = rx.loss_and_grad(base, Z, llr.astype(np.float64), syn, xa, al, ga, kappa=kappa)
    scale = FLOOR * max(np.abs(r_al).max(), np.abs(r_ga).max())
    eps = 1e-7
    for t, c in ((0, 0), (0, C - 1), (T // 2, C // 2), (T - 1, 0), (T - 1, C - 1), (5, min(1, C - 1))):
        for which, gpu, ref in (("alpha", g_al, r_al), ("gamma", g_ga, r_ga)):
            def L(sign):
                a2, g2 = al.copy(), ga.copy()
                (a2 if which == "alpha" else g2)[t, c] += sign * eps
                return rx.loss(base, Z, llr.astype(np.float64), syn, xa, T, a2, g2, kappa=kappa)
            fd = (L(1) - L(-1)) / (2 * eps)
            assert abs(fd - ref[t, c]) <= 1e-4 * max(abs(ref[t, c]), scale), (which, t, c, fd, ref[t, c])
            assert abs(gpu[t, c] - fd) <= 1e-3 * max(abs(fd), scale), (which, t, c, gpu[t, c], fd)

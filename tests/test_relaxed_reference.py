"""Pins of the FP64 relaxed-decoder reference (oracle/relaxed64.py) against
closed forms and finite differences."""
import numpy as np
import pytest

from oracle import relaxed64 as rx


def _gauss_case(Mb=3, Nb=9, Z=4, B=3, seed=0):
    from paper_1903_10107_gb300 import inputs
    base = inputs.qc_base_matrix(Mb, Nb, Z, 2, seed)
    g = np.random.default_rng(seed)
    n, m = Nb * Z, Mb * Z
    xa = g.integers(0, 2, size=(B, n))
    H = np.zeros((m, n), np.int64)
    for i in range(Mb):
        for k in range(Nb):
            if base[i, k] >= 0:
                for r in range(Z):
                    H[i * Z + r, k * Z + (r + base[i, k]) % Z] = 1
    syn = (xa @ H.T) % 2
    llr = (1 - 2 * xa) * 2.0 + g.normal(0, 1.5, size=(B, n))  # continuous: no sign/relu kinks
    return base, Z, llr, syn, xa


def test_single_check_equals_tanh_rule():
    """One check of degree d (Z = 1): after one iteration E_k = llr_k +
    (-1)^s prod_{k'!=k} sign * 2 atanh(prod tanh(|llr_k'|/2))  (Eqs. 1, 2, 9)."""
    g = np.random.default_rng(3)
    for d in (2, 3, 5, 7):
        base = np.zeros((1, d), np.int32)
        llr = g.normal(0, 3, size=(2, d))
        syn = np.array([[0], [1]])
        E = rx.decode(base, 1, llr, syn, 1)
        for f in range(2):
            for k in range(d):
                o = np.delete(llr[f], k)
                mag = 2 * np.arctanh(np.prod(np.tanh(np.abs(o) / 2)))
                sign = (-1) ** syn[f, 0] * np.prod(np.sign(o))
                assert abs(E[f, k] - (llr[f, k] + sign * mag)) < 1e-10


def test_tempered_boxplus_limits():
    g = np.random.default_rng(4)
    x, y = g.uniform(0, 10, 500), g.uniform(0, 10, 500)
    for kappa in (1.0, 0.5, 0.1, 0.01):
        b = rx.boxplus(x, y, kappa)
        assert np.all(b <= np.minimum(x, y) + 1e-12)
        assert np.all(b >= np.minimum(x, y) - kappa * np.log(2) - 1e-12)  # -> min-sum as kappa -> 0
    # kappa = 1 is Eq. 6's tanh form
    t = 2 * np.arctanh(np.tanh(x / 2) * np.tanh(y / 2))
    ok = t < 15
    assert np.allclose(rx.boxplus(x, y)[ok], t[ok], rtol=1e-9, atol=1e-12)


def test_numpy_and_torch_forms_agree():
    pytest.importorskip("torch")
    base, Z, llr, syn, xa = _gauss_case()
    T = 3
    C = len(rx.degree_classes(base)[1])
    g = np.random.default_rng(5)
    al, ga = g.uniform(0.7, 1.2, (T, C)), g.uniform(0.0, 0.3, (T, C))
    E_np = rx.decode(base, Z, llr, syn, T, al, ga, kappa=0.6)
    _, _, _, E_t = rx.loss_and_grad(base, Z, llr, syn, xa, al, ga, kappa=0.6)
    assert np.allclose(E_np, E_t, rtol=1e-12, atol=1e-12)


def test_reference_gradient_matches_finite_differences():
    pytest.importorskip("torch")
    base, Z, llr, syn, xa = _gauss_case(seed=7)
    T = 3
    C = len(rx.degree_classes(base)[1])
    g = np.random.default_rng(8)
    al, ga = g.uniform(0.7, 1.2, (T, C)), g.uniform(0.05, 0.3, (T, C))
    loss, g_al, g_ga, _ = rx.loss_and_grad(base, Z, llr, syn, xa, al, ga, kappa=0.7)
    eps = 1e-6
    for (t, c) in [(0, 0), (1, C - 1), (T - 1, 0)]:
        for which, grad in (("a", g_al), ("g", g_ga)):
            p, m = al.copy(), al.copy()
            q, r = ga.copy(), ga.copy()
            if which == "a":
                p[t, c] += eps; m[t, c] -= eps
                lp = rx.loss_and_grad(base, Z, llr, syn, xa, p, ga, kappa=0.7)[0]
                lm = rx.loss_and_grad(base, Z, llr, syn, xa, m, ga, kappa=0.7)[0]
            else:
                q[t, c] += eps; r[t, c] -= eps
                lp = rx.loss_and_grad(base, Z, llr, syn, xa, al, q, kappa=0.7)[0]
                lm = rx.loss_and_grad(base, Z, llr, syn, xa, al, r, kappa=0.7)[0]
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - grad[t, c]) <= 1e-6 + 1e-5 * abs(fd), (which, t, c, fd, grad[t, c])


def test_tree_code_converges_to_brute_force_posterior():
    """On a cycle-free Tanner graph belief propagation is exact: with kappa = 1
    and no scale or offset, the layered relaxation's soft values converge to
    the posterior LLRs log P(x_j = 0 | y, Hx = s) / P(x_j = 1 | y, Hx = s),
    computed here by enumerating the syndrome's coset (Eqs. 1, 2, 6, 9)."""
    import itertools
    # checks {0,1,2}, {2,3,4}, {4,5}, {1,6,7}: a tree over 8 variables (Z = 1)
    rows = [[0, 1, 2], [2, 3, 4], [4, 5], [1, 6, 7]]
    n = 8
    base = np.full((len(rows), n), -1, np.int32)
    for i, cols in enumerate(rows):
        base[i, cols] = 0
    H = (base >= 0).astype(np.int64)
    g = np.random.default_rng(11)
    B = 4
    llr = g.normal(0.5, 2.0, size=(B, n))
    syn = g.integers(0, 2, size=(B, len(rows)))
    E = rx.decode(base, 1, llr, syn, 12)
    words = np.array(list(itertools.product((0, 1), repeat=n)))
    for f in range(B):
        coset = words[np.all((words @ H.T) % 2 == syn[f], axis=1)]
        logw = (coset * -llr[f]).sum(axis=1)  # log P(y|x) up to a constant: bit 1 costs llr
        for j in range(n):
            l0 = np.logaddexp.reduce(logw[coset[:, j] == 0])
            l1 = np.logaddexp.reduce(logw[coset[:, j] == 1])
            assert abs(E[f, j] - (l0 - l1)) < 1e-9, (f, j, E[f, j], l0 - l1)


def _degree_one_case(Z=8, B=4, seed=21):
    """Rows of degree 1 (two of them), 2, 5 and 9 on 12 block columns."""
    g = np.random.default_rng(seed)
    Nb = 12
    base = np.full((5, Nb), -1, dtype=np.int32)
    for row, cols in ((0, [3]), (1, [7]), (2, [0, 5]), (3, [1, 2, 4, 8, 11]), (4, [0, 3, 5, 6, 7, 8, 9, 10, 11])):
        base[row, cols] = g.integers(0, Z, size=len(cols))
    from oracle import core as orc
    n = Nb * Z
    xa = g.integers(0, 2, size=(B, n)).astype(np.uint8)
    syn = orc.syndrome(base, Z, xa)
    llr = (1 - 2.0 * xa) * 1.5 + g.normal(0, 1.5, size=(B, n))
    return base, Z, llr, syn, xa


def test_empty_boxplus_stand_in_acts_as_infinity():
    """A degree-1 row sends EMPTY in place of the empty box-plus (+infinity).
    Beyond about 30 nats nothing else the decoder computes depends on the
    value: every soft value of a variable outside the degree-1 rows, the
    hard decisions and the loss agree to 1e-9 between EMPTY = 40, 50 and
    1000.  The degree-1 rows' own variables get soft values of magnitude
    about EMPTY whose sign does not depend on it (their check pins them).
    Far below the other magnitudes (EMPTY = 5) the stand-in is no longer
    neutral."""
    base, Z, llr, syn, xa = _degree_one_case()
    T, kappa = 6, 0.431
    C = len(rx.degree_classes(base)[1])
    al, ga = np.full((T, C), 0.9), np.full((T, C), 0.1)
    deg1 = np.zeros(base.shape[1] * Z, bool)
    for i in np.flatnonzero((base >= 0).sum(axis=1) == 1):
        k = int(np.flatnonzero(base[i] >= 0)[0])
        deg1[k * Z:(k + 1) * Z] = True
    E = {e: rx.decode(base, Z, llr, syn, T, al, ga, kappa=kappa, empty=e) for e in (5.0, 40.0, 50.0, 1000.0)}
    Ls = {e: rx.loss(base, Z, llr, syn, xa, T, al, ga, kappa=kappa, empty=e) for e in (40.0, 50.0, 1000.0)}
    for e in (40.0, 1000.0):
        assert np.allclose(E[e][:, ~deg1], E[50.0][:, ~deg1], rtol=1e-9, atol=1e-9)
        assert np.array_equal(E[e] < 0, E[50.0] < 0)
        assert abs(Ls[e] - Ls[50.0]) <= 1e-9 * Ls[50.0]
    # the degree-1 variables: |E| grows with the stand-in (their row pins them) and keeps its sign
    assert np.all(np.abs(E[1000.0][:, deg1]) > 500) and np.array_equal(E[1000.0][:, deg1] < 0, E[50.0][:, deg1] < 0)
    # far below the decoder's other magnitudes the stand-in is not neutral any more
    assert not np.allclose(E[5.0][:, ~deg1], E[50.0][:, ~deg1], rtol=1e-6, atol=1e-6)


def test_empty_stand_in_exceeds_the_integer_decoders_largest_message():
    """EMPTY is at least the integer decoder's MSG_max (127 LSB) in nats at
    the LLR steps the workloads use: the table's own 0.29 nat and 1/8 nat."""
    assert rx.EMPTY >= 127 * 0.29 and rx.EMPTY >= 127 / 8.0


def test_numpy_loss_equals_autograd_loss():
    base, Z, llr, syn, xa = _degree_one_case(seed=22)
    T = 4
    C = len(rx.degree_classes(base)[1])
    g = np.random.default_rng(5)
    al, ga = g.uniform(0.7, 1.1, (T, C)), g.uniform(0.0, 0.3, (T, C))
    l_np = rx.loss(base, Z, llr, syn, xa, T, al, ga, kappa=0.6)
    l_t, _, _, _ = rx.loss_and_grad(base, Z, llr, syn, xa, al, ga, kappa=0.6)
    assert abs(l_np - l_t) <= 1e-12 * abs(l_t)

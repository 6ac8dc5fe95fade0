"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test ties one part of the oracle to something other than itself:
hand-evaluated values of Algorithm 1, the box-plus function of Eq. 6, the
worked example of section 3.3, textbook min-sum as a special case, the
parity-check invariant, maximum-likelihood decoding by enumeration and the
closed form of the efficiency.
"""

import numpy as np
import pytest

from conftest import golden
from oracle import core, rate, tiny
from paper_1903_10107_gb300 import inputs


# ------------------------------------------------------------------ tau (Alg. 1)

def test_tau_hand_values():
    for p, q, mm, want in golden("tau_algorithm1_hand.txt"):
        assert core.tau(int(p), int(q), int(mm)) == int(want), (p, q, mm)


def test_tau_table_properties():
    T = core.tau_table()
    P, Q = np.meshgrid(np.arange(128), np.arange(128), indexing="ij")
    mn = np.minimum(P, Q)
    assert (T == T.T).all()                        # box-plus is symmetric
    assert (T <= mn).all() and (T >= mn - 2).all() and (T >= 0).all()
    far = np.abs(P - Q) >= 6
    assert (T[far] == mn[far]).all()               # correction vanishes for distant inputs
    assert (np.diff(T, axis=0) >= 0).all() and (np.diff(T, axis=1) >= 0).all()  # monotone like beta


def _beta(x, y):
    # Eq. 6 in a form that stays finite: min + ln(1+e^-(x+y)) - ln(1+e^-|x-y|)
    return np.minimum(x, y) + np.log1p(np.exp(-(x + y))) - np.log1p(np.exp(-np.abs(x - y)))


def test_tau_approximates_boxplus():
    """tau(p, q) is the integer representation of beta((p+1/2)D, (q+1/2)D)
    (section 3.2).  At the best-fitting step D = 0.29 nat every entry is within
    one LSB of floor(beta/D), and the mean error is small."""
    T = core.tau_table()
    P, Q = np.meshgrid(np.arange(128), np.arange(128), indexing="ij")
    D = 0.29
    ref = np.floor(_beta((P + 0.5) * D, (Q + 0.5) * D) / D)
    err = np.abs(T - ref)
    assert err.max() <= 1
    assert err.mean() < 0.05
    # with the correction switched off (tau = min) the same comparison is worse
    err_min = np.abs(np.minimum(P, Q) - ref)
    assert err_min.max() >= 2


def test_boxplus_forms_agree():
    """Eqs. 2, 3 and 6 describe one function: tanh form, phi form, stable form."""
    g = np.random.default_rng(0)
    x, y = g.uniform(0.05, 12, 1000), g.uniform(0.05, 12, 1000)
    tanh_form = 2 * np.arctanh(np.tanh(x / 2) * np.tanh(y / 2))
    phi = lambda z: -np.log(np.tanh(z / 2))
    phi_form = phi(phi(x) + phi(y))
    ok = tanh_form < 15  # arctanh loses precision close to 1
    assert np.allclose(tanh_form[ok], phi_form[ok], rtol=1e-9)
    assert np.allclose(_beta(x, y)[ok], tanh_form[ok], rtol=1e-9)


# --------------------------------------------------------- check-node magnitudes

@pytest.mark.parametrize("d", list(range(1, 9)))
def test_cn_forward_backward_matches_per_edge_definition(d):
    g = np.random.default_rng(d)
    for _ in range(300):
        a = g.integers(0, 128, size=d)
        if g.random() < 0.5:
            a = g.integers(0, 9, size=d)  # the small-magnitude region where tau corrects
        got = core.cn_magnitudes(a)
        want = tiny.brute_cn([int(x) for x in a])
        assert list(got) == want, a


@pytest.mark.parametrize("d", list(range(2, 9)))
def test_cn_min_mode_is_textbook_min_sum(d):
    g = np.random.default_rng(100 + d)
    for _ in range(300):
        a = g.integers(0, 128, size=d)
        got = core.cn_magnitudes(a, fold_mode=core.FOLD_MIN)
        want = [int(np.min(np.delete(a, k))) for k in range(d)]
        assert list(got) == want


def test_cn_bounds():
    g = np.random.default_rng(7)
    for d in range(2, 20):
        for _ in range(50):
            a = g.integers(0, 128, size=d)
            m = core.cn_magnitudes(a)
            for k in range(d):
                others = np.delete(a, k)
                lo = max(int(others.min()) - 2 * (d - 2), 0)
                assert lo <= m[k] <= others.min()


def test_cn_degree_one_is_msg_max():
    assert list(core.cn_magnitudes([5])) == [core.MSG_MAX]


def test_fold_order_matters():
    """tau is not associative, so the fold order is part of the method:
    ((5 [+] 6) [+] 7) = tau(3, 7) = 2 but ((5 [+] 7) [+] 6) = tau(4, 6) = 3."""
    assert core.tau(core.tau(5, 6), 7) == 2
    assert core.tau(core.tau(5, 7), 6) == 3


# ---------------------------------------------------------------- VN (Alg. 2)

def test_vn_worked_example():
    (row,) = golden("vn_saturation_example.txt")
    exact0, stored0, i1, i2, i3, exact1, naive1, alg2 = map(int, row)
    assert exact0 + i1 + i2 + i3 == exact1
    naive = stored0 + i1 + i2 + i3               # wrapping 8-bit arithmetic ignores saturation
    assert naive == naive1
    # Algorithm 2: L_ji = E - L_old, E <- L_ji + L_new, skipped while |E| = 127
    E, L_old = stored0, 0
    for inc in (i1, i2, i3):
        l_ji = max(-127, min(127, E - L_old))
        E = core.vn_update(E, l_ji, L_old + inc)
    assert E == alg2
    assert np.sign(E) == np.sign(exact1)


def test_vn_update_unsaturated():
    assert core.vn_update(10, 10 - 3, 20) == 27
    assert core.vn_update(-126, -120, -30) == -127   # saturates on the way in
    assert core.vn_update(-127, -100, 50) == -127    # then stays


# ------------------------------------------------------------------- LLRs

def test_llr_golden():
    for p, mag in golden("llr_quantisation.txt"):
        assert core.llr_magnitude(float(p)) == int(mag)


def test_llr_frame_states():
    y = np.array([[0, 1, 0, 1, 0, 1]], dtype=np.uint8)
    st = np.array([[0, 0, 1, 1, 2, 2]], dtype=np.uint8)
    kn = np.array([[0, 0, 0, 0, 1, 0]], dtype=np.uint8)
    llr = core.llr_frames(y, 0.02, st, kn)
    assert llr.tolist() == [[31, -31, 0, 0, -127, 127]]


# ------------------------------------------------------- code expansion / syndrome

def _small_code(seed, Mb=4, Nb=12, Z=8, deg=3):
    return inputs.qc_base_matrix(Mb, Nb, Z, deg, seed), Z


def test_expand_matches_dense_h():
    for seed in range(5):
        base, Z = _small_code(seed)
        H = tiny.dense_h(base, Z)
        row_ptr, vn = core.expand(base, Z)
        for c in range(H.shape[0]):
            assert list(vn[row_ptr[c]:row_ptr[c + 1]]) == list(np.nonzero(H[c])[0])


def test_syndrome_matches_dense_product():
    base, Z = _small_code(3)
    H = tiny.dense_h(base, Z)
    x = np.random.default_rng(0).integers(0, 2, size=(20, H.shape[1])).astype(np.uint8)
    assert np.array_equal(core.syndrome(base, Z, x), (x.astype(np.int64) @ H.T.astype(np.int64)) % 2)


# --------------------------------------------------------------- decoder

def _frames(base, Z, batch, q, seed):
    n = base.shape[1] * Z
    xa = inputs.unpack_bits(inputs.alice_keys(batch, n, seed), n)
    yb = inputs.unpack_bits(inputs.alice_keys(batch, n, seed) ^ inputs.bsc_noise(batch, n, q, seed), n)
    return xa, yb


def test_zero_error_frames_decode_in_one_iteration():
    base, Z = _small_code(11, Mb=8, Nb=32, Z=16)
    xa, _ = _frames(base, Z, 16, 0.0, 5)
    syn = core.syndrome(base, Z, xa)
    llr = core.llr_frames(xa, 0.02)
    bits, iters, ok, _ = core.decode(base, Z, llr, syn, 20)
    assert ok.all() and (iters == 1).all() and np.array_equal(bits, xa)


def test_syndrome_invariant_on_success():
    base, Z = _small_code(12, Mb=8, Nb=32, Z=32)
    H = tiny.dense_h(base, Z).astype(np.int64)
    xa, yb = _frames(base, Z, 64, 0.03, 6)
    syn = core.syndrome(base, Z, xa)
    bits, iters, ok, _ = core.decode(base, Z, core.llr_frames(yb, 0.03), syn, 30)
    assert ok.sum() > 0
    for f in range(len(ok)):
        par_ok = np.array_equal(H @ bits[f] % 2, syn[f])
        assert bool(ok[f]) == par_ok
        assert 1 <= iters[f] <= 30


def test_bp_never_beats_ml_and_corrects_single_errors():
    """n <= 20: on success the decoded word is a coset member no closer to
    Bob's key than the maximum-likelihood word; isolated single errors that
    ML corrects uniquely are corrected by the decoder too."""
    base = np.array([[0, 1, -1, 2, 0], [1, -1, 0, 3, 2]], dtype=np.int32)  # 2x5 base, Z=4 -> n=20
    Z = 4
    H = tiny.dense_h(base, Z)
    g = np.random.default_rng(1)
    fixed = 0
    for trial in range(40):
        xa = g.integers(0, 2, size=20).astype(np.uint8)
        y = xa.copy()
        y[g.integers(0, 20)] ^= 1
        syn = (H.astype(np.int64) @ xa % 2).astype(np.uint8)
        dml, words = tiny.ml_decode(H, syn, y)
        bits, it, ok, _ = core.decode(base, Z, core.llr_frames(y[None], 0.05), syn[None], 30)
        if ok[0]:
            assert np.array_equal(H.astype(np.int64) @ bits[0] % 2, syn)
            assert int(np.sum(bits[0] != y)) >= dml
        if len(words) == 1 and dml == 1 and ok[0] and np.array_equal(bits[0], words[0]):
            fixed += 1
    assert fixed >= 10


def test_fer_bp_at_least_fer_ml():
    base = np.array([[0, 1, -1, 2, 0], [1, -1, 0, 3, 2]], dtype=np.int32)
    Z = 4
    H = tiny.dense_h(base, Z)
    g = np.random.default_rng(2)
    err_ml = err_bp = 0
    for trial in range(60):
        xa = g.integers(0, 2, size=20).astype(np.uint8)
        y = xa ^ (g.random(20) < 0.08).astype(np.uint8)
        syn = (H.astype(np.int64) @ xa % 2).astype(np.uint8)
        _, words = tiny.ml_decode(H, syn, y)
        err_ml += not any(np.array_equal(w, xa) for w in words[:1])
        bits, _, ok, _ = core.decode(base, Z, core.llr_frames(y[None], 0.08), syn[None], 30)
        err_bp += not (ok[0] and np.array_equal(bits[0], xa))
    assert err_bp >= err_ml


def test_c_oracle_matches_python_decoder():
    """The C oracle and the independent pure-Python decoder agree on small
    codes, including strong (saturating) LLRs and random syndromes."""
    for seed, q, iters in ((21, 0.04, 15), (22, 0.08, 10), (23, 0.001, 5)):
        base, Z = _small_code(seed, Mb=4, Nb=16, Z=8, deg=3)
        xa, yb = _frames(base, Z, 6, q, seed)
        syn = core.syndrome(base, Z, xa)
        llr = core.llr_frames(yb, q)
        bits, it, ok, _ = core.decode(base, Z, llr, syn, iters)
        for f in range(6):
            b2, i2, o2 = tiny.decode(base, Z, llr[f], syn[f], iters)
            assert np.array_equal(bits[f], b2) and it[f] == i2 and ok[f] == o2


def test_min_mode_decoder_matches_python_min_sum():
    base, Z = _small_code(31, Mb=4, Nb=16, Z=8)
    xa, yb = _frames(base, Z, 6, 0.05, 31)
    syn = core.syndrome(base, Z, xa)
    llr = core.llr_frames(yb, 0.05)
    bits, it, ok, _ = core.decode(base, Z, llr, syn, 12, fold_mode=core.FOLD_MIN)
    for f in range(6):
        b2, i2, o2 = tiny.decode(base, Z, llr[f], syn[f], 12, op=min)
        assert np.array_equal(bits[f], b2) and it[f] == i2 and ok[f] == o2


def test_identity_tables_equal_plain_decoder():
    base, Z = _small_code(41, Mb=8, Nb=32, Z=16)
    xa, yb = _frames(base, Z, 32, 0.04, 41)
    syn = core.syndrome(base, Z, xa)
    llr = core.llr_frames(yb, 0.04)
    a = core.decode(base, Z, llr, syn, 25)
    b = core.decode(base, Z, llr, syn, 25, scale_q4=np.full((25, 8), 16, np.uint8),
                    offset_q=np.zeros((25, 8), np.int8))
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


def test_thread_count_does_not_change_results():
    base, Z = _small_code(51, Mb=8, Nb=32, Z=16)
    xa, yb = _frames(base, Z, 24, 0.05, 51)
    syn = core.syndrome(base, Z, xa)
    llr = core.llr_frames(yb, 0.05)
    a = core.decode(base, Z, llr, syn, 25, threads=1)
    b = core.decode(base, Z, llr, syn, 25, threads=4)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


# ------------------------------------------------------------- rate / efficiency

def test_efficiency_closed_form():
    for R, q, f in golden("efficiency_closed_form.txt"):
        R, q, f = float(R), float(q), float(f)
        assert abs((1 - R) / rate.binary_entropy(q) - f) < 5e-6
        # the same value through the punctured/shortened bookkeeping with p = s = 0
        n = 1000
        m = int(round((1 - R) * n))
        assert abs(rate.efficiency(n, m, 0, 0, q) - f) < 5e-6


@pytest.mark.parametrize("q", [0.01, 0.02, 0.03, 0.05, 0.08])
def test_rate_plan_hits_target_efficiency(q):
    n, m = 49152, 12288
    p, s = rate.rate_plan(n, m, q, 1.1)
    assert p == 0 or s == 0
    f = rate.efficiency(n, m, p, s, q)
    assert abs(f - 1.1) < 1e-3
    R = rate.effective_rate(n, m, p, s)
    assert abs((1 - R) / rate.binary_entropy(q) - f) < 1e-12


def test_position_rank_punctures_low_weight_first():
    base = inputs.qc_base_matrix(6, 12, 4, inputs.mixed_column_degrees(12, 0.3, 3, 6, 1), 1)
    Z = 4
    tb = inputs.tiebreak_permutation(48, 3)
    rk = rate.position_rank(base, Z, tb)
    assert sorted(rk.tolist()) == list(range(48))
    w = np.repeat((base >= 0).sum(axis=0), Z)
    order = np.argsort(rk)
    assert (np.diff(w[order]) >= 0).all()
    st = rate.position_states(rk, 5, 3)
    assert (st == 2).sum() == 3 and (st == 1).sum() == 5
    assert (rk[st == 2].max() < rk[st == 1].min())


def test_scale_offset_table_formula_through_the_decoder():
    """A single check on two variables: each edge receives the other edge's
    magnitude (degree 2: no box-plus at all), so one iteration from LLRs
    (40, -25) leaves E_0 = 40 - t(25) and E_1 = -25 + t(40) with the syndrome
    bit 0, the sign product negative and t(m) = clamp(((m s + 8) >> 4) - o, 0, 127)
    (reading R9).  The decoded bits after one iteration follow t across its
    rounding and its clamp at 0, for scales and offsets around each flip."""
    base = np.array([[0, 0]], dtype=np.int32)
    llr = np.array([[40, -25]], dtype=np.int8)
    syn = np.zeros((1, 1), dtype=np.uint8)

    def t(m, s, o):
        return min(max(((m * s + 8) >> 4) - o, 0), 127)

    for s in range(4, 33):
        for o in range(-3, 45):
            e0, e1 = 40 - t(25, s, o), -25 + t(40, s, o)
            bits, iters, ok, _ = core.decode(base, 1, llr, syn, 1, scale_q4=np.array([[s]], np.uint8),
                                            offset_q=np.array([[o]], np.int8))
            assert list(bits[0]) == [int(e0 < 0), int(e1 < 0)], (s, o)
            assert int(ok[0]) == int((e0 < 0) == (e1 < 0)) and iters[0] == 1


# ------------------------------------------------------------- stall rule

def _stop_iteration(u, K, max_iter):
    """Where the stall rule stops, by its definition, given the unsatisfied
    counts u[t-1] after each iteration t of the plain decoder."""
    best, t_best = None, 0
    for t in range(1, max_iter + 1):
        ut = int(u[t - 1])
        if ut == 0:
            return t, True
        if best is None or ut < best:
            best, t_best = ut, t
        elif t - t_best >= K:
            return t, False
    return max_iter, False


def test_stall_rule_truncates_the_plain_trajectory():
    """The stall rule changes no decoding step, only where it stops: with
    window K the oracle must return the plain decoder's state after the
    iteration the rule's definition picks from the counts of unsatisfied
    checks (taken here from the plain decoder's hard decisions after each
    iteration, stopped there by max_iter, and the dense H)."""
    base, Z = _small_code(21, Mb=8, Nb=32, Z=16)
    H = tiny.dense_h(base, Z).astype(np.int64)
    xa, yb = _frames(base, Z, 24, 0.075, 9)
    syn = core.syndrome(base, Z, xa)
    llr = core.llr_frames(yb, 0.075)
    T = 40
    # the plain decoder's hard decisions after t iterations, for every t
    traj = []
    for t in range(1, T + 1):
        b, it, ok, _ = core.decode(base, Z, llr, syn, t)
        traj.append(b)
    u = np.stack([((b.astype(np.int64) @ H.T) % 2 != syn).sum(axis=1) for b in traj], axis=1)  # [frame][t-1]
    stops = set()
    for K in (1, 3, 6, 12, 41):
        bits, iters, ok, _ = core.decode(base, Z, llr, syn, T, stall_window=K)
        for f in range(len(llr)):
            t_stop, success = _stop_iteration(u[f], K, T)
            assert iters[f] == t_stop and bool(ok[f]) == success, (K, f)
            assert np.array_equal(bits[f], traj[t_stop - 1][f])
            stops.add((K, t_stop < T and not success))
    assert (1, True) in stops and (41, True) not in stops  # both stall stops and none occurred
    # a window longer than the cap is the plain decoder
    b0, i0, o0, _ = core.decode(base, Z, llr, syn, T)
    b1, i1, o1, _ = core.decode(base, Z, llr, syn, T, stall_window=T)
    assert np.array_equal(b0, b1) and np.array_equal(i0, i1) and np.array_equal(o0, o1)

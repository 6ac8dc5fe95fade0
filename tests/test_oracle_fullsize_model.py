"""The C oracle's layered decoder against an independent vectorised model at
the benchmarks' own code sizes: n = 49152 (Z = 512, the PEG mother code of
rate 0.75 with 3/6 column degrees), frames rate-adapted by puncturing and
shortening, one batch that decodes (f = 1.36) and one that cannot (f = 1.1);
and the single-rate n = 40960 code (uniform row draw, rows of 6 to 25
edges) at its QBER of 3 %.  Bits, iteration counts and flags must be equal.

The model restates sections 2 and 3 over whole layers at once: Eq. 8 with
saturation, the row sign as the syndrome bit times the product of the
signs (Eq. 1), the magnitudes as the forward-backward fold of Algorithm 1's
tau (Eq. 7), and Eq. 9 under Algorithm 2.  It shares no code with the
oracle's decoder: tau is tabulated from the hand-pinned pure-Python
Algorithm 1 of ``oracle/tiny.py`` and the rows of H are read off the base
matrix here (row r of a block with shift s holds column (r + s) mod Z)."""
import numpy as np
import pytest

from oracle import core as orc
from oracle import rate as orate
from oracle import tiny
from paper_1903_10107_gb300 import inputs

MSG_MAX = 127


def _case(B, f_target, seed=5, Z=512, Mb=24, Nb=96, scale=1 / 0.29):
    degs = inputs.mixed_column_degrees(Nb, 0.3, 3, 6, seed)
    base = inputs.peg_base_matrix(Mb, Nb, Z, degs, seed)
    n, m = Nb * Z, Mb * Z
    q = inputs.frame_qbers(B, 0.01, 0.08, seed)
    xa = inputs.alice_keys(B, n, seed)
    yb = xa ^ inputs.bsc_noise(B, n, q, seed)
    rank = orate.position_rank(base, Z, inputs.tiebreak_permutation(n, seed))
    plans = [orate.rate_plan(n, m, float(x), f_target) for x in q]
    xa_u, yb_u = inputs.unpack_bits(xa, n), inputs.unpack_bits(yb, n)
    st = np.stack([orate.position_states(rank, int(p), int(s)) for p, s in plans])
    llr = orc.llr_frames(yb_u, q, st, xa_u, scale=scale)
    return base, Z, llr, orc.syndrome(base, Z, xa_u)


def _model(base, Z, llr, syn, max_iter):
    T = np.array([[tiny.tau(p, q) for q in range(128)] for p in range(128)], dtype=np.int32)
    Mb, Nb = base.shape
    B = llr.shape[0]
    r = np.arange(Z)
    layers = []
    for i in range(Mb):
        cols = [k for k in range(Nb) if base[i, k] >= 0]  # ascending variable order within a row
        idx = np.stack([k * Z + (r + int(base[i, k])) % Z for k in cols], axis=1) if cols else None
        layers.append((idx, syn[:, i * Z:(i + 1) * Z].astype(np.int32)))
    E = llr.astype(np.int32).copy()
    L = [None if idx is None else np.zeros((B, Z, idx.shape[1]), np.int32) for idx, _ in layers]
    live = np.ones(B, bool)
    iters = np.zeros(B, np.int32)
    ok = np.zeros(B, np.uint8)
    for it in range(1, max_iter + 1):
        for (idx, sy), Lr in zip(layers, L):
            if idx is None:
                continue
            d = idx.shape[1]
            e = E[:, idx]
            v = np.clip(e - Lr, -127, 127)                  # Eq. 8
            a = np.abs(v)
            neg = (v < 0).astype(np.int32)
            S = (sy + neg.sum(axis=2)) & 1                   # Eq. 1 with the syndrome sign
            F = np.empty_like(a)
            R = np.empty_like(a)
            F[..., 0] = a[..., 0]
            for k in range(1, d):
                F[..., k] = T[F[..., k - 1], a[..., k]]
            R[..., d - 1] = a[..., d - 1]
            for k in range(d - 2, -1, -1):
                R[..., k] = T[a[..., k], R[..., k + 1]]
            mag = np.empty_like(a)
            if d == 1:
                mag[..., 0] = MSG_MAX                        # box-plus over the empty set
            else:
                mag[..., 0] = R[..., 1]
                mag[..., d - 1] = F[..., d - 2]
                for k in range(1, d - 1):
                    mag[..., k] = T[F[..., k - 1], R[..., k + 1]]
            ln = np.where((S[..., None] ^ neg) == 1, -mag, mag)
            en = np.where(np.abs(e) == 127, e, np.clip(v + ln, -127, 127))  # Eq. 9 under Algorithm 2
            keep = ~live[:, None, None]
            E[:, idx] = np.where(keep, e, en)
            Lr[...] = np.where(keep, Lr, ln)
        hard = (E < 0).astype(np.int32)
        unsat = np.zeros(B, np.int64)
        for idx, sy in layers:
            if idx is not None:
                unsat += ((hard[:, idx].sum(axis=2) + sy) & 1).sum(axis=1)
            else:
                unsat += sy.sum(axis=1)
        done = live & (unsat == 0)
        ok[done] = 1
        iters[live] = it
        live &= ~done
        if not live.any():
            break
    return (E < 0).astype(np.uint8), iters, ok


def _plain_case(name, B):
    w = inputs.WORKLOADS[name]
    base = w.base()
    xa, yb, q = w.frames(B)
    xa_u, yb_u = inputs.unpack_bits(xa, w.n), inputs.unpack_bits(yb, w.n)
    return base, w.Z, orc.llr_frames(yb_u, q, scale=w.llr_scale), orc.syndrome(base, w.Z, xa_u)


def test_oracle_equals_vectorised_model_on_the_single_rate_code():
    base, Z, llr, syn = _plain_case("n40960_r080_q03", 2)
    assert (base >= 0).sum(axis=1).max() >= 20   # long rows: folds of 20+ magnitudes
    bits, iters, ok = _model(base, Z, llr, syn, 8)
    ob, oi, ook, _ = orc.decode(base, Z, llr, syn, 8)
    assert np.array_equal(iters, oi) and np.array_equal(ok, ook) and np.array_equal(bits, ob)


@pytest.mark.parametrize("B, f_target, max_iter", [(3, 1.36, 40), (2, 1.1, 12)])
def test_oracle_equals_vectorised_model_at_benchmark_size(B, f_target, max_iter):
    base, Z, llr, syn = _case(B, f_target)
    bits, iters, ok = _model(base, Z, llr, syn, max_iter)
    ob, oi, ook, _ = orc.decode(base, Z, llr, syn, max_iter)
    assert np.array_equal(iters, oi)
    assert np.array_equal(ok, ook)
    assert np.array_equal(bits, ob)
    if f_target > 1.3:
        assert ok.any()       # the decodable batch does decode
    else:
        assert not ok.any()   # below the code's threshold nothing does

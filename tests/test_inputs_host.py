"""The synthetic input recipe: seeded, per-frame reproducible draws with the
shapes and statistics of the workloads (no arithmetic of the method here)."""
import numpy as np
import pytest

from paper_1903_10107_gb300 import inputs


def test_every_frame_regenerates_alone():
    w = inputs.WORKLOADS["n49152_mixed_q01_08"]
    xa, yb, q = w.frames(6)
    for f in range(6):
        xa1, yb1, q1 = w.frames(1, first=f)
        assert np.array_equal(xa1[0], xa[f]) and np.array_equal(yb1[0], yb[f]) and q1[0] == q[f]


@pytest.mark.parametrize("Mb,Nb,Z,deg", [(8, 32, 128, 3), (16, 80, 512, 3), (6, 19, 7, 2)])
def test_base_matrix_column_degrees_and_shifts(Mb, Nb, Z, deg):
    base = inputs.qc_base_matrix(Mb, Nb, Z, deg, 1)
    assert base.shape == (Mb, Nb)
    assert np.all((base >= 0).sum(axis=0) == deg)
    assert base[base >= 0].min() >= 0 and base.max() < Z
    assert np.array_equal(base, inputs.qc_base_matrix(Mb, Nb, Z, deg, 1))  # seeded
    with pytest.raises(ValueError):
        inputs.qc_base_matrix(2, 4, Z, 3, 1)


def test_mixed_code_split_and_edges():
    w = inputs.WORKLOADS["n49152_mixed_q01_08"]
    base = w.base()
    cd = (base >= 0).sum(axis=0)
    assert sorted(set(cd.tolist())) == [3, 6] and (cd == 6).sum() == 29 and (cd == 3).sum() == 67
    assert int((base >= 0).sum()) * w.Z == 192000
    assert w.mask == "peg" and sorted(set((base >= 0).sum(axis=1).tolist())) == [15, 16]
    assert inputs.WORKLOADS["n40960_r080_q03"].mask == "uniform" and inputs.WORKLOADS["n4096_r075_q02"].mask == "uniform"


def _dense_h(base, Z):
    Mb, Nb = base.shape
    H = np.zeros((Mb * Z, Nb * Z), dtype=np.int64)
    for i in range(Mb):
        for j in range(Nb):
            if base[i, j] >= 0:
                for r in range(Z):
                    H[i * Z + r, j * Z + (r + base[i, j]) % Z] = 1
    return H


@pytest.mark.parametrize("Mb,Nb,Z,seed", [(6, 24, 64, 1), (4, 12, 16, 3), (24, 96, 512, 1)])
def test_peg_mask_degrees_and_girth(Mb, Nb, Z, seed):
    """PEG masks: the column degrees asked for, row degrees within one of
    each other, and a lifted graph without 4-cycles (no two rows of H share
    two columns: H H^T has no off-diagonal entry above 1), checked on the
    expanded matrix itself."""
    import scipy.sparse as sp
    degs = inputs.mixed_column_degrees(Nb, 0.3, 2 if Mb < 6 else 3, 4 if Mb < 6 else 6, seed)
    base = inputs.peg_base_matrix(Mb, Nb, Z, degs, seed)
    assert np.array_equal((base >= 0).sum(axis=0), degs)
    rd = (base >= 0).sum(axis=1)
    assert rd.max() - rd.min() <= 1
    assert base[base >= 0].min() >= 0 and base.max() < Z
    assert np.array_equal(base, inputs.peg_base_matrix(Mb, Nb, Z, degs, seed))  # seeded
    if Mb * Z <= 400:
        HH = _dense_h(base, Z) @ _dense_h(base, Z).T
    else:
        rows, cols = [], []
        for i, j in zip(*np.nonzero(base >= 0)):
            r = np.arange(Z)
            rows.append(i * Z + r)
            cols.append(j * Z + (r + base[i, j]) % Z)
        rows, cols = np.concatenate(rows), np.concatenate(cols)
        H = sp.csr_matrix((np.ones(rows.size, np.int64), (rows, cols)), shape=(Mb * Z, Nb * Z))
        HH = (H @ H.T).tocoo()
    if sp.issparse(HH):
        off = HH.row != HH.col
        assert HH.data[off].max() <= 1
    else:
        np.fill_diagonal(HH, 0)
        assert HH.max() <= 1


def test_uniform_draw_has_four_cycles_somewhere():
    """The 4-cycle check above can fail: a uniform draw of the small code
    with few shift values holds 4-cycles."""
    base = inputs.qc_base_matrix(6, 24, 4, 3, 1)
    HH = _dense_h(base, 4) @ _dense_h(base, 4).T
    np.fill_diagonal(HH, 0)
    assert HH.max() >= 2


def test_workload_shapes():
    W = inputs.WORKLOADS
    assert (W["n4096_r075_q02"].Mb, W["n4096_r075_q02"].Nb, W["n4096_r075_q02"].Z) == (8, 32, 128)
    assert (W["n4096_r075_q02"].batch, W["n4096_r075_q02"].max_iter, W["n4096_r075_q02"].qber) == (64, 50, 0.02)
    assert (W["n40960_r080_q03"].Mb, W["n40960_r080_q03"].Nb, W["n40960_r080_q03"].Z) == (16, 80, 512)
    assert (W["n40960_r080_q03"].batch, W["n40960_r080_q03"].max_iter, W["n40960_r080_q03"].qber) == (8192, 100, 0.03)
    m = W["n49152_mixed_q01_08"]
    assert (m.Mb, m.Nb, m.Z, m.batch, m.max_iter, m.qber) == (24, 96, 512, 16384, 200, (0.01, 0.08))
    q = m.qbers()
    assert q.min() >= 0.01 and q.max() < 0.08 and abs(q.mean() - 0.045) < 0.002
    r = W["n4096_relaxed_q02_04"]
    assert (r.n, r.batch, r.max_iter, r.qber) == (4096, 1024, 20, (0.02, 0.04))


def test_noise_rate_and_key_balance():
    w = inputs.WORKLOADS["n4096_r075_q02"]
    xa, yb, _ = w.frames(64)
    e = inputs.unpack_bits(xa ^ yb, w.n)
    k = e.size
    assert abs(e.sum() - 0.02 * k) < 5 * np.sqrt(0.02 * 0.98 * k)
    ones = inputs.unpack_bits(xa, w.n).sum()
    assert abs(ones - 0.5 * k) < 5 * np.sqrt(0.25 * k)


def test_packing_round_trip_and_padding():
    n = 133
    xa = inputs.alice_keys(5, n, 3)
    assert xa.shape == (5, 17) and np.all(xa[:, -1] >> (n % 8) == 0)  # bits past n are zero
    bits = inputs.unpack_bits(xa, n)
    assert bits.shape == (5, n) and np.array_equal(inputs.pack_bits(bits), xa)
    noise = inputs.bsc_noise(5, n, 0.3, 3)
    assert np.all(noise[:, -1] >> (n % 8) == 0)

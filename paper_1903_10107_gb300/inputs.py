"""Seeded synthetic inputs for the reconciliation decoder.

This module holds random draws and bit-format helpers only: quasi-cyclic base
matrices, Alice's keys, the binary-symmetric-channel noise that makes Bob's
keys, per-frame QBERs and tie-break permutations.  It contains none of the
decoder's arithmetic (no syndrome, no LLR quantisation, no check- or
variable-node rule), so both the CUDA path's harness and the CPU oracle's
tests can take their inputs from it without sharing any of the method.

Conventions
-----------
* A base matrix is ``int32[Mb][Nb]``; ``-1`` marks an all-zero Z x Z block,
  any other entry ``s`` in ``[0, Z)`` an identity matrix cyclically shifted by
  ``s`` (the QC-LDPC lifting of the paper's section 4.1).
* Bit vectors are packed LSB-first: bit ``j`` of a frame lives in byte
  ``j >> 3`` at bit position ``j & 7``.
* Every frame ``f`` draws from its own generator ``PCG64([seed, f])`` so any
  frame of a large batch can be regenerated alone.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "generator",
    "qc_base_matrix",
    "peg_base_matrix",
    "mixed_column_degrees",
    "alice_keys",
    "bsc_noise",
    "frame_qbers",
    "tiebreak_permutation",
    "pack_bits",
    "unpack_bits",
    "Workload",
    "WORKLOADS",
]


def generator(*seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(list(seed)))


def qc_base_matrix(Mb: int, Nb: int, Z: int, col_degrees, seed: int) -> np.ndarray:
    """Draw a base matrix whose column ``k`` has ``col_degrees[k]`` nonzero
    blocks in distinct rows chosen uniformly, each with a uniform shift."""
    col_degrees = np.broadcast_to(np.asarray(col_degrees, dtype=np.int64), (Nb,))
    if np.any(col_degrees > Mb) or np.any(col_degrees < 0):
        raise ValueError("column degree out of range")
    g = generator(seed, 0)
    base = np.full((Mb, Nb), -1, dtype=np.int32)
    for k in range(Nb):
        rows = g.choice(Mb, size=int(col_degrees[k]), replace=False)
        shifts = g.integers(0, Z, size=int(col_degrees[k]))
        base[rows, k] = shifts
    return base


def peg_base_matrix(Mb: int, Nb: int, Z: int, col_degrees, seed: int, max_draws: int = 1000) -> np.ndarray:
    """A base matrix whose mask is grown by progressive edge growth (PEG, Hu,
    Eleftheriou and Arnold 2005; the paper builds its masks this way,
    section 4.1) and whose shifts close no 4-cycle in the lifted graph.

    Mask: columns are taken in order of ascending degree (stable).  A
    column's first edge goes to a row of least current degree; each further
    edge to a row as far as possible from the column in the graph built so
    far: a row it cannot reach if there is one, else one of the rows reached
    last by a breadth-first expansion.  Among those the least-degree rows
    qualify; one is drawn uniformly.  This keeps the row degrees within one
    of each other.

    Shifts: edge by edge in the same order, a shift is drawn uniformly from
    ``[0, Z)`` and drawn again while, with two rows i, i' and two columns j,
    j' already holding nonzero blocks, ``s(i,j) - s(i',j) + s(i',j') -
    s(i,j') = 0 (mod Z)`` (the lifted graph would then hold a 4-cycle), so
    the code's girth is at least 6 like the finite-field codes of section 4.1.
    Raises if ``max_draws`` draws of one shift all close a 4-cycle."""
    col_degrees = np.broadcast_to(np.asarray(col_degrees, dtype=np.int64), (Nb,))
    if np.any(col_degrees > Mb) or np.any(col_degrees < 0):
        raise ValueError("column degree out of range")
    g = generator(seed, 7)
    row_deg = np.zeros(Mb, dtype=np.int64)
    col_rows = [[] for _ in range(Nb)]
    row_cols = [[] for _ in range(Mb)]
    order = np.argsort(col_degrees, kind="stable")
    for j in order:
        for k in range(int(col_degrees[j])):
            if k == 0:
                pool = np.arange(Mb)
            else:
                reached = set(col_rows[j])
                seen_cols = {int(j)}
                pool = None
                while True:
                    unreached = [i for i in range(Mb) if i not in reached]
                    if not unreached:
                        break
                    pool = unreached
                    cols = {c for i in reached for c in row_cols[i]} - seen_cols
                    seen_cols |= cols
                    new = {i for c in cols for i in col_rows[c]} - reached
                    if not new:
                        break
                    reached |= new
                pool = np.array(pool, dtype=np.int64)
            pool = pool[row_deg[pool] == row_deg[pool].min()]
            i = int(g.choice(pool))
            col_rows[j].append(i)
            row_cols[i].append(int(j))
            row_deg[i] += 1
    base = np.full((Mb, Nb), -1, dtype=np.int32)
    for j in order:
        for i in col_rows[j]:
            for _ in range(max_draws):
                s = int(g.integers(0, Z))
                if not any((s - base[i2, j] + base[i2, j2] - base[i, j2]) % Z == 0
                           for i2 in col_rows[j] if i2 != i and base[i2, j] >= 0
                           for j2 in row_cols[i] if j2 != j and base[i, j2] >= 0 and base[i2, j2] >= 0):
                    break
            else:
                raise RuntimeError(f"no 4-cycle-free shift for block ({i}, {j}) in {max_draws} draws")
            base[i, j] = s
    return base


def mixed_column_degrees(Nb: int, frac_high: float, d_low: int, d_high: int, seed: int) -> np.ndarray:
    """Column degrees with ``round(frac_high * Nb)`` columns of ``d_high``
    placed by a seeded permutation, the rest ``d_low``."""
    n_high = int(np.floor(frac_high * Nb + 0.5))
    g = generator(seed, 1)
    degs = np.full(Nb, d_low, dtype=np.int64)
    degs[g.permutation(Nb)[:n_high]] = d_high
    return degs


def alice_keys(batch: int, n: int, seed: int, first: int = 0) -> np.ndarray:
    """Uniform random keys, packed: ``uint8[batch][ceil(n/8)]``."""
    nb = (n + 7) // 8
    out = np.empty((batch, nb), dtype=np.uint8)
    for f in range(batch):
        out[f] = generator(seed, 2, first + f).integers(0, 256, size=nb, dtype=np.uint8)
    if n % 8:
        out[:, -1] &= np.uint8((1 << (n % 8)) - 1)
    return out


def bsc_noise(batch: int, n: int, qber, seed: int, first: int = 0) -> np.ndarray:
    """Bernoulli(qber_f) error patterns, packed: ``uint8[batch][ceil(n/8)]``.
    ``qber`` is a scalar or one value per frame."""
    q = np.broadcast_to(np.asarray(qber, dtype=np.float64), (batch,))
    nb = (n + 7) // 8
    out = np.empty((batch, nb), dtype=np.uint8)
    for f in range(batch):
        e = generator(seed, 3, first + f).random(n) < q[f]
        out[f] = np.packbits(e, bitorder="little")
    return out


def frame_qbers(batch: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Per-frame QBER drawn uniformly from ``[lo, hi)``."""
    return generator(seed, 4).uniform(lo, hi, size=batch)


def tiebreak_permutation(n: int, seed: int) -> np.ndarray:
    """A seeded permutation of ``range(n)`` used to break ties between
    positions of equal column weight when choosing punctured positions."""
    return generator(seed, 5).permutation(n).astype(np.int32)


def pack_bits(bits: np.ndarray) -> np.ndarray:
    return np.packbits(np.asarray(bits, dtype=np.uint8), axis=-1, bitorder="little")


def unpack_bits(packed: np.ndarray, n: int) -> np.ndarray:
    return np.unpackbits(np.asarray(packed, dtype=np.uint8), axis=-1, count=n, bitorder="little")


class Workload:
    """Shape and seeds of one synthetic workload (no arithmetic of the method)."""

    def __init__(self, name, Mb, Nb, Z, batch, max_iter, qber, col_degrees,
                 code_seed=1, frame_seed=2, mixed_rate=False, target_f=None, llr_scale=8.0, mask="uniform"):
        self.name = name
        self.Mb, self.Nb, self.Z = Mb, Nb, Z
        self.n, self.m = Nb * Z, Mb * Z
        self.batch, self.max_iter = batch, max_iter
        self.qber = qber            # float, or (lo, hi) for a per-frame uniform draw
        self.col_degrees = col_degrees
        self.code_seed, self.frame_seed = code_seed, frame_seed
        self.mixed_rate = mixed_rate
        self.target_f = target_f
        self.llr_scale = llr_scale  # channel LLR LSB per nat
        if mask not in ("uniform", "peg"):
            raise ValueError("mask must be 'uniform' or 'peg'")
        self.mask = mask            # base-matrix construction: qc_base_matrix or peg_base_matrix

    def base(self) -> np.ndarray:
        degs = self.col_degrees
        if callable(degs):
            degs = degs(self)
        make = peg_base_matrix if self.mask == "peg" else qc_base_matrix
        return make(self.Mb, self.Nb, self.Z, degs, self.code_seed)

    def qbers(self, batch=None, first: int = 0) -> np.ndarray:
        """QBER of frames ``first .. first+batch-1``."""
        b = self.batch if batch is None else batch
        if isinstance(self.qber, tuple):
            return frame_qbers(first + b, self.qber[0], self.qber[1], self.frame_seed)[first:first + b]
        return np.full(b, float(self.qber))

    def frames(self, batch=None, first: int = 0):
        """Alice's keys, Bob's keys (Alice XOR noise), both packed, and the QBERs."""
        b = self.batch if batch is None else batch
        q = self.qbers(b, first)
        xa = alice_keys(b, self.n, self.frame_seed, first)
        yb = xa ^ bsc_noise(b, self.n, q, self.frame_seed, first)
        return xa, yb, q


def _mixed_3_6(w: "Workload") -> np.ndarray:
    return mixed_column_degrees(w.Nb, 0.3, 3, 6, w.code_seed)


WORKLOADS = {
    # single column-3 code, rate 0.75, 64 frames at QBER 2 %
    "n4096_r075_q02": Workload("n4096_r075_q02", 8, 32, 128, 64, 50, 0.02, 3),
    # single column-3 code, rate 0.8, 8192 frames at QBER 3 %
    "n40960_r080_q03": Workload("n40960_r080_q03", 16, 80, 512, 8192, 100, 0.03, 3),
    # 3/6 mixed-degree mother code with a PEG mask (row degrees 15 and 16) and
    # 4-cycle-free shifts, per-frame QBER 1-8 %, per-frame rate for a common
    # efficiency target; LLRs quantised with the step at which the check-node
    # table represents the box-plus (0.29 nat per LSB)
    "n49152_mixed_q01_08": Workload("n49152_mixed_q01_08", 24, 96, 512, 16384, 200, (0.01, 0.08),
                                    _mixed_3_6, mixed_rate=True, target_f=1.7, llr_scale=1 / 0.29, mask="peg"),
    # the n=4096 code at QBER 2-4 %, for the FP32 relaxation
    "n4096_relaxed_q02_04": Workload("n4096_relaxed_q02_04", 8, 32, 128, 1024, 20, (0.02, 0.04), 3),
}

"""Pure-Python references for tiny codes (test infrastructure only).

* :func:`dense_h` -- H written out as a dense 0/1 matrix from the base matrix
  by placing rolled identity blocks (section 4.1), independent of the C
  oracle's row lists.
* :func:`ml_decode` -- maximum-likelihood syndrome decoding on a BSC by
  enumerating every coset member (n <= 20): the word closest to Bob's key
  among all x with H x = s.
* :func:`brute_cn` -- check-node output magnitudes computed edge by edge
  from their definition: for edge k, the left fold of the magnitudes before
  it, the right fold of those after it, and tau of the two (Eq. 7 under the
  forward-backward reading); ``op`` may be ``min`` for textbook min-sum.
* :func:`decode` -- the layered decoder in pure Python for n <= a few
  hundred, used to cross-check the C oracle.
"""
from __future__ import annotations

import numpy as np


def tau(p: int, q: int, msg_max: int = 127) -> int:
    """Algorithm 1, written out."""
    a, b = min(p, msg_max), min(q, msg_max)
    g, l = max(a, b), min(a, b)
    d = g - l
    if l > 2:
        return l - (d < 2) - (d < 6)
    return max(l - (d < 4), 0)


def dense_h(base: np.ndarray, Z: int) -> np.ndarray:
    base = np.asarray(base)
    Mb, Nb = base.shape
    H = np.zeros((Mb * Z, Nb * Z), dtype=np.uint8)
    I = np.eye(Z, dtype=np.uint8)
    for i in range(Mb):
        for k in range(Nb):
            s = int(base[i, k])
            if s >= 0:
                # row r has its one in column (r + s) mod Z
                H[i * Z:(i + 1) * Z, k * Z:(k + 1) * Z] = np.roll(I, s, axis=1)
    return H


_COSETS = {}


def _coset_table(H: np.ndarray):
    """Every word of length n <= 20 with its syndrome, as integers (cached per H)."""
    key = (H.shape, H.tobytes())
    if key not in _COSETS:
        m, n = H.shape
        assert n <= 20
        words = np.arange(1 << n, dtype=np.int64)
        bits = ((words[:, None] >> np.arange(n)) & 1).astype(np.int64)
        syn = (bits @ H.T.astype(np.int64)) % 2
        syn_int = syn @ (1 << np.arange(m, dtype=np.int64))
        _COSETS[key] = (bits.astype(np.uint8), syn_int)
    return _COSETS[key]


def ml_decode(H: np.ndarray, syn: np.ndarray, y: np.ndarray):
    """All minimum-distance coset members (and that distance), by enumerating
    every word of length n <= 20."""
    m, n = H.shape
    bits, syn_all = _coset_table(H)
    s_int = int(np.asarray(syn, dtype=np.int64) @ (1 << np.arange(m, dtype=np.int64)))
    members = bits[syn_all == s_int]
    dist = (members != np.asarray(y, dtype=np.uint8)[None, :]).sum(axis=1)
    best = int(dist.min())
    return best, [w for w in members[dist == best]]


def _fold_left(vals, op):
    acc = vals[0]
    for v in vals[1:]:
        acc = op(acc, v)
    return acc


def _fold_right(vals, op):
    acc = vals[-1]
    for v in reversed(vals[:-1]):
        acc = op(v, acc)
    return acc


def brute_cn(a, op=tau, msg_max: int = 127):
    d = len(a)
    if d == 1:
        return [msg_max]
    out = []
    for k in range(d):
        left, right = list(a[:k]), list(a[k + 1:])
        if not left:
            out.append(_fold_right(right, op))
        elif not right:
            out.append(_fold_left(left, op))
        else:
            out.append(op(_fold_left(left, op), _fold_right(right, op)))
    return out


def decode(base, Z, llr, syn, max_iter, op=tau, msg_max=127, e_max=127):
    """Layered decoding of one frame; returns (bits, iters, ok)."""
    base = np.asarray(base)
    Mb, Nb = base.shape
    E = [int(x) for x in llr]
    rows = []
    for i in range(Mb):
        for r in range(Z):
            rows.append([k * Z + (r + int(base[i, k])) % Z for k in range(Nb) if base[i, k] >= 0])
    L = [[0] * len(js) for js in rows]
    sat = lambda x: max(-127, min(127, x))
    sg = lambda x: -1 if x < 0 else 1
    for t in range(1, max_iter + 1):
        for c, js in enumerate(rows):
            if not js:
                continue
            v = [sat(E[j] - L[c][k]) for k, j in enumerate(js)]
            S = -1 if syn[c] else 1
            for x in v:
                S *= sg(x)
            mags = brute_cn([min(abs(x), msg_max) for x in v], op, msg_max)
            for k, j in enumerate(js):
                ln = S * sg(v[k]) * mags[k]
                if abs(E[j]) != e_max:
                    E[j] = sat(v[k] + ln)
                L[c][k] = ln
        bits = [1 if e < 0 else 0 for e in E]
        if all(sum(bits[j] for j in js) % 2 == syn[c] for c, js in enumerate(rows)):
            return np.array(bits, dtype=np.uint8), t, 1
    return np.array([1 if e < 0 else 0 for e in E], dtype=np.uint8), max_iter, 0

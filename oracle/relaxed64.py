"""FP64 reference of the relaxed (floating-point) layered decoder
(test infrastructure only).

The relaxation keeps the layered schedule of section 2 but computes in
floating point.  Algorithm 1's table is the integer representation of the
box-plus beta of Eq. 6 at its own quantisation step D_t (section 3.2); an
integer decoder fed channel LLRs at a finer step D therefore computes, in
nats, the tempered box-plus

    beta_k(x, y) = k * beta(x / k, y / k),   k = D / D_t,

which is exact belief propagation for k = 1 and tends to min-sum as k -> 0.
The relaxation folds beta_k over the other edges of the row in the same
forward-backward order as the integer decoder (Eq. 7), then scales and
offsets per iteration t and row-degree class c (the normalised/offset forms
listed in section 2):

    mag_k = alpha[t, c] * relu(fold_{k' != k} |L_k'i| - gamma[t, c])

There is no saturation, so Algorithm 2's guard does not apply and the
variable-node update is the plain Eq. 9.  The loss is the mean binary cross
entropy of the final soft values against Alice's bits (soft value E > 0
means bit 0).

A degree-1 row's check node has no other edge: its box-plus is over the
empty set, +infinity, and the integer decoder sends MSG_max (its largest
magnitude, 127 LSB).  +infinity cannot be carried in floating point through
the next E - L of the same edge (it would give infinity - infinity), so the
relaxation sends the finite stand-in EMPTY (a reading).  EMPTY = 50 nats
exceeds the integer decoder's MSG_max in nats at every LLR step used here
(127 * 0.29 = 36.8 at the table's own step, 127 / 8 = 15.9 at 8 LSB per
nat), and well before that nothing else the decoder computes depends on it:
box-plus against such a magnitude returns the other operand up to a term of
order exp(-(EMPTY - other)/kappa).  ``decode``, ``loss`` and
``loss_and_grad`` take it as a parameter so that tests can check that
independence.

``decode`` is numpy; ``loss_and_grad`` builds the same computation from
torch fp64 CPU operations so that autograd supplies a reference gradient.
"""
from __future__ import annotations

import numpy as np


EMPTY = 50.0


def boxplus(x, y, kappa=1.0):
    """beta_k(x, y) = k * beta(x/k, y/k), beta of Eq. 6, for x, y >= 0, in a
    form that stays finite."""
    return np.minimum(x, y) + kappa * (np.log1p(np.exp(-(x + y) / kappa)) - np.log1p(np.exp(-np.abs(x - y) / kappa)))


def layer_tables(base, Z):
    """Per layer: VN index array J[d][Z] (ascending block column), edge
    offset of the layer, degree."""
    base = np.asarray(base)
    Mb, Nb = base.shape
    out, off = [], 0
    r = np.arange(Z)
    for i in range(Mb):
        cols = [k for k in range(Nb) if base[i, k] >= 0]
        J = np.array([k * Z + (r + int(base[i, k])) % Z for k in cols], dtype=np.int64).reshape(len(cols), Z)
        out.append((J, off, len(cols)))
        off += len(cols) * Z
    return out, off


def degree_classes(base):
    """Row-degree class of every layer: index into the sorted distinct degrees."""
    deg = (np.asarray(base) >= 0).sum(axis=1)
    uniq = np.unique(deg[deg > 0])
    cls = np.array([int(np.searchsorted(uniq, d)) if d > 0 else 0 for d in deg])
    return cls, uniq


def _exclusive_boxplus(a, bp, xp):
    """a: [B][d][Z] magnitudes -> exclusive box-plus per edge, forward-backward."""
    d = a.shape[1]
    if d == 1:
        return xp.full_like(a, float("inf"))
    F = [a[:, 0]]
    for k in range(1, d - 1):
        F.append(bp(F[-1], a[:, k]))
    Bk = [None] * d
    Bk[d - 1] = a[:, d - 1]
    for k in range(d - 2, 0, -1):
        Bk[k] = bp(a[:, k], Bk[k + 1])
    outs = [Bk[1]]
    for k in range(1, d - 1):
        outs.append(bp(F[k - 1], Bk[k + 1]))
    outs.append(F[d - 2])
    return xp.stack(outs, axis=1)


def decode(base, Z, llr, syn, iters, alpha=None, gamma=None, stop=False, kappa=1.0, empty=EMPTY):
    """Relaxed layered decoding.  llr: float [B][n] (positive = bit 0),
    syn: 0/1 [B][m].  alpha, gamma: [iters][classes] or None (1, 0).
    Returns the final soft values E [B][n] (and, with stop=True, the
    iteration at which every parity check first held, or iters)."""
    tabs, edges = layer_tables(base, Z)
    cls, uniq = degree_classes(base)
    E = np.array(llr, dtype=np.float64)
    B = E.shape[0]
    L = np.zeros((B, edges))
    ssign = 1.0 - 2.0 * np.asarray(syn, dtype=np.float64)
    done = np.full(B, iters)
    for t in range(iters):
        for i, (J, off, d) in enumerate(tabs):
            if d == 0:
                continue
            sl = slice(off, off + d * Z)
            Lold = L[:, sl].reshape(B, d, Z)
            v = E[:, J] - Lold
            s = np.where(v < 0, -1.0, 1.0)
            S = ssign[:, i * Z:(i + 1) * Z][:, None, :] * np.prod(s, axis=1, keepdims=True)
            mag = _exclusive_boxplus(np.abs(v), lambda a, b: boxplus(a, b, kappa), np)
            al = 1.0 if alpha is None else alpha[t, cls[i]]
            ga = 0.0 if gamma is None else gamma[t, cls[i]]
            if d == 1:
                mag = np.full_like(mag, empty)
            mag = al * np.maximum(mag - ga, 0.0)
            Ln = S * s * mag
            E[:, J] = v + Ln
            L[:, sl] = Ln.reshape(B, d * Z)
        if stop:
            hard = (E < 0).astype(np.int64)
            ok = np.ones(B, dtype=bool)
            for i, (J, off, d) in enumerate(tabs):
                par = hard[:, J].sum(axis=1) % 2 if d else np.zeros((B, Z), np.int64)
                ok &= (par == np.asarray(syn)[:, i * Z:(i + 1) * Z]).all(axis=1)
            done = np.where(ok & (done == iters), t + 1, done)
            if (done < iters).all():
                break
    return (E, done) if stop else E


def loss_and_grad(base, Z, llr, syn, xa, alpha, gamma, kappa=1.0, empty=EMPTY):
    """Mean BCE of the final E against Alice's bits, and its gradient with
    respect to alpha and gamma, by torch fp64 autograd on the CPU."""
    import torch

    tabs, edges = layer_tables(base, Z)
    cls, _ = degree_classes(base)
    T = alpha.shape[0]
    al = torch.tensor(np.asarray(alpha, dtype=np.float64), requires_grad=True)
    ga = torch.tensor(np.asarray(gamma, dtype=np.float64), requires_grad=True)
    E = torch.tensor(np.asarray(llr, dtype=np.float64))
    B = E.shape[0]
    L = torch.zeros((B, edges), dtype=torch.float64)
    ssign = torch.tensor(1.0 - 2.0 * np.asarray(syn, dtype=np.float64))

    def bp(x, y):
        return torch.minimum(x, y) + kappa * (torch.log1p(torch.exp(-(x + y) / kappa))
                                              - torch.log1p(torch.exp(-(x - y).abs() / kappa)))

    for t in range(T):
        for i, (J, off, d) in enumerate(tabs):
            if d == 0:
                continue
            Jt = torch.from_numpy(J)
            Lold = L[:, off:off + d * Z].reshape(B, d, Z)
            v = E[:, Jt] - Lold
            s = torch.where(v < 0, -1.0, 1.0).to(torch.float64)
            S = ssign[:, i * Z:(i + 1) * Z][:, None, :] * torch.prod(s, dim=1, keepdim=True)
            if d == 1:
                mag = torch.full_like(v, empty)
            else:
                mag = _exclusive_boxplus(v.abs(), bp, torch)
            mag = al[t, cls[i]] * torch.relu(mag - ga[t, cls[i]])
            Ln = S * s * mag
            E = E.clone()
            E[:, Jt] = v + Ln
            L = L.clone()
            L[:, off:off + d * Z] = Ln.reshape(B, d * Z)
    sgn = torch.tensor(1.0 - 2.0 * np.asarray(xa, dtype=np.float64))
    loss = torch.nn.functional.softplus(-sgn * E).mean()
    loss.backward()
    return float(loss.detach()), al.grad.numpy().copy(), ga.grad.numpy().copy(), E.detach().numpy()


def loss(base, Z, llr, syn, xa, iters, alpha, gamma, kappa=1.0, empty=EMPTY):
    """The same mean cross entropy from ``decode`` (numpy fp64), for finite
    differences."""
    E = decode(base, Z, llr, syn, iters, alpha, gamma, kappa=kappa, empty=empty)
    x = -(1.0 - 2.0 * np.asarray(xa, dtype=np.float64)) * E
    return float(np.mean(np.maximum(x, 0.0) + np.log1p(np.exp(-np.abs(x)))))

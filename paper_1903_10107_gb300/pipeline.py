"""Bob's side of one reconciliation batch, end to end on the GPU.

``Reconciler`` holds one mother code and its puncturing order.  A call takes
Bob's keys, Alice's syndromes, the per-frame QBERs and the rate-adaptation
counts, quantises the channel LLRs (section 3.1, with the punctured and
shortened positions of section 4.1) and runs the layered int8 decoder
(sections 2 and 3).  ``reconcile_host`` does the same from host buffers,
including the host-device copies.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rate as _rate
from .decoder import QCCode


class Reconciler:
    def __init__(self, base, Z: int, tiebreak=None, device=None, llr_scale: float = 8.0):
        self.code = QCCode(base, Z, device)
        self.device = self.code.device
        self.llr_scale = float(llr_scale)
        self.rank = None
        if tiebreak is not None:
            rk = _rate.puncture_rank(base, Z, tiebreak)
            self.rank = torch.from_numpy(rk).to(self.device)

    @property
    def n(self):
        return self.code.n

    @property
    def m(self):
        return self.code.m

    def plan(self, qber, f_target: float = 1.1):
        return _rate.plan(self.n, self.m, qber, f_target)

    def reconcile(self, bob_bits, syndrome, qber, max_iter, n_punct=None, n_short=None, known=None, out=None):
        """Device tensors in, device tensors out: (bits, iters, ok)."""
        rank = self.rank if (n_punct is not None or n_short is not None) else None
        llr = self.code.llr_from_bsc(bob_bits, qber, rank=rank, n_short=n_short, n_punct=n_punct, known=known,
                                     scale=self.llr_scale)
        return self.code.decode(llr, syndrome, max_iter, out=out)

    def reconcile_host(self, bob_bits, syndrome, qber, max_iter, n_punct=None, n_short=None, known=None):
        """Host tensors (ideally pinned) in, host tensors out.  Returns
        ((bits, iters, ok), h2d_bytes, d2h_bytes)."""
        dev = self.device
        to = lambda t: None if t is None else t.to(dev, non_blocking=True)
        d_in = [to(t) for t in (bob_bits, syndrome, qber, n_punct, n_short, known)]
        h2d = sum(int(t.numel() * t.element_size()) for t in (bob_bits, syndrome, qber, n_punct, n_short, known)
                  if t is not None)
        bits, iters, ok = self.reconcile(d_in[0], d_in[1], d_in[2], max_iter, d_in[3], d_in[4], d_in[5])
        outs = []
        for t in (bits, iters, ok):
            h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
            h.copy_(t, non_blocking=True)
            outs.append(h)
        d2h = sum(int(t.numel() * t.element_size()) for t in outs)
        return tuple(outs), h2d, d2h


def corrected_frames(bits: np.ndarray, ok: np.ndarray, alice: np.ndarray) -> np.ndarray:
    """Frames whose decoder reported success and whose decoded word equals
    Alice's key (undetected errors do not count as corrected)."""
    return (ok.astype(bool)) & np.all(bits == alice, axis=1)

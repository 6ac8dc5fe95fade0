"""Differentiable FP32 relaxation of the layered decoder and learned
check-node tables.

``RelaxedDecodeFn`` is a ``torch.autograd.Function`` whose forward and
backward are the library's ``ldpc_relaxed_forward`` / ``ldpc_relaxed_backward``
kernels (the adjoint recomputes every iteration from iteration-boundary
checkpoints).  ``RelaxedDecoder`` holds one scale and one offset per
iteration and row-degree class.  ``integer_tables`` rounds them into the
integer decoder's tables (``ldpc_decode_batch_ex``):

    scale_q4[t][i] = round(16 * alpha[t][c(i)]),  offset_q[t][i] = round(gamma[t][c(i)] * LSB per nat)

so the integer magnitude becomes clamp(((m * s + 8) >> 4) - o, 0, 127).
"""
from __future__ import annotations

import numpy as np
import torch

from . import native

TABLE_STEP_NAT = 0.29  # step at which Algorithm 1's table represents the box-plus


def degree_classes(base):
    """Class of every layer: index into the sorted distinct row degrees."""
    deg = (np.asarray(base) >= 0).sum(axis=1)
    uniq = np.unique(deg[deg > 0])
    cls = np.array([int(np.searchsorted(uniq, d)) if d > 0 else 0 for d in deg], dtype=np.int32)
    return cls, uniq


def kappa_for_scale(llr_lsb_per_nat: float) -> float:
    """Temperature of the box-plus an integer decoder computes when its LLRs
    use ``llr_lsb_per_nat`` and its table the step TABLE_STEP_NAT."""
    return 1.0 / (llr_lsb_per_nat * TABLE_STEP_NAT)


class RelaxedDecodeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alpha, gamma, code, llr, syn, bits, cls, kappa):
        T, C = alpha.shape
        B, n = llr.shape
        dev = llr.device
        ckE = torch.empty((T + 1, B, n), dtype=torch.float32, device=dev)
        ckL = torch.empty((max(T, 1), B, code.edges), dtype=torch.float32, device=dev)
        loss = torch.zeros(1, dtype=torch.float32, device=dev)
        alpha = alpha.detach().contiguous().float()
        gamma = gamma.detach().contiguous().float()
        st = torch.cuda.current_stream(dev).cuda_stream
        native.ldpc_relaxed_forward(code.handle, llr.data_ptr(), syn.data_ptr(), bits.data_ptr(), B, T,
                                    alpha.data_ptr(), gamma.data_ptr(), cls.data_ptr(), C, float(kappa),
                                    ckE.data_ptr(), ckL.data_ptr(), loss.data_ptr(), st)
        ctx.save_for_backward(alpha, gamma, syn, bits, cls, ckE, ckL)
        ctx.code, ctx.kappa = code, float(kappa)
        final = ckE[T]
        ctx.mark_non_differentiable(final)
        return loss[0], final

    @staticmethod
    def backward(ctx, g_loss, g_final):
        alpha, gamma, syn, bits, cls, ckE, ckL = ctx.saved_tensors
        T, C = alpha.shape
        B = ckE.shape[1]
        dev = alpha.device
        code = ctx.code
        V = torch.empty((B, code.edges), dtype=torch.float32, device=dev)
        gL = torch.empty((B, code.edges), dtype=torch.float32, device=dev)
        ga = torch.empty((T, C), dtype=torch.float32, device=dev)
        gg = torch.empty((T, C), dtype=torch.float32, device=dev)
        st = torch.cuda.current_stream(dev).cuda_stream
        native.ldpc_relaxed_backward(code.handle, syn.data_ptr(), bits.data_ptr(), B, T, alpha.data_ptr(),
                                     gamma.data_ptr(), cls.data_ptr(), C, ctx.kappa, ckE.data_ptr(), ckL.data_ptr(),
                                     V.data_ptr(), gL.data_ptr(), ga.data_ptr(), gg.data_ptr(), None, st)
        return g_loss * ga, g_loss * gg, None, None, None, None, None, None


class RelaxedDecoder(torch.nn.Module):
    """Learnable per-iteration, per-degree-class scale and offset of the
    relaxed decoder for one code."""

    def __init__(self, code, iters: int, kappa: float = 1.0):
        super().__init__()
        self.code = code
        self.iters = int(iters)
        self.kappa = float(kappa)
        cls, uniq = degree_classes(code.base)
        self.degrees = uniq
        self.register_buffer("cls", torch.from_numpy(cls).to(code.device))
        C = len(uniq)
        self.alpha = torch.nn.Parameter(torch.ones((self.iters, C), device=code.device))
        self.gamma = torch.nn.Parameter(torch.zeros((self.iters, C), device=code.device))

    def forward(self, llr, syn, bits):
        """Mean cross entropy of the final soft values, and those values."""
        return RelaxedDecodeFn.apply(self.alpha, self.gamma, self.code, llr, syn, bits, self.cls, self.kappa)

    def integer_tables(self, llr_lsb_per_nat: float):
        """Round into ldpc_decode_batch_ex tables: (scale_q4 uint8[T][Mb], offset_q int8[T][Mb])."""
        cls = self.cls.cpu().numpy()
        a = self.alpha.detach().cpu().numpy()[:, cls]
        g = self.gamma.detach().cpu().numpy()[:, cls]
        rhaz = lambda x: np.sign(x) * np.floor(np.abs(x) + 0.5)
        sq = np.clip(rhaz(16.0 * a), 0, 255).astype(np.uint8)
        oq = np.clip(rhaz(g * llr_lsb_per_nat), -128, 127).astype(np.int8)
        return sq, oq


def bsc_llr_nats(bob_bits_unpacked: np.ndarray, qber) -> np.ndarray:
    """Unquantised channel LLRs (1 - 2y) ln((1-q)/q), float32, for training."""
    q = np.asarray(qber, dtype=np.float64).reshape(-1, 1)
    return ((1.0 - 2.0 * bob_bits_unpacked) * np.log((1.0 - q) / q)).astype(np.float32)

"""PyTorch front end of the decoder library.

``QCCode`` wraps one code handle.  Its methods check device, dtype, shape and
contiguity of torch tensors, allocate outputs with torch (so device memory
comes from PyTorch's caching allocator) and call the C ABI on the current
CUDA stream.  Every computation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import native


def _dev_ptr(t: torch.Tensor | None, name: str, dtype, device, shape=None) -> int:
    if t is None:
        return None
    if not t.is_cuda or t.device != device:
        raise ValueError(f"{name} must be a CUDA tensor on {device}")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def _host_ptr(t, name: str, dtype, shape=None) -> int:
    """Address of a contiguous host tensor (ideally pinned) or numpy array."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        t = torch.from_numpy(t)
    if t.is_cuda:
        raise ValueError(f"{name} must be in host memory")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def llr_magnitudes(qber, scale: float) -> np.ndarray:
    """Per-frame channel-LLR magnitudes (section 3.1), ``int8[B]``, computed
    on the host by the library (``ldpc_llr_magnitudes``) from host QBERs."""
    q = np.ascontiguousarray(np.atleast_1d(np.asarray(qber, dtype=np.float64)))
    out = np.empty(q.size, dtype=np.int8)
    native.ldpc_llr_magnitudes(q.ctypes.data, int(q.size), float(scale), out.ctypes.data)
    return out


class QCCode:
    """A quasi-cyclic LDPC code (section 4.1) resident on one GPU.

    ``base`` is ``int32[Mb][Nb]`` with ``-1`` for zero blocks and shifts in
    ``[0, Z)``; row ``r`` of block row ``i`` connects to variable
    ``k*Z + (r + base[i, k]) mod Z``."""

    def __init__(self, base, Z: int, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        base = np.ascontiguousarray(base, dtype=np.int32)
        if base.ndim != 2:
            raise ValueError("base must be a 2-D matrix")
        self.base = base
        self.Mb, self.Nb = base.shape
        self.Z = int(Z)
        with torch.cuda.device(self.device):
            self.handle = native.ldpc_code_create(base.ctypes.data, self.Mb, self.Nb, self.Z)
        self.n, self.m, self.edges, self.max_row_deg = native.ldpc_code_info(self.handle)
        self.nbytes = (self.n + 7) // 8
        self.mbytes = (self.m + 7) // 8

    def close(self):
        if getattr(self, "handle", None):
            native.ldpc_code_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def reserve(self, batch: int) -> None:
        with torch.cuda.device(self.device):
            native.ldpc_code_reserve(self.handle, int(batch))

    # ------------------------------------------------------------ kernels
    def syndrome(self, bits: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """H x mod 2 of packed bits ``uint8[B][ceil(n/8)]`` -> ``uint8[B][ceil(m/8)]``."""
        B = bits.shape[0]
        _dev_ptr(bits, "bits", torch.uint8, self.device, (B, self.nbytes))
        if out is None:
            out = torch.empty((B, self.mbytes), dtype=torch.uint8, device=self.device)
        _dev_ptr(out, "out", torch.uint8, self.device, (B, self.mbytes))
        native.ldpc_syndrome(self.handle, bits.data_ptr(), B, out.data_ptr(), self._stream())
        return out

    def llr_from_bsc(self, bob_bits, llr_mag, rank=None, n_short=None, n_punct=None, known=None,
                     out=None) -> torch.Tensor:
        """Quantised channel LLRs ``int8[B][n]`` (section 3.1) with punctured and
        shortened positions (section 4.1); ``llr_mag`` is the device copy of
        ``llr_magnitudes(qber, scale)``."""
        B = bob_bits.shape[0]
        _dev_ptr(bob_bits, "bob_bits", torch.uint8, self.device, (B, self.nbytes))
        _dev_ptr(llr_mag, "llr_mag", torch.int8, self.device, (B,))
        rp = _dev_ptr(rank, "rank", torch.int32, self.device, (self.n,))
        sp = _dev_ptr(n_short, "n_short", torch.int32, self.device, (B,))
        pp = _dev_ptr(n_punct, "n_punct", torch.int32, self.device, (B,))
        kp = _dev_ptr(known, "known", torch.uint8, self.device, (B, self.nbytes))
        if out is None:
            out = torch.empty((B, self.n), dtype=torch.int8, device=self.device)
        _dev_ptr(out, "out", torch.int8, self.device, (B, self.n))
        native.ldpc_llr_from_bsc(self.handle, bob_bits.data_ptr(), llr_mag.data_ptr(), rp, sp, pp, kp, B,
                                 out.data_ptr(), self._stream())
        return out

    def decode(self, llr: torch.Tensor, syndrome: torch.Tensor, max_iter: int, scale_q4=None, offset_q=None,
               words: int = 0, out=None):
        """Layered int8 decoding; returns ``(bits uint8[B][ceil(n/8)], iters
        int32[B], ok uint8[B])``."""
        B = llr.shape[0]
        _dev_ptr(llr, "llr", torch.int8, self.device, (B, self.n))
        _dev_ptr(syndrome, "syndrome", torch.uint8, self.device, (B, self.mbytes))
        sq = _dev_ptr(scale_q4, "scale_q4", torch.uint8, self.device, (max_iter, self.Mb))
        oq = _dev_ptr(offset_q, "offset_q", torch.int8, self.device, (max_iter, self.Mb))
        if out is None:
            out = (torch.empty((B, self.nbytes), dtype=torch.uint8, device=self.device),
                   torch.empty((B,), dtype=torch.int32, device=self.device),
                   torch.empty((B,), dtype=torch.uint8, device=self.device))
        bits, iters, ok = out
        _dev_ptr(bits, "out bits", torch.uint8, self.device, (B, self.nbytes))
        _dev_ptr(iters, "out iters", torch.int32, self.device, (B,))
        _dev_ptr(ok, "out ok", torch.uint8, self.device, (B,))
        st = self._stream()
        with torch.cuda.device(self.device):
            if sq is not None or oq is not None:
                if words:
                    raise ValueError("words cannot be combined with tables")
                native.ldpc_decode_batch_ex(self.handle, llr.data_ptr(), syndrome.data_ptr(), B, int(max_iter), sq, oq,
                                            bits.data_ptr(), iters.data_ptr(), ok.data_ptr(), st)
            elif words:
                native.ldpc_decode_batch_words(self.handle, llr.data_ptr(), syndrome.data_ptr(), B, int(max_iter),
                                               int(words), bits.data_ptr(), iters.data_ptr(), ok.data_ptr(), st)
            else:
                native.ldpc_decode_batch(self.handle, llr.data_ptr(), syndrome.data_ptr(), B, int(max_iter),
                                         bits.data_ptr(), iters.data_ptr(), ok.data_ptr(), st)
        return bits, iters, ok


    def reserve_persistent(self, list_len: int, words: int = 0, ctas_per_sm: int = 0, threads: int = 0) -> None:
        with torch.cuda.device(self.device):
            native.ldpc_code_reserve_persistent(self.handle, int(list_len), int(words), int(ctas_per_sm), int(threads))

    def reconcile_persistent(self, bob_bits, llr_mag, syndrome, max_iter: int, rank=None, n_short=None, n_punct=None,
                             known=None, frame_list=None, stall_window: int = 0, words: int = 0,
                             ctas_per_sm: int = 0, threads: int = 0, out=None):
        """Fused LLR quantisation + layered decoding in one persistent launch
        (frames indexed by id; ``frame_list`` selects which to decode).
        Returns ``(bits, iters, ok)`` indexed by frame id."""
        B = bob_bits.shape[0]
        _dev_ptr(bob_bits, "bob_bits", torch.uint8, self.device, (B, self.nbytes))
        _dev_ptr(llr_mag, "llr_mag", torch.int8, self.device, (B,))
        _dev_ptr(syndrome, "syndrome", torch.uint8, self.device, (B, self.mbytes))
        rp = _dev_ptr(rank, "rank", torch.int32, self.device, (self.n,))
        sp = _dev_ptr(n_short, "n_short", torch.int32, self.device, (B,))
        pp = _dev_ptr(n_punct, "n_punct", torch.int32, self.device, (B,))
        kp = _dev_ptr(known, "known", torch.uint8, self.device, (B, self.nbytes))
        if frame_list is not None:
            lp = _dev_ptr(frame_list, "frame_list", torch.int32, self.device)
            nl = int(frame_list.numel())
        else:
            lp, nl = None, B
        if out is None:
            out = (torch.zeros((B, self.nbytes), dtype=torch.uint8, device=self.device),
                   torch.zeros((B,), dtype=torch.int32, device=self.device),
                   torch.zeros((B,), dtype=torch.uint8, device=self.device))
        bits, iters, ok = out
        _dev_ptr(bits, "out bits", torch.uint8, self.device, (B, self.nbytes))
        _dev_ptr(iters, "out iters", torch.int32, self.device, (B,))
        _dev_ptr(ok, "out ok", torch.uint8, self.device, (B,))
        with torch.cuda.device(self.device):
            native.ldpc_reconcile_persistent(self.handle, bob_bits.data_ptr(), llr_mag.data_ptr(), rp, sp, pp, kp,
                                             syndrome.data_ptr(), B, lp, nl, int(max_iter), int(stall_window),
                                             int(words), int(ctas_per_sm), int(threads), bits.data_ptr(),
                                             iters.data_ptr(), ok.data_ptr(), self._stream())
        return bits, iters, ok


    def reconcile_interactive(self, bob_bits, llr_mag, syndrome, max_iter: int, rank, n_short, n_punct, known,
                              reveal, frame_list=None, stall_window: int = 0, words: int = 0, ctas_per_sm: int = 0,
                              threads: int = 0, out=None):
        """All interactive rounds in one persistent launch
        (``ldpc_reconcile_interactive``): ``n_short``/``n_punct`` are round
        0's counts, ``reveal`` ``int32[B][max_rounds + 1]`` the cumulative
        revealed bits per round.  Returns ``(bits, iters, ok, rounds)``
        indexed by frame id (iterations summed over rounds)."""
        B = bob_bits.shape[0]
        R = int(reveal.shape[1]) - 1
        _dev_ptr(bob_bits, "bob_bits", torch.uint8, self.device, (B, self.nbytes))
        _dev_ptr(llr_mag, "llr_mag", torch.int8, self.device, (B,))
        _dev_ptr(syndrome, "syndrome", torch.uint8, self.device, (B, self.mbytes))
        _dev_ptr(rank, "rank", torch.int32, self.device, (self.n,))
        _dev_ptr(n_short, "n_short", torch.int32, self.device, (B,))
        _dev_ptr(n_punct, "n_punct", torch.int32, self.device, (B,))
        _dev_ptr(known, "known", torch.uint8, self.device, (B, self.nbytes))
        _dev_ptr(reveal, "reveal", torch.int32, self.device, (B, R + 1))
        if frame_list is not None:
            lp = _dev_ptr(frame_list, "frame_list", torch.int32, self.device)
            nl = int(frame_list.numel())
        else:
            lp, nl = None, B
        if out is None:
            out = (torch.zeros((B, self.nbytes), dtype=torch.uint8, device=self.device),
                   torch.zeros((B,), dtype=torch.int32, device=self.device),
                   torch.zeros((B,), dtype=torch.uint8, device=self.device),
                   torch.zeros((B,), dtype=torch.int32, device=self.device))
        bits, iters, ok, rounds = out
        _dev_ptr(bits, "out bits", torch.uint8, self.device, (B, self.nbytes))
        _dev_ptr(iters, "out iters", torch.int32, self.device, (B,))
        _dev_ptr(ok, "out ok", torch.uint8, self.device, (B,))
        _dev_ptr(rounds, "out rounds", torch.int32, self.device, (B,))
        with torch.cuda.device(self.device):
            native.ldpc_reconcile_interactive(self.handle, bob_bits.data_ptr(), llr_mag.data_ptr(), rank.data_ptr(),
                                              n_short.data_ptr(), n_punct.data_ptr(), known.data_ptr(),
                                              syndrome.data_ptr(), B, lp, nl, int(max_iter), int(stall_window),
                                              reveal.data_ptr(), R, int(words), int(ctas_per_sm), int(threads),
                                              bits.data_ptr(), iters.data_ptr(), ok.data_ptr(), rounds.data_ptr(),
                                              self._stream())
        return bits, iters, ok, rounds

    def reconcile_interactive_host(self, bob_bits, llr_mag, syndrome, max_iter: int, rank, n_short, n_punct, known,
                                   reveal, frame_list=None, stall_window: int = 0, words: int = 0,
                                   ctas_per_sm: int = 0, threads: int = 0, out=None):
        """``reconcile_interactive`` from host buffers
        (``ldpc_reconcile_interactive_host``): every argument a contiguous
        host tensor or numpy array (pinned memory copies asynchronously), the
        copies to and from the device made by the library.  ``out``: host
        ``(bits, iters, ok, rounds)`` tensors, or None for new ones.
        Returns ``(bits, iters, ok, rounds, h2d_bytes, d2h_bytes)``."""
        B = int(bob_bits.shape[0])
        R = int(reveal.shape[1]) - 1
        args = [_host_ptr(bob_bits, "bob_bits", torch.uint8, (B, self.nbytes)),
                _host_ptr(llr_mag, "llr_mag", torch.int8, (B,)),
                _host_ptr(rank, "rank", torch.int32, (self.n,)),
                _host_ptr(n_short, "n_short", torch.int32, (B,)),
                _host_ptr(n_punct, "n_punct", torch.int32, (B,)),
                _host_ptr(known, "known", torch.uint8, (B, self.nbytes)),
                _host_ptr(syndrome, "syndrome", torch.uint8, (B, self.mbytes))]
        rv = _host_ptr(reveal, "reveal", torch.int32, (B, R + 1))
        if frame_list is not None:
            lp, nl = _host_ptr(frame_list, "frame_list", torch.int32), int(frame_list.shape[0])
        else:
            lp, nl = None, B
        if out is None:
            out = (torch.zeros((B, self.nbytes), dtype=torch.uint8), torch.zeros((B,), dtype=torch.int32),
                   torch.zeros((B,), dtype=torch.uint8), torch.zeros((B,), dtype=torch.int32))
        bits, iters, ok, rounds = out
        op = [_host_ptr(bits, "out bits", torch.uint8, (B, self.nbytes)),
              _host_ptr(iters, "out iters", torch.int32, (B,)), _host_ptr(ok, "out ok", torch.uint8, (B,)),
              _host_ptr(rounds, "out rounds", torch.int32, (B,))]
        h2d, d2h = ctypes.c_int64(0), ctypes.c_int64(0)
        with torch.cuda.device(self.device):
            native.ldpc_reconcile_interactive_host(self.handle, *args, B, lp, nl, int(max_iter), int(stall_window), rv,
                                                   R, int(words), int(ctas_per_sm), int(threads), *op,
                                                   ctypes.addressof(h2d), ctypes.addressof(d2h), self._stream())
        return bits, iters, ok, rounds, int(h2d.value), int(d2h.value)


    def epoch_state_bytes(self, words: int, ctas_per_sm: int = 0, threads: int = 0):
        """(bytes, grid) of the lane-state buffer of ``reconcile_epoch`` for a launch shape."""
        with torch.cuda.device(self.device):
            return native.ldpc_epoch_state_bytes(self.handle, int(words), int(ctas_per_sm), int(threads))

    def reconcile_epoch(self, bob_bits, llr_mag, syndrome, max_iter: int, lane_state, frame_list, list_len: int,
                        epoch_iters: int, resume: bool, out, claimed, rank=None, n_short=None, n_punct=None,
                        known=None, stall_window: int = 0, words: int = 1, ctas_per_sm: int = 0, threads: int = 0):
        """One epoch of the continuously batched decode (``ldpc_reconcile_epoch``):
        per-frame arrays indexed by pool slot; ``frame_list[:list_len]`` the
        slots this epoch may start; ``lane_state`` a uint8 device buffer of
        ``epoch_state_bytes`` bytes; ``out`` (bits, iters, ok) per slot;
        ``claimed`` int32[1] receives how many list entries lanes took."""
        B = bob_bits.shape[0]
        _dev_ptr(bob_bits, "bob_bits", torch.uint8, self.device, (B, self.nbytes))
        _dev_ptr(llr_mag, "llr_mag", torch.int8, self.device, (B,))
        _dev_ptr(syndrome, "syndrome", torch.uint8, self.device, (B, self.mbytes))
        rp = _dev_ptr(rank, "rank", torch.int32, self.device, (self.n,))
        sp = _dev_ptr(n_short, "n_short", torch.int32, self.device, (B,))
        pp = _dev_ptr(n_punct, "n_punct", torch.int32, self.device, (B,))
        kp = _dev_ptr(known, "known", torch.uint8, self.device, (B, self.nbytes))
        lp = _dev_ptr(frame_list, "frame_list", torch.int32, self.device)
        if int(list_len) > frame_list.numel():
            raise ValueError("list_len exceeds frame_list")
        _dev_ptr(lane_state, "lane_state", torch.uint8, self.device)
        bits, iters, ok = out
        _dev_ptr(bits, "out bits", torch.uint8, self.device, (B, self.nbytes))
        _dev_ptr(iters, "out iters", torch.int32, self.device, (B,))
        _dev_ptr(ok, "out ok", torch.uint8, self.device, (B,))
        _dev_ptr(claimed, "claimed", torch.int32, self.device, (1,))
        with torch.cuda.device(self.device):
            native.ldpc_reconcile_epoch(self.handle, bob_bits.data_ptr(), llr_mag.data_ptr(), rp, sp, pp, kp,
                                        syndrome.data_ptr(), B, lp, int(list_len), int(max_iter), int(stall_window),
                                        int(epoch_iters), 1 if resume else 0, lane_state.data_ptr(),
                                        int(lane_state.numel()), int(words), int(ctas_per_sm), int(threads),
                                        bits.data_ptr(), iters.data_ptr(), ok.data_ptr(), claimed.data_ptr(),
                                        self._stream())
        return out


def tau_table_device(device=None) -> torch.Tensor:
    """The decoder's byte-lane tau evaluated on the GPU for all (p, q) < 128."""
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    out = torch.empty(128 * 128, dtype=torch.uint8, device=device)
    with torch.cuda.device(device):
        native.ldpc_debug_tau_table(out.data_ptr(), torch.cuda.current_stream(device).cuda_stream)
    return out.view(128, 128)

"""Bob's side of one reconciliation batch, end to end on the GPU.

``Reconciler`` holds one mother code and its puncturing order.  A call takes
Bob's keys, Alice's syndromes, the per-frame QBERs and the rate-adaptation
counts, quantises the channel LLRs (section 3.1, with the punctured and
shortened positions of section 4.1) and runs the layered int8 decoder
(sections 2 and 3).  ``reconcile_host`` does the same from host buffers,
including the host-device copies; ``reconcile_host_stream`` does it for a
sequence of batches with the copies overlapped with decoding.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import rate as _rate
from .decoder import QCCode, llr_magnitudes


class Reconciler:
    def __init__(self, base, Z: int, tiebreak=None, device=None, llr_scale: float = 8.0):
        self.code = QCCode(base, Z, device)
        self.device = self.code.device
        self.llr_scale = float(llr_scale)
        self.rank = self.rank_host = None
        if tiebreak is not None:
            self.rank_host = np.ascontiguousarray(_rate.puncture_rank(base, Z, tiebreak), dtype=np.int32)
            self.rank = torch.from_numpy(self.rank_host).to(self.device)

    @property
    def n(self):
        return self.code.n

    @property
    def m(self):
        return self.code.m

    def plan(self, qber, f_target: float = 1.1):
        return _rate.plan(self.n, self.m, qber, f_target)

    def magnitudes(self, qber) -> np.ndarray:
        """Host int8 channel-LLR magnitudes of host QBERs at this reconciler's
        LSB-per-nat scale (computed by the library on the host)."""
        return llr_magnitudes(np.asarray(qber, dtype=np.float64), self.llr_scale)

    def reconcile(self, bob_bits, syndrome, llr_mag, max_iter, n_punct=None, n_short=None, known=None, out=None):
        """Device tensors in, device tensors out: (bits, iters, ok).
        ``llr_mag``: device int8 per-frame magnitudes (``magnitudes``)."""
        rank = self.rank if (n_punct is not None or n_short is not None) else None
        llr = self.code.llr_from_bsc(bob_bits, llr_mag, rank=rank, n_short=n_short, n_punct=n_punct, known=known)
        return self.code.decode(llr, syndrome, max_iter, out=out)

    def reconcile_persistent(self, bob_bits, syndrome, llr_mag, max_iter, n_punct=None, n_short=None, known=None,
                             frame_list=None, stall_window=0, words=0, ctas_per_sm=0, threads=0, out=None):
        """The same step as ``reconcile`` in one persistent launch with the LLR
        quantisation fused into the decoder."""
        rank = self.rank if (n_punct is not None or n_short is not None) else None
        return self.code.reconcile_persistent(bob_bits, llr_mag, syndrome, max_iter, rank=rank, n_short=n_short,
                                              n_punct=n_punct, known=known, frame_list=frame_list,
                                              stall_window=stall_window, words=words, ctas_per_sm=ctas_per_sm,
                                              threads=threads, out=out)

    def reconcile_host(self, bob_bits, syndrome, qber, max_iter, n_punct=None, n_short=None, known=None,
                       persistent=False, words=0, ctas_per_sm=0):
        """Host tensors (ideally pinned) in, host tensors out.  Returns
        ((bits, iters, ok), h2d_bytes, d2h_bytes).  The per-frame LLR
        magnitudes are computed on the host from ``qber`` and copied in with
        the other inputs.  The persistent launch claims frames hardest first
        (order computed here from the host-side rate counts and QBERs)."""
        dev = self.device
        order = None
        if persistent and n_punct is not None and n_short is not None:
            order = torch.from_numpy(hardest_first(n_punct.numpy(), n_short.numpy(), qber.numpy()))
        to = lambda t: None if t is None else t.to(dev, non_blocking=True)
        mag = torch.from_numpy(self.magnitudes(qber.numpy()))
        ins = (bob_bits, syndrome, mag, n_punct, n_short, known, order)
        d_in = [to(t) for t in ins]
        h2d = sum(int(t.numel() * t.element_size()) for t in ins if t is not None)
        if persistent:
            bits, iters, ok = self.reconcile_persistent(d_in[0], d_in[1], d_in[2], max_iter, d_in[3], d_in[4],
                                                        d_in[5], frame_list=d_in[6], words=words,
                                                        ctas_per_sm=ctas_per_sm)
        else:
            bits, iters, ok = self.reconcile(d_in[0], d_in[1], d_in[2], max_iter, d_in[3], d_in[4], d_in[5])
        outs = []
        for t in (bits, iters, ok):
            h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
            h.copy_(t, non_blocking=True)
            outs.append(h)
        d2h = sum(int(t.numel() * t.element_size()) for t in outs)
        return tuple(outs), h2d, d2h

    def reconcile_host_stream(self, batches, max_iter, persistent=False, words=0, ctas_per_sm=0):
        """``reconcile_host`` over a sequence of batches with the copies
        overlapped with decoding.  Each batch is a tuple of host tensors
        (ideally pinned) as for ``reconcile_host``: bob_bits, syndrome, qber
        and optionally n_punct, n_short, known, all batches of one shape.

        The LLR magnitudes of each batch are computed on the host from its
        QBERs and copied in with its other inputs (one byte per frame).

        Two device slots alternate.  Batch k's inputs are copied in on one
        copy stream while batch k-1 decodes; its results are copied out on a
        second copy stream while batch k+1 decodes; CUDA events order every
        reuse of a slot, the host never waits inside the loop.  Returns, per
        batch, ((bits, iters, ok) host tensors, h2d_bytes, d2h_bytes); all
        results are complete when the call returns."""
        dev = self.device
        comp = torch.cuda.current_stream(dev)
        h2d_s, d2h_s = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        slots = [None, None]    # (device inputs, device outputs) per slot
        freed = [None, None]    # slot's last decode done: its inputs may be overwritten
        drained = [None, None]  # slot's outputs copied out: they may be overwritten
        results = []
        for k, batch in enumerate(batches):
            s = k & 1
            bob, syn, q, npn, ns, kn = (tuple(batch) + (None,) * 6)[:6]
            order = None
            if persistent and npn is not None and ns is not None:
                order = torch.from_numpy(hardest_first(npn.numpy(), ns.numpy(), q.numpy())).pin_memory()
            mag = torch.from_numpy(self.magnitudes(q.numpy())).pin_memory()
            ins = (bob, syn, mag, npn, ns, kn, order)
            if slots[s] is None:
                d_in = [None if t is None else torch.empty(t.shape, dtype=t.dtype, device=dev) for t in ins]
                B = bob.shape[0]
                d_out = (torch.empty((B, self.code.nbytes), dtype=torch.uint8, device=dev),
                         torch.empty((B,), dtype=torch.int32, device=dev),
                         torch.empty((B,), dtype=torch.uint8, device=dev))
                slots[s] = (d_in, d_out)
            d_in, d_out = slots[s]
            with torch.cuda.stream(h2d_s):
                if freed[s] is not None:
                    h2d_s.wait_event(freed[s])
                for d, h in zip(d_in, ins):
                    if h is not None:
                        d.copy_(h, non_blocking=True)
                ready = torch.cuda.Event()
                ready.record(h2d_s)
            comp.wait_event(ready)
            if drained[s] is not None:
                comp.wait_event(drained[s])
            if persistent:
                self.reconcile_persistent(d_in[0], d_in[1], d_in[2], max_iter, d_in[3], d_in[4], d_in[5],
                                          frame_list=d_in[6], words=words, ctas_per_sm=ctas_per_sm, out=d_out)
            else:
                self.reconcile(d_in[0], d_in[1], d_in[2], max_iter, d_in[3], d_in[4], d_in[5], out=d_out)
            done = torch.cuda.Event()
            done.record(comp)
            freed[s] = done
            with torch.cuda.stream(d2h_s):
                d2h_s.wait_event(done)
                outs = []
                for t in d_out:
                    h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                    h.copy_(t, non_blocking=True)
                    outs.append(h)
                dr = torch.cuda.Event()
                dr.record(d2h_s)
                drained[s] = dr
            h2d = sum(int(t.numel() * t.element_size()) for t in ins if t is not None)
            d2h = sum(int(t.numel() * t.element_size()) for t in outs)
            results.append((tuple(outs), h2d, d2h))
        d2h_s.synchronize()
        h2d_s.synchronize()
        comp.synchronize()
        return results


def hardest_first(n_punct, n_short, qber) -> np.ndarray:
    """Frame order for the persistent launch: descending punctured count
    (puncturing is what makes a frame slow or fail at a given efficiency),
    then descending QBER."""
    return np.lexsort((-np.asarray(qber), -np.asarray(n_punct))).astype(np.int32)


def corrected_frames(bits: np.ndarray, ok: np.ndarray, alice: np.ndarray) -> np.ndarray:
    """Frames whose decoder reported success and whose decoded word equals
    Alice's key (undetected errors do not count as corrected)."""
    return (ok.astype(bool)) & np.all(bits == alice, axis=1)


class MixedRateBatch:
    """One persistent launch over a batch of frames of mixed rates, QBERs and
    iteration counts (section 4.1 rate adaptation on one mother code),
    replayed from a CUDA graph.

    ``bind`` fixes the device buffers (Bob's keys, Alice's syndromes, LLR
    magnitudes, rate counts, shortened values, outputs), picks the launch
    shape with the autotuner, reserves the scratch arena and captures the
    launch; ``run`` replays it on the current stream."""

    def __init__(self, rec: Reconciler, max_iter: int, use_graph: bool = True, tune: bool = True,
                 words: int = 0, ctas_per_sm: int = 0, threads: int = 0, stall_window: int = 0,
                 tune_tag: str = ""):
        self.rec = rec
        self.code = rec.code
        self.max_iter = int(max_iter)
        self.stall_window = int(stall_window)
        self.use_graph = use_graph
        self.tune, self.tune_tag = tune, tune_tag
        self.words, self.ctas, self.threads = words, ctas_per_sm, threads
        self.graph = None

    def _launch(self, words, ctas, threads, n_frames=None):
        b = self.buffers
        sl = (lambda t: t) if n_frames is None else (lambda t: None if t is None else t[:n_frames])
        out = self.out if n_frames is None else tuple(t[:n_frames] for t in self.out)
        order = self.order if n_frames is None else None
        return self.code.reconcile_persistent(sl(b["bob"]), sl(b["mag"]), sl(b["syn"]), self.max_iter,
                                              rank=self.rec.rank if b["n_punct"] is not None else None,
                                              n_short=sl(b["n_short"]), n_punct=sl(b["n_punct"]),
                                              known=sl(b["known"]), frame_list=order,
                                              stall_window=self.stall_window, words=words, ctas_per_sm=ctas,
                                              threads=threads, out=out)

    def bind(self, bob, syn, llr_mag, n_punct=None, n_short=None, known=None, order=None):
        """``llr_mag``: device int8 per-frame magnitudes.  ``order``: optional
        host array, the order in which lanes take the frames.  Frames likely
        to need many iterations (most punctured) should come first, so that
        their long decodes overlap the rest instead of running alone at the
        end of the launch."""
        from . import autotune
        B = bob.shape[0]
        self.buffers = dict(bob=bob, syn=syn, mag=llr_mag, n_punct=n_punct, n_short=n_short, known=known)
        self.order = None if order is None else torch.from_numpy(
            np.ascontiguousarray(order, dtype=np.int32)).to(self.code.device)
        dev = self.code.device
        self.out = (torch.zeros((B, self.code.nbytes), dtype=torch.uint8, device=dev),
                    torch.zeros((B,), dtype=torch.int32, device=dev),
                    torch.zeros((B,), dtype=torch.uint8, device=dev))
        if self.tune and not self.words:
            self.words, self.ctas, self.threads = autotune.tune_persistent(
                self.code, lambda w, c, t, nf: self._launch(w, c, t, nf), B, sample_frames=min(B, 4096),
                tag=self.tune_tag)
        self.code.reserve_persistent(B, self.words, self.ctas, self.threads)
        self._launch(self.words, self.ctas, self.threads)  # eager run: warms the kernel and checks arguments
        torch.cuda.synchronize(dev)
        if self.use_graph:
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream(dev)
            s.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.stream(s):
                with torch.cuda.graph(g, stream=s):
                    self._launch(self.words, self.ctas, self.threads)
            torch.cuda.current_stream(dev).wait_stream(s)
            self.graph = g
        return self

    def run(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._launch(self.words, self.ctas, self.threads)
        return self.out


class InteractiveProtocol:
    """Interactive rate adaptation (sections 4.1 and 4.2): every frame starts
    at the rate for ``f_start``; after each round the frames whose syndrome
    did not match get more bits revealed -- first the punctured positions,
    which become shortened, then key positions in the same order -- and are
    decoded again, up to ``max_rounds`` extra rounds.  Each reveal adds
    ``ceil(df * key_bits * h(q))`` bits.  While punctured positions remain
    this raises the frame's efficiency by about ``df``; revealed key positions
    leave the key instead of adding to the leak, which raises it by only about
    ``f * df * h(q)``.  The efficiency of a frame counts every revealed bit:
    leak = m - p0 + revealed punctured bits, key = n - p0 - s0 - revealed
    key bits, f = leak / (key * h(q)).

    The reveal schedule of a frame depends only on its QBER and starting
    counts, so it is computed up front (``reveal_table``).  By default all
    rounds run in one persistent launch (``ldpc_reconcile_interactive``): a
    frame that fails a round is rebuilt in its lane at the next round's
    state, so rounds of different frames overlap.  With ``fused=False``
    every round is its own launch over the frames still failing (the host
    reads the flags between rounds).  Both give the same per-frame results;
    frames are taken most punctured / highest QBER first.
    ``stall_window`` is the decoder's stall rule (0 = stop only at a syndrome
    match or max_iter).  With ``timing`` the launches are bracketed by CUDA
    events on the current stream and ``run`` reports their summed device
    time."""

    def __init__(self, rec: Reconciler, max_iter: int, f_start: float = 1.1, df: float = 0.1,
                 max_rounds: int = 6, stall_window: int = 0, words: int = 0, ctas_per_sm: int = 0,
                 threads: int = 0, fused: bool = True):
        self.rec, self.code = rec, rec.code
        self.max_iter = int(max_iter)
        self.f_start, self.df, self.max_rounds = float(f_start), float(df), int(max_rounds)
        self.stall_window = int(stall_window)
        self.words, self.ctas, self.threads = words, ctas_per_sm, threads
        self.fused = bool(fused)

    def tune(self, bob, syn, qber_host, known, sample_frames: int = 4096):
        """Pick the launch shape (words, CTAs per SM, threads) with the
        autotuner, timing the protocol's launch (every round, or the first
        one when rounds are separate launches) on the first
        ``sample_frames`` frames; cached per code shape, batch bucket,
        f_start, stall window and round form.  Returns the chosen triple."""
        from . import autotune
        dev = self.code.device
        q = np.asarray(qber_host, dtype=np.float64)
        B = q.size
        p0, s0, rev = self.reveal_table(q)
        c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        d_mag, d_p0, d_s0 = c(self.rec.magnitudes(q)), c(p0.astype(np.int32)), c(s0.astype(np.int32))
        d_rev = c(rev.astype(np.int32))
        out = (torch.zeros((B, self.code.nbytes), dtype=torch.uint8, device=dev),
               torch.zeros((B,), dtype=torch.int32, device=dev),
               torch.zeros((B,), dtype=torch.uint8, device=dev),
               torch.zeros((B,), dtype=torch.int32, device=dev))

        def launch(words, ctas, threads, nf):
            sl = lambda t: t[:nf]
            kw = dict(stall_window=self.stall_window, words=words, ctas_per_sm=ctas, threads=threads)
            if self.fused:
                self.code.reconcile_interactive(sl(bob), sl(d_mag), sl(syn), self.max_iter, self.rec.rank,
                                                sl(d_s0), sl(d_p0), sl(known), sl(d_rev),
                                                out=tuple(sl(t) for t in out), **kw)
            else:
                self.code.reconcile_persistent(sl(bob), sl(d_mag), sl(syn), self.max_iter, rank=self.rec.rank,
                                               n_short=sl(d_s0), n_punct=sl(d_p0), known=sl(known),
                                               out=tuple(sl(t) for t in out[:3]), **kw)
        tag = f"interactive_f{self.f_start}_k{self.stall_window}_{'fused' if self.fused else 'rounds'}"
        self.words, self.ctas, self.threads = autotune.tune_persistent(
            self.code, launch, B, sample_frames=min(B, sample_frames), tag=tag)
        return self.words, self.ctas, self.threads

    def reveal_table(self, qber_host):
        """(p0, s0, rev): round 0's punctured and shortened counts for f_start
        and rev[f][r], the bits revealed to frame f before round r
        (cumulative; each round adds ceil(df * key bits * h(q)), key bits
        being the frame's key length at that point)."""
        n, m = self.code.n, self.code.m
        q = np.asarray(qber_host, dtype=np.float64)
        p0, s0 = _rate.plan(n, m, q, self.f_start)
        key0 = _rate.key_bits(n, p0, s0)
        rev = np.zeros((q.size, self.max_rounds + 1), np.int64)
        for r in range(self.max_rounds):
            kb = key0 - np.maximum(rev[:, r] - p0, 0)
            rev[:, r + 1] = rev[:, r] + np.ceil(self.df * kb * _rate.h2(q)).astype(np.int64)
        return p0, s0, rev

    def _finish(self, q, p0, s0, revealed, bits, iters, okd, rounds, h2d, d2h, events):
        n, m = self.code.n, self.code.m
        key0 = _rate.key_bits(n, p0, s0)
        rp = np.minimum(revealed, p0)
        key = key0 - (revealed - rp)
        f = (m - p0 + rp) / (key * _rate.h2(q))
        res = dict(bits=bits, iters=iters, ok=okd, rounds=rounds, revealed=revealed, key_bits=key, f=f,
                   h2d_bytes=h2d, d2h_bytes=d2h)
        if events is not None:
            torch.cuda.synchronize(self.code.device)
            res["kernel_s"] = sum(a.elapsed_time(b) for a, b in events) / 1e3
            res["launches"] = len(events)
        return res

    def run(self, bob, syn, qber_host, known, timing: bool = False, bits_out=None):
        """bob, syn, known: device tensors for all frames; qber_host: numpy.
        Returns dict of host arrays: bits, iters (summed over rounds), ok,
        rounds (the last round decoded), revealed, key_bits, f; the
        host<->device bytes of the rounds' control (h2d_bytes, d2h_bytes);
        with ``timing`` also kernel_s (summed device time of the decoder
        launches) and launches.

        ``bits_out`` selects where the corrected keys go: None copies them
        to a new host array; ``"device"`` leaves them on the device
        (``res["bits"]`` is then the device tensor and d2h_bytes excludes
        them); a uint8 host tensor of shape (frames, ceil(n/8)), ideally
        pinned, receives them (``res["bits"]`` is its numpy view, valid
        until the buffer is reused)."""
        if self.fused:
            return self._run_fused(bob, syn, qber_host, known, timing, bits_out)
        return self._run_rounds(bob, syn, qber_host, known, timing, bits_out)

    @staticmethod
    def _bits_to(bits, bits_out):
        """(bits where ``bits_out`` asks, bytes copied to the host)."""
        if isinstance(bits_out, str):
            if bits_out != "device":
                raise ValueError(f"bits_out must be None, 'device' or a host tensor, not {bits_out!r}")
            return bits, 0
        if bits_out is None:
            h = bits.cpu().numpy()
            return h, h.nbytes
        if tuple(bits_out.shape) != tuple(bits.shape) or bits_out.dtype != bits.dtype or bits_out.is_cuda:
            raise ValueError("bits_out must be a host uint8 tensor of shape (frames, ceil(n/8))")
        bits_out.copy_(bits, non_blocking=bits.is_cuda and bits_out.is_pinned())
        if bits.is_cuda:
            torch.cuda.current_stream(bits.device).synchronize()
        return bits_out.numpy(), int(bits.numel())

    def _stage(self, key, a):
        """Numpy array ``a`` copied into a page-locked host tensor kept per
        key (reused while the shape and type stay), so that the control
        arrays of a step move by DMA.  Every caller synchronises before the
        next step, so a buffer is never overwritten while a copy reads it."""
        a = np.ascontiguousarray(a)
        cache = self.__dict__.setdefault("_pinned", {})
        t = cache.get(key)
        if t is None or tuple(t.shape) != a.shape or t.numpy().dtype != a.dtype:
            t = torch.from_numpy(np.empty_like(a))
            if torch.cuda.is_available():
                t = t.pin_memory()
            cache[key] = t
        t.numpy()[...] = a
        return t

    def _run_fused(self, bob, syn, qber_host, known, timing, bits_out=None):
        dev = self.code.device
        q = np.asarray(qber_host, dtype=np.float64)
        B = q.size
        p0, s0, rev = self.reveal_table(q)
        c = lambda k, a: self._stage(k, a).to(dev, non_blocking=True)
        d_mag, d_p0 = c("mag", self.rec.magnitudes(q)), c("p0", p0.astype(np.int32))
        d_s0, d_rev = c("s0", s0.astype(np.int32)), c("rev", rev.astype(np.int32))
        d_list = c("list", hardest_first(p0, s0, q).astype(np.int32))
        h2d = B + 8 * B + 4 * rev.size + 4 * B
        events = None
        if timing:
            stream = torch.cuda.current_stream(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        bits, iters, ok, rounds = self.code.reconcile_interactive(
            bob, d_mag, syn, self.max_iter, self.rec.rank, d_s0, d_p0, known, d_rev, frame_list=d_list,
            stall_window=self.stall_window, words=self.words, ctas_per_sm=self.ctas, threads=self.threads)
        if timing:
            e1.record(stream)
            events = [(e0, e1)]
        iters, ok, rounds = (t.cpu().numpy() for t in (iters, ok, rounds))
        bits, d2h = self._bits_to(bits, bits_out)
        d2h += 4 * B + B + 4 * B
        revealed = rev[np.arange(B), rounds]
        return self._finish(q, p0, s0, revealed, bits, iters.astype(np.int64), ok, rounds, h2d, d2h, events)

    def _run_fused_host(self, bob_h, syn_h, qber_host, known_h, timing, bits_out):
        """All rounds in one launch from host buffers through
        ``ldpc_reconcile_interactive_host``: the library copies the inputs in
        and the results out."""
        q = np.asarray(qber_host, dtype=np.float64)
        B = q.size
        p0, s0, rev = self.reveal_table(q)
        out = (bits_out if bits_out is not None else torch.zeros((B, self.code.nbytes), dtype=torch.uint8),
               torch.zeros((B,), dtype=torch.int32), torch.zeros((B,), dtype=torch.uint8),
               torch.zeros((B,), dtype=torch.int32))
        if timing:
            t0 = time.perf_counter()
        bits, iters, ok, rounds, h2d, d2h = self.code.reconcile_interactive_host(
            bob_h, self._stage("mag", self.rec.magnitudes(q)), syn_h, self.max_iter,
            self._stage("rank", self.rec.rank_host), self._stage("s0", s0.astype(np.int32)),
            self._stage("p0", p0.astype(np.int32)), known_h, self._stage("rev", rev.astype(np.int32)),
            frame_list=self._stage("list", hardest_first(p0, s0, q).astype(np.int32)),
            stall_window=self.stall_window, words=self.words, ctas_per_sm=self.ctas, threads=self.threads, out=out)
        iters, ok, rounds = iters.numpy(), ok.numpy(), rounds.numpy()
        revealed = rev[np.arange(B), rounds]
        res = self._finish(q, p0, s0, revealed, bits.numpy(), iters.astype(np.int64), ok, rounds, 0, 0, None)
        if timing:
            res["call_s"] = time.perf_counter() - t0
            res["launches"] = 1
        return res, h2d, d2h

    def _run_rounds(self, bob, syn, qber_host, known, timing: bool = False, bits_out=None):
        dev = self.code.device
        n, m = self.code.n, self.code.m
        q = np.asarray(qber_host, dtype=np.float64)
        B = q.size
        p0, s0 = _rate.plan(n, m, q, self.f_start)
        n_punct, n_short = p0.astype(np.int32).copy(), s0.astype(np.int32).copy()
        revealed = np.zeros(B, np.int64)
        rounds = np.zeros(B, np.int32)
        iters_total = np.zeros(B, np.int64)
        d_mag = torch.from_numpy(self.rec.magnitudes(q)).to(dev)
        h2d, d2h = B, 0  # control traffic of the rounds: magnitudes, counts and lists in; flags out
        out = (torch.zeros((B, self.code.nbytes), dtype=torch.uint8, device=dev),
               torch.zeros((B,), dtype=torch.int32, device=dev),
               torch.zeros((B,), dtype=torch.uint8, device=dev))
        todo = np.arange(B, dtype=np.int32)
        key0 = _rate.key_bits(n, p0, s0)
        stream = torch.cuda.current_stream(dev) if timing else None
        events = []
        for rnd in range(self.max_rounds + 1):
            d_np = torch.from_numpy(n_punct).to(dev)
            d_ns = torch.from_numpy(n_short).to(dev)
            # the frames still to decode, most punctured / highest QBER first
            d_list = torch.from_numpy(np.ascontiguousarray(
                todo[hardest_first(n_punct[todo], n_short[todo], q[todo])])).to(dev)
            h2d += 8 * B + 4 * todo.size
            if timing:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            self.code.reconcile_persistent(bob, d_mag, syn, self.max_iter, rank=self.rec.rank, n_short=d_ns,
                                           n_punct=d_np, known=known, frame_list=d_list,
                                           stall_window=self.stall_window, words=self.words,
                                           ctas_per_sm=self.ctas, threads=self.threads, out=out)
            if timing:
                e1.record(stream)
                events.append((e0, e1))
            ok = out[2].cpu().numpy()[todo].astype(bool)
            it = out[1].cpu().numpy()[todo]
            d2h += 5 * B
            iters_total[todo] += it
            rounds[todo] = rnd
            todo = todo[~ok]
            if todo.size == 0 or rnd == self.max_rounds:
                break
            # reveal more bits for the frames still failing
            kb = key0[todo] - np.maximum(revealed[todo] - p0[todo], 0)
            r = np.ceil(self.df * kb * _rate.h2(q[todo])).astype(np.int64)
            revealed[todo] += r
            n_short[todo] = (s0[todo] + revealed[todo]).astype(np.int32)
            n_punct[todo] = np.maximum(p0[todo] - revealed[todo], 0).astype(np.int32)
        okd = out[2].cpu().numpy()
        bits, nb = self._bits_to(out[0], bits_out)
        d2h += nb + 5 * B
        return self._finish(q, p0, s0, revealed, bits, iters_total, okd, rounds, h2d, d2h,
                            events if timing else None)

    def run_host(self, bob_h, syn_h, qber_host, known_h, timing: bool = False, bits_out=None):
        """``run`` from host buffers (ideally pinned): Bob's keys, Alice's
        syndromes and the values Alice reveals (her key; only revealed and
        shortened positions are read) are copied to the device, the rounds
        run, and the final bits, iteration counts and flags come back (the
        bits into ``bits_out`` when given, a host uint8 tensor of shape
        (frames, ceil(n/8))).  Returns (result dict as for ``run``,
        h2d_bytes, d2h_bytes).  With all rounds in one launch (the default)
        the library makes the copies itself, through its host-buffer entry
        point ``ldpc_reconcile_interactive_host``; with one launch per round
        the copies are torch copies issued by this Python layer around the
        C-ABI launches."""
        if isinstance(bits_out, str):
            raise ValueError("run_host returns the bits to the host: bits_out must be None or a host tensor")
        if self.fused:
            return self._run_fused_host(bob_h, syn_h, qber_host, known_h, timing, bits_out)
        dev = self.code.device
        d = [t.to(dev, non_blocking=True) for t in (bob_h, syn_h, known_h)]
        h2d = sum(int(t.numel() * t.element_size()) for t in (bob_h, syn_h, known_h))
        res = self.run(d[0], d[1], qber_host, d[2], timing=timing, bits_out=bits_out)
        return res, h2d + res["h2d_bytes"], res["d2h_bytes"]

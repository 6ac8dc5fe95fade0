"""Reconciliation serving loop with continuous batching.

Requests (one key block each) arrive over time.  Every request is decoded in
both directions, as in the bi-directional protocol the paper uses (section
4.1): Bob decodes his key against Alice's syndrome, Alice decodes hers
against Bob's; the block is reconciled if either direction recovers the
other party's key.  Shortened positions hold values both parties know;
punctured positions are the other party's filler (LLR 0).

Scheduling:
  * each code has ``slots_per_code`` slots, each with its own code handle
    (message scratch) and CUDA stream;
  * arrived requests are admitted while the device has free memory for their
    buffers (``torch.cuda.mem_get_info`` minus a reserve, and an optional
    byte budget); the rest wait in arrival order;
  * whenever a slot is idle, the requests admitted for its code are packed
    into one persistent launch (two frames per request, hardest first) with
    their copies in and out on the slot's stream; launches of different
    slots overlap on the device while new requests keep arriving.
  * message state stays on the device for all iterations of a launch.

Per-request results are deterministic: a block decodes to the same bits
whether it runs alone or in a mix.
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import inputs, rate
from .decoder import QCCode, llr_magnitudes
from .pipeline import hardest_first


@dataclass
class Request:
    rid: int
    n: int
    qber: float
    xa: np.ndarray          # Alice's key, packed
    yb: np.ndarray          # Bob's key, packed (shortened positions equal Alice's)
    n_punct: int
    n_short: int
    t_arrival: float
    t_done: float = -1.0
    ok: bool = False
    key_bits: int = 0
    dirs: tuple = ()        # (bob_ok, alice_ok, bob_iters, alice_iters)
    bits: tuple = ()        # decoded (bob, alice), packed


@dataclass
class _Slot:
    code: QCCode
    stream: torch.cuda.Stream
    busy: list = field(default_factory=list)
    event: object = None
    host_out: tuple = ()
    nbytes_held: int = 0
    keep: tuple = ()        # device tensors of the launch in flight


class CodeEntry:
    def __init__(self, name, base, Z, tiebreak, slots, device):
        self.name, self.base, self.Z = name, base, Z
        self.slots = [_Slot(QCCode(base, Z, device), torch.cuda.Stream(device)) for _ in range(slots)]
        code = self.slots[0].code
        self.n, self.m, self.nbytes, self.mbytes = code.n, code.m, code.nbytes, code.mbytes
        self.rank = torch.from_numpy(rate.puncture_rank(base, Z, tiebreak)).to(device)
        self.queue: list = []


class ReconciliationServer:
    def __init__(self, codes, llr_scale: float, max_iter: int, slots_per_code: int = 2, max_batch: int = 512,
                 mem_budget: int = 0, reserve: int = 512 << 20, device=None):
        """codes: {name: (base, Z, tiebreak)}."""
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.codes = {name: CodeEntry(name, b, Z, tb, slots_per_code, self.device) for name, (b, Z, tb) in codes.items()}
        self.by_n = {e.n: e for e in self.codes.values()}
        self.llr_scale, self.max_iter, self.max_batch = float(llr_scale), int(max_iter), int(max_batch)
        self.mem_budget, self.reserve = int(mem_budget), int(reserve)
        self.held = 0

    # ------------------------------------------------------------ memory
    def _need(self, e: CodeEntry, k: int) -> int:
        """Device bytes for the buffers of k requests (2 frames each): keys,
        shortened values, syndromes, per-frame parameters, outputs.  The
        message scratch belongs to the slot's code handle and is reserved once
        (at warm-up), not per request."""
        frames = 2 * k
        return frames * (4 * e.nbytes + 2 * e.mbytes + 8 + 4 + 4 + 4 + 4 + 1)

    def _admissible(self, e: CodeEntry, k: int) -> bool:
        need = self._need(e, k)
        if self.mem_budget and self.held + need > self.mem_budget:
            return False
        free, _ = torch.cuda.mem_get_info(self.device)
        return free - self.reserve >= need

    # ------------------------------------------------------------ launch
    def _launch(self, e: CodeEntry, slot: _Slot, reqs):
        dev = self.device
        k = len(reqs)
        B = 2 * k  # frame 2i: Bob decodes (target s_A); 2i+1: Alice decodes (target s_B)
        with torch.cuda.stream(slot.stream):
            obs = np.empty((B, e.nbytes), np.uint8)
            truth_other = np.empty((B, e.nbytes), np.uint8)
            known = np.empty((B, e.nbytes), np.uint8)
            q = np.empty(B, np.float64)
            npn = np.empty(B, np.int32)
            nsh = np.empty(B, np.int32)
            for i, r in enumerate(reqs):
                obs[2 * i], obs[2 * i + 1] = r.yb, r.xa
                truth_other[2 * i], truth_other[2 * i + 1] = r.xa, r.yb
                known[2 * i] = known[2 * i + 1] = r.xa
                q[2 * i] = q[2 * i + 1] = r.qber
                npn[2 * i] = npn[2 * i + 1] = r.n_punct
                nsh[2 * i] = nsh[2 * i + 1] = r.n_short
            pin = lambda a: torch.from_numpy(a).pin_memory()
            d_obs = pin(obs).to(dev, non_blocking=True)
            d_other = pin(truth_other).to(dev, non_blocking=True)  # the other party's key, for its syndrome
            d_known = pin(known).to(dev, non_blocking=True)
            d_mag = pin(llr_magnitudes(q, self.llr_scale)).to(dev, non_blocking=True)
            d_np = pin(npn).to(dev, non_blocking=True)
            d_ns = pin(nsh).to(dev, non_blocking=True)
            order = torch.from_numpy(hardest_first(npn, nsh, q)).pin_memory().to(dev, non_blocking=True)
            syn = slot.code.syndrome(d_other)  # the syndrome each side receives from the other
            bits, iters, ok = slot.code.reconcile_persistent(d_obs, d_mag, syn, self.max_iter, rank=e.rank,
                                                             n_short=d_ns, n_punct=d_np, known=d_known,
                                                             frame_list=order)
            h_bits = torch.empty(bits.shape, dtype=torch.uint8, pin_memory=True)
            h_iters = torch.empty(iters.shape, dtype=torch.int32, pin_memory=True)
            h_ok = torch.empty(ok.shape, dtype=torch.uint8, pin_memory=True)
            h_bits.copy_(bits, non_blocking=True)
            h_iters.copy_(iters, non_blocking=True)
            h_ok.copy_(ok, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
            # keep device tensors alive until the launch completes
            slot.keep = (d_obs, d_other, d_known, d_mag, d_np, d_ns, order, syn, bits, iters, ok)
        slot.busy, slot.event, slot.host_out = list(reqs), ev, (h_bits, h_iters, h_ok, truth_other)
        slot.nbytes_held = self._need(e, k)
        self.held += slot.nbytes_held

    def _finish(self, e: CodeEntry, slot: _Slot, now: float):
        h_bits, h_iters, h_ok, truth = slot.host_out
        bits, iters, ok = h_bits.numpy(), h_iters.numpy(), h_ok.numpy()
        n = e.n
        for i, r in enumerate(slot.busy):
            res = []
            for d in (0, 1):
                f = 2 * i + d
                good = bool(ok[f]) and np.array_equal(bits[f], truth[f])
                res.append(good)
            r.ok = res[0] or res[1]
            r.key_bits = n - r.n_punct - r.n_short
            r.dirs = (res[0], res[1], int(iters[2 * i]), int(iters[2 * i + 1]))
            r.bits = (bits[2 * i].copy(), bits[2 * i + 1].copy())
            r.t_done = now
        self.held -= slot.nbytes_held
        slot.busy, slot.event, slot.host_out, slot.keep = [], None, (), ()

    # ------------------------------------------------------------ loop
    def serve(self, requests, realtime: bool = True):
        """Serve requests (sorted by t_arrival, seconds from start).  Returns
        the requests with their results and completion times."""
        pending = list(requests)
        t0 = time.perf_counter()
        nxt = 0
        inflight = 0
        while nxt < len(pending) or inflight or any(e.queue for e in self.codes.values()):
            now = time.perf_counter() - t0
            # arrivals
            while nxt < len(pending) and (not realtime or pending[nxt].t_arrival <= now):
                r = pending[nxt]
                if not realtime:
                    r.t_arrival = now
                self.by_n[r.n].queue.append(r)
                nxt += 1
            progressed = False
            # completions
            for e in self.codes.values():
                for s in e.slots:
                    if s.event is not None and s.event.query():
                        self._finish(e, s, time.perf_counter() - t0)
                        inflight -= 1
                        progressed = True
            # launches: admitted requests of a code go to its idle slots
            for e in self.codes.values():
                for s in e.slots:
                    if s.event is None and e.queue:
                        k = min(len(e.queue), self.max_batch)
                        while k > 0 and not self._admissible(e, k):
                            k //= 2
                        if k == 0:
                            continue
                        batch, e.queue = e.queue[:k], e.queue[k:]
                        self._launch(e, s, batch)
                        inflight += 1
                        progressed = True
            if not progressed:
                if inflight == 0:
                    for e in self.codes.values():
                        if e.queue and not self._admissible(e, 1):
                            # nothing in flight will free memory: this request can never start
                            raise RuntimeError(
                                f"serving: a request of code {e.name} needs {self._need(e, 1)} device bytes; "
                                f"the budget ({self.mem_budget or 'none'}) or free memory minus the reserve "
                                f"({self.reserve}) is smaller")
                time.sleep(0.0002)
        torch.cuda.synchronize(self.device)
        return pending


# ---------------------------------------------------------------- workload
SERVING_CODES = {
    "n4096": ("n4096_r075_q02",),
    "n40960": ("n40960_r080_q03",),
    "n49152": ("n49152_mixed_q01_08",),
}


def make_codes():
    out = {}
    for name, (wname,) in SERVING_CODES.items():
        w = inputs.WORKLOADS[wname]
        out[name] = (w.base(), w.Z, inputs.tiebreak_permutation(w.n, w.code_seed))
    return out


def make_requests(count: int, rate_per_s: float, f_target: float, seed: int = 7, codes=None):
    """Poisson arrivals; code uniform over the three lengths; QBER U(1 %, 8 %);
    rate per request for f_target; shortened positions of Bob's key set to
    Alice's values (both know them)."""
    codes = codes or make_codes()
    names = sorted(codes, key=lambda k: codes[k][0].shape[1] * codes[k][1])
    g = inputs.generator(seed, 9)
    gaps = g.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps) - gaps[0]
    which = g.integers(0, len(names), size=count)
    q = g.uniform(0.01, 0.08, size=count)
    reqs = []
    ranks = {}
    for i in range(count):
        name = names[which[i]]
        base, Z, tb = codes[name]
        n, m = base.shape[1] * Z, base.shape[0] * Z
        p, s = rate.plan(n, m, q[i], f_target)
        xa = inputs.alice_keys(1, n, seed + 100, i)[0]
        yb = xa ^ inputs.bsc_noise(1, n, q[i], seed + 100, i)[0]
        if s[0] > 0:
            if name not in ranks:
                ranks[name] = rate.puncture_rank(base, Z, tb)
            sh = inputs.pack_bits((ranks[name] < s[0]).astype(np.uint8))
            yb = (yb & ~sh) | (xa & sh)
        reqs.append(Request(i, n, float(q[i]), xa, yb, int(p[0]), int(s[0]), float(t[i])))
    return reqs


def summarize(reqs, wall_s):
    lat = np.array([r.t_done - r.t_arrival for r in reqs]) * 1e3
    key = sum(r.key_bits for r in reqs if r.ok)
    return {
        "requests": len(reqs), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "max_ms": float(lat.max()), "corrected_key_mbps": key / wall_s / 1e6,
        "fer": 1.0 - float(np.mean([r.ok for r in reqs])),
        "bidirectional_gain": int(sum(1 for r in reqs if r.ok and not r.dirs[0])),
    }


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--duration", type=float, default=3.0)
    ap.add_argument("--f", type=float, default=1.7)
    ap.add_argument("--max-iter", type=int, default=200)
    ap.add_argument("--slots", type=int, default=2)
    args = ap.parse_args(argv)
    codes = make_codes()
    count = int(args.rate * args.duration)
    reqs = make_requests(count, args.rate, args.f, codes=codes)
    srv = ReconciliationServer(codes, llr_scale=1 / 0.29, max_iter=args.max_iter, slots_per_code=args.slots)
    srv.serve(make_requests(64, 1e9, args.f, seed=99, codes=codes), realtime=False)  # warm-up
    t0 = time.perf_counter()
    srv.serve(reqs, realtime=True)
    wall = time.perf_counter() - t0
    out = {"offered_rate_per_s": args.rate, "duration_s": args.duration, "f_target": args.f, "max_iter": args.max_iter,
           "slots_per_code": args.slots, "wall_s": wall, **summarize(reqs, wall)}
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()

"""Reconciliation serving loop: continuous batching with resident decoder state.

Requests (one key block each) arrive over time.  Every request is decoded in
both directions, as in the bi-directional protocol the paper uses (section
4.1): Bob decodes his key against Alice's syndrome, Alice decodes hers
against Bob's; the block is reconciled if either direction recovers the
other party's key.  Shortened positions hold values both parties know;
punctured positions are the other party's filler (LLR 0).

Each code has one ``EpochEngine``: a device-resident pool of frame slots
(inputs and outputs, two slots per request), one code handle whose message
arena holds the lanes' messages, a lane-state buffer, a CUDA stream and
pinned staging buffers, all allocated once.  The engine runs the persistent
decoder in epochs (``ldpc_reconcile_epoch``): every epoch runs a bounded
number of iterations, leaves every unfinished frame's soft values, syndrome
bits and iteration state in device memory and the messages in the arena,
and the next epoch continues them while the lanes that came free take the
requests admitted in between.  So a request that arrives while others are
decoding joins at the next epoch boundary, its work overlaps theirs on the
device, and the engines of the different codes overlap on their streams.

Admission is by device memory: an engine's pool is sized once from the free
device memory (minus a reserve, or an explicit byte budget); a request waits
while its code's pool has no two free slots.

Per-request results are deterministic: a block decodes to the same bits and
iteration counts whether it runs alone or in a mix, whatever epochs its
decode is split into.
"""
from __future__ import annotations

import argparse
import gc
import json
import time
from collections import deque
from dataclasses import dataclass

import numpy as np
import torch

from . import inputs, rate
from .decoder import QCCode, llr_magnitudes


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


def pool_bytes_per_frame(nbytes: int, mbytes: int) -> int:
    """Device bytes of one frame slot: observed key, known values, the other
    party's key (for the syndrome it sends), syndrome, magnitude, two rate
    counts, decoded bits, iteration count, flag; plus the staging row."""
    return 2 * (3 * nbytes + mbytes + 1 + 8) + nbytes + 4 + 1


class EpochEngine:
    """Continuously batched decoding of one code (see the module docstring)."""

    def __init__(self, name, base, Z, tiebreak, device, capacity: int, llr_scale: float, max_iter: int,
                 epoch_iters: int = 8, stall_window: int = 0, words: int = 1, ctas_per_sm: int = 1,
                 threads: int = 0):
        self.name = name
        self.device = torch.device(device)
        self.code = QCCode(base, Z, self.device)
        c = self.code
        self.n, self.m, self.nbytes, self.mbytes = c.n, c.m, c.nbytes, c.mbytes
        self.rank = torch.from_numpy(rate.puncture_rank(base, Z, tiebreak)).to(self.device)
        self.llr_scale, self.max_iter = float(llr_scale), int(max_iter)
        self.epoch_iters, self.stall_window = int(epoch_iters), int(stall_window)
        self.words, self.ctas, self.threads = int(words), int(ctas_per_sm), int(threads)
        P = 2 * max(1, int(capacity) // 2)
        self.capacity = P
        dev = self.device
        z8 = lambda *sh: torch.zeros(sh, dtype=torch.uint8, device=dev)
        z32 = lambda *sh: torch.zeros(sh, dtype=torch.int32, device=dev)
        nb, mb = self.nbytes, self.mbytes
        # the pool (frame slots) and the same-shaped staging rows of one admission
        self.obs, self.known, self.syn = z8(P, nb), z8(P, nb), z8(P, mb)
        self.mag = torch.zeros((P,), dtype=torch.int8, device=dev)
        self.ns, self.np_ = z32(P), z32(P)
        self.out = (z8(P, nb), z32(P), z8(P))
        self.st_obs, self.st_known, self.st_other = z8(P, nb), z8(P, nb), z8(P, nb)
        self.st_mag = torch.zeros((P,), dtype=torch.int8, device=dev)
        self.st_ns, self.st_np = z32(P), z32(P)
        self.d_list, self.d_claimed = z32(P), z32(1)
        pin8 = lambda *sh: torch.zeros(sh, dtype=torch.uint8).pin_memory()
        self.h_obs, self.h_known, self.h_other = pin8(P, nb), pin8(P, nb), pin8(P, nb)
        self.h_mag = torch.zeros((P,), dtype=torch.int8).pin_memory()
        self.h_ns = torch.zeros((P,), dtype=torch.int32).pin_memory()
        self.h_np = torch.zeros((P,), dtype=torch.int32).pin_memory()
        self.h_list = torch.zeros((P,), dtype=torch.int32).pin_memory()
        self.h_slots = torch.zeros((P,), dtype=torch.int64).pin_memory()
        self.h_iters = torch.zeros((P,), dtype=torch.int32).pin_memory()
        self.h_ok = torch.zeros((P,), dtype=torch.uint8).pin_memory()
        self.h_claimed = torch.zeros((1,), dtype=torch.int32).pin_memory()
        self.h_rows = torch.zeros((P,), dtype=torch.int64).pin_memory()  # slots of finished frames
        self.d_rows = torch.zeros((P,), dtype=torch.int64, device=dev)
        self.d_done_bits = z8(P, nb)
        self.h_done_bits = pin8(P, nb)
        state_bytes, self.grid = c.epoch_state_bytes(self.words, self.ctas, self.threads)
        self.lane_state = z8(state_bytes)
        self.stream = torch.cuda.Stream(dev)
        self.free_pairs = deque(range(P // 2))   # request slots: frame slots 2k (Bob) and 2k + 1 (Alice)
        self.queue: deque = deque()              # requests waiting for admission
        self.pending: list = []                  # frame slots admitted but not yet taken by a lane
        self.inflight: dict = {}                 # request slot -> request
        self.event = None
        self.started = False
        self.epochs = 0

    @staticmethod
    def bytes_for(nbytes: int, mbytes: int, frames: int) -> int:
        return frames * pool_bytes_per_frame(nbytes, mbytes)

    # ------------------------------------------------------------ admission
    def admit(self) -> int:
        """Move waiting requests into free slots: stage their rows in pinned
        memory, copy them in, compute each direction's syndrome from the other
        party's key, and place everything in the pool.  Returns how many."""
        k = min(len(self.queue), len(self.free_pairs))
        if k == 0:
            return 0
        reqs = [self.queue.popleft() for _ in range(k)]
        pairs = [self.free_pairs.popleft() for _ in range(k)]
        F = 2 * k
        # frame 2i: Bob decodes his key against s_A; 2i + 1: Alice decodes hers against s_B
        yb = np.stack([r.yb for r in reqs])
        xa = np.stack([r.xa for r in reqs])
        ho, hx, hk = self.h_obs.numpy(), self.h_other.numpy(), self.h_known.numpy()
        ho[0:F:2], ho[1:F:2] = yb, xa
        hx[0:F:2], hx[1:F:2] = xa, yb
        hk[0:F:2], hk[1:F:2] = xa, xa
        two = lambda attr, dt: np.repeat(np.fromiter((getattr(r, attr) for r in reqs), dt, k), 2)
        q = two("qber", np.float64)
        self.h_ns.numpy()[:F] = two("n_short", np.int32)
        self.h_np.numpy()[:F] = two("n_punct", np.int32)
        self.h_mag.numpy()[:F] = llr_magnitudes(q, self.llr_scale)
        slots = np.empty(F, np.int64)
        slots[0::2] = 2 * np.asarray(pairs)
        slots[1::2] = 2 * np.asarray(pairs) + 1
        self.h_slots[:F] = torch.from_numpy(slots)
        with torch.cuda.stream(self.stream):
            for d, h in ((self.st_obs, self.h_obs), (self.st_known, self.h_known), (self.st_other, self.h_other),
                         (self.st_mag, self.h_mag), (self.st_ns, self.h_ns), (self.st_np, self.h_np)):
                d[:F].copy_(h[:F], non_blocking=True)
            d_slots = self.h_slots[:F].to(self.device, non_blocking=True)
            st_syn = self.code.syndrome(self.st_other[:F])  # the syndrome each side receives from the other
            for pool, st in ((self.obs, self.st_obs), (self.known, self.st_known), (self.mag, self.st_mag),
                             (self.ns, self.st_ns), (self.np_, self.st_np)):
                pool.index_copy_(0, d_slots, st[:F])
            self.syn.index_copy_(0, d_slots, st_syn)
            self.out[1].index_fill_(0, d_slots, 0)  # iterations 0 = not finished
        for r, p in zip(reqs, pairs):
            self.inflight[p] = r
        self.pending.extend(slots.tolist())
        return k

    # ------------------------------------------------------------ epochs
    def launch(self) -> bool:
        """Start the next epoch if any frame is waiting or in flight."""
        if self.event is not None or not self.inflight:
            return False
        L = len(self.pending)
        if L:
            self.h_list[:L] = torch.tensor(self.pending, dtype=torch.int32)
        with torch.cuda.stream(self.stream):
            if L:
                self.d_list[:L].copy_(self.h_list[:L], non_blocking=True)
            self.code.reconcile_epoch(self.obs, self.mag, self.syn, self.max_iter, self.lane_state, self.d_list, L,
                                      self.epoch_iters, self.started, self.out, self.d_claimed, rank=self.rank,
                                      n_short=self.ns, n_punct=self.np_, known=self.known,
                                      stall_window=self.stall_window, words=self.words, ctas_per_sm=self.ctas,
                                      threads=self.threads)
            self.h_iters.copy_(self.out[1], non_blocking=True)
            self.h_ok.copy_(self.out[2], non_blocking=True)
            self.h_claimed.copy_(self.d_claimed, non_blocking=True)
            self.event = torch.cuda.Event()
            self.event.record(self.stream)
        self.started = True
        self.epochs += 1
        self._launched = L
        return True

    def poll(self, now: float) -> list:
        """If the epoch in flight has ended: the requests it completed (their
        results filled in), after freeing their slots.  Else []."""
        if self.event is None or not self.event.query():
            return []
        self.event = None
        taken = min(int(self.h_claimed[0]), self._launched)
        self.pending = self.pending[taken:]  # the rest were not reached: next epoch
        iters, ok = self.h_iters.numpy(), self.h_ok.numpy()
        keys = np.fromiter(self.inflight.keys(), np.int64, len(self.inflight))
        fin = keys[(iters[2 * keys] > 0) & (iters[2 * keys + 1] > 0)]
        if fin.size == 0:
            return []
        R = 2 * fin.size
        rows = self.h_rows.numpy()
        rows[0:R:2], rows[1:R:2] = 2 * fin, 2 * fin + 1
        with torch.cuda.stream(self.stream):  # the finished frames' bits, gathered into one copy out
            self.d_rows[:R].copy_(self.h_rows[:R], non_blocking=True)
            torch.index_select(self.out[0], 0, self.d_rows[:R], out=self.d_done_bits[:R])
            self.h_done_bits[:R].copy_(self.d_done_bits[:R], non_blocking=True)
            self.stream.synchronize()
        bits = self.h_done_bits.numpy()[:R].copy()
        reqs = [self.inflight.pop(p) for p in fin.tolist()]
        # a direction succeeds when its decoder matched the syndrome and recovered the other party's key
        good0 = ok[2 * fin].astype(bool) & (bits[0::2] == np.stack([r.xa for r in reqs])).all(axis=1)
        good1 = ok[2 * fin + 1].astype(bool) & (bits[1::2] == np.stack([r.yb for r in reqs])).all(axis=1)
        it0, it1 = iters[2 * fin].tolist(), iters[2 * fin + 1].tolist()
        g0, g1 = good0.tolist(), good1.tolist()
        for i, r in enumerate(reqs):
            r.ok = g0[i] or g1[i]
            r.key_bits = r.n - r.n_punct - r.n_short
            r.dirs = (g0[i], g1[i], it0[i], it1[i])
            r.bits = (bits[2 * i], bits[2 * i + 1])
            r.t_done = now
        self.free_pairs.extend(fin.tolist())
        return reqs

    def idle(self) -> bool:
        return self.event is None and not self.inflight and not self.queue


class ReconciliationServer:
    def __init__(self, codes, llr_scale: float, max_iter: int, epoch_iters: int = 8, stall_window: int = 0,
                 capacity: int = 1024, mem_budget: int = 0, reserve: int = 1 << 30, ctas_per_sm: int = 1,
                 max_epoch_iters: int = 64, device=None):
        """codes: {name: (base, Z, tiebreak)}.  Every code's engine gets a pool
        of up to ``capacity`` frames, fewer if the free device memory minus
        ``reserve`` (or ``mem_budget`` bytes, split over the codes) holds
        fewer; requests beyond the pools wait for admission.  The code with
        the most edges runs ``epoch_iters`` iterations per epoch, the others
        as many more as their iterations are cheaper (the same edge updates
        per epoch), at most ``max_epoch_iters``: an epoch then lasts about as
        long on every code, and a short code's long decodes are not cut into
        many epochs whose host round trips would dominate their latency."""
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        free, _ = torch.cuda.mem_get_info(self.device)
        budget = (free - int(reserve)) if not mem_budget else int(mem_budget)
        share = max(0, budget) // max(1, len(codes))
        edges = {name: int((np.asarray(b) >= 0).sum()) * Z for name, (b, Z, tb) in codes.items()}
        e_max = max(edges.values())
        self.engines = {}
        for name, (b, Z, tb) in codes.items():
            Mb, Nb = np.asarray(b).shape
            iters = int(min(max_epoch_iters, max(1, round(epoch_iters * e_max / max(1, edges[name])))))
            nb, mb = (Nb * Z + 7) // 8, (Mb * Z + 7) // 8
            frames = min(int(capacity), share // pool_bytes_per_frame(nb, mb))
            if frames < 2:
                raise RuntimeError(f"serving: the device memory left for code {name} holds no request "
                                   f"({share} bytes, {2 * pool_bytes_per_frame(nb, mb)} needed)")
            self.engines[name] = EpochEngine(name, b, Z, tb, self.device, frames, llr_scale, max_iter,
                                             epoch_iters=iters, stall_window=stall_window,
                                             ctas_per_sm=ctas_per_sm)
        self.by_n = {e.n: e for e in self.engines.values()}

    def serve(self, requests, realtime: bool = True):
        """Serve requests (sorted by t_arrival, seconds from start).  Returns
        the requests with their results and completion times."""
        pending = list(requests)
        gc_was_on = gc.isenabled()
        gc.disable()  # a cyclic collection in the loop would stall every request in flight
        try:
            self._loop(pending, realtime)
        finally:
            if gc_was_on:
                gc.enable()
        torch.cuda.synchronize(self.device)
        return pending

    def _loop(self, pending, realtime):
        t0 = time.perf_counter()
        nxt = 0
        while nxt < len(pending) or not all(e.idle() for e in self.engines.values()):
            now = time.perf_counter() - t0
            while nxt < len(pending) and (not realtime or pending[nxt].t_arrival <= now):
                r = pending[nxt]
                if not realtime:
                    r.t_arrival = now
                self.by_n[r.n].queue.append(r)
                nxt += 1
            progressed = False
            for e in self.engines.values():
                if e.poll(time.perf_counter() - t0):
                    progressed = True
                if e.event is None:
                    if e.admit():
                        progressed = True
                    if e.launch():
                        progressed = True
            if not progressed:
                time.sleep(0.00005)


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
    ap.add_argument("--epoch-iters", type=int, default=8, help="iterations per epoch of the largest code")
    ap.add_argument("--stall-window", type=int, default=0)
    ap.add_argument("--capacity", type=int, default=1024, help="frame slots per code (two per request)")
    ap.add_argument("--out", default="", help="append the JSON line to this file")
    args = ap.parse_args(argv)
    codes = make_codes()
    count = int(args.rate * args.duration)
    reqs = make_requests(count, args.rate, args.f, codes=codes)
    srv = ReconciliationServer(codes, llr_scale=1 / 0.29, max_iter=args.max_iter, epoch_iters=args.epoch_iters,
                               stall_window=args.stall_window, capacity=args.capacity)
    srv.serve(make_requests(64, 1e9, args.f, seed=99, codes=codes), realtime=False)  # warm-up
    epochs0 = {k: e.epochs for k, e in srv.engines.items()}
    t0 = time.perf_counter()
    srv.serve(reqs, realtime=True)
    wall = time.perf_counter() - t0
    out = {"command": "python -m paper_1903_10107_gb300.serving " + " ".join(argv or []),
           "offered_rate_per_s": args.rate, "duration_s": args.duration, "f_target": args.f,
           "max_iter": args.max_iter, "epoch_iters": {k: e.epoch_iters for k, e in srv.engines.items()},
           "stall_window": args.stall_window,
           "capacity_frames": {k: e.capacity for k, e in srv.engines.items()},
           "epochs": {k: e.epochs - epochs0[k] for k, e in srv.engines.items()},
           "wall_s": wall, **summarize(reqs, wall)}
    print(json.dumps(out), flush=True)
    if args.out:
        with open(args.out, "a") as fh:
            fh.write(json.dumps(out) + "\n")
    return out


if __name__ == "__main__":
    import sys
    main(sys.argv[1:])

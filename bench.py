#!/usr/bin/env python
"""Throughput of Bob's reconciliation step on GB300: corrected-key Mbps.

One step = one pass of the whole hot path over one batch: channel-LLR
quantisation with the batch's punctured/shortened positions, then layered
int8 decoding with per-frame early termination.  Inputs (Bob's keys, Alice's
syndromes, QBERs, rate counts) are resident in device memory when the timed
region starts; ``e2e`` repeats the measurement from pinned host buffers with
the host<->device copies inside the timed region.

Corrected-key Mbps = sum, over frames whose syndrome matched and whose
decoded word equals Alice's key, of the key bits n - p - s, divided by the
step time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the CPU oracle on the same workload
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1903_10107_gb300 import inputs, rate, sharding  # noqa: E402

DEFAULT_WORKLOAD = "n49152_mixed_q01_08"
METRIC = "corrected-key Mbps on 1 GB300 at FER<=1e-2 and f~1.1 (QBER 1-8%); % HBM roofline"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--batch", type=int, default=0, help="override the workload's batch (for small runs)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--max-iter", type=int, default=0, help="override the workload's iteration cap")
    ap.add_argument("--target-f", type=float, default=0.0,
                    help="override the mixed-rate workload's target efficiency (rate plan per frame)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-order", action="store_true", help="persistent launch takes frames in index order")
    ap.add_argument("--protocol", choices=["fixed", "interactive"], default="fixed",
                    help="fixed: one rate per frame for the workload's target f; interactive: rounds of reveal")
    ap.add_argument("--f-start", type=float, default=1.1)
    ap.add_argument("--df", type=float, default=0.1)
    ap.add_argument("--max-rounds", type=int, default=8)
    return ap.parse_args()


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ workload

class Batch:
    """Host-side arrays of one rank's share of the workload."""

    def __init__(self, w, batch, first):
        self.w = w
        self.base = w.base()
        self.xa, self.yb, self.q = w.frames(batch, first)
        self.B = batch
        if w.mixed_rate:
            self.n_punct, self.n_short = rate.plan(w.n, w.m, self.q, w.target_f)
            self.tiebreak = inputs.tiebreak_permutation(w.n, w.code_seed)
        else:
            self.n_punct = np.zeros(batch, np.int32)
            self.n_short = np.zeros(batch, np.int32)
            self.tiebreak = None
        self.key_bits = rate.key_bits(w.n, self.n_punct, self.n_short)
        self.f = rate.efficiency(w.n, w.m, self.n_punct, self.n_short, self.q)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_sources_sha():
    """Hash of the decoder kernels' code, comments and whitespace removed (a
    profile taken before a comment-only edit still describes the kernel)."""
    h = hashlib.sha256()
    for fn in ("decode_int8.cu", "decode_int8.cuh", "decode_persistent.cu", "decode_persistent.cuh", "maxh.cuh",
               "row_update.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1903_10107_gb300", "csrc", fn)) as fh:
            txt = fh.read()
        txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", " ", txt)
        h.update(" ".join(txt.split()).encode())
    return h.hexdigest()[:16]


# Integer work of the method per edge and frame-iteration, in byte operations:
# Eq. 8 (difference, saturation), the sign product of Eq. 1, three box-plus
# evaluations of Algorithm 1 in the forward-backward fold (min, |difference|,
# five range tests, corrections: about 10 each) and Eq. 9 with Algorithm 2's
# guard; about 40 in all.
ALU_OPS_PER_EDGE = 40


def roofline_alu(it_sum, edges, seconds, clk):
    """The integer-issue roofline of the decoder: byte operations of the method
    per second against what the SMs can issue, 152 SMs x 4 schedulers x 32
    lanes x the SM clock seen during the run x 4 byte lanes per 32-bit
    operation (the ALU and FMA pipes each take 16 lanes per scheduler and
    cycle, the scheduler issues one 32-lane instruction per cycle)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    peak = sms * 4 * 32 * float(mhz) * 1e6 * 4 / 1e12
    achieved = ALU_OPS_PER_EDGE * float(edges) * float(it_sum) / seconds / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T byte-op/s", "frac": achieved / peak,
            "ops_per_edge_frame_iteration": ALU_OPS_PER_EDGE,
            "peak_basis": f"{sms} SMs x 4 schedulers x 32 lanes x {float(mhz):.0f} MHz x 4 byte lanes"}


def profiled_traffic(kernel: str, workload: str, launch_frames: int, key: str = "dram_bytes_per_frame"):
    """Bytes per launch from the committed ncu summary of the kernel (DRAM by
    default, ``l2_bytes_per_frame`` for the L2 slices), if it was taken on the
    current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    msha = re.search(r"kernel_sha:\s*([0-9a-f]+)", txt)
    mtr = re.search(key + r":\s*([0-9.eE+]+)", txt)
    if not msha or not mtr or msha.group(1) != kernel_sources_sha():
        return None
    return float(mtr.group(1)) * launch_frames


def measure_l2_copy_gbs(dev, mbytes: int = 24, reps: int = 20) -> float:
    """Copy bandwidth of a buffer that stays in L2 (bytes read + written per
    second, best of five batches of ``reps`` copies, CUDA events): the L2
    counterpart of the HBM copy peak, for kernels whose traffic L2 serves."""
    import torch
    a = torch.ones((mbytes << 20) // 4, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    for _ in range(5):
        b.copy_(a)
    st = torch.cuda.current_stream(dev)
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            b.copy_(a)
        e1.record(st)
        torch.cuda.synchronize(dev)
        best = max(best, 2.0 * a.numel() * 4 * reps / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


# ----------------------------------------------------------------- reference

def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import core as orc
    w = inputs.WORKLOADS[args.workload]
    if args.max_iter:
        w.max_iter = args.max_iter
    if args.target_f and w.mixed_rate:
        w.target_f = args.target_f
    B = args.batch or w.batch
    # size a per-step sample of about (cpu_seconds / (steps + warmup)) of oracle time
    per_step = max(2.0, args.cpu_seconds * 4 / max(1, args.steps + args.warmup))
    res = cpu_oracle_measure(w, B, per_step, orc, steps=args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": res["value"], "unit": "Mbps", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": {"workload": w.name, "frames": B * world, "n": w.n, "m": w.m, "Z": w.Z, "max_iter": w.max_iter,
                   "qber": list(w.qber) if isinstance(w.qber, tuple) else w.qber, "target_f": w.target_f,
                   "llr_lsb_per_nat": round(w.llr_scale, 4), "sample_frames_per_step": res["frames"]},
        "cpu_baseline": {"value": res["value"], "unit": "Mbps", "cores": res["cores"], "kind": "oracle",
                         "sample": res["sample"]},
        "e2e": {"value": res["value"], "unit": "Mbps", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_oracle_measure(w, B, seconds, orc, steps=1, warmup=0):
    """Time the oracle on the first frames of the workload, sized to ~seconds per step."""
    probe = min(B, max(1, orc.num_cores()))
    bt = Batch(w, probe, 0)
    n = w.n
    t0 = time.time()
    _oracle_decode(bt, orc)
    dt = max(time.time() - t0, 1e-3)
    k = int(min(B, max(probe, probe * seconds / dt)))
    bt = Batch(w, k, 0)
    for _ in range(warmup if warmup else 0):
        _oracle_decode(bt, orc, limit=min(k, probe))
    times, corr_bits, cores = [], 0, 1
    for _ in range(max(1, steps)):
        t0 = time.time()
        bits, iters, ok, cores = _oracle_decode(bt, orc)
        times.append(time.time() - t0)
    xa_u = inputs.unpack_bits(bt.xa, n)
    corr = ok.astype(bool) & np.all(bits == xa_u, axis=1)
    corr_bits = int(bt.key_bits[corr].sum())
    t = float(np.mean(times))
    return {"value": corr_bits / t / 1e6, "ms_per_step": t * 1e3, "cores": int(cores), "frames": k,
            "sample": f"first {k} of {B} frames of {w.name}, {len(times)} timed pass(es), "
                      f"mean {t:.2f} s/pass, FER {1 - corr.mean():.3f}"}


def _oracle_decode(bt, orc, limit=None):
    from oracle import rate as orate
    w = bt.w
    k = bt.B if limit is None else limit
    xa_u = inputs.unpack_bits(bt.xa[:k], w.n)
    yb_u = inputs.unpack_bits(bt.yb[:k], w.n)
    syn = orc.syndrome(bt.base, w.Z, xa_u)
    st = kn = None
    if w.mixed_rate:
        rk = orate.position_rank(bt.base, w.Z, bt.tiebreak) if not hasattr(bt, "_orank") else bt._orank
        bt._orank = rk
        st = np.stack([orate.position_states(rk, int(bt.n_punct[f]), int(bt.n_short[f])) for f in range(k)])
        kn = xa_u
    llr = orc.llr_frames(yb_u, bt.q[:k], st, kn, scale=w.llr_scale)
    bits, iters, ok, used = orc.decode(bt.base, w.Z, llr, syn, w.max_iter)
    return bits, iters, ok, used


# ---------------------------------------------------------------------- ours

def measure_e2e(args, rec, bt, d_syn, xa_bits, dev, words=0, ctas=0):
    """Same step through Reconciler.reconcile_host_stream from pinned host buffers."""
    import torch
    w = bt.w
    mixed = w.mixed_rate
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_yb, h_syn, h_q = pin(bt.yb), pin(d_syn.cpu().numpy()), pin(bt.q)
    h_np = pin(bt.n_punct) if mixed else None
    h_ns = pin(bt.n_short) if mixed else None
    h_kn = pin(bt.xa) if mixed else None
    batch = (h_yb, h_syn, h_q, h_np, h_ns, h_kn)
    rec.reconcile_host_stream([batch] * max(2, args.warmup), w.max_iter, persistent=mixed, words=words,
                              ctas_per_sm=ctas)
    torch.cuda.synchronize()
    e2e_steps = max(2, min(args.steps, 5))
    # every step copies its inputs in from pinned host memory and its results
    # out; the copies of one step overlap the decode of its neighbours
    t0 = time.perf_counter()
    out = rec.reconcile_host_stream([batch] * e2e_steps, w.max_iter, persistent=mixed, words=words,
                                    ctas_per_sm=ctas)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    res, h2d, d2h = out[-1]
    e_bits = inputs.unpack_bits(res[0].numpy(), w.n)
    e_corr = res[2].numpy().astype(bool) & np.all(e_bits == xa_bits, axis=1)
    e_key = float(bt.key_bits[e_corr].sum())
    return e2e_s, e_key, h2d, d2h


def run_ours(args, rank, world, dist):
    import torch
    from paper_1903_10107_gb300 import native
    from paper_1903_10107_gb300.pipeline import MixedRateBatch, Reconciler, hardest_first

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = inputs.WORKLOADS[args.workload]
    if args.max_iter:
        w.max_iter = args.max_iter
    if args.target_f and w.mixed_rate:
        w.target_f = args.target_f
    first, B = sharding.weak_shard(args.batch or w.batch, rank, world)  # every rank its own frames
    bt = Batch(w, B, first)
    rec = Reconciler(bt.base, w.Z, bt.tiebreak, dev, llr_scale=w.llr_scale)
    code = rec.code
    # Alice's syndromes (her side of the protocol; computed once, outside the step)
    d_xa = torch.from_numpy(bt.xa).to(dev)
    d_syn = code.syndrome(d_xa)
    d_yb = torch.from_numpy(bt.yb).to(dev)
    d_q = torch.from_numpy(bt.q).to(dev)
    mixed = w.mixed_rate
    d_np = torch.from_numpy(bt.n_punct).to(dev) if mixed else None
    d_ns = torch.from_numpy(bt.n_short).to(dev) if mixed else None
    d_kn = d_xa if mixed else None
    xa_bits = inputs.unpack_bits(bt.xa, w.n)

    if args.protocol == "interactive":
        return run_interactive(args, rank, world, dist, w, bt, rec, d_yb, d_syn, d_xa, xa_bits, dev)

    if mixed:
        # one persistent launch (LLR quantisation fused), replayed from a CUDA graph
        order = None if args.no_order else hardest_first(bt.n_punct, bt.n_short, bt.q)
        mrb = MixedRateBatch(rec, w.max_iter).bind(d_yb, d_syn, d_q, d_np, d_ns, d_kn, order=order)
        l0 = native.ldpc_launch_count()
        mrb._launch(mrb.words, mrb.ctas)
        torch.cuda.synchronize()
        launches_per_step = native.ldpc_launch_count() - l0
        out = mrb.out
        step = mrb.run
        kernel_name = "persistent_kernel"
        shape = {"words_per_cta": mrb.words, "ctas_per_sm": mrb.ctas, "cuda_graph": mrb.graph is not None,
                 "work_order": "given" if order is None else "hardest first"}
    else:
        code.reserve(B)
        out = (torch.empty((B, code.nbytes), dtype=torch.uint8, device=dev),
               torch.empty((B,), dtype=torch.int32, device=dev),
               torch.empty((B,), dtype=torch.uint8, device=dev))

        def step():
            return rec.reconcile(d_yb, d_syn, d_q, w.max_iter, out=out)
        launches_per_step = 2
        kernel_name = "decode_kernel"
        shape = {"cuda_graph": False}

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.current_stream(dev)
    # Bytes one step touches on the device: inputs, message scratch, outputs.
    if mixed:
        msg_bytes = torch.cuda.get_device_properties(dev).multi_processor_count * mrb.ctas * 4 * mrb.words * code.edges
        in_bytes = B * (2 * code.nbytes + code.mbytes + 4 + 16)
    else:
        msg_bytes = B * code.edges
        in_bytes = B * (code.nbytes + code.mbytes + 4 + w.n)
    out_bytes = B * (code.nbytes + 5)
    work_set = in_bytes + msg_bytes + out_bytes
    l2_bytes = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = work_set < 2 * l2_bytes
    flush_buf = torch.empty(2 * l2_bytes if flush else 0, dtype=torch.uint8, device=dev)

    def timed(fn, reps):
        # Device time of `reps` calls of fn on the launching stream.  With a small
        # working set every call runs after a write of twice the L2 size, outside
        # the timed events, so that no call finds its inputs cached by the last.
        if not flush:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / 1e3 / reps
        pairs = []
        for k in range(reps):
            flush_buf.fill_(k & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            pairs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in pairs) / 1e3 / reps

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    l0 = native.ldpc_launch_count()
    step_s = timed(step, args.steps)
    eager_launches = native.ldpc_launch_count() - l0
    barrier()
    clk = clocks.stop()
    # graph replays bypass the library's launch counter: count the kernels the graph holds
    launches = eager_launches if eager_launches else launches_per_step * args.steps

    bits, iters, ok = (t.cpu().numpy() for t in out)
    got_bits = inputs.unpack_bits(bits, w.n)
    corr = ok.astype(bool) & np.all(got_bits == xa_bits, axis=1)
    corr_key = float(bt.key_bits[corr].sum())
    all_key = float(bt.key_bits.sum())

    # the dominant kernel alone, for the roofline (same stream, CUDA events)
    if mixed:
        dec_s = step_s  # the step is the single persistent kernel
    else:
        llr = code.llr_from_bsc(d_yb, d_q)
        for _ in range(2):
            code.decode(llr, d_syn, w.max_iter, out=out)
        torch.cuda.synchronize()
        dec_s = timed(lambda: code.decode(llr, d_syn, w.max_iter, out=out), max(3, args.steps))
    it_sum = float(iters.astype(np.int64).sum())
    if mixed:  # Bob's bits, syndrome, shortened values in; bits, iterations, flag out
        io_bytes = B * (2 * code.nbytes + code.mbytes + code.nbytes + 4 + 1 + 16)
    else:      # int8 LLRs, syndrome in; bits, iterations, flag out
        io_bytes = B * (w.n + code.mbytes + code.nbytes + 4 + 1)
    alg_bytes = it_sum * 2.0 * code.edges + io_bytes
    peak, peak_kind = peaks()
    achieved = alg_bytes / dec_s / 1e9

    # end to end through the public API from pinned host buffers
    e2e_s, e_key, h2d, d2h = float("nan"), 0.0, 0, 0
    if not args.no_e2e:
        e2e_s, e_key, h2d, d2h = measure_e2e(args, rec, bt, d_syn, xa_bits, dev,
                                             shape.get("words_per_cta", 0), shape.get("ctas_per_sm", 0))

    # max over ranks (times), sums over ranks (key bits)
    vals_max, vals_sum = sharding.reduce_max_sum([step_s, e2e_s, dec_s], [corr_key, all_key, e_key], dist, dev)
    step_max, e2e_max = vals_max[0], vals_max[1]
    corr_tot, all_tot, e_tot = vals_sum[0], vals_sum[1], vals_sum[2]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import core as orc
        r = cpu_oracle_measure(w, B, args.cpu_seconds, orc)
        cpu = {"value": r["value"], "unit": "Mbps", "cores": r["cores"], "kind": "oracle", "sample": r["sample"]}

    if rank != 0:
        return
    traffic = profiled_traffic(kernel_name, w.name, B)
    l2_traffic = profiled_traffic(kernel_name, w.name, B, "l2_bytes_per_frame")
    l2 = None
    if l2_traffic is not None:  # the messages are partly served from L2: its share against a measured L2 copy
        l2_peak = measure_l2_copy_gbs(dev)
        l2 = {"achieved": l2_traffic / dec_s / 1e9, "peak": l2_peak, "unit": "GB/s",
              "frac": l2_traffic / dec_s / 1e9 / l2_peak, "traffic": l2_traffic,
              "traffic_source": "lts__t_bytes.sum per launch, committed ncu summary of this kernel source",
              "peak_kind": "measured in this run: device copy of a 24 MB buffer held in L2, best of 5 x 20"}
    line = {
        "metric": METRIC,
        "value": corr_tot / step_max / 1e6,
        "unit": "Mbps",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step_max * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int8",
        "data": "synthetic",
        "config": {
            "workload": w.name, "frames": B * world, "n": w.n, "m": w.m, "Z": w.Z, "max_iter": w.max_iter,
            "qber": list(w.qber) if isinstance(w.qber, tuple) else w.qber,
            "target_f": w.target_f, "llr_lsb_per_nat": round(w.llr_scale, 4),
            "l2": (("L2 flushed before every timed step (%.0f MB write); working set %.1f MB per rank"
                    % (2 * l2_bytes / 1e6, work_set / 1e6)) if flush else
                   ("working set larger than L2, no flush: inputs %.0f MB + message scratch %.0f MB + outputs %.0f MB per rank"
                    % (in_bytes / 1e6, msg_bytes / 1e6, out_bytes / 1e6))),
            "parallelism": f"frames sharded over {world} GPU(s), no collective on the data path",
            **shape,
        },
        "processed_key_mbps": all_tot / step_max / 1e6,
        "fer": 1.0 - float(corr.mean()),
        "efficiency_f_mean": float(np.mean(bt.f)),
        "iters_mean": float(iters.mean()),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": kernel_name, "kernel_ms": dec_s * 1e3,
                     "algorithmic_bytes": alg_bytes, "l2": l2},
        "roofline_alu": roofline_alu(it_sum, code.edges, dec_s, clk),
        "e2e": {"value": e_tot / e2e_max / 1e6, "unit": "Mbps", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "cpu_baseline": cpu,
        "paper_context": "60 Mbps at f~1.1 on an Intel i7-6700HQ (section 4.2, Table 2), other codes and hardware",
    }
    print(json.dumps(line), flush=True)


def run_interactive(args, rank, world, dist, w, bt, rec, d_yb, d_syn, d_xa, xa_bits, dev):
    """Interactive rate adaptation from f_start: rounds of decode + reveal."""
    import torch
    from paper_1903_10107_gb300.pipeline import InteractiveProtocol
    proto = InteractiveProtocol(rec, w.max_iter, f_start=args.f_start, df=args.df, max_rounds=args.max_rounds)
    for _ in range(max(1, args.warmup)):
        proto.run(d_yb, d_syn, bt.q, d_xa)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res = proto.run(d_yb, d_syn, bt.q, d_xa)
    torch.cuda.synchronize()
    step_s = (time.perf_counter() - t0) / args.steps
    got = inputs.unpack_bits(res["bits"], w.n)
    corr = res["ok"].astype(bool) & np.all(got == xa_bits, axis=1)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "protocol": "interactive", "value": float(res["key_bits"][corr].sum()) / step_s / 1e6,
        "unit": "Mbps", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": {"workload": w.name, "frames": bt.B, "f_start": args.f_start, "df": args.df,
                   "max_rounds": args.max_rounds, "max_iter": w.max_iter},
        "fer": 1.0 - float(corr.mean()), "efficiency_f_mean": float(res["f"][corr].mean()) if corr.any() else None,
        "rounds_mean": float(res["rounds"].mean()), "iters_mean_total": float(res["iters"].mean()),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    run_ours(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

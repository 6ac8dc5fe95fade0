#!/usr/bin/env python
"""Throughput of Bob's reconciliation on GB300: corrected-key Mbps.

Default step: the paper's rate-adaptive, interactive protocol (sections 4.1
and 4.2) over one batch of the mixed-rate workload (n = 49152 mother code,
16384 frames, per-frame QBER uniform in 1-8 %).  Every frame starts at the
rate for efficiency f_start = 1.1; each round is one persistent launch of
the layered int8 decoder (channel-LLR quantisation fused) over the frames
still failing, after which those frames have more of their puncturing order
revealed (punctured positions first, then key positions) and are decoded
again.  One step = every round for every frame.  Inputs (Bob's keys,
Alice's syndromes, the values she reveals) are resident in device memory
when the timed region starts; ``e2e`` repeats the step from pinned host
buffers with the host<->device copies inside the timed region.

Corrected-key Mbps = sum, over frames whose syndrome matched and whose
decoded word equals Alice's key, of their final key bits (n - p - s minus
the key positions revealed), divided by the step time.

``--protocol fixed`` times one persistent launch at a fixed rate per frame
for ``--target-f`` instead (also reported as ``fixed_rate`` beside the
default line); the other workloads (``--workload``) are single-code
fixed-rate batches.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--protocol interactive|fixed]
    python bench.py --impl reference ...   # the CPU oracle on the same workload and protocol
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
STALL_WINDOW = 10  # decoder stall rule of the default interactive rounds (0 = off)
METRIC = "corrected-key Mbps on 1 GB300 at FER<=1e-2 and f~1.1 (QBER 1-8%); % HBM roofline"
L2_BYTES = 129 * 10**6  # GB300 L2 (for the flush decision's statement; the device's own size decides the flush)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--batch", type=int, default=0, help="override the workload's batch (for small runs)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--max-iter", type=int, default=0, help="override the workload's iteration cap")
    ap.add_argument("--protocol", choices=["interactive", "fixed"], default="interactive",
                    help="interactive: rounds of decode + reveal from --f-start (mixed-rate workload only); "
                         "fixed: one rate per frame for --target-f")
    ap.add_argument("--f-start", type=float, default=1.1)
    ap.add_argument("--df", type=float, default=0.1)
    ap.add_argument("--max-rounds", type=int, default=8)
    ap.add_argument("--stall-window", type=int, default=STALL_WINDOW,
                    help="decoder stall rule of the interactive rounds (0 = stop only at a match or max_iter)")
    ap.add_argument("--target-f", type=float, default=0.0,
                    help="fixed protocol: the mixed-rate workload's target efficiency (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the fixed-rate line and the second starting efficiency beside the default")
    ap.add_argument("--alt-f-start", type=float, default=1.25,
                    help="a second starting efficiency for the interactive protocol, reported beside the default "
                         "(0 = none)")
    ap.add_argument("--no-order", action="store_true", help="persistent launch takes frames in index order")
    ap.add_argument("--separate-rounds", action="store_true",
                    help="interactive: one launch per round (host reads the flags between rounds)")
    ap.add_argument("--launch", default="", metavar="W,C,T",
                    help="launch shape words,ctas_per_sm,threads instead of the autotuner's (profiling runs)")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ workload

class Batch:
    """Host-side arrays of one rank's share of the workload."""

    def __init__(self, w, batch, first, target_f=None):
        self.w = w
        self.base = w.base()
        self.xa, self.yb, self.q = w.frames(batch, first)
        self.B = batch
        if w.mixed_rate:
            self.target_f = w.target_f if target_f is None else target_f
            self.n_punct, self.n_short = rate.plan(w.n, w.m, self.q, self.target_f)
            self.tiebreak = inputs.tiebreak_permutation(w.n, w.code_seed)
        else:
            self.target_f = None
            self.n_punct = np.zeros(batch, np.int32)
            self.n_short = np.zeros(batch, np.int32)
            self.tiebreak = None
        self.key_bits = rate.key_bits(w.n, self.n_punct, self.n_short)
        self.f = rate.efficiency(w.n, w.m, self.n_punct, self.n_short, self.q)


def interactive_mode(args, w) -> bool:
    return args.protocol == "interactive" and w.mixed_rate


def workload_config(args, w, frames, world):
    """The workload's description, identical for both arms of the bench."""
    cfg = {"workload": w.name, "frames": frames, "n": w.n, "m": w.m, "Z": w.Z, "max_iter": w.max_iter,
           "qber": list(w.qber) if isinstance(w.qber, tuple) else w.qber,
           "llr_lsb_per_nat": round(w.llr_scale, 4)}
    if interactive_mode(args, w):
        cfg.update({"protocol": "interactive rate-adaptive (sections 4.1, 4.2)", "f_start": args.f_start,
                    "reveal_df": args.df, "max_extra_rounds": args.max_rounds, "stall_window": args.stall_window,
                    "efficiency_note": "every frame starts at the rate for f_start; on these seeded random codes no "
                                       "decoder reaches FER <= 1e-2 at f = 1.1 (exact FP64 belief propagation "
                                       "fails every frame there), so frames end at the f their last round reached "
                                       "(efficiency_f_mean)"})
    else:
        cfg.update({"protocol": "fixed rate per frame" if w.mixed_rate else "single code, no rate adaptation",
                    "target_f": (args.target_f or w.target_f) if w.mixed_rate else None})
    # bytes one step touches per rank: inputs (Bob's key, known values, syndrome, per-frame counts), outputs,
    # and for the batch decoder every frame's messages (the persistent launch keeps only its lanes')
    nb, mb = (w.n + 7) // 8, (w.m + 7) // 8
    edges = int((np.asarray(w.base()) >= 0).sum()) * w.Z
    ws = frames / world * (3 * nb + mb + 37 + (0 if w.mixed_rate else edges))
    if ws > 2 * L2_BYTES:
        cfg["l2"] = "working set %.0f MB per rank, above twice the L2: no flush" % (ws / 1e6)
    else:
        cfg["l2"] = "L2 flushed (a write of twice its size) before every timed step"
    cfg["parallelism"] = f"frames sharded over {world} GPU(s), no collective on the data path"
    return cfg


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
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


def roofline_alu(it_sum, edges, seconds, clk, sms=152):
    """The integer-issue roofline of the decoder: byte operations of the method
    per second against what the SMs can issue, SMs x 4 schedulers x 32 lanes
    x the SM clock seen during the run x 4 byte lanes per 32-bit operation
    (the ALU and FMA pipes each take 16 lanes per scheduler and cycle, the
    scheduler issues one 32-lane instruction per cycle)."""
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    peak = sms * 4 * 32 * float(mhz) * 1e6 * 4 / 1e12
    achieved = ALU_OPS_PER_EDGE * float(edges) * float(it_sum) / seconds / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T byte-op/s", "frac": achieved / peak,
            "ops_per_edge_frame_iteration": ALU_OPS_PER_EDGE,
            "peak_basis": f"{sms} SMs x 4 schedulers x 32 lanes x {float(mhz):.0f} MHz x 4 byte lanes"}


def profile_value(kernel: str, workload: str, key: str):
    """A per-unit figure from the committed ncu summary of the kernel on the
    workload (``profiles/<kernel>_<workload>.md``), if it was taken on the
    current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    msha = re.search(r"kernel_sha:\s*([0-9a-f]+)", txt)
    mtr = re.search(key + r":\s*([0-9.eE+]+)", txt)
    if not msha or not mtr or msha.group(1) != kernel_sources_sha():
        return None
    return float(mtr.group(1))


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


def persistent_io_bytes(code, frame_decodes):
    """Bytes a persistent launch moves per decoded frame besides the message
    stream: Bob's key and the shortened values (2 n/8), the syndrome (m/8),
    the decoded bits (n/8), iterations, flag, magnitude, rate counts and the
    work-list entry."""
    return float(frame_decodes) * (2 * code.nbytes + code.mbytes + code.nbytes + 4 + 1 + 1 + 8 + 4)


def roofline_hbm(alg_bytes, kernel_s, kernel, traffic, extra=None):
    peak, peak_kind = peaks()
    achieved = alg_bytes / kernel_s / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic, "peak_kind": peak_kind, "kernel": kernel, "kernel_ms": kernel_s * 1e3,
           "algorithmic_bytes": alg_bytes}
    if extra:
        out.update(extra)
    return out


# ----------------------------------------------------------------- reference

def _oracle_fixed(bt, orc, k):
    from oracle import rate as orate
    w = bt.w
    xa_u = inputs.unpack_bits(bt.xa[:k], w.n)
    yb_u = inputs.unpack_bits(bt.yb[:k], w.n)
    syn = orc.syndrome(bt.base, w.Z, xa_u)
    st = kn = None
    if w.mixed_rate:
        rk = orate.position_rank(bt.base, w.Z, bt.tiebreak)
        st = np.stack([orate.position_states(rk, int(bt.n_punct[f]), int(bt.n_short[f])) for f in range(k)])
        kn = xa_u
    llr = orc.llr_frames(yb_u, bt.q[:k], st, kn, scale=w.llr_scale)
    bits, iters, ok, used = orc.decode(bt.base, w.Z, llr, syn, w.max_iter)
    corr = ok.astype(bool) & np.all(bits == xa_u, axis=1)
    return float(bt.key_bits[:k][corr].sum()), corr, used


def _oracle_interactive(bt, args, k):
    from oracle import core as orc
    from oracle import protocol as oproto
    w = bt.w
    xa_u = inputs.unpack_bits(bt.xa[:k], w.n)
    res = oproto.interactive(bt.base, w.Z, bt.tiebreak, xa_u, inputs.unpack_bits(bt.yb[:k], w.n), bt.q[:k],
                             args.f_start, args.df, args.max_rounds, w.max_iter, w.llr_scale,
                             stall_window=args.stall_window)
    corr = res["ok"].astype(bool) & np.all(res["bits"] == xa_u, axis=1)
    return float(res["key_bits"][corr].sum()), corr, orc.num_cores(), res


def oracle_sample(args, w, B, seconds, steps=1, warmup=0):
    """Time the oracle (the same protocol) on the first frames of the
    workload, the prefix sized for about ``seconds`` of CPU time per pass."""
    from oracle import core as orc
    inter = interactive_mode(args, w)
    run = (lambda bt, k: _oracle_interactive(bt, args, k)[:3]) if inter else (lambda bt, k: _oracle_fixed(bt, orc, k))
    probe = min(B, max(1, orc.num_cores()))
    bt = Batch(w, probe, 0, args.target_f or None)
    t0 = time.time()
    run(bt, probe)
    dt = max(time.time() - t0, 1e-3)
    k = int(min(B, max(probe, probe * seconds / dt)))
    bt = Batch(w, k, 0, args.target_f or None)
    for _ in range(warmup):
        run(bt, min(k, probe))
    times, cores = [], 1
    for _ in range(max(1, steps)):
        t0 = time.time()
        key, corr, cores = run(bt, k)
        times.append(time.time() - t0)
    t = float(np.mean(times))
    what = ("the interactive protocol from f = %.2f" % args.f_start) if inter else "one fixed-rate decode"
    return {"value": key / t / 1e6, "ms_per_step": t * 1e3, "cores": int(cores), "frames": k,
            "sample": f"first {k} of {B} frames of {w.name}, {what}, {len(times)} timed pass(es), "
                      f"mean {t:.2f} s/pass, FER {1 - corr.mean():.3f}"}


def run_reference(args, rank, world):
    """The oracle (the tier's reference) on the machine's host cores: each step a
    bounded sample of the same workload and protocol."""
    if rank != 0:
        return
    w = inputs.WORKLOADS[args.workload]
    if args.max_iter:
        w.max_iter = args.max_iter
    B = args.batch or w.batch
    per_step = max(2.0, args.cpu_seconds * 4 / max(1, args.steps + args.warmup))
    res = oracle_sample(args, w, B, per_step, steps=args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": res["value"], "unit": "Mbps", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": workload_config(args, w, B * world, world),
        "cpu_baseline": {"value": res["value"], "unit": "Mbps", "cores": res["cores"], "kind": "oracle",
                         "sample": res["sample"]},
        "e2e": {"value": res["value"], "unit": "Mbps", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------- ours

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
        return parse_clock_lines(self.lines)


def parse_clock_lines(lines):
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
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


def event_time(stream, fn, reps, flush_buf=None):
    """Mean device time of ``fn`` over ``reps`` calls, CUDA events on the
    launching stream.  With ``flush_buf`` every call runs after a write of
    that buffer (twice the L2), outside the timed events."""
    import torch
    pairs = []
    for k in range(reps):
        if flush_buf is not None:
            flush_buf.fill_(k & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        pairs.append((e0, e1))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in pairs) / 1e3 / reps


def fixed_rate_run(args, w, bt, rec, dv, dev, steps, warmup, flush_buf=None):
    """One persistent launch at a fixed rate per frame (mixed workload, CUDA
    graph) or one LLR + batch decode (single-code workloads), device-timed."""
    import torch
    from paper_1903_10107_gb300 import native
    from paper_1903_10107_gb300.pipeline import MixedRateBatch, hardest_first
    code = rec.code
    B = bt.B
    stream = torch.cuda.current_stream(dev)
    if w.mixed_rate:
        order = None if args.no_order else hardest_first(bt.n_punct, bt.n_short, bt.q)
        shape = [int(x) for x in args.launch.split(",")] if args.launch else [0, 0, 0]
        mrb = MixedRateBatch(rec, w.max_iter, tune_tag="fixed", tune=not args.launch, words=shape[0],
                             ctas_per_sm=shape[1], threads=shape[2]).bind(
            dv["yb"], dv["syn"], dv["mag"], dv["np"], dv["ns"], dv["xa"], order=order)
        out, step = mrb.out, mrb.run
        kernel = "persistent_kernel"
        launch = {"words_per_cta": mrb.words, "ctas_per_sm": mrb.ctas, "threads_per_cta": mrb.threads,
                  "cuda_graph": mrb.graph is not None, "work_order": "index" if order is None else "hardest first"}
        launches_per_step = 1
    else:
        code.reserve(B)
        out = (torch.empty((B, code.nbytes), dtype=torch.uint8, device=dev),
               torch.empty((B,), dtype=torch.int32, device=dev),
               torch.empty((B,), dtype=torch.uint8, device=dev))
        step = lambda: rec.reconcile(dv["yb"], dv["syn"], dv["mag"], w.max_iter, out=out)
        kernel = "decode_kernel"
        launch = {"cuda_graph": False}
        launches_per_step = 2
        mrb = None
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    l0 = native.ldpc_launch_count()
    step_s = event_time(stream, step, steps, flush_buf)
    eager = native.ldpc_launch_count() - l0
    launches = eager if eager else launches_per_step * steps  # graph replays bypass the library's counter
    bits, iters, ok = (t.cpu().numpy() for t in out)
    xa_bits = inputs.unpack_bits(bt.xa, w.n)
    corr = ok.astype(bool) & np.all(inputs.unpack_bits(bits, w.n) == xa_bits, axis=1)
    if w.mixed_rate:
        dec_s = step_s  # the step is the single persistent kernel
        io = persistent_io_bytes(code, B)
    else:
        llr = code.llr_from_bsc(dv["yb"], dv["mag"])
        for _ in range(2):
            code.decode(llr, dv["syn"], w.max_iter, out=out)
        dec_s = event_time(stream, lambda: code.decode(llr, dv["syn"], w.max_iter, out=out), max(3, steps), flush_buf)
        io = float(B) * (w.n + code.mbytes + code.nbytes + 5)
    it_sum = float(iters.astype(np.int64).sum())
    alg = it_sum * 2.0 * code.edges + io
    per_fi = profile_value(kernel, w.name if not w.mixed_rate else w.name + "_fixed", "dram_bytes_per_frame_iteration")
    traffic = None if per_fi is None else per_fi * it_sum
    return dict(step_s=step_s, dec_s=dec_s, corr=corr, iters=iters, it_sum=it_sum, alg=alg, kernel=kernel,
                traffic=traffic, launch=launch, launches=launches, corr_key=float(bt.key_bits[corr].sum()),
                all_key=float(bt.key_bits.sum()), mrb=mrb)


def measure_fixed_e2e(args, rec, bt, d_syn, dev, launch):
    """The fixed-rate step through Reconciler.reconcile_host_stream from
    pinned host buffers (copies issued by the Python layer)."""
    import torch
    w = bt.w
    mixed = w.mixed_rate
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_yb, h_syn, h_q = pin(bt.yb), pin(d_syn.cpu().numpy()), pin(bt.q)
    batch = (h_yb, h_syn, h_q, pin(bt.n_punct) if mixed else None, pin(bt.n_short) if mixed else None,
             pin(bt.xa) if mixed else None)
    kw = dict(persistent=mixed, words=launch.get("words_per_cta", 0), ctas_per_sm=launch.get("ctas_per_sm", 0))
    rec.reconcile_host_stream([batch] * max(2, args.warmup), w.max_iter, **kw)
    torch.cuda.synchronize()
    e2e_steps = max(2, min(args.steps, 5))
    t0 = time.perf_counter()
    out = rec.reconcile_host_stream([batch] * e2e_steps, w.max_iter, **kw)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    res, h2d, d2h = out[-1]
    e_bits = inputs.unpack_bits(res[0].numpy(), w.n)
    e_corr = res[2].numpy().astype(bool) & np.all(e_bits == inputs.unpack_bits(bt.xa, w.n), axis=1)
    return e2e_s, float(bt.key_bits[e_corr].sum()), h2d, d2h


def run_ours(args, rank, world, dist):
    import torch
    from paper_1903_10107_gb300 import native
    from paper_1903_10107_gb300.pipeline import InteractiveProtocol, Reconciler

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = inputs.WORKLOADS[args.workload]
    if args.max_iter:
        w.max_iter = args.max_iter
    inter = interactive_mode(args, w)
    first, B = sharding.weak_shard(args.batch or w.batch, rank, world)  # every rank its own frames
    bt = Batch(w, B, first, args.target_f or None)
    rec = Reconciler(bt.base, w.Z, bt.tiebreak, dev, llr_scale=w.llr_scale)
    code = rec.code
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    dv = {"xa": c(bt.xa), "yb": c(bt.yb), "mag": c(rec.magnitudes(bt.q)),
          "np": c(bt.n_punct) if w.mixed_rate else None, "ns": c(bt.n_short) if w.mixed_rate else None}
    dv["syn"] = code.syndrome(dv["xa"])  # Alice's syndromes (her side of the protocol; outside the step)
    if not w.mixed_rate:
        dv["xa"] = None
    xa_bits = inputs.unpack_bits(bt.xa, w.n)
    stream = torch.cuda.current_stream(dev)
    cfg = workload_config(args, w, B * world, world)
    flush = cfg["l2"].startswith("L2 flushed")
    flush_buf = torch.empty(2 * torch.cuda.get_device_properties(dev).L2_cache_size, dtype=torch.uint8,
                            device=dev) if flush else None

    def barrier():
        if dist is not None:
            dist.barrier()

    secondary = None
    if inter and not args.no_secondary:
        # the fixed-rate launch at the workload's own target f, beside the default line
        bt_f = Batch(w, B, first)
        dv_f = {**dv, "np": c(bt_f.n_punct), "ns": c(bt_f.n_short)}
        fr = fixed_rate_run(args, w, bt_f, rec, dv_f, dev, max(3, min(args.steps, 10)), 3)
        secondary = {
            "value": fr["corr_key"] / fr["step_s"] / 1e6, "unit": "Mbps", "ms_per_step": fr["step_s"] * 1e3,
            "target_f": w.target_f, "efficiency_f_mean": float(np.mean(bt_f.f)),
            "fer": 1.0 - float(fr["corr"].mean()), "iters_mean": float(fr["iters"].mean()), "launch": fr["launch"],
            "roofline": roofline_hbm(fr["alg"], fr["dec_s"], fr["kernel"], fr["traffic"]),
            "note": "one persistent launch per step (CUDA graph), every frame at the rate for target_f; "
                    "plain stopping rule (syndrome match or max_iter)"}
        del fr, dv_f

    clocks = ClockSampler(local)
    if inter:
        proto = InteractiveProtocol(rec, w.max_iter, f_start=args.f_start, df=args.df, max_rounds=args.max_rounds,
                                    stall_window=args.stall_window, fused=not args.separate_rounds)
        if args.launch:
            words, ctas, threads = (int(x) for x in args.launch.split(","))
            proto.words, proto.ctas, proto.threads = words, ctas, threads
        else:
            words, ctas, threads = proto.tune(dv["yb"], dv["syn"], bt.q, c(bt.xa))
        d_known = c(bt.xa)
        for _ in range(args.warmup):
            proto.run(dv["yb"], dv["syn"], bt.q, d_known)
        torch.cuda.synchronize()
        barrier()
        clocks.start()
        time.sleep(0.3)
        torch.cuda.synchronize()
        l0 = native.ldpc_launch_count()
        step_times, kern = [], []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = proto.run(dv["yb"], dv["syn"], bt.q, d_known, timing=True, bits_out="device")
            e1.record(stream)
            torch.cuda.synchronize()
            step_times.append(e0.elapsed_time(e1) / 1e3)
            kern.append(res["kernel_s"])
        launches = native.ldpc_launch_count() - l0
        barrier()
        clk = clocks.stop()
        step_s = float(np.mean(step_times))
        dec_s = float(np.mean(kern))
        got = inputs.unpack_bits(res["bits"].cpu().numpy(), w.n)
        corr = res["ok"].astype(bool) & np.all(got == xa_bits, axis=1)
        corr_key, all_key = float(res["key_bits"][corr].sum()), float(res["key_bits"].sum())
        it_sum = float(res["iters"].sum())
        decodes = float((res["rounds"] + 1).sum())
        alg = it_sum * 2.0 * code.edges + persistent_io_bytes(code, decodes)
        per_fi = profile_value("persistent_kernel", w.name + "_interactive", "dram_bytes_per_frame_iteration")
        traffic = None if per_fi is None else per_fi * it_sum
        extra = {"launches_per_step": int(res["launches"]), "per": "step: the launches of all rounds",
                 "kernel_ms_is": "summed CUDA-event time of the step's persistent launches"}
        l2_per_fi = profile_value("persistent_kernel", w.name + "_interactive", "l2_bytes_per_frame_iteration")
        if l2_per_fi is not None:
            l2_peak = measure_l2_copy_gbs(dev)
            l2t = l2_per_fi * it_sum
            extra["l2"] = {"achieved": l2t / dec_s / 1e9, "peak": l2_peak, "unit": "GB/s",
                           "frac": l2t / dec_s / 1e9 / l2_peak, "traffic": l2t,
                           "traffic_source": "lts__t_bytes.sum per frame-iteration, committed ncu summary",
                           "peak_kind": "measured in this run: device copy of a 24 MB buffer held in L2"}
        roof = roofline_hbm(alg, dec_s, "persistent_kernel", traffic, extra)
        fer = 1.0 - float(corr.mean())
        by_qber = []
        for lo in np.arange(0.01, 0.08, 0.01):
            sel = (bt.q >= lo) & (bt.q < lo + 0.01)
            if sel.any():
                by_qber.append({"qber": [round(float(lo), 2), round(float(lo) + 0.01, 2)], "frames": int(sel.sum()),
                                "fer": 1.0 - float(corr[sel].mean()), "f_mean": float(res["f"][sel].mean()),
                                "rounds_mean": float(res["rounds"][sel].mean()),
                                "iters_mean": float(res["iters"][sel].mean()),
                                "key_share": float(res["key_bits"][sel & corr].sum()) / max(corr_key, 1.0)})
        extra_keys = {"fer": fer, "efficiency_f_mean": float(res["f"][corr].mean()) if corr.any() else None,
                      "by_qber": by_qber,
                      "efficiency_f_all_frames": float(res["f"].mean()),
                      "rounds_mean": float(res["rounds"].mean()), "rounds_max": int(res["rounds"].max()),
                      "iters_mean_total": float(res["iters"].mean()),
                      "frames_decoded_per_round": np.bincount(res["rounds"]).tolist(),
                      "processed_key_mbps": all_key / step_s / 1e6}
        launch = {"words_per_cta": words, "ctas_per_sm": ctas, "threads_per_cta": threads, "cuda_graph": False,
                  "rounds": ("one persistent launch per round" if args.separate_rounds else
                             "all in one persistent launch (ldpc_reconcile_interactive)"),
                  "work_order": "hardest first (most punctured, highest QBER)"}
        # end to end from pinned host buffers through InteractiveProtocol.run_host
        e2e = None
        e2e_each = []
        if not args.no_e2e:
            pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            h_yb, h_syn, h_kn = pin(bt.yb), dv["syn"].cpu().pin_memory(), pin(bt.xa)
            h_bits = torch.empty((B, code.nbytes), dtype=torch.uint8, pin_memory=True)
            proto.run_host(h_yb, h_syn, bt.q, h_kn, bits_out=h_bits)
            torch.cuda.synchronize()
            e2e_steps = max(2, min(args.steps, 5))
            e2e_each = []
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                ts = time.perf_counter()
                eres, h2d, d2h = proto.run_host(h_yb, h_syn, bt.q, h_kn, bits_out=h_bits)
                e2e_each.append(time.perf_counter() - ts)
            torch.cuda.synchronize()
            e2e_s = (time.perf_counter() - t0) / e2e_steps
            ecorr = eres["ok"].astype(bool) & np.all(inputs.unpack_bits(eres["bits"], w.n) == xa_bits, axis=1)
            e2e = (e2e_s, float(eres["key_bits"][ecorr].sum()), h2d, d2h)
        if not args.no_secondary and args.alt_f_start > 0:
            # the same protocol from a second starting efficiency, device-timed like the default
            alt = InteractiveProtocol(rec, w.max_iter, f_start=args.alt_f_start, df=args.df,
                                      max_rounds=args.max_rounds, stall_window=args.stall_window, words=words,
                                      ctas_per_sm=ctas, threads=threads)
            for _ in range(2):
                alt.run(dv["yb"], dv["syn"], bt.q, d_known, bits_out="device")
            torch.cuda.synchronize()
            a_steps, a_kern = [], []
            for _ in range(max(3, min(args.steps, 5))):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ares = alt.run(dv["yb"], dv["syn"], bt.q, d_known, timing=True, bits_out="device")
                e1.record(stream)
                torch.cuda.synchronize()
                a_steps.append(e0.elapsed_time(e1) / 1e3)
                a_kern.append(ares["kernel_s"])
            acorr = ares["ok"].astype(bool) & np.all(inputs.unpack_bits(ares["bits"].cpu().numpy(), w.n) == xa_bits,
                                                     axis=1)
            a_s, a_it = float(np.mean(a_steps)), float(ares["iters"].sum())
            a_alg = a_it * 2.0 * code.edges + persistent_io_bytes(code, float((ares["rounds"] + 1).sum()))
            extra_keys["alt_start"] = {
                "f_start": args.alt_f_start, "value": float(ares["key_bits"][acorr].sum()) / a_s / 1e6, "unit": "Mbps",
                "ms_per_step": a_s * 1e3, "fer": 1.0 - float(acorr.mean()),
                "efficiency_f_mean": float(ares["f"][acorr].mean()) if acorr.any() else None,
                "rounds_mean": float(ares["rounds"].mean()), "iters_mean_total": float(ares["iters"].mean()),
                "roofline": roofline_hbm(a_alg, float(np.mean(a_kern)), "persistent_kernel", None),
                "note": "the default protocol started from f_start instead of 1.1: the same final efficiency "
                        "range is reached with fewer hopeless rounds"}
    else:
        barrier()
        clocks.start()
        time.sleep(0.3)
        torch.cuda.synchronize()
        fr = fixed_rate_run(args, w, bt, rec, dv, dev, args.steps, args.warmup, flush_buf)
        barrier()
        clk = clocks.stop()
        step_s, dec_s, corr = fr["step_s"], fr["dec_s"], fr["corr"]
        corr_key, all_key, it_sum, launches = fr["corr_key"], fr["all_key"], fr["it_sum"], fr["launches"]
        roof = roofline_hbm(fr["alg"], dec_s, fr["kernel"], fr["traffic"])
        extra_keys = {"fer": 1.0 - float(corr.mean()), "efficiency_f_mean": float(np.mean(bt.f)),
                      "iters_mean": float(fr["iters"].mean()), "processed_key_mbps": all_key / step_s / 1e6}
        launch = fr["launch"]
        e2e = None
        e2e_each = []
        if not args.no_e2e:
            e2e = measure_fixed_e2e(args, rec, bt, dv["syn"], dev, launch)

    e2e_s, e_key, h2d, d2h = e2e if e2e is not None else (float("nan"), 0.0, 0, 0)
    # max over ranks (times), sums over ranks (key bits)
    vals_max, vals_sum = sharding.reduce_max_sum([step_s, e2e_s, dec_s], [corr_key, all_key, e_key], dist, dev)
    step_max, e2e_max = vals_max[0], vals_max[1]
    corr_tot, e_tot = vals_sum[0], vals_sum[2]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_sample(args, w, B, args.cpu_seconds)
        cpu = {"value": r["value"], "unit": "Mbps", "cores": r["cores"], "kind": "oracle", "sample": r["sample"]}
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": corr_tot / step_max / 1e6, "unit": "Mbps", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_max * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic", "config": cfg,
        "launch": launch, **extra_keys,
        "roofline": roof,
        "roofline_alu": roofline_alu(it_sum, code.edges, dec_s, clk,
                                     torch.cuda.get_device_properties(dev).multi_processor_count),
        "e2e": {"value": e_tot / e2e_max / 1e6 if e2e is not None else None, "unit": "Mbps",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "step_ms": [round(1e3 * x, 2) for x in e2e_each] if e2e_each else None,
                "path": ("the C-ABI host-buffer call ldpc_reconcile_interactive_host (via InteractiveProtocol."
                         "run_host): pinned host buffers in and out, the library's own copies around its one "
                         "launch" if inter and not args.separate_rounds else
                         ("InteractiveProtocol.run_host" if inter else "Reconciler.reconcile_host_stream") +
                         ": torch copies from pinned host buffers, issued by the Python layer around the C-ABI "
                         "launches (the C ABI takes device pointers)")},
        "gpu_launches": int(launches), "clocks": clk, "cpu_baseline": cpu,
        "paper_context": "60 Mbps at f~1.1 on an Intel i7-6700HQ (section 4.2, Table 2), other codes and hardware",
    }
    if secondary is not None:
        line["fixed_rate"] = secondary
    print(json.dumps(line), flush=True)


def main(argv=None):
    args = parse_args(argv)
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

"""Autotuner for the persistent mixed-rate decoder.

The launch shape of ``ldpc_reconcile_persistent`` has three knobs: the
number of 32-bit lane words per CTA (``words``: 4, 8 or 16 frames per CTA),
the number of resident CTAs per SM, and the threads per CTA (one thread
pair per check row of a layer, or half as many threads, each pair then
taking two rows of a layer: fewer warps to hide latency, but less
per-row bookkeeping and half the shuffles and barrier arrivals).  Which is
fastest depends on the code (n bytes of soft values per frame must fit in
shared memory, row degrees set the register budget) and on how uneven the
frames' iteration counts are.  The tuner times every candidate that fits on
a sample of the real batch with CUDA events and caches the winner per code
shape in a JSON file next to the built library.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import build as _build

_CACHE_PATH = os.path.join(_build.OUT_DIR, "autotune.json")
_lock = threading.Lock()


def _key(code, batch: int, tag: str = "") -> str:
    bucket = 1 << max(0, (int(batch) - 1).bit_length())
    key = f"Mb{code.Mb}_Nb{code.Nb}_Z{code.Z}_e{code.edges}_d{code.max_row_deg}_b{bucket}"
    return f"{key}_{tag}" if tag else key


def _load():
    try:
        with open(_CACHE_PATH) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store(cache):
    os.makedirs(os.path.dirname(_CACHE_PATH), exist_ok=True)
    tmp = _CACHE_PATH + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE_PATH)


def default_threads(code, words: int) -> int:
    """Threads per CTA of the automatic launch: one thread pair per check row
    of a layer, capped at 1024 (512 for rows of more than 32 edges), rounded
    up to whole warps."""
    cap = 1024 if (code.max_row_deg + 1) // 2 <= 16 else 512
    t = min(code.Z * words * 2, cap)
    return (t + 31) // 32 * 32


def candidates(code):
    """(words, ctas_per_sm, threads) triples whose shared-memory state fits
    one SM and whose registers fit (64 per thread)."""
    props = torch.cuda.get_device_properties(code.device)
    smem_sm = getattr(props, "shared_memory_per_multiprocessor", 228 * 1024)
    smem_blk = getattr(props, "shared_memory_per_block_optin", 227 * 1024)
    regs_sm = getattr(props, "regs_per_multiprocessor", 65536)
    tab = 4 * (((2 * code.Mb + 1 + 1) & ~1) + 2 * (code.edges // code.Z))
    out = []
    for words in (1, 2, 4):
        per_cta = 4 * code.n * words + tab + code.m * words + 1024
        if per_cta > smem_blk:
            continue
        t0 = default_threads(code, words)
        threads = [t0]
        if t0 // 2 >= 64 and (t0 // 2) % (32 * words) == 0:
            threads.append(t0 // 2)
        for t in threads:
            for ctas in (1, 2, 3, 4):
                if ctas * per_cta > smem_sm or ctas * t * 64 > regs_sm:
                    break
                out.append((words, ctas, t))
    return out


def tune_persistent(code, run, batch: int, sample_frames: int = 0, reps: int = 2, force: bool = False,
                    tag: str = ""):
    """Pick (words, ctas_per_sm, threads) for ``run(words, ctas_per_sm,
    threads, n_frames)``, a callable that launches one persistent decode of
    the first ``n_frames`` frames on the current stream.  Returns the chosen
    triple.  ``tag`` separates workloads of one code shape whose frames
    behave differently (their rates, and so their iteration counts)."""
    key = _key(code, batch, tag)
    with _lock:
        cache = _load()
    if not force and key in cache and len(cache[key]["choice"]) == 3:
        return tuple(cache[key]["choice"])
    cands = candidates(code)
    if len(cands) == 1:
        choice = cands[0]
        timings = {}
    else:
        nf = batch if sample_frames <= 0 else min(batch, sample_frames)
        timings = {}
        st = torch.cuda.current_stream(code.device)
        for words, ctas, threads in cands:
            run(words, ctas, threads, nf)  # warm-up (also grows the scratch arena)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                run(words, ctas, threads, nf)
            e1.record(st)
            torch.cuda.synchronize(code.device)
            timings[f"{words}x{ctas}x{threads}"] = e0.elapsed_time(e1) / reps
        best = min(timings, key=timings.get)
        choice = tuple(int(x) for x in best.split("x"))
    with _lock:
        cache = _load()
        cache[key] = {"choice": list(choice), "timings_ms": timings}
        _store(cache)
    return choice

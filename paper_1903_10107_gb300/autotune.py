"""Autotuner for the persistent mixed-rate decoder.

The launch shape of ``ldpc_reconcile_persistent`` has two knobs: the number
of 32-bit lane words per CTA (``words``: 4, 8 or 16 frames per CTA) and the
number of resident CTAs per SM.  Which is fastest depends on the code (n
bytes of soft values per frame must fit in shared memory, row degrees set the
register budget) and on how uneven the frames' iteration counts are.  The
tuner times every candidate that fits on a sample of the real batch with
CUDA events and caches the winner per code shape in a JSON file next to the
built library.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import build as _build

_CACHE_PATH = os.path.join(_build.OUT_DIR, "autotune.json")
_lock = threading.Lock()


def _key(code, batch: int) -> str:
    bucket = 1 << max(0, (int(batch) - 1).bit_length())
    return f"Mb{code.Mb}_Nb{code.Nb}_Z{code.Z}_e{code.edges}_d{code.max_row_deg}_b{bucket}"


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


def candidates(code):
    """(words, ctas_per_sm) pairs whose shared-memory state fits one SM."""
    props = torch.cuda.get_device_properties(code.device)
    smem_sm = getattr(props, "shared_memory_per_multiprocessor", 228 * 1024)
    smem_blk = getattr(props, "shared_memory_per_block_optin", 227 * 1024)
    tab = 4 * (((2 * code.Mb + 1 + 1) & ~1) + 2 * (code.edges // code.Z))
    out = []
    for words in (1, 2, 4):
        per_cta = 4 * code.n * words + tab + code.m * words + 1024
        if per_cta > smem_blk:
            continue
        for ctas in (1, 2, 3, 4):
            if ctas * per_cta > smem_sm:
                break
            out.append((words, ctas))
    return out


def tune_persistent(code, run, batch: int, sample_frames: int = 0, reps: int = 2, force: bool = False):
    """Pick (words, ctas_per_sm) for ``run(words, ctas_per_sm, n_frames)``, a
    callable that launches one persistent decode of the first ``n_frames``
    frames on the current stream.  Returns the chosen pair."""
    key = _key(code, batch)
    with _lock:
        cache = _load()
    if not force and key in cache:
        return tuple(cache[key]["choice"])
    cands = candidates(code)
    if len(cands) == 1:
        choice = cands[0]
        timings = {}
    else:
        nf = batch if sample_frames <= 0 else min(batch, sample_frames)
        timings = {}
        st = torch.cuda.current_stream(code.device)
        for words, ctas in cands:
            run(words, ctas, nf)  # warm-up (also grows the scratch arena)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                run(words, ctas, nf)
            e1.record(st)
            torch.cuda.synchronize(code.device)
            timings[f"{words}x{ctas}"] = e0.elapsed_time(e1) / reps
        best = min(timings, key=timings.get)
        choice = tuple(int(x) for x in best.split("x"))
    with _lock:
        cache = _load()
        cache[key] = {"choice": list(choice), "timings_ms": timings}
        _store(cache)
    return choice

"""Learn check-node scale/offset tables with the relaxed decoder and measure
what they do to the integer decoder.

    python -m paper_1903_10107_gb300.train_tables [--steps 60] [--batch 1024]

Training: the FP32 relaxation (tempered box-plus at the temperature the
integer decoder's LLR scale implies) unrolled for ``iters`` iterations on
fresh seeded frames each step, Adam on one scale and one offset per
iteration and row-degree class, loss = cross entropy of the final soft
values against Alice's bits.  Evaluation: the learned parameters rounded
into ``ldpc_decode_batch_ex`` tables, against the untuned tables (scale 16,
offset 0), on the same fresh frames of the same code (equal rate), with the
same iteration cap.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import inputs
from .decoder import QCCode, llr_magnitudes
from .relaxed import RelaxedDecoder, bsc_llr_nats, kappa_for_scale


def frames(w, B, seed_offset, qlo, qhi):
    q = inputs.frame_qbers(B, qlo, qhi, w.frame_seed + 1000 + seed_offset)
    xa = inputs.alice_keys(B, w.n, w.frame_seed + 1000 + seed_offset)
    yb = xa ^ inputs.bsc_noise(B, w.n, q, w.frame_seed + 1000 + seed_offset)
    return xa, yb, q


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="n4096_relaxed_q02_04")
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=0.02)
    ap.add_argument("--eval-frames", type=int, default=16384)
    ap.add_argument("--llr-scale", type=float, default=8.0)
    args = ap.parse_args(argv)

    w = inputs.WORKLOADS[args.workload]
    qlo, qhi = w.qber
    dev = torch.device("cuda", torch.cuda.current_device())
    code = QCCode(w.base(), w.Z, dev)
    model = RelaxedDecoder(code, w.max_iter, kappa=kappa_for_scale(args.llr_scale))
    opt = torch.optim.Adam(model.parameters(), lr=args.lr)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    losses, t_fwd, t_bwd = [], 0.0, 0.0
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for step in range(args.steps):
        xa, yb, q = frames(w, args.batch, step, qlo, qhi)
        llr = c(bsc_llr_nats(inputs.unpack_bits(yb, w.n), q))
        syn = code.syndrome(c(xa))
        bits = c(xa)
        opt.zero_grad()
        ev[0].record()
        loss, _ = model(llr, syn, bits)
        ev[1].record()
        loss.backward()
        ev[2].record()
        opt.step()
        with torch.no_grad():
            model.alpha.clamp_(0.0, 15.9)
            model.gamma.clamp_(-2.0, 4.0)
        torch.cuda.synchronize()
        if step > 0:
            t_fwd += ev[0].elapsed_time(ev[1])
            t_bwd += ev[1].elapsed_time(ev[2])
        losses.append(float(loss))

    # evaluation on fresh frames: integer decoder, untuned vs learned tables
    sq, oq = model.integer_tables(args.llr_scale)
    xa, yb, q = frames(w, args.eval_frames, 10_000, qlo, qhi)
    d_xa = c(xa)
    syn = code.syndrome(d_xa)
    llr_q = code.llr_from_bsc(c(yb), c(llr_magnitudes(q, args.llr_scale)))
    res = {}
    for name, tabs in (("untuned", (None, None)), ("learned", (c(sq), c(oq)))):
        bits, iters, ok = code.decode(llr_q, syn, w.max_iter, scale_q4=tabs[0], offset_q=tabs[1])
        got = inputs.unpack_bits(bits.cpu().numpy(), w.n)
        corr = ok.cpu().numpy().astype(bool) & np.all(got == inputs.unpack_bits(xa, w.n), axis=1)
        res[name] = {"fer": 1.0 - float(corr.mean()), "iters_mean": float(iters.float().mean())}
    steps_timed = max(1, args.steps - 1)
    ck_bytes = 4.0 * args.batch * ((w.max_iter + 1) * w.n + w.max_iter * code.edges)
    line = {
        "workload": w.name, "n": w.n, "iters": w.max_iter, "qber": [qlo, qhi], "batch": args.batch,
        "steps": args.steps, "kappa": model.kappa, "llr_lsb_per_nat": args.llr_scale,
        "loss_first": losses[0], "loss_last": losses[-1],
        "forward_ms": t_fwd / steps_timed, "backward_ms": t_bwd / steps_timed,
        "forward_checkpoint_GBps": ck_bytes / (t_fwd / steps_timed * 1e-3) / 1e9,
        "eval_frames": args.eval_frames, "fer_untuned": res["untuned"]["fer"], "fer_learned": res["learned"]["fer"],
        "iters_untuned": res["untuned"]["iters_mean"], "iters_learned": res["learned"]["iters_mean"],
        "scale_q4_range": [int(sq.min()), int(sq.max())], "offset_q_range": [int(oq.min()), int(oq.max())],
        "alpha_mean": float(model.alpha.mean()), "gamma_mean": float(model.gamma.mean()),
    }
    print(json.dumps(line), flush=True)
    return line


if __name__ == "__main__":
    main()

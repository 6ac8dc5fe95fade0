"""Learn check-node scale/offset tables with the relaxed decoder and measure
what they do to the integer decoder.

    python -m paper_1903_10107_gb300.train_tables [--steps 60] [--batch 1024] [--train-qber LO HI]
                                                 [--target-fer 0.03] [--out FILE]

Training: the FP32 relaxation (tempered box-plus at the temperature the
integer decoder's LLR scale implies) unrolled for ``iters`` iterations on
fresh seeded frames each step, Adam on one scale and one offset per
iteration and row-degree class, loss = cross entropy of the final soft
values against Alice's bits.  Evaluation: the learned parameters rounded
into ``ldpc_decode_batch_ex`` tables, against the untuned tables (scale 16,
offset 0), on the same fresh frames of the same code (equal rate), with the
same iteration cap: over the training QBER range, and at an operating point
where the comparison says something -- the fixed QBER (equal efficiency f
for both tables) of a grid at which the untuned decoder's FER, measured on
a separate selection set, is closest to ``--target-fer`` (default 0.03,
inside 1e-2 .. 1e-1).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json

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
    ap.add_argument("--target-fer", type=float, default=0.03, help="untuned FER of the operating point")
    ap.add_argument("--train-qber", type=float, nargs=2, default=None, metavar=("LO", "HI"),
                    help="training QBER range (default: the workload's)")
    ap.add_argument("--out", default="", help="append the JSON line to this file")
    args = ap.parse_args(argv)

    w = inputs.WORKLOADS[args.workload]
    qlo, qhi = w.qber if args.train_qber is None else tuple(args.train_qber)
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
    tables = {"untuned": (None, None), "learned": (c(sq), c(oq))}

    def evaluate(B, seed_offset, lo, hi, names=("untuned", "learned")):
        xa, yb, q = frames(w, B, seed_offset, lo, hi)
        syn = code.syndrome(c(xa))
        llr_q = code.llr_from_bsc(c(yb), c(llr_magnitudes(q, args.llr_scale)))
        xa_u = inputs.unpack_bits(xa, w.n)
        out = {}
        for name in names:
            sq_d, oq_d = tables[name]
            bits, iters, ok = code.decode(llr_q, syn, w.max_iter, scale_q4=sq_d, offset_q=oq_d)
            got = inputs.unpack_bits(bits.cpu().numpy(), w.n)
            corr = ok.cpu().numpy().astype(bool) & np.all(got == xa_u, axis=1)
            fails = int((~corr).sum())
            out[name] = {"fer": fails / B, "frame_errors": fails, "iters_mean": float(iters.float().mean()),
                         "fer_95ci": wilson(fails, B)}
        return out

    wlo, whi = w.qber
    res = evaluate(args.eval_frames, 10_000, wlo, whi)  # the workload's own QBER range
    # operating point: the grid QBER whose untuned FER (selection set, other seeds) is closest to the target
    grid = np.round(np.arange(0.010, 0.0301, 0.0025), 4)
    sel = {float(g): evaluate(4096, 20_000 + k, g, g, ("untuned",))["untuned"]["fer"] for k, g in enumerate(grid)}
    q_op = min(sel, key=lambda g: abs(np.log(max(sel[g], 1e-6)) - np.log(args.target_fer)))
    op = evaluate(args.eval_frames, 30_000, q_op, q_op)
    R = 1.0 - code.m / code.n
    h = -q_op * np.log2(q_op) - (1 - q_op) * np.log2(1 - q_op)
    steps_timed = max(1, args.steps - 1)
    ck_bytes = 4.0 * args.batch * ((w.max_iter + 1) * w.n + w.max_iter * code.edges)
    line = {
        "workload": w.name, "n": w.n, "iters": w.max_iter, "train_qber": [qlo, qhi], "eval_qber": [wlo, whi],
        "batch": args.batch,
        "steps": args.steps, "kappa": model.kappa, "llr_lsb_per_nat": args.llr_scale,
        "loss_first": losses[0], "loss_last": losses[-1],
        "forward_ms": t_fwd / steps_timed, "backward_ms": t_bwd / steps_timed,
        "forward_checkpoint_GBps": ck_bytes / (t_fwd / steps_timed * 1e-3) / 1e9,
        "eval_frames": args.eval_frames, "fer_untuned": res["untuned"]["fer"], "fer_learned": res["learned"]["fer"],
        "fer_95ci_untuned": res["untuned"]["fer_95ci"], "fer_95ci_learned": res["learned"]["fer_95ci"],
        "iters_untuned": res["untuned"]["iters_mean"], "iters_learned": res["learned"]["iters_mean"],
        "operating_point": {"qber": q_op, "efficiency_f": (1 - R) / h, "selection_untuned_fer_by_qber": sel,
                            "target_untuned_fer": args.target_fer, "frames": args.eval_frames,
                            "untuned": op["untuned"], "learned": op["learned"]},
        "scale_q4_range": [int(sq.min()), int(sq.max())], "offset_q_range": [int(oq.min()), int(oq.max())],
        "alpha_mean": float(model.alpha.mean()), "gamma_mean": float(model.gamma.mean()),
    }
    print(json.dumps(line), flush=True)
    if args.out:
        with open(args.out, "a") as fh:
            fh.write(json.dumps(line) + "\n")
    return line


def wilson(k: int, n: int, z: float = 1.96):
    """95 % Wilson score interval of a binomial proportion k / n."""
    if n == 0:
        return [0.0, 1.0]
    p = k / n
    d = 1 + z * z / n
    c = (p + z * z / (2 * n)) / d
    r = z * np.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return [float(max(0.0, c - r)), float(min(1.0, c + r))]


if __name__ == "__main__":
    main()

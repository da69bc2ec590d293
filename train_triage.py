#!/usr/bin/env python
"""Train and judge the learned sky triage on the GPU.

Training set: method-generated events at the shapes of the plain 2-detector
workload (10^4 segments x 10^4 bins, T_SFT = 4 s, 500-3000 Hz, 1024
Fibonacci-sphere skies), each with one injected track of SNR uniform in
[6, 12] whose template comes from the workload's 2e5-template uniform-random
bank; one example per sky patch (32 Doppler-sorted skies), label 1 for the
patches within one patch of an injected sky: 3125 events give 1.0e5
examples.  The features come from the library's coarse pass (every segment)
and the network is trained by the library's own forward/backward/Adam
kernels.

Judge (Sec. 3): the detection threshold is the largest Psi of exhaustive
searches of noise-only events with the same bank; on held-out events the
triaged search (best 35 % of patches, each contributing its best 1.2 % of
templates by coarse Psi) is compared with the exhaustive search of every
sky; an injection counts as found when its template is within the first 10
entries, with Psi above the threshold, of a searched sky within 64
Doppler-sorted positions of the injected sky.

  python train_triage.py [--train-events 3125] [--valid-events 100]
                         [--frac 0.35] [--templates-permille 12] [--judge-only]
                         [--out paper_2507_07816_gb300/triage_weights.npz]
                         [--report triage_report.json]

--judge-only skips the training and judges the weights in --out.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-events", type=int, default=3125)   # x 32 patches = 1.0e5 examples
    ap.add_argument("--valid-events", type=int, default=100)
    ap.add_argument("--noise-events", type=int, default=4)
    ap.add_argument("--n-tmpl", type=int, default=200000)
    ap.add_argument("--stride", type=int, default=None)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--frac", type=float, default=None)
    ap.add_argument("--patch-size", type=int, default=32)
    ap.add_argument("--injections", type=int, default=1)
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_2507_07816_gb300", "triage_weights.npz"))
    ap.add_argument("--report", default=None)
    ap.add_argument("--templates-permille", type=int, default=None)
    ap.add_argument("--judge-only", action="store_true")
    args = ap.parse_args()

    import torch
    import paper_2507_07816_gb300 as tcw
    from paper_2507_07816_gb300 import triage as TR
    import tcw_synth as syn

    dev = torch.device("cuda:0")
    bank_seed, train_seed, valid_seed = 20250715, 30_000_000, 40_000_000
    bank = syn.random_bank(syn.rng(bank_seed), args.n_tmpl, f0_range=(500.0, 3000.0))
    tpm = TR.TEMPLATES_PERMILLE if args.templates_permille is None else args.templates_permille
    if args.frac is None:
        args.frac = TR.FRAC
    stride = TR.STRIDE if args.stride is None else args.stride

    def make(seed0, n_inj=None):
        n = args.injections if n_inj is None else n_inj
        return lambda i: syn.training_event(seed0 + i, bank, n_inj=n, snr_range=(6.0, 12.0), device=dev)

    noise_seed = valid_seed + 500_000
    t0 = time.perf_counter()
    psi_det = TR.noise_threshold(make(noise_seed, 0), args.noise_events, bank)
    print(f"noise-only threshold {psi_det:.4f} from {args.noise_events} events in "
          f"{time.perf_counter() - t0:.0f} s", flush=True)

    if args.judge_only:
        mlp = tcw.Mlp.load(args.out, device=dev)
        untrained = tcw.Mlp(seed=1, device=dev)
        t0 = time.perf_counter()
        judged = TR.evaluate(mlp, make(valid_seed + 1000), args.valid_events, bank, psi_det, frac=args.frac,
                             patch_size=args.patch_size, templates_permille=tpm, stride=stride)
        # the literal form: the best 10 % of the patches, every template
        judged_all = TR.evaluate(mlp, make(valid_seed + 1000), min(args.valid_events, 200), bank, psi_det,
                                 frac=0.1, patch_size=args.patch_size, templates_permille=1000, stride=stride)
        judged_un = TR.evaluate(untrained, make(valid_seed + 1000), min(args.valid_events, 50), bank, psi_det,
                                frac=args.frac, patch_size=args.patch_size, templates_permille=tpm, stride=stride)
        report = {"weights": os.path.relpath(args.out, ROOT), "psi_det": psi_det, "judged_trained": judged,
                  "judged_trained_top10pct_all_templates": judged_all, "judged_untrained": judged_un,
                  "valid_s": time.perf_counter() - t0}
        print(json.dumps(report), flush=True)
        if args.report:
            os.makedirs(os.path.dirname(os.path.abspath(args.report)), exist_ok=True)
            with open(args.report, "w") as f:
                json.dump(report, f, indent=1)
        return 0

    t0 = time.perf_counter()
    X, y, sizes = TR.collect(make(train_seed), args.train_events, bank, patch_size=args.patch_size, stride=stride)
    t_collect = time.perf_counter() - t0
    print(f"collected {X.shape[0]} examples ({int(y.sum().item())} positive) in {t_collect:.0f} s", flush=True)
    Xh, yh, sizes_h = TR.collect(make(valid_seed), 64, bank, patch_size=args.patch_size, stride=stride)
    untrained = tcw.Mlp(seed=1, device=dev)
    t0 = time.perf_counter()
    mlp, losses = TR.train(X, y, steps=args.steps, batch=args.batch, lr=args.lr, seed=1,
                           log_every=max(1, args.steps // 20))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    rec = {f: TR.recall_at(mlp, Xh, yh, sizes_h, f) for f in (0.05, 0.1, 0.2)}
    rec_un = {f: TR.recall_at(untrained, Xh, yh, sizes_h, f) for f in (0.05, 0.1, 0.2)}
    print(f"trained in {t_train:.0f} s; loss {losses[0][1]:.4f} -> {losses[-1][1]:.4f}; "
          f"patch recall trained {rec} untrained {rec_un}", flush=True)
    np.savez(args.out, theta=mlp.parameters(), bank_seed=bank_seed, n_tmpl=args.n_tmpl,
             patch_size=args.patch_size, frac=args.frac, psi_lo=TR.PSI_LO, psi_hi=TR.PSI_HI,
             valid_seed=valid_seed, train_events=args.train_events, train_examples=int(X.shape[0]),
             injections=args.injections, stride=stride, psi_det=psi_det, noise_seed=noise_seed,
             noise_events=args.noise_events)
    t0 = time.perf_counter()
    judged = TR.evaluate(mlp, make(valid_seed + 1000), args.valid_events, bank, psi_det, frac=args.frac,
                         patch_size=args.patch_size, templates_permille=tpm, stride=stride)
    judged_un = TR.evaluate(untrained, make(valid_seed + 1000), min(args.valid_events, 50), bank, psi_det,
                            frac=args.frac, patch_size=args.patch_size, templates_permille=tpm, stride=stride)
    # the literal form: the best 10 % of the patches, every template
    judged_lit = TR.evaluate(mlp, make(valid_seed + 1000), args.valid_events, bank, psi_det, frac=0.1,
                             patch_size=args.patch_size, templates_permille=1000, stride=stride)
    t_valid = time.perf_counter() - t0
    report = {"psi_det": psi_det, "stride": stride,
              "train_examples": int(X.shape[0]), "train_positive": int(y.sum().item()),
              "train_events": args.train_events, "n_tmpl": args.n_tmpl, "steps": args.steps,
              "batch": args.batch, "lr": args.lr, "losses": losses, "collect_s": t_collect,
              "train_s": t_train, "valid_s": t_valid, "patch_recall_trained": rec,
              "patch_recall_untrained": rec_un, "judged_trained": judged,
              "judged_untrained": judged_un, "judged_trained_top10pct_all_templates": judged_lit}
    print(json.dumps(report), flush=True)
    if args.report:
        os.makedirs(os.path.dirname(os.path.abspath(args.report)), exist_ok=True)
        with open(args.report, "w") as f:
            json.dump(report, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())

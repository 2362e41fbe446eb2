#!/usr/bin/env python3
"""Train the learned block screen and calibrate its skip threshold.

Training data are (grid batch, shell pair) blocks that the plain FP64 method
computes for fresh 96-atom clusters (the 96-atom workload's recipe: 1:2
heavy:light atoms, scale basis up to d, 50 x 8 x 20 points per atom, 200
occupied columns) with seeds that no benchmark workload uses.  Each block's
features and label come from snk_learn_collect on a handle with the rigorous
sn-LinK screen at 1e-10, the screen the learned one runs behind.  The MLP is
trained by snk_mlp_train (the library's FP32 forward/backward/Adam kernels).

Calibration: on one more fresh instance, K with the learned screen is
compared with K of the same form without it (rigorous screen at 1e-10, FP32
integrals below an estimate of 3e-4, double-FP32 integrals above it,
split GEMMs) for a ladder of thresholds: first the skip threshold (the
largest whose max|dK| stays within a fifth of the 1e-8 tolerance), then, with
that skip threshold, the tier threshold below which a double-FP32 block moves
to the FP32 tier (the largest keeping skip and moves together within 0.3 of
the tolerance).  Both are stored with the weights.

    python -m paper_2303_14280_gb300.train_screen [--instances 20] [--out PATH]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "screen_mlp.npz")
TRAIN_SEED0 = 3000
TOLERANCE = 1e-8
THRESHOLDS = (-12.0, -11.5, -11.0, -10.75, -10.5, -10.25, -10.0, -9.75, -9.5)
BUDGET = 0.2  # share of the tolerance the skipped blocks may use
FP32_THRESHOLDS = (-6.0, -5.5, -5.0, -4.75, -4.5, -4.25, -4.0, -3.75, -3.5)
FP32_BUDGET = 0.3  # share of the tolerance skipped and moved blocks may use together


def instance(seed, device):
    sys.path.insert(0, os.path.dirname(HERE))
    import synth
    return synth.cluster(96, seed, n_occ=200, device=device)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--instances", type=int, default=20)
    ap.add_argument("--stride", type=int, default=24, help="sample every stride-th grid batch")
    ap.add_argument("--cap", type=int, default=300000, help="blocks per instance at most")
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--under-weight", type=float, default=8.0)
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--calibrate-only", action="store_true",
                    help="keep the weights of --out and redo the calibration")
    args = ap.parse_args(argv)

    import torch
    import paper_2303_14280_gb300 as snk

    dev = torch.device("cuda", torch.cuda.current_device())
    if args.calibrate_only:
        w, _, meta = snk.trained_screen(args.out)
        calibrate(snk, w, meta, args, dev)
        return 0
    feats, labs = [], []
    t0 = time.perf_counter()
    for k in range(args.instances):
        p = instance(TRAIN_SEED0 + k, dev)
        eng = snk.Engine(p.basis, p.grid, eps=1e-10)
        eng.set_density(p.P)
        f, lab = eng.learn_collect(stride=args.stride, cap=args.cap)
        eng.close()
        feats.append(f)
        labs.append(lab)
        print(f"instance {k}: {f.shape[0]} blocks", flush=True)
    F, L = np.concatenate(feats), np.concatenate(labs)
    t_collect = time.perf_counter() - t0
    t0 = time.perf_counter()
    w, hist = snk.mlp_train(F, L, epochs=args.epochs, batch=args.batch, lr=args.lr,
                            under_weight=args.under_weight, seed=0)
    t_train = time.perf_counter() - t0
    print(f"{F.shape[0]} blocks collected in {t_collect:.1f} s, trained in {t_train:.1f} s, "
          f"loss {hist[0]:.4g} -> {hist[-1]:.4g}", flush=True)

    meta = {"train_seeds": [TRAIN_SEED0, TRAIN_SEED0 + args.instances - 1], "blocks": int(F.shape[0]),
            "stride": args.stride, "cap": args.cap, "epochs": args.epochs, "batch": args.batch, "lr": args.lr,
            "under_weight": args.under_weight, "loss_history": [float(x) for x in hist]}
    calibrate(snk, w, meta, args, dev)
    return 0


def calibrate(snk, w, meta, args, dev):
    """Skip and tier thresholds on a held-out instance (see the module text)."""
    p = instance(TRAIN_SEED0 + args.instances, dev)
    form = dict(eps=1e-10, precision="mixed", fp32_bound=3e-4, gemm="split", ds_integrals=1)
    rig = snk.Engine(p.basis, p.grid, **form)
    rig.set_density(p.P)
    K0 = rig.build_K()
    s0 = rig.stats()
    rig.close()

    def run(skip, fp32):
        e = snk.Engine(p.basis, p.grid, screen="learned", learned_skip=skip, learned_fp32=fp32, **form)
        e.screen_load(w)
        e.set_density(p.P)
        K1 = e.build_K()
        s = e.stats()
        e.close()
        return {"skip": skip, "fp32": fp32, "max_abs_dK": float(np.max(np.abs(K1 - K0))),
                "skipped": int(s["pairs_learned_skipped"]), "fp32_pairs": int(s["pairs_kept_fp32"]),
                "kept_rigorous": int(s0["pairs_kept"]), "fp32_pairs_rigorous": int(s0["pairs_kept_fp32"])}

    table, chosen = [], THRESHOLDS[0]
    for t in THRESHOLDS:
        table.append(run(t, -99.0))
        print(json.dumps(table[-1]), flush=True)
        if table[-1]["max_abs_dK"] > BUDGET * TOLERANCE:
            break
        chosen = t
    table32, chosen32 = [], -99.0
    for t in FP32_THRESHOLDS:
        table32.append(run(chosen, t))
        print(json.dumps(table32[-1]), flush=True)
        if table32[-1]["max_abs_dK"] > FP32_BUDGET * TOLERANCE:
            break
        chosen32 = t
    meta.update(holdout_seed=TRAIN_SEED0 + args.instances, calibration=table, calibration_fp32=table32,
                tolerance=TOLERANCE, budget=BUDGET, fp32_budget=FP32_BUDGET, form=form,
                fp32_threshold=chosen32)
    np.savez(args.out, weights=w, threshold=np.float32(chosen), meta=json.dumps(meta))
    print(f"skip threshold {chosen}, tier threshold {chosen32}; wrote {args.out}", flush=True)


if __name__ == "__main__":
    sys.exit(main())

"""Train the config-5 temperature-field surrogate and write its weights.

Generates the training fields with the library's own batched solver
(`surr_solve`, FP32, 2000 ADI steps at dt = 50 tau_exp of a k = 400, C = 1e6
cell), trains the FNO with `surr_train` (minibatch 64, Adam, cosine decay),
measures the rise-relative max error on held-out solver runs (`surr_errors`)
and writes the FP32 weights (`.npy`) plus a JSON summary beside them.  Every
step runs on the GPU through the C ABI; this script only orchestrates.

    python -m paper_1912_03744_gb300.train_surrogate --n-train 20480 --epochs 250 \\
        --out paper_1912_03744_gb300/weights/fno_config5.npy
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-train", type=int, default=20480)
    ap.add_argument("--n-eval", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=250)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--seed", type=int, default=5, help="seed of the training parameter draws")
    ap.add_argument("--out", required=True)
    args = ap.parse_args(argv)

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    from paper_1912_03744_gb300 import HeatSolver, Surrogate
    from workloads import fno as F
    from workloads import heat as H

    D = F.FnoDims()
    ref = H.config5_reference_problem()
    probe = HeatSolver(ref, 1.0, precision="fp64")
    dt = H.DT_FACTOR * probe.tau_exp
    probe.close()
    train = H.config5_params(args.n_train, seed=args.seed)
    held = H.config5_params(args.n_eval, seed=args.seed + 1000)
    s = Surrogate(H.config5_problem(train[0]), D, heater=H.HEATER, dt=dt, steps=2000, max_batch=args.batch)
    s.set_params(F.init_params(D, 7).astype(np.float32))
    fields = torch.empty((args.n_train + args.n_eval, D.Nz, D.Nr), dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    s.solve(np.concatenate([train, held]), out=fields)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    loss = s.train(train, fields[:args.n_train], epochs=args.epochs, batch=args.batch, lr=args.lr,
                   lr_min_frac=0.02, seed=1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    err = s.errors(held, fields[args.n_train:])
    w = s.get_params()
    s.close()
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.save(args.out, w)
    summary = {"dims": {"Nz": D.Nz, "Nr": D.Nr, "C": D.C, "mz": D.mz, "mr": D.mr, "L": D.L},
               "steps": 2000, "dt": dt, "n_train": args.n_train, "train_seed": args.seed, "epochs": args.epochs,
               "lr": args.lr, "batch": args.batch, "final_loss": loss, "data_s": t_data, "train_s": t_train,
               "held_out": {"n": args.n_eval, "seed": args.seed + 1000,
                            "p50": float(np.percentile(err, 50)), "p90": float(np.percentile(err, 90)),
                            "p99": float(np.percentile(err, 99)), "max": float(err.max()),
                            "frac_le_1pct": float(np.mean(err <= 0.01))}}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()

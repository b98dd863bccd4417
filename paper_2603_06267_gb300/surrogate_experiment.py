"""Surrogate experiment: simulate steering patterns with the batched DG-SEM
solver, train the surrogate with the project's kernels, and report its
held-out error against the solver and its speed in patterns per second.

    python -m paper_2603_06267_gb300.surrogate_experiment [--train 4096 --test 512 --epochs 60]

Prints one JSON line.  Everything runs on cuda:0.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=4096)
    ap.add_argument("--test", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--n-out", type=int, default=512)
    ap.add_argument("--hidden", type=int, default=2048)
    args = ap.parse_args()
    import torch
    import workloads as W
    from paper_2603_06267_gb300 import surrogate as S

    torch.cuda.set_device(0)
    n = args.train + args.test
    t0 = time.perf_counter()
    X, Y, t_solve = S.generate_dataset(W.surrogate_array, n, batch=64, seed=11, n_out=args.n_out)
    t_data = time.perf_counter() - t0
    scale = float(np.abs(Y[:args.train]).max())
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.tensor(Y / scale, device="cuda")
    d_in = X.shape[1]
    t_out = args.n_out
    t0_len = t_out // 16
    net = S.Surrogate(d_in=d_in, hidden=args.hidden, n_hidden=3, c0=256, t0=t0_len, conv_ch=(128, 128, 64, 64),
                      max_batch=max(args.batch, 64 * ((args.test + 63) // 64)), seed=12)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = S.train(net, Xd[:args.train], Yd[:args.train], epochs=args.epochs, batch=args.batch, lr=args.lr,
                   lr_decay=0.96)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    nt = 64 * (args.test // 64)
    pred = torch.zeros((nt, 64, t_out), dtype=torch.float32, device="cuda")
    net.forward(Xd[args.train:args.train + nt], pred)
    torch.cuda.synchronize()
    reps = 20
    t2 = time.perf_counter()
    for _ in range(reps):
        net.forward(Xd[args.train:args.train + nt], pred)
    torch.cuda.synchronize()
    t_inf = (time.perf_counter() - t2) / reps
    truth = Yd[args.train:args.train + nt].cpu().numpy().astype(np.float64)
    p = pred.cpu().numpy().astype(np.float64)
    rel = float(np.linalg.norm(p - truth) / np.linalg.norm(truth))
    per = [float(np.linalg.norm(p[i] - truth[i]) / np.linalg.norm(truth[i])) for i in range(nt)]
    const = Yd[:args.train].mean(dim=0, keepdim=True).cpu().numpy().astype(np.float64)
    rel_const = float(np.linalg.norm(np.broadcast_to(const, truth.shape) - truth) / np.linalg.norm(truth))
    out = {
        "experiment": "surrogate_screening", "workload": "surrogate_array (8x8 PMUTs, 1.91M nodes, 2950 steps)",
        "train_patterns": args.train, "test_patterns": nt, "features": d_in, "output": [64, t_out],
        "params": net.n, "epochs": args.epochs, "final_train_loss": hist[-1],
        "test_rel_l2": rel, "test_rel_l2_median_pattern": float(np.median(per)),
        "constant_prediction_rel_l2": rel_const,
        "solver_patterns_per_s": n / t_solve, "surrogate_patterns_per_s": nt / t_inf,
        "speedup": (nt / t_inf) / (n / t_solve),
        "seconds": {"data": t_data, "solver": t_solve, "train": t_train, "inference_per_batch": t_inf},
    }
    print(json.dumps(out), flush=True)
    net.close()


if __name__ == "__main__":
    main()

"""Surrogate experiment: simulate steering patterns with the batched DG-SEM
solver, train the surrogate with the project's kernels, and report its
held-out error against the solver and its speed in patterns per second.

    python -m paper_2603_06267_gb300.surrogate_experiment [--train 4096 --test 512 --epochs 60]
    python -m paper_2603_06267_gb300.surrogate_experiment --timing [--d-in 2048 --batch 512]
    python -m paper_2603_06267_gb300.surrogate_experiment --gemm 512 2048 2048

--timing measures the forward pass and one training step of the network at
the given width on random inputs (no solver data); --gemm the rate of one
dense-layer product C = A B^T on the tensor cores.  Prints one JSON line.
Everything runs on cuda:0.
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
    ap.add_argument("--d-in", type=int, default=2048)
    ap.add_argument("--timing", action="store_true")
    ap.add_argument("--gemm", type=int, nargs=3, default=None, metavar=("M", "N", "K"))
    args = ap.parse_args()
    import torch
    import workloads as W
    from paper_2603_06267_gb300 import surrogate as S

    torch.cuda.set_device(0)
    if args.gemm:
        M, N, K = args.gemm
        tf = S.gemm_tflops(M, N, K, reps=20)
        print(json.dumps({"experiment": "dense_product_rate", "M": M, "N": N, "K": K, "tflops": tf}), flush=True)
        return
    if args.timing:
        timing(args, torch, S)
        return
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


def timing(args, torch, S):
    """Forward and training-step time of the experiment-width network on
    random inputs, with the flop counts of its dense and convolution parts."""
    B = args.batch
    conv = (128, 128, 64, 64)
    net = S.Surrogate(d_in=args.d_in, hidden=args.hidden, n_hidden=3, c0=256, t0=32, conv_ch=conv, max_batch=B,
                      seed=13)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((B, args.d_in), device="cuda", generator=g)
    t = torch.randn((B, net.c_out, net.t_out), device="cuda", generator=g)
    y = torch.zeros((B, net.c_out, net.t_out), device="cuda")
    for _ in range(3):
        net.forward(x, y)
        net.backward(x, t)
    torch.cuda.synchronize()
    reps = 20
    t0 = time.perf_counter()
    for _ in range(reps):
        net.forward(x, y)
    torch.cuda.synchronize()
    t_fwd = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        net.backward(x, t)
        net.adam(1e-4)
    torch.cuda.synchronize()
    t_step = (time.perf_counter() - t0) / reps
    H, nd = args.hidden, 256 * 32
    dense = 2.0 * B * (args.d_in * H + 2 * H * H + H * nd)
    ci, ti, convf = 256, 32, 0.0
    for co in conv:
        convf += 2.0 * B * co * (2 * ti) * ci * 2          # two of the four taps reach each output sample
        ci, ti = co, 2 * ti
    out = {"experiment": "surrogate_timing", "batch": B, "d_in": args.d_in, "hidden": H, "params": net.n,
           "forward_ms": t_fwd * 1e3, "train_step_ms": t_step * 1e3,
           "forward_gflop": {"dense": dense / 1e9, "transposed_conv": convf / 1e9},
           "forward_tflops": (dense + convf) / t_fwd / 1e12,
           "patterns_per_s": B / t_fwd}
    print(json.dumps(out), flush=True)
    net.close()


if __name__ == "__main__":
    main()

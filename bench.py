#!/usr/bin/env python
"""Benchmark of the explicit DG-SEM + reduced-order PMUT time step.

Metric: DG-SEM Gdof-steps/s = (unique GLL nodes) x (drive patterns) x (time
steps) / seconds, at FP64 or FP32/mixed precision, on synthetic inputs with
the shapes of the paper's problem class (see workloads/).

Default workload: 64 beam-steering drive patterns on the 1024-PMUT mesh
(primary 128x128x16 hexes N=4 + secondary 64x64x96 hexes N=6, 2:1 interface,
102.6M nodes), FP32/mixed precision, one launch sequence for all patterns.

`python bench.py --gpus N --steps K --warmup W` prints one JSON line.  Under
torchrun (N > 1) every rank runs its own batch of patterns (replicas; the
path needs no data exchange) and rank 0 reports the max time over ranks.
`--impl reference` times the CPU oracle on a bounded sample of the same
workload instead.  `--workload hex_c3_like` (or hex_c2_like) measures the
general-hexahedron path (include/dghex.h) on the same mesh class with
displaced vertices and a bent interface.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

# DRAM bytes per launch of the dominant kernel measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by
# (workload, precision, kernel kind); see profiles/.  None: not measured for
# the current kernel.
NCU_TRAFFIC_PER_LAUNCH = {
    # profiles/vol_kernel_f32_N6_dram_traffic_config3.md (variant 9, the one
    # the autotuner picks): 707.4 MB read + 640.8 MB written per launch at batch 1
    # on the config-3 mesh (secondary box); the traffic scales with the number of
    # patterns (each has its own state, the operator lives in the parameter block)
    ("config4_batched", "fp32", "vol_secondary"): 1.3482e9 * 64,
    ("config3_array32", "fp32", "vol_secondary"): 1.3482e9,
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="config4_batched",
                    choices=["config4_batched", "config4b_uneven", "config3_array32", "config2_array16",
                             "config1_single_pmut", "hex_c3_like", "hex_c2_like"])
    ap.add_argument("--precision", default=None, choices=["fp32", "fp64"])
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-parity", action="store_true",
                    help="skip the FP32-vs-FP64 check of the benchmarked configuration (FP32 lines)")
    ap.add_argument("--tiles", default=None,
                    help="comma-separated volume-kernel tile variant per box, or element-stiffness variant per "
                         "domain on general hexahedra (skips the autotuner)")
    ap.add_argument("--layers", default=None,
                    help="comma-separated element layers per CTA of the volume kernel, per box (0 = automatic): "
                         "profiles a one-pattern case in the launch shape of a many-pattern run")
    return ap.parse_args(argv)


def make_workload(name, batch):
    if name == "config4_batched":
        return W.config4_batched(nsteps=1, batch=batch or 64)
    if name == "config3_array32":
        return W.config3_array32(nsteps=1, batch=batch or 1)
    if name == "config2_array16":
        w = W.config2_array16(nsteps=1)
    else:
        w = W.config1_single_pmut(nsteps=1)
    if batch and batch > 1:
        w.batch = batch
        w.drive_delay = np.repeat(w.drive_delay, batch, axis=0)
        w.drive_amp = np.repeat(w.drive_amp, batch, axis=0)
    return w


def replica_workload(name, batch, rank, world):
    """The workload rank `rank` of `world` runs.  The path shards as replicas:
    every rank advances its own batch of independent drive patterns and no
    data moves between ranks (config 4: its own seeded steering angles)."""
    w = make_workload(name, batch)
    if w.batch > 1 and world > 1 and name == "config4_batched":
        w.drive_delay, w.drive_amp, _ = W.steering_patterns(w.pmuts.centers, w.batch, seed=4 + 1000 * rank)
    return w


def max_over_ranks(x, dist, device="cuda"):
    """The largest value of x over all ranks (x itself on one rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ndof, batch, steps, world, seconds):
    """Gdof-steps/s of the whole job: every rank advanced batch patterns of
    ndof nodes by steps steps within `seconds` (the slowest rank's time)."""
    return ndof * batch * steps * world / seconds / 1e9


def default_precision(name):
    return "fp32" if name in ("config4_batched", "config4b_uneven", "config3_array32", "hex_c3_like",
                              "hex_c2_like") else "fp64"


def is_hex(name):
    return name.startswith("hex_")


def make_hex_workload(name, batch):
    from workloads import hex as H
    if name == "hex_c3_like":
        return H.hex_c3_like(nsteps=1, batch=batch or 64)
    return H.hex_c2_like(nsteps=1, batch=batch or 8)


def oracle_sample(name):
    """Bounded sample of the workload for the CPU oracle: the same element
    types, orders and PMUT model on a crop the oracle assembles in seconds."""
    if is_hex(name):
        from workloads import hex as H
        return H.distorted_two_domain(nx_p=8, nz_p=4, nx_s=4, nz_s=6, n_pmut_side=2, nsteps=1)
    if name == "config1_single_pmut":
        return W.config1_single_pmut(nsteps=1)
    return W.small_two_domain(nx_p=8, nz_p=4, nx_s=4, nz_s=8, n_pmut_side=2, nsteps=1)


def _loop_seconds(P, nsteps, dt):
    """Wall time of the oracle's time loop alone: the run's per-step callback
    marks the end of step 0 and of the last step, so setup inside run() (the
    receiver matrix, the drive array, the initial state) stays outside; the
    first step's share is added back from the per-step mean."""
    marks = {}

    def cb(n, **_):
        if n == 0 or n == nsteps - 1:
            marks[n] = time.perf_counter()

    P.run(nsteps=nsteps, dt=dt, batch=1, callback=cb)
    return (marks[nsteps - 1] - marks[0]) * nsteps / (nsteps - 1)


def _oracle_worker_init(name):
    global _WORKER
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    w = oracle_sample(name)
    P = _oracle_problem(w)
    _WORKER = (P, P.stable_dt())


def _oracle_worker_run(nsteps):
    P, dt = _WORKER
    return _loop_seconds(P, nsteps, dt)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def time_oracle(name, seconds=15.0, chunk=None, parallel=True):
    """Oracle Gdof-steps/s on the bounded sample, time loop only: on one host
    thread (scipy's sparse mat-vec and numpy's element-wise kernels run on one
    core), and on every host core as independent processes, one drive pattern
    each (the patterns of a batch are independent problems).  Returns the
    all-core figure (and the one-thread figure inside the sample text)."""
    w = oracle_sample(name)
    P = _oracle_problem(w)
    dt = P.stable_dt()
    n = 8
    while True:
        el = _loop_seconds(P, n, dt)
        if el > 0.5 or n >= 1 << 20:
            break
        n *= 4
    per_step = el / n
    S = max(2, int(seconds / 2 / per_step)) if chunk is None else max(2, chunk)
    el = _loop_seconds(P, S, dt)
    one = P.nh * S / el / 1e9
    sample = (f"{w.name}: primary {_nelem(w.domains[0])} N={w.domains[0].order}"
              + (f" + secondary {_nelem(w.domains[1])} N={w.domains[1].order}" if len(w.domains) > 1 else "")
              + f", {P.nh} nodes, {S} steps per pattern, time loop only")
    cores = host_cores()
    if not parallel or cores < 2:
        return one, sample + f"; 1 thread: {one:.4g} Gdof-steps/s", 1, one
    import multiprocessing as mp
    ctx = mp.get_context("spawn")           # no fork after the GPU is in use
    with ctx.Pool(cores, initializer=_oracle_worker_init, initargs=(name,)) as pool:
        pool.map(_oracle_worker_run, [2] * cores, chunksize=1)      # every worker built and warm
        t0 = time.perf_counter()
        pool.map(_oracle_worker_run, [S] * cores, chunksize=1)
        wall = time.perf_counter() - t0
    allc = P.nh * S * cores / wall / 1e9
    sample += (f"; {cores} processes x 1 pattern each (wall time of the pool, loops only); "
               f"1 thread: {one:.4g} Gdof-steps/s")
    return allc, sample, cores, one


def _oracle_problem(w):
    if hasattr(w, "pmut_faces"):
        from oracle import hex_oracle as HO
        return HO.HexOracleProblem(w)
    from oracle import dgsem_oracle as O
    return O.OracleProblem(w)


def _nelem(d):
    return tuple(d.nelem) if hasattr(d, "nelem") else tuple(d.lattice)


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, gpu_index):
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return None
        rows = [[x.strip() for x in r] for r in rows if len(r) >= 9 and r[0].strip() == str(gpu_index)]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# arithmetic peaks derived from unit counts and the maximum SM clock (no measured figure):
# FP32 152 SMs x 128 lanes x 2 flop (FMA) x 2.070 GHz; FP64 the nominal GB300 rate
FP32_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_TFLOPS = 1.25


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def run_reference(args):
    """Reference arm: the CPU oracle as it stands on a bounded sample of the
    workload, on every host core (one process and one drive pattern per core;
    time loops only, setup outside), K timed steps of about 0.5 s each."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = args.workload
    w = oracle_sample(name)
    P = _oracle_problem(w)
    dt = P.stable_dt()
    per = _loop_seconds(P, 8, dt) / 8
    chunk = max(2, int(0.5 / per))
    cores = host_cores()
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_oracle_worker_init, initargs=(name,)) as pool:
        for _ in range(max(1, args.warmup)):
            pool.map(_oracle_worker_run, [chunk] * cores, chunksize=1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.map(_oracle_worker_run, [chunk] * cores, chunksize=1)
        el = time.perf_counter() - t0
    value = P.nh * chunk * cores * args.steps / el / 1e9
    sample = (f"{w.name}: {P.nh} nodes, {chunk} oracle time steps per bench step on each of {cores} processes "
              f"(one drive pattern each; same element sizes/orders/PMUT model as {name}; time loops only)")
    out = {"impl": "reference", "metric": "DG-SEM Gdof-steps/s", "value": value, "unit": "Gdof-steps/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": name, "precision": "fp64 (oracle)", "sample": sample},
           "cpu_baseline": {"value": value, "unit": "Gdof-steps/s", "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "Gdof-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2603_06267_gb300 import dgsem

    name = args.workload
    if is_hex(name):
        main_hex(args, torch, dist, rank, world, local)
        return
    if name == "config4b_uneven":
        main_multi(args, torch, dist, rank, world, local)
        return
    prec_name = args.precision or default_precision(name)
    prec = dgsem.DGSEM_FP32_MIXED if prec_name == "fp32" else dgsem.DGSEM_FP64
    w = replica_workload(name, args.batch, rank, world)
    B = w.batch
    sol = dgsem.Solver(w)
    ndof = sol.ndof
    # untimed setup: pick the volume-kernel tile shape per box for this batch
    if args.tiles:
        tiles = [int(t) for t in args.tiles.split(",")]
        dgsem.dgsem_set_tiles(sol.ctx, prec, tiles)
    else:
        tiles = dgsem.dgsem_autotune(sol.ctx, prec, B, len(w.domains), reps=2)
    if args.layers:
        dgsem.dgsem_set_layers(sol.ctx, [int(t) for t in args.layers.split(",")])
    K_p = w.pmuts.n_pmut if w.pmuts is not None else 0
    R = w.receivers.shape[0]
    S_tot = args.warmup + args.steps
    drive_all = w.drive(sol.dt, S_tot + args.steps, B)
    stream = torch.cuda.current_stream()
    d_warm = torch.tensor(np.ascontiguousarray(drive_all[:, :, :args.warmup]), device="cuda")
    d_time = torch.tensor(np.ascontiguousarray(drive_all[:, :, args.warmup:S_tot]), device="cuda")
    tr_warm = torch.zeros((B, R, args.warmup), dtype=torch.float64, device="cuda")
    tr_time = torch.zeros((B, R, args.steps), dtype=torch.float64, device="cuda")

    # warm-up from rest
    sol.run(drive=d_warm, precision=prec, nsteps=args.warmup, traces=tr_warm)
    torch.cuda.synchronize()
    clocks_dir = os.environ.get("DGSEM_BENCH_CLOCKS_DIR", tempfile.gettempdir())
    clocks_path = os.path.join(clocks_dir, f".bench_clocks_{rank}.csv")
    dgsem.dgsem_profile(sol.ctx, False)      # reset launch counters
    with ClockSampler(clocks_path) as cs:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sol.run(drive=d_time, precision=prec, nsteps=args.steps, traces=tr_time, flags=dgsem.DGSEM_RUN_CONTINUE,
                stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ms = e0.elapsed_time(e1)
        launches = sum(dgsem.dgsem_kernel_stats(sol.ctx, k)[1] for k in range(5))
        # per-kernel timing pass (CUDA events around each launch)
        dgsem.dgsem_profile(sol.ctx, True)
        sol.run(drive=d_time, precision=prec, nsteps=args.steps, traces=tr_time, flags=dgsem.DGSEM_RUN_CONTINUE,
                stream=stream.cuda_stream)
        kstats = [dgsem.dgsem_kernel_stats(sol.ctx, k) for k in range(5)]
        dgsem.dgsem_profile(sol.ctx, False)
        # end to end through host buffers (pinned), copies inside the timed region
        e2e = None
        if not args.no_e2e:
            h_drive = torch.from_numpy(np.ascontiguousarray(drive_all[:, :, S_tot:S_tot + args.steps])).pin_memory()
            h_tr = torch.zeros((B, R, args.steps), dtype=torch.float64).pin_memory()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sol.run(drive=h_drive, precision=prec, nsteps=args.steps, traces=h_tr,
                    flags=dgsem.DGSEM_RUN_CONTINUE, stream=stream.cuda_stream)
            e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
            e2e = {"value": whole_job_rate(ndof, B, args.steps, world, e2e_s), "unit": "Gdof-steps/s",
                   "h2d_bytes_per_step": int(B * K_p * 8), "d2h_bytes_per_step": int(B * R * 8)}
    finite = bool(torch.isfinite(tr_time).all().item())
    ms = max_over_ranks(ms, dist)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    value = whole_job_rate(ndof, B, args.steps, world, ms / 1e3)
    # roofline of the dominant kernel
    names = BOX_KERNELS
    es = 4 if prec == dgsem.DGSEM_FP32_MIXED else 8
    peaks = measured_peaks()
    alu = alu_peaks(dgsem, stream)
    roof = box_roofline(kstats, w.domains, B, prec == dgsem.DGSEM_FP32_MIXED, peaks["hbm_gbs"] if peaks else None,
                        lambda kernel: NCU_TRAFFIC_PER_LAUNCH.get((name, prec_name, kernel)),
                        fp64_peak=alu.get("fp64_tflops"))
    parity = None
    if not args.no_parity and prec == dgsem.DGSEM_FP32_MIXED and w.pmuts is not None:
        parity = live_parity(dgsem, sol, w, torch)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, sample, cores, one = time_oracle(name, seconds=15.0)
        cpu = {"value": v, "unit": "Gdof-steps/s", "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread_value": one}
    clocks = cs.summary(local)
    out = {
        "metric": "DG-SEM Gdof-steps/s", "value": value, "unit": "Gdof-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == dgsem.DGSEM_FP32_MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": name, "precision": "fp32-mixed" if prec == dgsem.DGSEM_FP32_MIXED else "fp64",
                   "ndof": ndof, "batch_per_gpu": B, "n_pmut": K_p, "receivers": R,
                   "parallelism": f"replicas x{world}" if world > 1 else "single-gpu",
                   "tiles": [int(t) for t in tiles],
                   **({"layers_per_cta": [int(t) for t in args.layers.split(",")]} if args.layers else {}),
                   "l2": "state larger than L2" if ndof * B * 3 * es > 129e6 else "state fits in L2"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        "kernels": {names[k]: {"ms_total": kstats[k][0], "launches": kstats[k][1]} for k in range(5) if kstats[k][1]},
        "alu_peaks": alu, "parity": parity,
        "finite": finite,
    }
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


BOX_KERNELS = ["pmut_recv", "iface", "vol_primary", "vol_secondary", "pml"]

# oracle-parity tests of the benchmarked kernels and configuration (run by
# `pytest -m gpu`); their measured errors are printed by the tests
PARITY_TESTS = [
    "tests/test_gpu_fullsize_sampled.py: config-4 mesh, 64 patterns FP32 / 8 FP64, every tile variant, "
    "sampled receivers vs the oracle on local crops",
    "tests/test_gpu_launch_shape.py: every CTA through all layers of its box, 64 patterns, every tile "
    "variant, each pattern vs its own oracle column",
    "tests/test_gpu_config3_crop.py: cropped config 3 (6.5M nodes), 8000 steps vs the stored oracle run; "
    "traces, q(t), energy",
    "tests/test_gpu_precision_scale.py: config 3 (8000 steps) and config 4 (8 patterns) FP32 vs FP64",
]


def alu_peaks(dgsem, stream):
    """FP64 and packed-FP32 FMA rates of this GPU, measured now (untimed)."""
    out = {}
    for key, prec in (("fp64_tflops", dgsem.DGSEM_FP64), ("fp32_tflops", dgsem.DGSEM_FP32_MIXED)):
        try:
            out[key] = dgsem.dgsem_measure_peak(prec, stream.cuda_stream)
        except Exception as e:  # the line still reports, against nominal figures
            out[key + "_error"] = str(e)
    return out


def live_parity(dgsem, sol32, w, torch, nsteps=400, nb=8):
    """FP32 (the benchmarked batch) against FP64 (its first nb patterns) on
    the benchmarked mesh from rest over nsteps steps, at 64 receivers 0.15 mm
    above the array (the 2 mm receivers see nothing that early): relative L2
    per pattern."""
    pm = w.pmuts
    lo, hi = pm.centers.min(axis=0), pm.centers.max(axis=0)
    gx = np.linspace(lo[0], hi[0], 8)
    gy = np.linspace(lo[1], hi[1], 8)
    X, Y = np.meshgrid(gx, gy, indexing="ij")
    rec = np.stack([X.ravel(), Y.ravel(), np.full(64, 0.15e-3)], axis=1)
    drive = w.drive(sol32.dt, nsteps, w.batch)
    t32 = sol32.run(drive=drive, precision=dgsem.DGSEM_FP32_MIXED, nsteps=nsteps, receivers=rec)
    sol64 = dgsem.Solver(w)
    t64 = sol64.run(drive=np.ascontiguousarray(drive[:nb]), precision=dgsem.DGSEM_FP64, batch=nb, nsteps=nsteps,
                    receivers=rec)
    sol64.close()
    errs = [float(np.linalg.norm(t32[b] - t64[b]) / np.linalg.norm(t64[b])) for b in range(nb)]
    return {"fp32_vs_fp64_gpu": {"patterns": nb, "steps": nsteps, "receivers": "8x8 over the array at z = 0.15 mm",
                                 "rel_l2_max": max(errs), "rel_l2_median": float(np.median(errs))},
            "oracle_parity_tests": PARITY_TESTS}


def box_roofline(kstats, domains, B, fp32, hbm_gbs, traffic_of, fp64_peak=None):
    """Roofline block of the box path for its dominant volume kernel, from
    per-kind (total ms, launches).  Algorithmic bytes per launch: p read, v
    read and written, p_next written once per node of the box and pattern
    (4 words); FP32 reports against the copy bandwidth, FP64 against the FP64
    rate with 2 (3 (N + 2) + 4) flops per node (the three assembled 1-D
    stencils and the update).  traffic_of(kernel) gives the ncu DRAM bytes
    per launch where a capture of this kernel exists (None otherwise)."""
    kdom = max(range(4), key=lambda k: kstats[k][0])
    if kdom < 2 or kstats[kdom][1] == 0:
        return None
    es = 4 if fp32 else 8
    name = BOX_KERNELS[kdom]
    d = domains[kdom - 2]
    nodes = int(np.prod([d.nelem[i] * d.order + 1 for i in range(3)]))
    alg_bytes = nodes * B * 4 * es
    avg_s = kstats[kdom][0] / kstats[kdom][1] / 1e3
    achieved = alg_bytes / avg_s / 1e9
    if fp32:
        peak = hbm_gbs if hbm_gbs else 6800.0
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_of(name) if B in (1, 64) else None, "kernel": name,
                "peak_source": "measured" if hbm_gbs else "fallback", "alg_bytes_per_launch": alg_bytes}
    flop_per_node = 2 * (3 * (d.order + 2) + 4)
    achieved_f = nodes * B * flop_per_node / avg_s / 1e12
    peak = fp64_peak if fp64_peak else FP64_TFLOPS
    return {"bound": "alu", "achieved": achieved_f, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved_f / peak, "traffic": traffic_of(name), "kernel": name,
            "peak_source": "measured in this run: DFMA probe (dgsem_measure_peak)" if fp64_peak
            else "nominal FP64 (no measured FP64 peak)", "hbm_achieved_gbs": achieved}


HEX_KERNELS = ["pmut", "vol", "iface", "update", "tail", "pml"]


def hex_roofline(kstats, orders, nelem, ndof, B, fp32, hbm_gbs, alu_peaks=None):
    """Roofline block of the general-hexahedron step for its dominant kernel
    (element stiffness or update), from per-kind (total ms, launches).

    Algorithmic bytes per launch: stiffness (per launch averaged over the
    domains) p once per node, the element-local residual slots written, the
    geometric factors and node ids once; update: p in, p out, v in and out,
    the slots read, M^-1 and the node's slot list.  Algorithmic flops of the
    stiffness per element and member: 12 n^4 + 18 n^3 (reference gradient and
    transposed derivative along three directions, 2 x 3 n^4 FMA; geometric-
    factor product, 9 n^3 FMA).  Above the ridge point the arithmetic pipe
    bounds the kernel and the block reports TFLOP/s against it."""
    es = 4 if fp32 else 8
    peak = hbm_gbs if hbm_gbs else 6800.0
    nl = [(o + 1) ** 3 for o in orders]
    ploc = sum(a * b for a, b in zip(nl, nelem))              # element-local nodes = volume slots
    vol_bytes = (ndof * B * es + ploc * B * es + ploc * (6 * es + 4)) / len(orders)
    upd_bytes = ndof * B * 4 * es + ploc * B * es + ndof * (es + 4) + ploc * 4
    alg = {"vol": vol_bytes, "update": upd_bytes}
    kdom = max((1, 3), key=lambda k: kstats[k][0])
    name = HEX_KERNELS[kdom]
    avg_s = kstats[kdom][0] / kstats[kdom][1] / 1e3
    achieved = alg[name] / avg_s / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "kernel": name, "peak_source": "measured" if hbm_gbs else "fallback",
            "alg_bytes_per_launch": alg[name]}
    if name == "vol":
        vol_flops = sum(e * B * (12 * (o + 1) ** 4 + 18 * (o + 1) ** 3) for e, o in zip(nelem, orders)) / len(orders)
        measured = (alu_peaks or {}).get("fp32_tflops" if fp32 else "fp64_tflops")
        alu_peak = measured or (FP32_TFLOPS if fp32 else FP64_TFLOPS)
        achieved_f = vol_flops / avg_s / 1e12
        if vol_flops / vol_bytes > alu_peak * 1e12 / (peak * 1e9):
            roof = {"bound": "alu", "achieved": achieved_f, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved_f / alu_peak, "traffic": None, "kernel": "vol",
                    "peak_source": ("measured in this run: packed FP32 FMA probe (dgsem_measure_peak)"
                                    if fp32 else "measured in this run: DFMA probe (dgsem_measure_peak)")
                    if measured else ("derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"
                                      if fp32 else "nominal FP64 (no measured FP64 peak)"),
                    "alg_flops_per_launch": vol_flops, "alg_bytes_per_launch": vol_bytes,
                    "hbm_achieved_gbs": achieved, "hbm_frac": achieved / peak}
    return roof


def multi_roofline(ndofs, B, fp32, ms_per_step, hbm_gbs):
    """Roofline block of a several-mesh launch: the algorithmic bytes of one
    step of every mesh (p read, v read and written, p_next written: 4 words
    per node and pattern) over the measured step time, against the copy
    bandwidth (FP32).  The meshes' volume launches run as parallel graph
    branches, so the step, not one kernel, is the unit."""
    es = 4 if fp32 else 8
    alg = sum(ndofs) * B * 4 * es
    achieved = alg / (ms_per_step / 1e3) / 1e9
    peak = hbm_gbs if hbm_gbs else 6800.0
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "kernel": "whole step (volume, interface and PMUT launches of every mesh)",
            "peak_source": "measured" if hbm_gbs else "fallback", "alg_bytes_per_step": alg}


def main_multi(args, torch, dist, rank, world, local):
    """Uneven PMUT arrays (8x8, 16x16, 24x24, 32x32, primary N=4 + secondary
    N=6 boxes) advanced together: dgsem_run_multi captures every mesh's step
    as a parallel branch of one CUDA graph; tile shapes from the autotuner."""
    from paper_2603_06267_gb300 import dgsem
    name = args.workload
    prec_name = args.precision or default_precision(name)
    prec = dgsem.DGSEM_FP32_MIXED if prec_name == "fp32" else dgsem.DGSEM_FP64
    B = args.batch or 64
    ws = W.config4b_uneven(nsteps=1, batch=B)
    if world > 1:
        for w in ws:
            w.drive_delay, w.drive_amp, _ = W.steering_patterns(w.pmuts.centers, B, seed=4 + 1000 * rank)
    sols = [dgsem.Solver(w) for w in ws]
    ctxs = [s_.ctx for s_ in sols]
    ndofs = [s_.ndof for s_ in sols]
    tiles = []
    for s_, w in zip(sols, ws):
        if args.tiles:
            t = [int(v) for v in args.tiles.split(",")]
            dgsem.dgsem_set_tiles(s_.ctx, prec, t)
        else:
            t = dgsem.dgsem_autotune(s_.ctx, prec, B, len(w.domains), reps=2)
        tiles.append([int(v) for v in t])
    S_tot = args.warmup + args.steps
    drives = [w.drive(s_.dt, S_tot + args.steps, B) for s_, w in zip(sols, ws)]
    recvs = [w.receivers for w in ws]
    R = [r.shape[0] for r in recvs]
    stream = torch.cuda.current_stream()
    d_warm = [torch.tensor(np.ascontiguousarray(d[:, :, :args.warmup]), device="cuda") for d in drives]
    d_time = [torch.tensor(np.ascontiguousarray(d[:, :, args.warmup:S_tot]), device="cuda") for d in drives]
    tr_warm = [torch.zeros((B, r, args.warmup), dtype=torch.float64, device="cuda") for r in R]
    tr_time = [torch.zeros((B, r, args.steps), dtype=torch.float64, device="cuda") for r in R]
    Bs = [B] * len(ws)
    dgsem.dgsem_run_multi(ctxs, prec, Bs, args.warmup, d_warm, recvs, traces=tr_warm, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    clocks_dir = os.environ.get("DGSEM_BENCH_CLOCKS_DIR", tempfile.gettempdir())
    clocks_path = os.path.join(clocks_dir, f".bench_clocks_{rank}.csv")
    for c in ctxs:
        dgsem.dgsem_profile(c, False)
    with ClockSampler(clocks_path) as cs:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dgsem.dgsem_run_multi(ctxs, prec, Bs, args.steps, d_time, recvs, traces=tr_time,
                              flags=dgsem.DGSEM_RUN_CONTINUE, stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ms = e0.elapsed_time(e1)
        launches = sum(dgsem.dgsem_kernel_stats(c, k)[1] for c in ctxs for k in range(5))
        e2e = None
        if not args.no_e2e:
            h_drive = [torch.from_numpy(np.ascontiguousarray(d[:, :, S_tot:S_tot + args.steps])).pin_memory()
                       for d in drives]
            h_tr = [torch.zeros((B, r, args.steps), dtype=torch.float64).pin_memory() for r in R]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dgsem.dgsem_run_multi(ctxs, prec, Bs, args.steps, h_drive, recvs, traces=h_tr,
                                  flags=dgsem.DGSEM_RUN_CONTINUE, stream=stream.cuda_stream)
            e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
            e2e = {"value": whole_job_rate(sum(ndofs), B, args.steps, world, e2e_s), "unit": "Gdof-steps/s",
                   "h2d_bytes_per_step": int(sum(B * w.pmuts.n_pmut * 8 for w in ws)),
                   "d2h_bytes_per_step": int(sum(B * r * 8 for r in R))}
    finite = all(bool(torch.isfinite(t).all().item()) for t in tr_time)
    ms = max_over_ranks(ms, dist)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    value = whole_job_rate(sum(ndofs), B, args.steps, world, ms / 1e3)
    peaks = measured_peaks()
    es = 4 if prec == dgsem.DGSEM_FP32_MIXED else 8
    roof = multi_roofline(ndofs, B, prec == dgsem.DGSEM_FP32_MIXED, ms / args.steps,
                          peaks["hbm_gbs"] if peaks else None)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, sample, cores, one = time_oracle("config4_batched", seconds=15.0)
        cpu = {"value": v, "unit": "Gdof-steps/s", "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread_value": one}
    out = {
        "metric": "DG-SEM Gdof-steps/s", "value": value, "unit": "Gdof-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == dgsem.DGSEM_FP32_MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": name, "precision": "fp32-mixed" if prec == dgsem.DGSEM_FP32_MIXED else "fp64",
                   "meshes": [w.name for w in ws], "ndof": ndofs, "ndof_total": sum(ndofs), "batch_per_mesh": B,
                   "n_pmut": [w.pmuts.n_pmut for w in ws], "receivers": R,
                   "parallelism": f"replicas x{world}" if world > 1 else "single-gpu, one graph, 4 branches",
                   "tiles": tiles,
                   "l2": "state larger than L2" if sum(ndofs) * B * 3 * es > 129e6 else "state fits in L2"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": cs.summary(local),
        "finite": finite,
    }
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main_hex(args, torch, dist, rank, world, local):
    """General hexahedra (include/dghex.h): the same step on distorted
    trilinear meshes with a bent 2:1 interface."""
    from paper_2603_06267_gb300 import dghex
    name = args.workload
    prec_name = args.precision or default_precision(name)
    prec = dghex.DGSEM_FP32_MIXED if prec_name == "fp32" else dghex.DGSEM_FP64
    w = make_hex_workload(name, args.batch)
    B = w.batch
    t0 = time.perf_counter()
    sol = dghex.HexSolver(w)
    setup_s = time.perf_counter() - t0
    ndof = sol.ndof
    # untimed setup: pick the element-stiffness launch variant per domain for this batch
    if args.tiles:
        variants = [int(t) for t in args.tiles.split(",")]
        dghex.dghex_set_volume_variant(sol.ctx, prec, variants)
    else:
        variants = dghex.dghex_autotune(sol.ctx, prec, B, len(w.domains), reps=2)
    K_p = w.pmuts.n_pmut
    R = w.receivers.shape[0]
    S_tot = args.warmup + args.steps
    drive_all = w.drive(sol.dt, S_tot + args.steps, B)
    stream = torch.cuda.current_stream()
    d_warm = torch.tensor(np.ascontiguousarray(drive_all[:, :, :args.warmup]), device="cuda")
    d_time = torch.tensor(np.ascontiguousarray(drive_all[:, :, args.warmup:S_tot]), device="cuda")
    tr_warm = torch.zeros((B, R, args.warmup), dtype=torch.float64, device="cuda")
    tr_time = torch.zeros((B, R, args.steps), dtype=torch.float64, device="cuda")
    sol.run(drive=d_warm, precision=prec, nsteps=args.warmup, traces=tr_warm)
    torch.cuda.synchronize()
    clocks_dir = os.environ.get("DGSEM_BENCH_CLOCKS_DIR", tempfile.gettempdir())
    clocks_path = os.path.join(clocks_dir, f".bench_clocks_{rank}.csv")
    dghex.dghex_profile(sol.ctx, False)
    with ClockSampler(clocks_path) as cs:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sol.run(drive=d_time, precision=prec, nsteps=args.steps, traces=tr_time, flags=dghex._dg.DGSEM_RUN_CONTINUE,
                stream=stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = sum(dghex.dghex_kernel_stats(sol.ctx, k)[1] for k in range(6))
        dghex.dghex_profile(sol.ctx, True)
        sol.run(drive=d_time, precision=prec, nsteps=args.steps, traces=tr_time, flags=dghex._dg.DGSEM_RUN_CONTINUE,
                stream=stream.cuda_stream)
        kstats = [dghex.dghex_kernel_stats(sol.ctx, k) for k in range(6)]
        dghex.dghex_profile(sol.ctx, False)
        e2e = None
        if not args.no_e2e:
            h_drive = torch.from_numpy(np.ascontiguousarray(drive_all[:, :, S_tot:S_tot + args.steps])).pin_memory()
            h_tr = torch.zeros((B, R, args.steps), dtype=torch.float64).pin_memory()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sol.run(drive=h_drive, precision=prec, nsteps=args.steps, traces=h_tr,
                    flags=dghex._dg.DGSEM_RUN_CONTINUE, stream=stream.cuda_stream)
            e2e_s = time.perf_counter() - t0
            e2e = {"value": whole_job_rate(ndof, B, args.steps, 1, e2e_s), "unit": "Gdof-steps/s",
                   "h2d_bytes_per_step": int(B * K_p * 8), "d2h_bytes_per_step": int(B * R * 8)}
    finite = bool(torch.isfinite(tr_time).all().item())
    value = whole_job_rate(ndof, B, args.steps, 1, ms / 1e3)
    peaks = measured_peaks()
    from paper_2603_06267_gb300 import dgsem as _dgsem
    alu = alu_peaks(_dgsem, stream)
    roof = hex_roofline(kstats, [d.order for d in w.domains], [d.elements.shape[0] for d in w.domains], ndof, B,
                        prec == dghex.DGSEM_FP32_MIXED, peaks["hbm_gbs"] if peaks else None, alu_peaks=alu)
    names = HEX_KERNELS
    es = 4 if prec == dghex.DGSEM_FP32_MIXED else 8
    cpu = None
    if not args.no_cpu_baseline:
        v, sample, cores, one = time_oracle(name, seconds=15.0)
        cpu = {"value": v, "unit": "Gdof-steps/s", "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread_value": one}
    out = {
        "metric": "DG-SEM Gdof-steps/s", "value": value, "unit": "Gdof-steps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == dghex.DGSEM_FP32_MIXED else "f64",
        "data": "synthetic",
        "config": {"workload": name, "precision": "fp32-mixed" if prec == dghex.DGSEM_FP32_MIXED else "fp64",
                   "ndof": ndof, "batch_per_gpu": B, "n_pmut": K_p, "receivers": R,
                   "elements": [int(d.elements.shape[0]) for d in w.domains],
                   "orders": [d.order for d in w.domains], "setup_s": setup_s,
                   "vol_variants": variants,
                   "parallelism": "single-gpu",
                   "l2": "state larger than L2" if ndof * B * 3 * es > 129e6 else "state fits in L2"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": cs.summary(local),
        "kernels": {names[k]: {"ms_total": kstats[k][0], "launches": kstats[k][1]} for k in range(6) if kstats[k][1]},
        "alu_peaks": alu,
        "finite": finite,
    }
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

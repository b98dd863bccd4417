"""Thin ctypes binding of the learned surrogate (include/surrogate.h) and the
helpers that feed it: drive-pattern features, trace resampling, dataset
generation with the DG-SEM solver, and the training loop.  All network
arithmetic runs in the CUDA kernels of libdgsem.so."""
from __future__ import annotations

import ctypes
import time
from ctypes import POINTER, byref, c_double, c_float, c_int, c_size_t, c_uint64, c_void_p

import numpy as np

from . import dgsem

SRG_EXPORTED = ["srg_create", "srg_num_params", "srg_get_params", "srg_set_params", "srg_get_grads",
                "srg_forward", "srg_backward", "srg_adam_step", "srg_train_step", "srg_gemm_bench",
                "srg_last_error", "srg_destroy"]


class SrgConfig(ctypes.Structure):
    _fields_ = [("d_in", c_int), ("hidden", c_int), ("n_hidden", c_int), ("c0", c_int), ("t0", c_int),
                ("n_conv", c_int), ("conv_ch", c_int * 8)]


_lib = None


def load():
    global _lib
    if _lib is not None:
        return _lib
    lib = dgsem.load_library()
    vp = c_void_p
    lib.srg_create.argtypes = [POINTER(SrgConfig), c_int, c_uint64, POINTER(vp)]
    lib.srg_num_params.argtypes = [vp]
    lib.srg_num_params.restype = c_size_t
    for n in ("srg_get_params", "srg_set_params", "srg_get_grads"):
        getattr(lib, n).argtypes = [vp, vp, c_size_t]
    lib.srg_forward.argtypes = [vp, vp, c_int, vp, vp]
    lib.srg_backward.argtypes = [vp, vp, vp, c_int, POINTER(c_double), vp]
    lib.srg_adam_step.argtypes = [vp, c_float, c_float, c_float, c_float, vp]
    lib.srg_train_step.argtypes = [vp, vp, vp, c_int, c_float, POINTER(c_double), vp]
    lib.srg_gemm_bench.argtypes = [c_int, c_int, c_int, c_int, POINTER(c_double), vp]
    lib.srg_last_error.restype = ctypes.c_char_p
    lib.srg_destroy.argtypes = [vp]
    lib.srg_destroy.restype = None
    for n in ("srg_create", "srg_get_params", "srg_set_params", "srg_get_grads", "srg_forward", "srg_backward",
              "srg_adam_step", "srg_train_step", "srg_gemm_bench"):
        getattr(lib, n).restype = c_int
    _lib = lib
    return lib


def _check(code, where):
    if code != 0:
        raise dgsem.DgsemError(code, where, _lib.srg_last_error().decode())


def gemm_tflops(M, N, K, reps=20, stream=None):
    """TFLOP/s of the dense-layer product C = A B^T (A [M][K], B [N][K]) on the
    tensor cores, timed with CUDA events."""
    lib = load()
    v = c_double()
    if stream is None:
        stream = dgsem._current_stream()
    _check(lib.srg_gemm_bench(M, N, K, reps, byref(v), stream), "srg_gemm_bench")
    return v.value


class Surrogate:
    """Owns one network.  x, y, target: torch CUDA float32 tensors."""

    def __init__(self, d_in, hidden=2048, n_hidden=3, c0=256, t0=32, conv_ch=(128, 128, 64, 64), max_batch=256,
                 seed=1):
        lib = load()
        cfg = SrgConfig()
        cfg.d_in, cfg.hidden, cfg.n_hidden, cfg.c0, cfg.t0 = d_in, hidden, n_hidden, c0, t0
        cfg.n_conv = len(conv_ch)
        cfg.conv_ch = (c_int * 8)(*list(conv_ch), *([0] * (8 - len(conv_ch))))
        self.cfg = dict(d_in=d_in, hidden=hidden, n_hidden=n_hidden, c0=c0, t0=t0, conv_ch=list(conv_ch))
        self.c_out = conv_ch[-1]
        self.t_out = t0 * 2 ** len(conv_ch)
        self.max_batch = max_batch
        self.net = c_void_p()
        _check(lib.srg_create(byref(cfg), max_batch, seed, byref(self.net)), "srg_create")
        self.n = int(lib.srg_num_params(self.net))

    def params(self):
        out = np.zeros(self.n, dtype=np.float32)
        _check(_lib.srg_get_params(self.net, out.ctypes.data, self.n), "srg_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(_lib.srg_set_params(self.net, p.ctypes.data, self.n), "srg_set_params")

    def grads(self):
        out = np.zeros(self.n, dtype=np.float32)
        _check(_lib.srg_get_grads(self.net, out.ctypes.data, self.n), "srg_get_grads")
        return out

    def forward(self, x, y):
        _check(_lib.srg_forward(self.net, x.data_ptr(), x.shape[0], y.data_ptr(), dgsem._current_stream()),
               "srg_forward")
        return y

    def backward(self, x, target):
        loss = c_double()
        _check(_lib.srg_backward(self.net, x.data_ptr(), target.data_ptr(), x.shape[0], byref(loss),
                                 dgsem._current_stream()), "srg_backward")
        return loss.value

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(_lib.srg_adam_step(self.net, lr, beta1, beta2, eps, dgsem._current_stream()), "srg_adam_step")

    def train_step(self, x, target, lr):
        loss = c_double()
        _check(_lib.srg_train_step(self.net, x.data_ptr(), target.data_ptr(), x.shape[0], lr, byref(loss),
                                   dgsem._current_stream()), "srg_train_step")
        return loss.value

    def close(self):
        if self.net:
            _lib.srg_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------- data helpers
def features(delay, amp, d_in=None, delay_scale=100e-9, amp_scale=10.0):
    """Per-PMUT (delay / 100 ns, amplitude / 10 V) pairs, zero-padded to d_in."""
    delay = np.atleast_2d(delay)
    amp = np.atleast_2d(amp)
    x = np.concatenate([delay / delay_scale, amp / amp_scale], axis=1)
    if d_in is not None and x.shape[1] < d_in:
        x = np.pad(x, ((0, 0), (0, d_in - x.shape[1])))
    return x.astype(np.float32)


def resample(traces, n_out):
    """Linear interpolation of [.., S] traces (samples at t = (s+1) dt) onto
    n_out uniform samples of [dt, S dt]."""
    S = traces.shape[-1]
    src = np.arange(1, S + 1, dtype=np.float64)
    dst = np.linspace(1.0, float(S), n_out)
    flat = traces.reshape(-1, S)
    out = np.stack([np.interp(dst, src, r) for r in flat])
    return out.reshape(traces.shape[:-1] + (n_out,))


def generate_dataset(workload_fn, n_patterns, batch=64, seed=0, n_out=512, precision=dgsem.DGSEM_FP32_MIXED):
    """Simulate n_patterns steering patterns with the batched solver.
    Returns (X features, Y traces [n, R, n_out], seconds of solver time)."""
    import torch
    w = workload_fn(batch=batch, seed=seed)
    sol = dgsem.Solver(w)
    dgsem.dgsem_autotune(sol.ctx, precision, batch, len(w.domains), reps=1)
    import workloads as W
    xs, ys = [], []
    t_solve = 0.0
    for i in range((n_patterns + batch - 1) // batch):
        d, a, _ = W.steering_patterns(w.pmuts.centers, batch, seed=seed * 1000 + i)
        w.drive_delay, w.drive_amp = d, a
        drive = torch.tensor(w.drive(sol.dt, w.nsteps, batch), device="cuda")
        tr = torch.zeros((batch, w.receivers.shape[0], w.nsteps), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sol.run(drive=drive, precision=precision, traces=tr)
        torch.cuda.synchronize()
        t_solve += time.perf_counter() - t0
        xs.append(features(d, a))
        ys.append(resample(tr.cpu().numpy(), n_out))
    sol.close()
    X = np.concatenate(xs)[:n_patterns]
    Y = np.concatenate(ys)[:n_patterns].astype(np.float32)
    return X, Y, t_solve


def train(net, X, Y, epochs=50, batch=128, lr=1e-3, seed=0, lr_decay=0.97):
    """Adam on mini-batches (X, Y torch CUDA float32); returns per-epoch mean losses."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0] - X.shape[0] % batch
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(X.shape[0], generator=g)[:n].to(X.device)
        tot = 0.0
        for i in range(0, n, batch):
            idx = perm[i:i + batch]
            tot += net.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr)
        hist.append(tot / (n // batch))
        lr *= lr_decay
    return hist

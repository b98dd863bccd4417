"""Plain FP64 CPU reference of the learned surrogate (test infrastructure only).

Only tests, ``__graft_entry__.smoke()`` and ``bench.py`` may import this
module.  The surrogate is not part of the paper; it maps an array drive
pattern (per-PMUT delay and amplitude) to receiver pressure traces:

    x [d_in] -> (Linear + GELU) x n_hidden (width H) -> Linear -> [c0, t0]
             -> (ConvTranspose1d k=4 s=2 p=1 + GELU) ... -> last ConvTranspose1d
             -> y [c_last, t0 * 2^n_conv]

Loss: mean squared error over all outputs.  Optimiser: Adam.
Parameters are one flat FP32 vector in the order W_1, b_1, ..., W_dec, b_dec,
Wc_1, bc_1, ... with Linear weights [out][in] and transposed-convolution
weights [c_in][c_out][4].

``quant=True`` rounds to bfloat16 (round to nearest even) at the points
where the GPU path stores bfloat16: weights used in products, the network
input, hidden activations after GELU, the decoder output, transposed-
convolution activations after GELU, and pre-activation gradients before
the matrix products.  Everything else is FP64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

GELU_S = math.sqrt(2.0 / math.pi)
GELU_C = 0.044715


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    """tanh form: 0.5 z (1 + tanh(s (z + c z^3)))."""
    return 0.5 * z * (1.0 + np.tanh(GELU_S * (z + GELU_C * z ** 3)))


def gelu_grad(z):
    t = np.tanh(GELU_S * (z + GELU_C * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_S * (1.0 + 3.0 * GELU_C * z * z)


def convt_fwd(u, W, b):
    """ConvTranspose1d, kernel 4, stride 2, padding 1:
    v[n, co, t] = b[co] + sum_{ci, k: t = 2 i - 1 + k} u[n, ci, i] W[ci, co, k]."""
    n, ci, ti = u.shape
    co = W.shape[1]
    to = 2 * ti
    v = np.zeros((n, co, to)) + b[None, :, None]
    for k in range(4):
        for i in range(ti):
            t = 2 * i - 1 + k
            if 0 <= t < to:
                v[:, :, t] += u[:, :, i] @ W[:, :, k]
    return v


def convt_bwd(u, W, dv):
    """Gradients of convt_fwd: (du, dW, db)."""
    n, ci, ti = u.shape
    to = dv.shape[2]
    du = np.zeros_like(u)
    dW = np.zeros_like(W)
    for k in range(4):
        for i in range(ti):
            t = 2 * i - 1 + k
            if 0 <= t < to:
                du[:, :, i] += dv[:, :, t] @ W[:, :, k].T
                dW[:, :, k] += u[:, :, i].T @ dv[:, :, t]
    db = dv.sum(axis=(0, 2))
    return du, dW, db


@dataclass
class SurrogateConfig:
    d_in: int
    hidden: int = 2048
    n_hidden: int = 3
    c0: int = 256
    t0: int = 32
    conv_ch: List[int] = field(default_factory=lambda: [128, 128, 64, 64])

    @property
    def t_out(self):
        return self.t0 * 2 ** len(self.conv_ch)

    @property
    def c_out(self):
        return self.conv_ch[-1]

    def shapes(self):
        """(name, shape) of every parameter block in flat order."""
        out = []
        fan = self.d_in
        for l in range(self.n_hidden):
            out += [(f"W{l}", (self.hidden, fan)), (f"b{l}", (self.hidden,))]
            fan = self.hidden
        out += [("Wdec", (self.c0 * self.t0, fan)), ("bdec", (self.c0 * self.t0,))]
        ci = self.c0
        for j, co in enumerate(self.conv_ch):
            out += [(f"Wc{j}", (ci, co, 4)), (f"bc{j}", (co,))]
            ci = co
        return out

    def num_params(self):
        return sum(int(np.prod(s)) for _, s in self.shapes())


def unflatten(cfg: SurrogateConfig, flat):
    out, o = {}, 0
    for name, shp in cfg.shapes():
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def flatten(cfg: SurrogateConfig, d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in cfg.shapes()])


class SurrogateRef:
    def __init__(self, cfg: SurrogateConfig, quant: bool = True):
        self.cfg = cfg
        self.q = bf16 if quant else (lambda a: np.asarray(a, dtype=np.float64))

    def forward(self, params, x, keep=False):
        cfg, q = self.cfg, self.q
        P = unflatten(cfg, params)
        a = q(x)
        acts, pre = [a], []
        for l in range(cfg.n_hidden):
            z = a @ q(P[f"W{l}"]).T + P[f"b{l}"]
            pre.append(z)
            a = q(gelu(z))
            acts.append(a)
        zd = a @ q(P["Wdec"]).T + P["bdec"]
        u = q(zd).reshape(-1, cfg.c0, cfg.t0)
        us, vs = [u], []
        for j in range(len(cfg.conv_ch)):
            v = convt_fwd(u, q(P[f"Wc{j}"]), P[f"bc{j}"])
            vs.append(v)
            if j < len(cfg.conv_ch) - 1:
                u = q(gelu(v))
                us.append(u)
        y = vs[-1]
        if keep:
            self._cache = (P, acts, pre, us, vs)
        return y

    def loss_and_grad(self, params, x, target):
        """MSE loss and its gradient with respect to the flat parameters."""
        cfg, q = self.cfg, self.q
        y = self.forward(params, x, keep=True)
        P, acts, pre, us, vs = self._cache
        nel = y.size
        loss = float(np.sum((y - target) ** 2) / nel)
        G = {}
        dv = 2.0 * (y - target) / nel
        for j in range(len(cfg.conv_ch) - 1, -1, -1):
            # the products read dv rounded like the other pre-activation
            # gradients; the bias gradient sums it as it is
            du, dW, _ = convt_bwd(us[j], q(P[f"Wc{j}"]), q(dv))
            G[f"Wc{j}"], G[f"bc{j}"] = dW, dv.sum(axis=(0, 2))
            if j > 0:
                dv = du * gelu_grad(vs[j - 1])
        dzd = q(du.reshape(du.shape[0], -1))
        G["Wdec"] = dzd.T @ acts[-1]
        G["bdec"] = du.reshape(du.shape[0], -1).sum(axis=0)
        da = dzd @ q(P["Wdec"])
        for l in range(cfg.n_hidden - 1, -1, -1):
            dz = da * gelu_grad(pre[l])
            G[f"b{l}"] = dz.sum(axis=0)
            dzq = q(dz)
            G[f"W{l}"] = dzq.T @ acts[l]
            if l > 0:
                da = dzq @ q(P[f"W{l}"])
        return loss, flatten(cfg, G)


def adam_step(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), returns (params, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v

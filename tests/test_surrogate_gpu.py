"""The learned surrogate's CUDA kernels against the CPU reference (same
bfloat16 rounding points), and what the trained network gains over running
the solver for every candidate pattern."""
import time

import numpy as np
import pytest

import workloads as W
from oracle import surrogate_ref as R

pytestmark = pytest.mark.gpu

SMALL = dict(d_in=64, hidden=128, n_hidden=2, c0=16, t0=8, conv_ch=(8, 4))


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def _net_and_ref(seed=3, max_batch=128):
    from paper_2603_06267_gb300 import surrogate as S
    net = S.Surrogate(max_batch=max_batch, seed=seed, **SMALL)
    cfg = R.SurrogateConfig(d_in=SMALL["d_in"], hidden=SMALL["hidden"], n_hidden=SMALL["n_hidden"],
                            c0=SMALL["c0"], t0=SMALL["t0"], conv_ch=list(SMALL["conv_ch"]))
    assert net.n == cfg.num_params()
    return net, R.SurrogateRef(cfg, quant=True), cfg


def test_forward_matches_reference():
    import torch
    net, ref, cfg = _net_and_ref()
    rng = np.random.default_rng(0)
    x = rng.normal(size=(64, cfg.d_in)).astype(np.float32)
    y = torch.zeros((64, cfg.c_out, cfg.t_out), dtype=torch.float32, device="cuda")
    net.forward(torch.tensor(x, device="cuda"), y)
    yr = ref.forward(net.params().astype(np.float64), x)
    assert _rel(y.cpu().numpy(), yr) < 5e-3
    net.close()


def test_gradients_match_reference():
    import torch
    net, ref, cfg = _net_and_ref(seed=4)
    rng = np.random.default_rng(1)
    x = rng.normal(size=(64, cfg.d_in)).astype(np.float32)
    t = rng.normal(size=(64, cfg.c_out, cfg.t_out)).astype(np.float32)
    loss = net.backward(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    lr_, gr = ref.loss_and_grad(net.params().astype(np.float64), x, t.astype(np.float64))
    assert abs(loss - lr_) <= 1e-3 * lr_
    g = net.grads()
    o = 0
    for name, shp in cfg.shapes():
        n = int(np.prod(shp))
        assert _rel(g[o:o + n], gr[o:o + n]) < 2e-2, name
        o += n


def test_adam_step_matches_reference():
    import torch
    net, ref, cfg = _net_and_ref(seed=5)
    rng = np.random.default_rng(2)
    x = torch.tensor(rng.normal(size=(64, cfg.d_in)).astype(np.float32), device="cuda")
    t = torch.tensor(rng.normal(size=(64, cfg.c_out, cfg.t_out)).astype(np.float32), device="cuda")
    p0 = net.params().astype(np.float64)
    m = np.zeros_like(p0)
    v = np.zeros_like(p0)
    p = p0
    for step in range(1, 4):
        net.backward(x, t)
        g = net.grads().astype(np.float64)
        net.adam(1e-3)
        p, m, v = R.adam_step(p, g, m, v, step, 1e-3)
    np.testing.assert_allclose(net.params(), p, rtol=1e-4, atol=1e-6)
    net.close()


FULL = dict(d_in=2048, hidden=2048, n_hidden=3, c0=256, t0=32, conv_ch=(128, 128, 64, 64))


def _check_widths(widths, seed):
    import torch
    from paper_2603_06267_gb300 import surrogate as S
    net = S.Surrogate(max_batch=64, seed=seed, **widths)
    cfg = R.SurrogateConfig(d_in=widths["d_in"], hidden=widths["hidden"], n_hidden=widths["n_hidden"],
                            c0=widths["c0"], t0=widths["t0"], conv_ch=list(widths["conv_ch"]))
    assert net.n == cfg.num_params()
    ref = R.SurrogateRef(cfg, quant=True)
    rng = np.random.default_rng(seed + 1)
    x = rng.normal(size=(64, cfg.d_in)).astype(np.float32)
    t = rng.normal(size=(64, cfg.c_out, cfg.t_out)).astype(np.float32)
    y = torch.zeros((64, cfg.c_out, cfg.t_out), dtype=torch.float32, device="cuda")
    net.forward(torch.tensor(x, device="cuda"), y)
    p = net.params().astype(np.float64)
    assert _rel(y.cpu().numpy(), ref.forward(p, x)) < 5e-3
    loss = net.backward(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    lr_, gr = ref.loss_and_grad(p, x, t.astype(np.float64))
    assert abs(loss - lr_) <= 1e-3 * lr_
    g = net.grads()
    o = 0
    for name, shp in cfg.shapes():
        n = int(np.prod(shp))
        assert _rel(g[o:o + n], gr[o:o + n]) < 2e-2, name
        o += n
    net.close()


def test_forward_and_gradients_at_experiment_widths():
    """The experiment's network (1024 PMUTs x 2 features, three hidden layers
    of 2048, decoder 2048 -> 256 x 32, four transposed convolutions to 64 x
    512): forward, loss and every gradient block against the CPU reference
    at 64 patterns.  Every convolution has 64 or 128 output channels and
    takes both output parities in one tensor-core product."""
    _check_widths(FULL, 11)


def test_convolution_with_192_output_channels():
    """A convolution with 192 output channels takes the two-product form (one
    product per output parity) on the tensor cores; the next one, 192 -> 64,
    the paired form."""
    _check_widths(dict(d_in=128, hidden=256, n_hidden=1, c0=64, t0=32, conv_ch=(192, 64)), 21)


@pytest.mark.parametrize("M,N,K,what", [(512, 2048, 2048, "hidden layer forward / dA"),
                                        (512, 8192, 2048, "decoder forward"),
                                        (2048, 2048, 512, "hidden layer dW")])
def test_dense_product_rate(M, N, K, what):
    """Tensor-core rate of the dense-layer products at the experiment's
    shapes (512 patterns), against the measured BF16 peak."""
    import json
    import os
    from paper_2603_06267_gb300 import surrogate as S
    tf = S.gemm_tflops(M, N, K, reps=50)
    peak = None
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(path):
        peak = json.load(open(path)).get("bf16_tflops")
    frac = f" = {tf / peak:.3f} of the measured {peak:.0f} TFLOP/s" if peak else ""
    print(f"{what}: {M} x {N} x {K}: {tf:.1f} TFLOP/s{frac}")
    assert tf > 50.0


def test_training_reduces_loss():
    import torch
    from paper_2603_06267_gb300 import surrogate as S
    net, _, cfg = _net_and_ref(seed=6)
    rng = np.random.default_rng(3)
    x = rng.normal(size=(128, cfg.d_in)).astype(np.float32)
    # a smooth target: fixed random linear map of x, then a tanh
    A = rng.normal(size=(cfg.d_in, cfg.c_out * cfg.t_out)) / np.sqrt(cfg.d_in)
    y = np.tanh(x @ A).reshape(128, cfg.c_out, cfg.t_out).astype(np.float32)
    X = torch.tensor(x, device="cuda")
    Y = torch.tensor(y, device="cuda")
    hist = S.train(net, X, Y, epochs=150, batch=64, lr=2e-3, lr_decay=0.99)
    assert hist[-1] < 0.2 * hist[0], hist[::15]
    net.close()


def test_screening_gain_over_solver():
    """Train a small surrogate on solver-generated steering patterns and
    screen held-out patterns: its error beats the best constant prediction
    and it evaluates patterns at least 100x faster than the solver."""
    import torch
    from paper_2603_06267_gb300 import surrogate as S
    n_train, n_test = 320, 64
    X, Y, t_solve = S.generate_dataset(W.surrogate_array, n_train + n_test, batch=64, seed=7, n_out=64)
    scale = float(np.abs(Y[:n_train]).max())
    Xd = torch.tensor(X, device="cuda")               # [n, 2 x 64 PMUTs] = 128 features
    Yd = torch.tensor(Y / scale, device="cuda")
    net = S.Surrogate(d_in=128, hidden=256, n_hidden=2, c0=32, t0=8, conv_ch=(64, 64, 64), max_batch=64, seed=8)
    S.train(net, Xd[:n_train], Yd[:n_train], epochs=300, batch=64, lr=2e-3, lr_decay=0.995)
    pred = torch.zeros((n_test, 64, 64), dtype=torch.float32, device="cuda")
    net.forward(Xd[n_train:], pred)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(20):
        net.forward(Xd[n_train:], pred)
    torch.cuda.synchronize()
    t_inf = (time.perf_counter() - t0) / 20
    truth = Yd[n_train:].cpu().numpy()
    err = _rel(pred.cpu().numpy(), truth)
    mean_pred = Yd[:n_train].mean(dim=0, keepdim=True).cpu().numpy()
    err_const = _rel(np.broadcast_to(mean_pred, truth.shape), truth)
    solver_pps = (n_train + n_test) / t_solve
    surr_pps = n_test / t_inf
    print(f"surrogate rel-L2 {err:.3f} (constant {err_const:.3f}); {surr_pps:.0f} vs {solver_pps:.1f} patterns/s")
    assert err < 0.8 * err_const
    assert surr_pps > 100 * solver_pps
    net.close()


def test_forward_into_unaligned_output_buffer():
    """The forward writes the last layer straight into an aligned output
    buffer; a buffer that starts one float off 16 bytes gets the same values
    through the network's own buffer."""
    import torch
    from paper_2603_06267_gb300 import surrogate as S
    w = dict(d_in=128, hidden=256, n_hidden=1, c0=64, t0=32, conv_ch=(128, 64))
    net = S.Surrogate(max_batch=64, seed=5, **w)
    x = torch.randn((64, 128), device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    shape = (64, net.c_out, net.t_out)
    n = 64 * net.c_out * net.t_out
    y0 = torch.zeros(shape, device="cuda")
    net.forward(x, y0)
    big = torch.full((n + 1,), float("nan"), device="cuda")
    y1 = big[1:].view(shape)
    assert y1.data_ptr() % 16 == 4
    net.forward(x, y1)
    assert torch.equal(y0, y1)
    assert torch.isnan(big[0])
    net.close()

"""Pins of the CPU surrogate reference: library routines for the building
blocks (torch CPU conv_transpose1d, GELU tanh form, Adam, bfloat16 rounding)
and central finite differences for the whole backward pass."""
import numpy as np
import pytest

from oracle import surrogate_ref as S

torch = pytest.importorskip("torch")


def test_convt_matches_torch():
    rng = np.random.default_rng(0)
    u = rng.normal(size=(3, 5, 7))
    W = rng.normal(size=(5, 4, 4))
    b = rng.normal(size=4)
    ref = torch.nn.functional.conv_transpose1d(torch.tensor(u), torch.tensor(W), torch.tensor(b), stride=2,
                                               padding=1).numpy()
    np.testing.assert_allclose(S.convt_fwd(u, W, b), ref, rtol=1e-12, atol=1e-12)


def test_convt_backward_matches_autograd():
    rng = np.random.default_rng(1)
    u = rng.normal(size=(2, 3, 6))
    W = rng.normal(size=(3, 5, 4))
    dv = rng.normal(size=(2, 5, 12))
    tu = torch.tensor(u, requires_grad=True)
    tW = torch.tensor(W, requires_grad=True)
    tb = torch.zeros(5, dtype=torch.float64, requires_grad=True)
    out = torch.nn.functional.conv_transpose1d(tu, tW, tb, stride=2, padding=1)
    out.backward(torch.tensor(dv))
    du, dW, db = S.convt_bwd(u, W, dv)
    np.testing.assert_allclose(du, tu.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dW, tW.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(db, tb.grad.numpy(), rtol=1e-12, atol=1e-12)


def test_gelu_and_derivative():
    z = np.linspace(-6, 6, 101)
    ref = torch.nn.functional.gelu(torch.tensor(z), approximate="tanh").numpy()
    np.testing.assert_allclose(S.gelu(z), ref, rtol=1e-12, atol=1e-14)
    h = 1e-6
    np.testing.assert_allclose(S.gelu_grad(z), (S.gelu(z + h) - S.gelu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(2).normal(size=1000) * 10 ** np.random.default_rng(3).uniform(-5, 5, 1000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(S.bf16(x), ref)


def test_adam_step_matches_torch():
    rng = np.random.default_rng(4)
    p = rng.normal(size=10)
    tp = torch.tensor(p, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2)
    m = np.zeros(10)
    v = np.zeros(10)
    for t in range(1, 4):
        g = rng.normal(size=10)
        tp.grad = torch.tensor(g)
        opt.step()
        p, m, v = S.adam_step(p, g, m, v, t, 1e-2)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-10, atol=1e-12)


def test_full_backward_finite_differences():
    """Unquantised FP64 network: analytic gradient = central differences."""
    cfg = S.SurrogateConfig(d_in=6, hidden=8, n_hidden=2, c0=4, t0=3, conv_ch=[3, 2])
    ref = S.SurrogateRef(cfg, quant=False)
    rng = np.random.default_rng(5)
    theta = rng.normal(size=cfg.num_params()) * 0.5
    x = rng.normal(size=(4, 6))
    target = rng.normal(size=(4, cfg.c_out, cfg.t_out))
    loss, g = ref.loss_and_grad(theta, x, target)
    idx = rng.choice(theta.size, size=40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (ref.loss_and_grad(theta + e, x, target)[0] - ref.loss_and_grad(theta - e, x, target)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_forward_shapes_and_param_count():
    cfg = S.SurrogateConfig(d_in=128)
    assert cfg.t_out == 512 and cfg.c_out == 64
    n = cfg.num_params()
    expect = (128 * 2048 + 2048) + 2 * (2048 * 2048 + 2048) + (2048 * 8192 + 8192) \
        + (256 * 128 * 4 + 128) + (128 * 128 * 4 + 128) + (128 * 64 * 4 + 64) + (64 * 64 * 4 + 64)
    assert n == expect

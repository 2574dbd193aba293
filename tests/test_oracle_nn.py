"""Pins of the U-Net oracle: conv3d against the library routine
torch.nn.functional.conv3d (CPU, FP64), and every gradient against central
finite differences of the loss (no GPU)."""
import numpy as np
import pytest

from oracle import nn


def test_conv3d_matches_torch_cpu():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 5, 4, 6))
    for k in (3, 1):
        w = rng.standard_normal((4, 3, k, k, k))
        b = rng.standard_normal(4)
        ref = torch.nn.functional.conv3d(torch.tensor(x[None]), torch.tensor(w), torch.tensor(b),
                                         padding=k // 2)[0].numpy()
        assert np.abs(nn.conv3d(x, w, b) - ref).max() <= 1e-12


def test_pool_up_adjoint():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 4, 6, 8))
    y = rng.standard_normal((2, 2, 3, 4))
    assert abs((nn.pool(x) * y).sum() - (x * nn.pool_backward(y)).sum()) <= 1e-12
    assert abs((nn.up(y) * x).sum() - (y * nn.up_backward(x)).sum()) <= 1e-12


def test_param_count_about_one_million():
    specs = nn.layer_specs(base=14, levels=4)
    n = sum(co * ci * k ** 3 + co for _, ci, co, k in specs)
    assert 0.8e6 <= n <= 1.3e6


def test_gradients_central_differences():
    specs = nn.layer_specs(in_ch=4, out_ch=3, base=2, levels=4)
    params = nn.init_params(specs, seed=3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((4, 8, 8, 8))
    t = rng.standard_normal((3, 8, 8, 8))
    mask = (rng.random((3, 8, 8, 8)) > 0.2).astype(float)
    for k in params:                                 # nonzero biases exercise the ReLU masks
        if k.endswith(".b"):
            params[k] = rng.normal(0, 0.1, params[k].shape)
    out, cache = nn.forward(params, x)
    loss, dout = nn.mse_loss(out, t, mask)
    grads = nn.backward(params, cache, dout)
    eps = 1e-6
    for name in ["enc0a.w", "enc1b.w", "bota.w", "dec2a.w", "dec0b.b", "out.w", "out.b"]:
        flat = params[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = nn.mse_loss(nn.forward(params, x)[0], t, mask)
            flat[idx] = old - eps
            lm, _ = nn.mse_loss(nn.forward(params, x)[0], t, mask)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = grads[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, idx, fd, an)

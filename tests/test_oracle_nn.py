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


def test_node_density_closed_forms():
    # uniform density: every real node sees the same mean, padding is zero
    D, H, W = nn.grid_dims(3, 2, 2)
    assert (D, H, W) == (8, 8, 8)
    dens = nn.node_density(np.full(12, 0.4), 3, 2, 2)
    assert np.allclose(dens[:3, :3, :4], np.float32(0.4))
    assert not dens[3:].any() and not dens[:, 3:].any() and not dens[:, :, 4:].any()
    # one solid element in a void grid: its corner nodes average it with the
    # elements around them (1 / number of elements touching the node)
    rho = np.zeros(2 * 2 * 2)
    rho[0] = 1.0                      # element (0, 0, 0)
    dens = nn.node_density(rho, 2, 2, 2)
    assert dens[0, 0, 0] == np.float32(1.0)           # corner node: 1 element
    assert dens[0, 0, 1] == np.float32(0.5)           # edge node: 2 elements
    assert dens[0, 1, 1] == np.float32(0.25)          # face node: 4 elements
    assert dens[1, 1, 1] == np.float32(0.125)         # interior node: 8 elements
    assert dens[2, 2, 2] == 0.0


def test_dof_channels_and_inverse_map():
    rng = np.random.default_rng(7)
    nelx, nely, nelz = 5, 3, 2
    n_dof = 3 * (nelx + 1) * (nely + 1) * (nelz + 1)
    a = rng.standard_normal(n_dof)
    ch = nn.dof_channels(a, nelx, nely, nelz)
    assert np.abs(ch).max() == np.float32(1.0)
    # node (i, j, k) = (4, 2, 1), component 1
    n = 4 + (nelx + 1) * (2 + (nely + 1) * 1)
    assert abs(ch[1, 1, 2, 4] - a[3 * n + 1] / np.abs(a).max()) <= 1e-7
    fixed = np.zeros(n_dof, dtype=bool)
    fixed[:9] = True
    back = nn.to_dofs(ch, fixed, nelx, nely, nelz)
    assert not back[:9].any()
    assert np.allclose(back[9:], (a / np.abs(a).max())[9:], rtol=1e-6, atol=1e-7)
    mask = nn.target_mask(fixed, nelx, nely, nelz)
    assert mask.sum() == n_dof - 9


def test_energy_loss_closed_forms_and_gradient():
    from oracle import fem
    rng = np.random.default_rng(3)
    nelx, nely, nelz = 4, 2, 2
    n_dof = 3 * (nelx + 1) * (nely + 1) * (nelz + 1)
    fixed_nodes = np.zeros((nelx + 1) * (nely + 1) * (nelz + 1), dtype=np.uint8)
    fixed_nodes[::nelx + 1] = 7                      # x = 0 face clamped
    fd = fem.dof_mask(fixed_nodes)
    E = rng.uniform(0.2, 1.0, nelx * nely * nelz)
    edof = fem.edof_table_fast(nelx, nely, nelz)
    K = fem.assemble_masked(fem.ke_exact(), E, edof, n_dof, fd)
    f = np.zeros(n_dof)
    f[-2] = -1.0
    u = np.linalg.solve(K, f)
    S = f @ u
    # the exact solution (any scale) has loss 0; a direction K-orthogonal to it, loss 1
    assert abs(onn_loss(-3.0 * u, f, K, S)) <= 1e-12
    w = rng.standard_normal(n_dof)
    w[fd] = 0
    w -= (w @ K @ u) / (u @ K @ u) * u
    assert abs(onn_loss(w, f, K, S) - 1.0) <= 1e-12
    # gradient against central differences
    c = u + 0.3 * w
    _, g = nn.energy_loss(c, f, K @ c, S)
    for idx in rng.choice(np.flatnonzero(~fd), 5, replace=False):
        e = np.zeros(n_dof)
        e[idx] = 1e-6
        fdiff = (onn_loss(c + e, f, K, S) - onn_loss(c - e, f, K, S)) / 2e-6
        assert abs(fdiff - g[idx]) <= 1e-6 * max(1.0, abs(g[idx]))
    # dofs_to_grid is the adjoint of to_dofs
    y = rng.standard_normal((3,) + nn.grid_dims(nelx, nely, nelz))
    assert abs((nn.to_dofs(y, fd, nelx, nely, nelz) * g).sum()
               - (y * nn.dofs_to_grid(g, fd, nelx, nely, nelz)).sum()) <= 1e-10


def onn_loss(c, f, K, S):
    return nn.energy_loss(c, f, K @ c, S)[0]

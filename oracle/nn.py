"""Oracle: the 3D convolutional U-Net of the learned solver, forward and
backward, in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

The paper has no learned component; the network is the one the library
defines for its learned initial guess and flexible-PCG correction (a
4-level 3D U-Net on the node grid).  Definitions, in the order the library
applies them:
  conv(x; W, b)[o, v] = b[o] + sum_i sum_k W[o, i, k] x[i, v + d_k]
      (k over the 3x3x3 offsets d = (dz, dy, dx) in {-1, 0, 1}^3 with
       k = 9 (dz+1) + 3 (dy+1) + (dx+1); zero outside the grid), or a 1x1x1
       conv for the output head;
  relu(x) = max(x, 0);
  pool(x)[c, v] = mean of the 2x2x2 children of v;
  up(x)[c, v] = x[c, v // 2] (nearest);
  encoder level l (l = 0 .. L-2): e_l = relu(conv(relu(conv(in_l)))),
      in_0 = input, in_l = pool(e_{l-1}); channels c 2^l;
  bottleneck: relu(conv(relu(conv(pool(e_{L-2}))))), channels c 2^(L-1);
  decoder level l (L-2 .. 0): d_l = relu(conv(relu(conv([up(d_{l+1}), e_l])))),
      [a, b] = channel concatenation, channels c 2^l;
  output = conv1x1(d_0) (3 channels, no activation);
  loss = sum over unmasked entries of (output - target)^2 / (number of them).
Arrays are [channels, nz, ny, nx]; grid sizes are multiples of 2^(L-1).

Network input and target on the node grid of a mesh (nelx, nely, nelz),
padded with zeros to multiples of 2^(L-1) per axis:
  density channel: the mean physical density of the (up to 8) elements
      around a node;
  load channels:   a[3 n + c] / max |a| (a = load or residual), float32;
  target:          u[3 n + c] / max |u|, mask 1 on free DOFs of real nodes;
  to_dofs:         the inverse map, zero on fixed DOFs.

Energy loss of a predicted direction c for the load f (no displacement
needed): with a = f.c and b = c.Kc, the optimally scaled prediction (a/b) c
has potential energy -a^2 / (2b); against the solution's -S/2 (S = f.u*,
the compliance) the squared relative energy-norm error is
  loss = 1 - a^2 / (b S),   d loss / d c = (2 a^2 / b^2 Kc - 2 a / b f) / S.
"""
from __future__ import annotations

import numpy as np


def layer_specs(in_ch=4, out_ch=3, base=14, levels=4):
    """(name, c_in, c_out, k) of every convolution, in forward order."""
    specs = []
    ch = [base * 2 ** l for l in range(levels)]
    prev = in_ch
    for l in range(levels - 1):
        specs += [(f"enc{l}a", prev, ch[l], 3), (f"enc{l}b", ch[l], ch[l], 3)]
        prev = ch[l]
    specs += [("bota", prev, ch[-1], 3), ("botb", ch[-1], ch[-1], 3)]
    below = ch[-1]
    for l in range(levels - 2, -1, -1):
        specs += [(f"dec{l}a", below + ch[l], ch[l], 3), (f"dec{l}b", ch[l], ch[l], 3)]
        below = ch[l]
    specs += [("out", ch[0], out_ch, 1)]
    return specs


def init_params(specs, seed=0):
    """He-normal weights, zero biases (float64)."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, ci, co, k in specs:
        fan_in = ci * k ** 3
        params[name + ".w"] = rng.normal(0.0, np.sqrt(2.0 / fan_in), (co, ci, k, k, k))
        params[name + ".b"] = np.zeros(co)
    return params


def conv3d(x, w, b):
    co, ci, k = w.shape[:3]
    pad = k // 2
    D, H, W = x.shape[1:]
    xp = np.pad(x, ((0, 0), (pad, pad), (pad, pad), (pad, pad)))
    out = np.broadcast_to(b[:, None, None, None], (co, D, H, W)).astype(np.float64).copy()
    for dz in range(k):
        for dy in range(k):
            for dx in range(k):
                out += np.einsum("oi,idhw->odhw", w[:, :, dz, dy, dx],
                                 xp[:, dz:dz + D, dy:dy + H, dx:dx + W])
    return out


def conv3d_backward(x, w, dout):
    """(dx, dw, db) of conv3d."""
    co, ci, k = w.shape[:3]
    pad = k // 2
    D, H, W = x.shape[1:]
    xp = np.pad(x, ((0, 0), (pad, pad), (pad, pad), (pad, pad)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for dz in range(k):
        for dy in range(k):
            for dx in range(k):
                sl = (slice(None), slice(dz, dz + D), slice(dy, dy + H), slice(dx, dx + W))
                dw[:, :, dz, dy, dx] = np.einsum("odhw,idhw->oi", dout, xp[sl])
                dxp[sl] += np.einsum("oi,odhw->idhw", w[:, :, dz, dy, dx], dout)
    dx_ = dxp[:, pad:pad + D, pad:pad + H, pad:pad + W]
    return dx_, dw, dout.sum(axis=(1, 2, 3))


def pool(x):
    c, D, H, W = x.shape
    return x.reshape(c, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(dout):
    return np.repeat(np.repeat(np.repeat(dout, 2, 1), 2, 2), 2, 3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 1), 2, 2), 2, 3)


def up_backward(dout):
    c, D, H, W = dout.shape
    return dout.reshape(c, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(2, 4, 6))


def forward(params, x, levels=4):
    """Returns (output, cache of every layer input and activation)."""
    cache = {}

    def block(name, inp):
        za = conv3d(inp, params[name + "a.w"], params[name + "a.b"])
        a = np.maximum(za, 0.0)
        zb = conv3d(a, params[name + "b.w"], params[name + "b.b"])
        bb = np.maximum(zb, 0.0)
        cache[name] = (inp, a, bb)
        return bb

    skips = []
    h = x
    for l in range(levels - 1):
        e = block(f"enc{l}", h)
        skips.append(e)
        h = pool(e)
    h = block("bot", h)
    for l in range(levels - 2, -1, -1):
        cat = np.concatenate([up(h), skips[l]], axis=0)
        h = block(f"dec{l}", cat)
    out = conv3d(h, params["out.w"], params["out.b"])
    cache["out"] = h
    return out, cache


def backward(params, cache, dout, levels=4):
    """Gradients of every parameter for the output gradient dout."""
    g = {}

    def block_back(name, dbb):
        inp, a, bb = cache[name]
        dzb = dbb * (bb > 0)
        da, g[name + "b.w"], g[name + "b.b"] = conv3d_backward(a, params[name + "b.w"], dzb)
        dza = da * (a > 0)
        dinp, g[name + "a.w"], g[name + "a.b"] = conv3d_backward(inp, params[name + "a.w"], dza)
        return dinp

    dh, g["out.w"], g["out.b"] = conv3d_backward(cache["out"], params["out.w"], dout)
    dskips = {}
    for l in range(0, levels - 1):          # decoder blocks, last applied first
        dcat = block_back(f"dec{l}", dh)
        c_up = dcat.shape[0] - cache[f"enc{l}"][2].shape[0]
        dskips[l] = dcat[c_up:]
        dh = up_backward(dcat[:c_up])
    dh = block_back("bot", dh)
    for l in range(levels - 2, -1, -1):
        de = pool_backward(dh) + dskips[l]
        dh = block_back(f"enc{l}", de)
    return g


def mse_loss(pred, target, mask):
    """loss and d loss / d pred; mask [3, ...] is 1 where an entry counts."""
    n = max(float(mask.sum()), 1.0)
    diff = (pred - target) * mask
    return float((diff ** 2).sum() / n), 2.0 * diff / n


def grid_dims(nelx, nely, nelz, levels=4):
    """Padded node grid (D, H, W) = (z, y, x)."""
    m = 2 ** (levels - 1)
    up = lambda a: -(-a // m) * m
    return up(nelz + 1), up(nely + 1), up(nelx + 1)


def node_density(rho_phys, nelx, nely, nelz, levels=4):
    """[D, H, W] float32: mean density of the elements around each node."""
    D, H, W = grid_dims(nelx, nely, nelz, levels)
    rho = np.asarray(rho_phys, dtype=np.float64).reshape(nelz, nely, nelx)
    out = np.zeros((D, H, W), dtype=np.float32)
    for k in range(nelz + 1):
        for j in range(nely + 1):
            for i in range(nelx + 1):
                vals = [rho[ek, ej, ei]
                        for ek in (k - 1, k) for ej in (j - 1, j) for ei in (i - 1, i)
                        if 0 <= ek < nelz and 0 <= ej < nely and 0 <= ei < nelx]
                out[k, j, i] = np.float32(np.mean(vals))
    return out


def dof_channels(a, nelx, nely, nelz, levels=4):
    """[3, D, H, W] float32: a[3 n + c] / max |a| on the real nodes."""
    D, H, W = grid_dims(nelx, nely, nelz, levels)
    a32 = np.asarray(a, dtype=np.float64).astype(np.float32)
    m = np.float32(np.abs(a32).max()) if a32.size else np.float32(0)
    inv = np.float32(1.0) / m if m > 0 else np.float32(0)
    out = np.zeros((3, D, H, W), dtype=np.float32)
    out[:, :nelz + 1, :nely + 1, :nelx + 1] = (
        a32.reshape(nelz + 1, nely + 1, nelx + 1, 3).transpose(3, 0, 1, 2) * inv)
    return out


def features(rho_phys, load, nelx, nely, nelz, levels=4):
    return np.concatenate([node_density(rho_phys, nelx, nely, nelz, levels)[None],
                           dof_channels(load, nelx, nely, nelz, levels)])


def target_mask(fixed_dofs_mask, nelx, nely, nelz, levels=4):
    """[3, D, H, W] float32 mask: 1 on free DOFs of real nodes.
    fixed_dofs_mask: bool [n_dof] (True = fixed)."""
    D, H, W = grid_dims(nelx, nely, nelz, levels)
    out = np.zeros((3, D, H, W), dtype=np.float32)
    free = (~np.asarray(fixed_dofs_mask, dtype=bool)).astype(np.float32)
    out[:, :nelz + 1, :nely + 1, :nelx + 1] = free.reshape(
        nelz + 1, nely + 1, nelx + 1, 3).transpose(3, 0, 1, 2)
    return out


def to_dofs(y, fixed_dofs_mask, nelx, nely, nelz):
    """[3, D, H, W] -> DOF vector, zero on fixed DOFs."""
    c = np.asarray(y)[:, :nelz + 1, :nely + 1, :nelx + 1].transpose(1, 2, 3, 0).reshape(-1)
    c = c.astype(np.float64)
    c[np.asarray(fixed_dofs_mask, dtype=bool)] = 0.0
    return c


def energy_loss(c, f, Kc, S):
    """(loss, d loss / d c) of the energy loss above."""
    a = float(f @ c)
    b = float(c @ Kc)
    return 1.0 - a * a / (b * S), (2 * a * a / (b * b) * Kc - 2 * a / b * f) / S


def dofs_to_grid(g, fixed_dofs_mask, nelx, nely, nelz, levels=4):
    """DOF vector -> [3, D, H, W] (zero on fixed DOFs and padding): the
    adjoint of to_dofs."""
    D, H, W = grid_dims(nelx, nely, nelz, levels)
    g = np.array(g, dtype=np.float64)
    g[np.asarray(fixed_dofs_mask, dtype=bool)] = 0.0
    out = np.zeros((3, D, H, W))
    out[:, :nelz + 1, :nely + 1, :nelx + 1] = g.reshape(
        nelz + 1, nely + 1, nelx + 1, 3).transpose(3, 0, 1, 2)
    return out

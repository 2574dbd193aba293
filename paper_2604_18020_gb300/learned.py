"""Training data and training for the learned solve (the U-Net of nn.cu).

Samples are (density, load, displacement) triples that the SIMP loop
itself produces: for each SIMP iteration of a cantilever run, the filtered
density, the load and the solved displacement, and, from the same state,
the residual and error of partly converged Jacobi-PCG iterates (k
iterations from zero).  Every array is built on the device by the library
(mfto_nn_sample); this module only orders the calls and keeps the tensors.

    python -m paper_2604_18020_gb300.learned --out weights.npz
trains the default network (base 14, 4 levels) on SIMP runs at 64x32x32 and
128x64x64 and writes its FP32 parameters.
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import mfto, workloads as W

LEVELS = 4


def simp_samples(nelx, nely, nelz, volfrac, iters, ks=(0, 10, 50, 200), every=1, cuda="cuda",
                 rtol=1e-8, seed=0):
    """List of (x, y, mask, dims) device tensors from one SIMP run of the
    cantilever (mixed-precision solver), `iters` iterations, a sample set
    every `every` iterations, one sample per k in ks."""
    import torch
    P = W.cantilever(nelx, nely, nelz)
    m = P.mesh
    prm = mfto.default_params(volfrac=volfrac, rtol=rtol, maxit=20000)
    dims = mfto.nn_grid(nelx, nely, nelz, LEVELS)
    V = int(np.prod(dims))
    out = []
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed, prm) as h:
        h.set_solver(mfto.FORM_F32, inner_tol=1e-2)
        rho = torch.full((m.n_elem,), volfrac, dtype=torch.float64, device=cuda)
        rho_phys = torch.zeros_like(rho)
        E = torch.zeros_like(rho)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        f = torch.tensor(P.f, device=cuda)
        for it in range(iters):
            h.simp_step(rho, u, f, rho_phys)   # u solves K(E(rho_phys)) u = f
            if it % every:
                continue
            h.simp_modulus(rho_phys, E)
            for k in ks:
                x = torch.empty(4 * V, dtype=torch.float32, device=cuda)
                y = torch.empty(3 * V, dtype=torch.float32, device=cuda)
                mk = torch.empty(3 * V, dtype=torch.float32, device=cuda)
                h.nn_sample(E, rho_phys, f, u, k, x, y, mk, LEVELS)
                out.append((x, y, mk, dims))
    return out


def train(net, samples, steps, lr=1e-3, lr_final=1e-4, seed=0, log_every=0):
    """Adam on single samples drawn in a seeded order, learning rate decayed
    geometrically from lr to lr_final.  Returns the loss history."""
    rng = np.random.default_rng(seed)
    hist = []
    for s in range(steps):
        x, y, mk, dims = samples[int(rng.integers(len(samples)))]
        cur = lr * (lr_final / lr) ** (s / max(steps - 1, 1))
        want = log_every and (s % log_every == 0 or s == steps - 1)
        loss = net.train_step(x, y, mk, dims, lr=cur, want_loss=bool(want))
        if want:
            hist.append((s, loss))
    return hist


def save(net, path):
    np.savez(path, params=net.get_params(), base=net.base, levels=net.levels)


def load(path, max_voxels, stream=None):
    d = np.load(path)
    net = mfto.Net(base=int(d["base"]), levels=int(d["levels"]), max_voxels=max_voxels,
                   stream=stream)
    net.set_params(d["params"])
    return net


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--base", type=int, default=14)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--small-iters", type=int, default=40)
    ap.add_argument("--large-iters", type=int, default=20)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    import torch
    t0 = time.time()
    samples = []
    for vf in (0.12, 0.2):
        samples += simp_samples(64, 32, 32, vf, a.small_iters, every=2)
        samples += simp_samples(128, 64, 64, vf, a.large_iters, every=2)
    torch.cuda.synchronize()
    t1 = time.time()
    big = max(int(np.prod(s[3])) for s in samples)
    net = mfto.Net(base=a.base, levels=LEVELS, max_voxels=big, max_train_voxels=big, seed=a.seed)
    hist = train(net, samples, a.steps, lr=a.lr, seed=a.seed, log_every=max(a.steps // 20, 1))
    torch.cuda.synchronize()
    t2 = time.time()
    save(net, a.out)
    print(f"samples {len(samples)} in {t1 - t0:.1f} s; {a.steps} steps in {t2 - t1:.1f} s; "
          f"params {net.num_params}")
    for s, l in hist:
        print(f"step {s:6d} loss {l:.4e}")


if __name__ == "__main__":
    main()

"""Training data and training for the learned solve (the U-Net of nn.cu).

Training data comes from the SIMP loop itself.  The default (energy) loss
needs, per SIMP iteration of a cantilever run, the state (modulus E, filtered
density rho_phys) and its compliance f.u, and trains the network to minimise
the energy-norm error of its optimally scaled prediction
(mfto_nn_train_energy).  The MSE loss instead fits (density, load,
displacement) triples: the solved displacement, and the residual and error
of partly converged Jacobi-PCG iterates (mfto_nn_sample).  Every array is
built on the device by the library; this module only orders the calls and
keeps the tensors.

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


class StateSet:
    """SIMP states (E, rho_phys, compliance) of one mesh, with its handle."""

    def __init__(self, nelx, nely, nelz, volfracs, iters, cuda="cuda", every=1):
        import torch
        P = W.cantilever(nelx, nely, nelz)
        m = P.mesh
        self.dims = mfto.nn_grid(nelx, nely, nelz, LEVELS)
        self.h = mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed,
                             mfto.default_params(rtol=1e-8, maxit=20000))
        self.h.set_solver(mfto.FORM_F32, inner_tol=1e-2)
        self.f = torch.tensor(P.f, device=cuda)
        self.states = []
        for vf in volfracs:
            self.h.set_params(mfto.default_params(volfrac=vf, rtol=1e-8, maxit=20000))
            rho = torch.full((m.n_elem,), vf, dtype=torch.float64, device=cuda)
            u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
            for it in range(iters):
                rp = torch.zeros_like(rho)
                st = self.h.simp_step(rho, u, self.f, rp)
                if it % every == 0:
                    E = torch.zeros_like(rho)
                    self.h.simp_modulus(rp, E)
                    self.states.append((E, rp, st.compliance))

    @property
    def voxels(self):
        return int(np.prod(self.dims))


def train_energy(net, sets, steps, lr=1e-3, lr_final=1e-4, seed=0, log_every=0):
    """Adam on the energy loss (mfto_nn_train_energy) of states drawn in a
    seeded order from the StateSets, learning rate decayed geometrically.
    Returns [(step, loss)] every log_every steps."""
    rng = np.random.default_rng(seed)
    pool = [(s, i) for s in sets for i in range(len(s.states))]
    hist = []
    for k in range(steps):
        ss, i = pool[int(rng.integers(len(pool)))]
        E, rp, c = ss.states[i]
        cur = lr * (lr_final / lr) ** (k / max(steps - 1, 1))
        want = bool(log_every) and (k % log_every == 0 or k == steps - 1)
        loss = ss.h.nn_train_energy(net, E, rp, ss.f, c, lr=cur, want_loss=want)
        if want:
            hist.append((k, loss))
    return hist


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


WEIGHTS = mfto.HERE / "weights" / "unet_b14_l4_cantilever.npz"


def _to_bf16_bits(p):
    """float32 -> bfloat16 bit patterns, round to nearest even (the rounding
    the network applies to its working copy of the weights)."""
    b = np.ascontiguousarray(p, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def save(net, path, bf16=True):
    """Parameters, compressed; bf16=True keeps only the BF16 values the
    forward pass uses (the FP32 master copy is dropped)."""
    p = net.get_params()
    if bf16:
        np.savez_compressed(path, params_bf16=_to_bf16_bits(p), base=net.base, levels=net.levels)
    else:
        np.savez_compressed(path, params=p, base=net.base, levels=net.levels)


def load(path=WEIGHTS, max_voxels=1, max_train_voxels=0, stream=None):
    d = np.load(path)
    if "params_bf16" in d:
        params = (d["params_bf16"].astype(np.uint32) << 16).view(np.float32)
    else:
        params = d["params"]
    net = mfto.Net(base=int(d["base"]), levels=int(d["levels"]), max_voxels=max_voxels,
                   max_train_voxels=max_train_voxels, stream=stream)
    net.set_params(params)
    return net


def evaluate(path=WEIGHTS, sizes=((64, 32, 32), (128, 64, 64)), simp_iters=25, cuda="cuda"):
    """Compare, on the state after `simp_iters` SIMP iterations of each
    cantilever size (V_f 0.12), the trained network with an untrained one and
    with no network: the energy-norm error of the optimally scaled initial
    guess, and the inner iterations and wall time of the solve from u = 0 to
    rtol 1.5e-2 (one refinement step) and 1e-8.  Prints one line per case."""
    import torch
    rows = []
    for nx, ny, nz in sizes:
        P = W.cantilever(nx, ny, nz)
        m = P.mesh
        dims = mfto.nn_grid(nx, ny, nz, LEVELS)
        V = int(np.prod(dims))
        nets = {"trained": load(path, V), "untrained": mfto.Net(base=14, levels=LEVELS,
                                                               max_voxels=V, seed=123)}
        h = mfto.Handle(nx, ny, nz, P.fixed, mfto.default_params(volfrac=0.12, rtol=1e-8,
                                                                  maxit=100000))
        h.set_solver(mfto.FORM_F32, inner_tol=1e-2)
        rho = torch.full((m.n_elem,), 0.12, dtype=torch.float64, device=cuda)
        rp, E = torch.zeros_like(rho), torch.zeros_like(rho)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        f = torch.tensor(P.f, device=cuda)
        for _ in range(simp_iters):
            st = h.simp_step(rho, u, f, rp)
        h.filter(rho, rp)
        h.simp_modulus(rp, E)
        # compliance of the current state from a tight solve
        us = u.clone()
        h.set_params(mfto.default_params(volfrac=0.12, rtol=1e-11, maxit=100000))
        h.ir_solve(E, f, us, inner=mfto.FORM_F32, inner_tol=1e-2)
        S = float(torch.dot(f, us))
        x = torch.zeros(4 * V, dtype=torch.float32, device=cuda)
        y = torch.zeros(3 * V, dtype=torch.float32, device=cuda)
        c, Kc = torch.zeros_like(u), torch.zeros_like(u)
        h.nn_features(rp, f, x, LEVELS)
        for name, net in nets.items():
            net.forward(x, y, dims)
            h.nn_to_dofs(y, c, LEVELS)
            h.kv(E, c, Kc)
            a, b = float(torch.dot(f, c)), float(torch.dot(c, Kc))
            err = float(np.sqrt(max(1.0 - a * a / (b * S), 0.0))) if b > 0 else 1.0
            rows.append({"mesh": f"{nx}x{ny}x{nz}", "net": name, "guess_energy_error": err})
        for tol in (1.5e-2, 1e-8):
            h.set_params(mfto.default_params(volfrac=0.12, rtol=tol, maxit=100000))
            for name in ("none", "untrained", "trained"):
                uu = torch.zeros_like(u)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if name == "none":
                    h.set_learned(None)
                    s2 = h.ir_solve(E, f, uu, inner=mfto.FORM_F32, inner_tol=1e-2)
                else:
                    h.set_learned(nets[name], every=0)
                    s2 = h.learned_solve(E, rp, f, uu)
                torch.cuda.synchronize()
                rows.append({"mesh": f"{nx}x{ny}x{nz}", "rtol": tol, "net": name,
                             "outer": s2.outer_iterations, "inner": s2.inner_iterations,
                             "status": mfto.STATUS_NAMES[s2.status],
                             "ms": 1e3 * (time.perf_counter() - t0)})
        h.set_learned(None)
        h.close()
    for r in rows:
        print(r)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out")
    ap.add_argument("--eval", metavar="WEIGHTS", help="evaluate a trained network and exit")
    ap.add_argument("--base", type=int, default=14)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--small-iters", type=int, default=40)
    ap.add_argument("--large-iters", type=int, default=20)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--loss", choices=("energy", "mse"), default="energy")
    a = ap.parse_args(argv)
    if a.eval:
        evaluate(a.eval)
        return
    if not a.out:
        ap.error("--out is required for training")
    import torch
    t0 = time.time()
    if a.loss == "energy":
        sets = [StateSet(64, 32, 32, (0.12, 0.2, 0.3), a.small_iters),
                StateSet(128, 64, 64, (0.12, 0.2), a.large_iters)]
        n_samples = sum(len(s.states) for s in sets)
        big = max(s.voxels for s in sets)
    else:
        samples = []
        for vf in (0.12, 0.2):
            samples += simp_samples(64, 32, 32, vf, a.small_iters, every=2)
            samples += simp_samples(128, 64, 64, vf, a.large_iters, every=2)
        n_samples = len(samples)
        big = max(int(np.prod(s[3])) for s in samples)
    torch.cuda.synchronize()
    t1 = time.time()
    net = mfto.Net(base=a.base, levels=LEVELS, max_voxels=big, max_train_voxels=big, seed=a.seed)
    log = max(a.steps // 20, 1)
    if a.loss == "energy":
        hist = train_energy(net, sets, a.steps, lr=a.lr, seed=a.seed, log_every=log)
    else:
        hist = train(net, samples, a.steps, lr=a.lr, seed=a.seed, log_every=log)
    torch.cuda.synchronize()
    t2 = time.time()
    save(net, a.out)
    print(f"samples {n_samples} in {t1 - t0:.1f} s; {a.steps} steps in {t2 - t1:.1f} s; "
          f"params {net.num_params}")
    for s, l in hist:
        print(f"step {s:6d} loss {l:.4e}")


if __name__ == "__main__":
    main()

"""The learned part on the GPU against the FP64 oracle: the U-Net forward
pass and every parameter gradient (BF16 weights on both sides, FP32 against
FP64 arithmetic: max error <= 1e-4 of the largest reference value per
tensor), the network input/target builders, training, and the learned
solve (accepted only at the FP64 residual tolerance, checked by the
oracle's own residual)."""
import numpy as np
import pytest

from oracle import fem, nn as onn
from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def bf16_values(a):
    """float32 values of a rounded to bfloat16 (nearest, ties to even)."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


def oracle_params(base, levels, seed):
    specs = onn.layer_specs(in_ch=4, out_ch=3, base=base, levels=levels)
    params = onn.init_params(specs, seed=seed)
    rng = np.random.default_rng(seed + 1)
    for name, _, _, _ in specs:
        params[name + ".w"] = bf16_values(params[name + ".w"]).astype(np.float64)
        params[name + ".b"] = rng.normal(0, 0.1, params[name + ".b"].shape).astype(
            np.float32).astype(np.float64)
    flat = np.concatenate([np.concatenate([params[n + ".w"].reshape(-1), params[n + ".b"]])
                           for n, _, _, _ in specs]).astype(np.float32)
    return specs, params, flat


def rel_err(got, ref):
    return np.abs(np.asarray(got, np.float64) - ref).max() / max(np.abs(ref).max(), 1e-30)


@pytest.mark.parametrize("base,dims", [(3, (8, 16, 24)), (2, (16, 16, 24))])
def test_forward_matches_oracle(cuda, base, dims):
    import torch
    from paper_2604_18020_gb300 import mfto
    specs, params, flat = oracle_params(base, 4, seed=11)
    D, H, Wd = dims
    x = np.random.default_rng(2).standard_normal((4, D, H, Wd)).astype(np.float32)
    ref, _ = onn.forward(params, x.astype(np.float64), levels=4)
    net = mfto.Net(base=base, levels=4, max_voxels=D * H * Wd)
    net.set_params(flat)
    assert net.num_params == flat.size
    assert np.array_equal(net.get_params(), flat)
    out = torch.zeros(3 * D * H * Wd, dtype=torch.float32, device=cuda)
    net.forward(torch.tensor(x, device=cuda).reshape(-1), out, dims)
    got = out.cpu().numpy().reshape(3, D, H, Wd)
    assert rel_err(got, ref) <= 1e-4


def test_forward_tensor_cores_match_fma_pipe(cuda):
    """The tcgen05 implicit-GEMM convolutions (activations split into BF16 hi +
    lo) against the FP32 FMA-pipe ones, on a grid whose tiles are ragged in x
    and y, at the learned part's width (14 .. 112 channels: one and several
    output-channel slices, one and several 16-channel input stages); both
    within 1e-4 of each other, the tensor-core pass bit-identical on repeat
    and without a given-up wait."""
    import torch
    from paper_2604_18020_gb300 import mfto
    dims = (16, 40, 24)
    D, H, Wd = dims
    V = D * H * Wd
    net = mfto.Net(base=14, levels=4, max_voxels=V, seed=3)
    x = torch.randn(4 * V, generator=torch.Generator().manual_seed(4)).to(cuda)
    outs = []
    for tc in (True, True, False):
        net.set_tensor_cores(tc)
        out = torch.zeros(3 * V, dtype=torch.float32, device=cuda)
        net.forward(x, out, dims)
        outs.append(out.cpu().numpy())
    assert not net.tc_gave_up()
    assert np.array_equal(outs[0], outs[1])
    assert rel_err(outs[0], outs[2].astype(np.float64)) <= 1e-4
    assert np.abs(outs[2]).max() > 0


# Gradient tolerance of the tensor-core convolutions (relative to the largest
# value of each parameter tensor).  Each convolution carries its FP32 input as
# BF16 hi + lo, exact to about 2^-17 of each value, and the gradient of the
# first layer passes through the 14 forward and 13 adjoint convolutions of the
# net; 27 such roundings, compounded, give a few times 1e-4 at most, against
# about 1e-6 for the FMA-pipe path, whose tolerance stays 1e-4.
TC_GRAD_TOL = 5e-4


def test_gradients_tensor_cores_match_fma_pipe(cuda):
    """The data gradient as the adjoint tcgen05 convolution (adjoint weights,
    ReLU gate in its epilogue) against the FMA-pipe backward pass, at the
    learned part's width on a grid ragged in x and y: every parameter
    gradient within TC_GRAD_TOL of the largest value of its tensor,
    bit-identical on repeat, no given-up wait."""
    import torch
    from paper_2604_18020_gb300 import mfto
    dims = (16, 40, 24)
    D, H, Wd = dims
    V = D * H * Wd
    net = mfto.Net(base=14, levels=4, max_voxels=V, max_train_voxels=V, seed=7)
    g = torch.Generator().manual_seed(8)
    x = torch.randn(4 * V, generator=g).to(cuda)
    t = torch.randn(3 * V, generator=g).to(cuda)
    mask = (torch.rand(3 * V, generator=g) > 0.3).float().to(cuda)
    grads = []
    for tc in (True, True, False):
        net.set_tensor_cores(tc)
        loss, gr = net.gradient(x, t, mask, dims)
        grads.append((loss, gr))
    assert not net.tc_gave_up()
    assert grads[0][0] == grads[1][0] and np.array_equal(grads[0][1], grads[1][1])
    specs = onn.layer_specs(in_ch=4, out_ch=3, base=14, levels=4)
    off, worst = 0, 0.0
    for name, ci, co, k in specs:
        for n in (co * ci * k ** 3, co):
            a, b = grads[0][1][off:off + n], grads[2][1][off:off + n].astype(np.float64)
            worst = max(worst, rel_err(a, b))
            assert rel_err(a, b) <= TC_GRAD_TOL, name
            off += n
    print(f"tensor-core vs FMA-pipe gradients: worst tensor {worst:.2e}")
    assert off == grads[0][1].size
    assert abs(grads[0][0] - grads[2][0]) <= 1e-5 * abs(grads[2][0])


@pytest.mark.parametrize("tensor_cores", [False, True])
def test_gradients_match_oracle(cuda, tensor_cores):
    """Every parameter gradient and the loss against the FP64 oracle, with the
    convolutions on the FMA pipe (1e-4) and on the tensor cores
    (TC_GRAD_TOL)."""
    import torch
    from paper_2604_18020_gb300 import mfto
    base, dims = 2, (16, 16, 24)            # 6144 voxels: 2 gradient chunks at level 0
    specs, params, flat = oracle_params(base, 4, seed=5)
    D, H, Wd = dims
    rng = np.random.default_rng(6)
    x = rng.standard_normal((4, D, H, Wd)).astype(np.float32)
    t = rng.standard_normal((3, D, H, Wd)).astype(np.float32)
    mask = (rng.random((3, D, H, Wd)) > 0.3).astype(np.float32)
    out, cache = onn.forward(params, x.astype(np.float64))
    loss_ref, dout = onn.mse_loss(out, t.astype(np.float64), mask.astype(np.float64))
    g_ref = onn.backward(params, cache, dout)
    net = mfto.Net(base=base, levels=4, max_voxels=D * H * Wd, max_train_voxels=D * H * Wd)
    net.set_params(flat)
    net.set_tensor_cores(tensor_cores)
    tol = TC_GRAD_TOL if tensor_cores else 1e-4
    dev = lambda a: torch.tensor(a, device=cuda).reshape(-1)
    loss, g = net.gradient(dev(x), dev(t), dev(mask), dims)
    assert abs(loss - loss_ref) <= 1e-5 * abs(loss_ref)
    off, worst = 0, 0.0
    for name, ci, co, k in specs:
        nw = co * ci * k ** 3
        ew = rel_err(g[off:off + nw], g_ref[name + ".w"].reshape(-1))
        assert ew <= tol, name
        off += nw
        eb = rel_err(g[off:off + co], g_ref[name + ".b"])
        assert eb <= tol, name
        off += co
        worst = max(worst, ew, eb)
    print(f"gradients vs oracle (tensor cores {tensor_cores}): worst tensor {worst:.2e}")
    assert off == g.size
    # fixed reduction order: a second evaluation is bit-identical
    loss2, g2 = net.gradient(dev(x), dev(t), dev(mask), dims)
    assert loss2 == loss and np.array_equal(g2, g)


def test_features_targets_match_oracle(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(13, 6, 5)
    m = P.mesh
    rng = np.random.default_rng(9)
    rho = rng.uniform(0.01, 1.0, m.n_elem)
    u = rng.standard_normal(m.n_dof)
    fd = fem.dof_mask(P.fixed)
    u[fd] = 0.0
    dims = onn.grid_dims(m.nelx, m.nely, m.nelz)
    V = int(np.prod(dims))
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        assert h.nn_grid() == dims
        x = torch.zeros(4 * V, dtype=torch.float32, device=cuda)
        y = torch.zeros(3 * V, dtype=torch.float32, device=cuda)
        mk = torch.zeros(3 * V, dtype=torch.float32, device=cuda)
        h.nn_features(torch.tensor(rho, device=cuda), torch.tensor(P.f, device=cuda), x)
        h.nn_target(torch.tensor(u, device=cuda), y, mk)
        c = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        h.nn_to_dofs(y, c)
        xg = x.cpu().numpy().reshape(4, *dims)
        yg = y.cpu().numpy().reshape(3, *dims)
    xr = onn.features(rho, P.f, m.nelx, m.nely, m.nelz)
    assert np.abs(xg[0] - xr[0]).max() <= 1e-7
    assert np.abs(xg[1:] - xr[1:]).max() <= 1e-6
    yr = onn.dof_channels(u, m.nelx, m.nely, m.nelz)
    assert np.abs(yg - yr).max() <= 1e-6
    assert np.array_equal(mk.cpu().numpy().reshape(3, *dims),
                          onn.target_mask(fd, m.nelx, m.nely, m.nelz))
    assert np.array_equal(c.cpu().numpy(), onn.to_dofs(yg, fd, m.nelx, m.nely, m.nelz))


def test_training_reduces_loss(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(16, 8, 8)
    m = P.mesh
    dims = onn.grid_dims(m.nelx, m.nely, m.nelz)
    V = int(np.prod(dims))
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        rho = torch.tensor(W.rho_random(m, seed=3, lo=0.1, hi=1.0), device=cuda)
        E = torch.zeros(m.n_elem, dtype=torch.float64, device=cuda)
        h.simp_modulus(rho, E)
        f = torch.tensor(P.f, device=cuda)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        assert h.pcg(E, f, u).status == mfto.OK
        x = torch.zeros(4 * V, dtype=torch.float32, device=cuda)
        y = torch.zeros(3 * V, dtype=torch.float32, device=cuda)
        mk = torch.zeros(3 * V, dtype=torch.float32, device=cuda)
        h.nn_sample(E, rho, f, u, 0, x, y, mk)
        net = mfto.Net(base=4, levels=4, max_voxels=V, max_train_voxels=V, seed=1)
        losses = [net.train_step(x, y, mk, dims, lr=3e-3) for _ in range(80)]
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.3 * losses[0], (losses[0], losses[-1])


def _setup_solve(cuda, P, seed):
    import torch
    from paper_2604_18020_gb300 import mfto
    m = P.mesh
    h = mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed)
    rho = torch.tensor(W.rho_random(m, seed=seed, lo=0.05, hi=1.0), device=cuda)
    E = torch.zeros(m.n_elem, dtype=torch.float64, device=cuda)
    h.simp_modulus(rho, E)
    return h, rho, E, torch.tensor(P.f, device=cuda)


def _true_rel(P, E, u):
    m = P.mesh
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    r = P.f - fem.kv(fem.ke_exact(), E, edof, u, fd)
    return np.linalg.norm(r) / np.linalg.norm(P.f)


@pytest.mark.parametrize("every", [0, 25])
def test_learned_solve_accepts_only_at_rtol(cuda, every):
    """An untrained network: the flexible PCG must still reach the FP64
    tolerance (the line search makes a poor direction harmless)."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(24, 12, 12)
    h, rho, E, f = _setup_solve(cuda, P, seed=21)
    dims = h.nn_grid()
    net = mfto.Net(base=4, levels=4, max_voxels=int(np.prod(dims)), seed=2)
    h.set_learned(net, every=every)
    h.set_solver(mfto.FORM_F32, inner_tol=1e-2)
    u = torch.zeros(P.mesh.n_dof, dtype=torch.float64, device=cuda)
    st = h.learned_solve(E, rho, f, u)
    assert st.status == mfto.OK, (st.status, st.fallback, st.rel_residual)
    assert st.nn_calls >= 1 and st.outer_iterations >= 1
    assert st.rel_residual <= 1e-8
    assert _true_rel(P, E.cpu().numpy(), u.cpu().numpy()) <= 1.5e-8
    h.close()


def test_learned_solve_fallback_chain(cuda):
    """One inner iteration per outer step cannot reduce the residual by 10 %
    twice in a row: the network is switched off, then FP64 Jacobi-PCG
    finishes; the result is still accepted only at rtol."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(16, 8, 8)
    h, rho, E, f = _setup_solve(cuda, P, seed=4)
    dims = h.nn_grid()
    net = mfto.Net(base=2, levels=4, max_voxels=int(np.prod(dims)), seed=3)
    h.set_learned(net, every=0)
    h.set_solver(mfto.FORM_F32, inner_tol=1e-2, inner_maxit=1, max_outer=200)
    u = torch.zeros(P.mesh.n_dof, dtype=torch.float64, device=cuda)
    st = h.learned_solve(E, rho, f, u)
    assert st.fallback == 2
    assert st.fp64_iterations > 0
    assert st.status == mfto.OK
    assert _true_rel(P, E.cpu().numpy(), u.cpu().numpy()) <= 1.5e-8
    h.close()


def test_set_learned_checks_size(cuda):
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(24, 12, 12)
    m = P.mesh
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        net = mfto.Net(base=2, levels=4, max_voxels=1000)
        with pytest.raises(mfto.MftoError) as e:
            h.set_learned(net)
        assert e.value.code == mfto.TOO_LARGE


def test_energy_training_step_matches_oracle(cuda):
    """One Adam step on the energy loss: the loss equals the oracle's
    1 - (f.c)^2 / (c.Kc f.u*) of the oracle network's prediction, and every
    parameter with a clear gradient moves by -lr sign(gradient) (the first
    Adam step), the gradient being the oracle's back-propagated energy
    gradient."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(13, 6, 5)
    m = P.mesh
    specs, params, flat = oracle_params(2, 4, seed=8)
    rng = np.random.default_rng(12)
    rho = rng.uniform(0.05, 1.0, m.n_elem)
    E = fem.simp_modulus(rho, 3.0)
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    K = fem.assemble(KE, E, edof, m.n_dof).toarray()
    K[fd, :] = 0
    K[:, fd] = 0
    K[fd, fd] = 1
    S = float(P.f @ np.linalg.solve(K, P.f))
    x = onn.features(rho, P.f, m.nelx, m.nely, m.nelz)
    out, cache = onn.forward(params, x.astype(np.float64))
    c = onn.to_dofs(out, fd, m.nelx, m.nely, m.nelz)
    loss_ref, gc = onn.energy_loss(c, P.f, fem.kv(KE, E, edof, c, fd), S)
    g_ref = onn.backward(params, cache, onn.dofs_to_grid(gc, fd, m.nelx, m.nely, m.nelz))
    gflat = np.concatenate([np.concatenate([g_ref[n + ".w"].reshape(-1), g_ref[n + ".b"]])
                            for n, _, _, _ in specs])
    V = int(np.prod(onn.grid_dims(m.nelx, m.nely, m.nelz)))
    net = mfto.Net(base=2, levels=4, max_voxels=V, max_train_voxels=V)
    net.set_params(flat)
    lr = 1e-3
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        loss = h.nn_train_energy(net, torch.tensor(E, device=cuda), torch.tensor(rho, device=cuda),
                                 torch.tensor(P.f, device=cuda), S, lr=lr)
    assert abs(loss - loss_ref) <= 1e-4, (loss, loss_ref)
    delta = net.get_params().astype(np.float64) - flat
    sel = np.abs(gflat) > 1e-2 * np.abs(gflat).max()
    assert sel.sum() > 20
    assert np.all(np.sign(delta[sel]) == -np.sign(gflat[sel]))
    assert np.allclose(np.abs(delta[sel]), lr, rtol=0.02)


def test_trained_network_gain(cuda):
    """What training gains, on a SIMP state held out of training: the
    energy-norm error of the network's optimally scaled initial guess drops
    from ~1 (untrained: no better than u = 0) to well below, and the learned
    solve reaches the first refinement tolerance (1.5e-2) in fewer inner
    iterations than the solve without the network.  At rtol 1e-8 the learned
    solve is accepted with the oracle's residual."""
    import torch
    from paper_2604_18020_gb300 import learned as L, mfto
    nelx, nely, nelz = 32, 16, 16
    P = W.cantilever(nelx, nely, nelz)
    m = P.mesh
    ss = L.StateSet(nelx, nely, nelz, (0.12,), 14)
    train, held = ss.states[:10], ss.states[13]
    V = ss.voxels
    net = mfto.Net(base=8, levels=4, max_voxels=V, max_train_voxels=V, seed=0)
    untrained = mfto.Net(base=8, levels=4, max_voxels=V, seed=0)
    steps = 400
    for k in range(steps):
        E, rp, c = train[k % len(train)]
        ss.h.nn_train_energy(net, E, rp, ss.f, c, lr=2e-3 * 0.1 ** (k / steps), want_loss=False)
    E, rp, S = held
    edof = fem.edof_table_fast(nelx, nely, nelz)
    fd = fem.dof_mask(P.fixed)
    En = E.cpu().numpy()

    def energy_error(nt):
        x = torch.zeros(4 * V, dtype=torch.float32, device=cuda)
        y = torch.zeros(3 * V, dtype=torch.float32, device=cuda)
        cv = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        ss.h.nn_features(rp, ss.f, x)
        nt.forward(x, y, ss.dims)
        ss.h.nn_to_dofs(y, cv)
        c = cv.cpu().numpy()
        loss, _ = onn.energy_loss(c, P.f, fem.kv(fem.ke_exact(), En, edof, c, fd), S)
        return np.sqrt(max(loss, 0.0))

    err_t, err_u = energy_error(net), energy_error(untrained)
    iters = {}
    ss.h.set_params(mfto.default_params(volfrac=0.12, rtol=1.5e-2, maxit=20000))
    u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
    iters["plain"] = ss.h.ir_solve(E, ss.f, u, inner=mfto.FORM_F32, inner_tol=1e-2).inner_iterations
    for name, nt in (("untrained", untrained), ("trained", net)):
        ss.h.set_learned(nt, every=0)
        u.zero_()
        iters[name] = ss.h.learned_solve(E, rp, ss.f, u).inner_iterations
    print(f"energy error of the initial guess: trained {err_t:.3f}, untrained {err_u:.3f}; "
          f"inner iterations to 1.5e-2: {iters}")
    assert err_u > 0.95
    assert err_t < 0.8
    assert iters["trained"] < 0.9 * iters["plain"]
    ss.h.set_params(mfto.default_params(volfrac=0.12, rtol=1e-8, maxit=20000))
    ss.h.set_learned(net, every=0)
    u.zero_()
    st = ss.h.learned_solve(E, rp, ss.f, u)
    assert st.status == mfto.OK
    assert _true_rel(P, En, u.cpu().numpy()) <= 1.5e-8

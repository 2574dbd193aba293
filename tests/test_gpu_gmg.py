"""Geometric multigrid on the GPU against the oracle (oracle/gmg.py): the
level hierarchy, every level's Galerkin operator applied to a vector, one
V-cycle, the V-cycle CG solve and SIMP steps with it, on meshes with odd
(ragged) element counts; the argument checks."""
import numpy as np
import pytest

from oracle import fem, gmg, solve, simp as osimp, filter as cone
from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _setup(shape, seed=3, **kw):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(*shape)
    m = P.mesh
    fd = fem.dof_mask(P.fixed)
    E = fem.simp_modulus(W.rho_random(m, seed=seed, lo=0.1, hi=1.0), 3.0)
    h = mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed)
    Ed = torch.tensor(E, device="cuda:0")
    h.gmg_setup(Ed, mfto.default_gmg_params(**kw))
    prm = h.gmg_params_in_use()                   # automatic choices resolved
    H = gmg.build(fem.ke_exact(), E, *shape, fd, max_levels=prm.max_levels,
                  coarse_max_dofs=prm.coarse_max_dofs, omega=prm.omega, nu_pre=prm.nu_pre,
                  nu_post=prm.nu_post, cheb_degree=prm.cheb_degree)
    return P, m, fd, E, Ed, h, H


@pytest.mark.parametrize("matfree", [-1, 1])
@pytest.mark.parametrize("shape", [(24, 12, 12), (13, 7, 5)])
def test_levels_and_operators_match_oracle(cuda, shape, matfree):
    """Every level's operator against the oracle's Galerkin product; level 1
    from its element matrices (-1) and as Phat^T K Phat (1)."""
    import torch
    P, m, fd, E, Ed, h, H = _setup(shape, matfree_level1=matfree)
    with h:
        assert h.gmg_levels() == [lev.dims for lev in H.levels]
        rng = np.random.default_rng(7)
        for li, lev in enumerate(H.levels):
            x = rng.uniform(-1, 1, lev.A.shape[0])
            y = torch.empty(len(x), dtype=torch.float32, device=cuda)
            h.gmg_apply(li, torch.tensor(x, dtype=torch.float32, device=cuda), y)
            ref = lev.A @ x
            got = y.cpu().numpy().astype(np.float64)
            assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max(), li


@pytest.mark.parametrize("shape,nu,matfree,cheb", [((24, 12, 12), 2, -1, 0), ((13, 7, 5), 1, -1, 0),
                                                   ((9, 6, 4), 0, -1, 0), ((24, 12, 12), 1, 1, 0),
                                                   ((13, 7, 5), 2, 1, 0), ((24, 12, 12), 1, -1, 2),
                                                   ((13, 7, 5), 2, 1, 3), ((13, 7, 5), 2, -1, 2),
                                                   ((9, 6, 4), 0, -1, 2)])
def test_vcycle_matches_oracle(cuda, shape, nu, matfree, cheb):
    """One V-cycle against the oracle's: l1-Jacobi (cheb 0) and Chebyshev
    sweeps, 0-2 sweeps each side (two sweeps start the second from the
    current iterate, the fused kernels' second-buffer path), level 1 from
    its matrices (-1) or as Phat^T K Phat (1)."""
    import torch
    P, m, fd, E, Ed, h, H = _setup(shape, nu_pre=nu, nu_post=nu, matfree_level1=matfree,
                                   cheb_degree=cheb)
    with h:
        r = W.vec_random(m.n_dof, seed=11)
        r[fd] = 0.0
        z = torch.empty(m.n_dof, dtype=torch.float32, device=cuda)
        h.gmg_vcycle(torch.tensor(r, dtype=torch.float32, device=cuda), z)
        ref = gmg.vcycle(H, r)
        got = z.cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


def test_single_level_is_dense_solve(cuda):
    import torch
    P, m, fd, E, Ed, h, H = _setup((4, 2, 2), coarse_max_dofs=1000)
    with h:
        assert h.gmg_levels() == [(4, 2, 2)]
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        st = h.gmg_solve(Ed, torch.tensor(P.f, device=cuda), u)
        assert st.status == 0 and st.iterations <= 4


def _simp_state(shape, n_iter=6):
    P = W.cantilever(*shape)
    rho, _, _ = osimp.simp(*shape, P.f, P.fixed, 0.3, 1.5, n_iter)
    return P, cone.filter_fwd(rho, *shape, 1.5)


@pytest.mark.parametrize("mixed,matfree,cont,cheb", [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 0, 0),
                                                    (1, 0, 1, 0), (1, 0, 1, 2), (0, 0, 0, 2)])
def test_gmg_solve_matches_oracle(cuda, mixed, matfree, cont, cheb):
    """A SIMP state of the 24 x 12 x 12 cantilever (E from 1e-9 to 1): the
    V-cycle CG (FP64, or FP64 refinement around FP32 CGs) reaches the
    tolerance with the oracle's true residual, the oracle's compliance, and
    about the oracle's iteration count."""
    import torch
    from paper_2604_18020_gb300 import mfto
    shape = (24, 12, 12)
    P, rho_phys = _simp_state(shape)
    m = P.mesh
    fd = fem.dof_mask(P.fixed)
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(*shape)
    E = fem.simp_modulus(rho_phys, 3.0)
    K = lambda v: fem.kv(KE, E, edof, v, fd)
    u_j, _ = solve.pcg(K, fem.jacobi_diag(KE, E, edof, fd), P.f, np.zeros(m.n_dof), 1e-10)
    prm = mfto.default_gmg_params(mixed=mixed, matfree_level1=matfree, continue_dir=cont,
                                  cheb_degree=cheb)
    H = gmg.build(KE, E, *shape, fd, max_levels=prm.max_levels,
                  coarse_max_dofs=prm.coarse_max_dofs, omega=prm.omega, nu_pre=prm.nu_pre,
                  nu_post=prm.nu_post, cheb_degree=prm.cheb_degree)
    _, st_o = gmg.pcg(H, K, P.f, np.zeros(m.n_dof), 1e-8)
    with mfto.Handle(*shape, P.fixed) as h:
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        h.set_gmg_solver(False, prm)
        st = h.gmg_solve(torch.tensor(E, device=cuda), torch.tensor(P.f, device=cuda), u)
        assert h.gmg_levels() == [lev.dims for lev in H.levels]
    ug = u.cpu().numpy()
    assert st.status == 0 and st.rel_residual <= 1e-8
    assert np.linalg.norm(P.f - K(ug)) / np.linalg.norm(P.f) <= 1.5e-8
    assert abs(P.f @ ug - P.f @ u_j) <= 1e-7 * abs(P.f @ u_j)
    assert st.iterations <= (1.5 if mixed == 0 else 2.0) * st_o.iterations + 3


@pytest.mark.parametrize("form", ["tf32", "bf16", "f16", "bf16x3"])
def test_tensor_core_smoother(cuda, form):
    """The level-0 sweeps on a tensor-core K.v (the paper's proposal of a BF16
    smoother inside a V-cycle): the solve still reaches the oracle's solution,
    in a bounded number of iterations."""
    import torch
    from paper_2604_18020_gb300 import mfto
    shape = (24, 12, 12)
    P, rho_phys = _simp_state(shape)
    m = P.mesh
    fd = fem.dof_mask(P.fixed)
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(*shape)
    E = fem.simp_modulus(rho_phys, 3.0)
    K = lambda v: fem.kv(KE, E, edof, v, fd)
    u_j, _ = solve.pcg(K, fem.jacobi_diag(KE, E, edof, fd), P.f, np.zeros(m.n_dof), 1e-10)
    its = {}
    with mfto.Handle(*shape, P.fixed) as h:
        for name in ("f32", form):
            u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
            h.set_gmg_solver(False, mfto.default_gmg_params(smoother_form=mfto.FORMS[name]))
            st = h.gmg_solve(torch.tensor(E, device=cuda), torch.tensor(P.f, device=cuda), u)
            assert st.status == 0 and st.rel_residual <= 1e-8, name
            ug = u.cpu().numpy()
            assert np.linalg.norm(P.f - K(ug)) / np.linalg.norm(P.f) <= 1.5e-8
            assert abs(P.f @ ug - P.f @ u_j) <= 1e-7 * abs(P.f @ u_j)
            its[name] = st.iterations
    assert its[form] <= 3 * its["f32"] + 5


@pytest.mark.parametrize("mixed", [0, 1])
def test_simp_steps_with_gmg_solver(cuda, mixed):
    """Three SIMP iterations on 16 x 8 x 8 with the V-cycle CG as the solver
    against the oracle's SIMP loop (Jacobi-PCG): the same compliances."""
    import torch
    from paper_2604_18020_gb300 import mfto
    shape = (16, 8, 8)
    P = W.cantilever(*shape)
    m = P.mesh
    _, _, hist = osimp.simp(*shape, P.f, P.fixed, 0.3, 1.5, 3)
    with mfto.Handle(*shape, P.fixed, params=mfto.default_params(volfrac=0.3, rmin=1.5)) as h:
        h.set_gmg_solver(True, mfto.default_gmg_params(mixed=mixed))
        rho = torch.full((m.n_elem,), 0.3, dtype=torch.float64, device=cuda)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        f = torch.tensor(P.f, device=cuda)
        cs = [h.simp_step(rho, u, f) for _ in range(3)]
    for st, c_ref in zip(cs, hist.compliance):
        assert st.cg_status == 0
        assert abs(st.compliance - c_ref) <= 1e-6 * abs(c_ref)


def test_gmg_argument_checks(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(24, 12, 12)
    m = P.mesh
    E = torch.ones(m.n_elem, dtype=torch.float64, device=cuda)
    with mfto.Handle(24, 12, 12, P.fixed) as h:
        z = torch.empty(m.n_dof, dtype=torch.float32, device=cuda)
        with pytest.raises(mfto.MftoError):          # no hierarchy yet
            h.gmg_vcycle(torch.zeros(m.n_dof, dtype=torch.float32, device=cuda), z)
        with pytest.raises(mfto.MftoError):          # weight outside (0, 2)
            h.gmg_setup(E, mfto.default_gmg_params(omega=2.0))
        with pytest.raises(mfto.MftoError):          # FP64 is no smoother form
            h.gmg_setup(E, mfto.default_gmg_params(smoother_form=mfto.FORM_F64))
        with pytest.raises(mfto.MftoError) as ei:    # a single 4,875-DOF level is too large
            h.gmg_setup(E, mfto.default_gmg_params(max_levels=1))
        assert ei.value.code == mfto.TOO_LARGE


def test_gmg_on_singular_mbb(cuda):
    """The MBB preset's free z translation and rotation make the coarsest
    operator rank deficient; the shifted coarsest inverse keeps the V-cycle
    SPD and the solve reaches the oracle's compliance (both precisions)."""
    import torch
    from paper_2604_18020_gb300 import mfto
    shape = (30, 10, 5)
    P = W.mbb(*shape)
    m = P.mesh
    fd = fem.dof_mask(P.fixed)
    E = fem.simp_modulus(np.full(m.n_elem, P.volfrac), 3.0)
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(*shape)
    K = lambda v: fem.kv(KE, E, edof, v, fd)
    u_j, _ = solve.pcg(K, fem.jacobi_diag(KE, E, edof, fd), P.f, np.zeros(m.n_dof), 1e-10)
    with mfto.Handle(*shape, P.fixed) as h:
        for mixed in (0, 1):
            u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
            h.set_gmg_solver(False, mfto.default_gmg_params(mixed=mixed))
            st = h.gmg_solve(torch.tensor(E, device=cuda), torch.tensor(P.f, device=cuda), u)
            ug = u.cpu().numpy()
            assert st.status == 0 and st.rel_residual <= 1e-8, mixed
            assert np.linalg.norm(P.f - K(ug)) / np.linalg.norm(P.f) <= 1.5e-8
            assert abs(P.f @ ug - P.f @ u_j) <= 1e-7 * abs(P.f @ u_j)


def test_device_bytes_accounts_for_the_hierarchy(cuda):
    """mfto_device_bytes: at least the handle's DOF vectors after creation,
    and exactly the hierarchy's arrays more after a multigrid setup (element
    matrices, masks, vectors of every level, the coarsest inverse)."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(24, 12, 12)
    m = P.mesh
    with mfto.Handle(24, 12, 12, P.fixed) as h:
        b0 = h.device_bytes()
        assert b0 >= m.n_dof * (6 * 8 + 7 * 4) + m.n_elem * (6 * 8 + 4)
        h.gmg_setup(torch.ones(m.n_elem, dtype=torch.float64, device=cuda))
        dims = h.gmg_levels()
        cheb = h.gmg_params_in_use().cheb_degree
        exp = 8 * 576 * 4 + m.n_elem * 4                        # G table, FP32 moduli
        for l, (nx, ny, nz) in enumerate(dims):
            n_node = (nx + 1) * (ny + 1) * (nz + 1)
            exp += 2 * 4 * 3 * n_node
            if cheb > 0 and l + 1 < len(dims):
                exp += 2 * 4 * 3 * n_node                         # Chebyshev step, residual
            if cheb != 1 and l == 0:
                exp += 2 * 4 * 3 * n_node                         # fused-sweep scratch
            if l > 0:
                exp += n_node + 4 * (576 * nx * ny * nz + 3 * 3 * n_node)
        nx, ny, nz = dims[-1]
        n_c = 3 * (nx + 1) * (ny + 1) * (nz + 1)
        exp += 4 * n_c * n_c
        grown = h.device_bytes() - b0
        assert exp <= grown <= exp + 256                          # plus two scalar blocks


def test_gmg_is_bit_reproducible(cuda):
    """No atomics anywhere in the hierarchy, the cycle or the CG sums: two
    setups, V-cycles and solves from the same inputs agree bit for bit."""
    import torch
    from paper_2604_18020_gb300 import mfto
    shape = (20, 10, 10)
    P, rho_phys = _simp_state(shape, n_iter=4)
    m = P.mesh
    E = torch.tensor(fem.simp_modulus(rho_phys, 3.0), device=cuda)
    f = torch.tensor(P.f, device=cuda)
    r = torch.tensor(W.vec_random(m.n_dof, seed=9), dtype=torch.float32, device=cuda)
    outs = []
    for _ in range(2):
        with mfto.Handle(*shape, P.fixed) as h:
            h.gmg_setup(E)
            z = torch.empty_like(r)
            h.gmg_vcycle(r, z)
            u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
            st = h.gmg_solve(E, f, u)
            outs.append((z.clone(), u.clone(), st.iterations))
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1]) and outs[0][2] == outs[1][2]


def test_gmg_full_size_bench_configuration(cuda):
    """120x60x30 (216,000 elements, 686,433 DOFs), the configuration and
    solver settings the benchmark's multigrid leg uses, on a filtered random
    design (E from 1e-9 to 1): the hierarchy equals the oracle's, the solve's
    true residual (the oracle's K.v of the GPU solution) holds the tolerance,
    and its compliance f.u equals the sum of the oracle's element energies."""
    import torch
    from paper_2604_18020_gb300 import mfto
    from oracle import simp as osimp
    shape = (120, 60, 30)
    P = W.cantilever(*shape)
    m = P.mesh
    fd = fem.dof_mask(P.fixed)
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(*shape)
    rho = cone.filter_fwd(W.rho_binary(m, seed=2, volfrac=0.3), *shape, 1.5)
    E = fem.simp_modulus(rho, 3.0)
    with mfto.Handle(*shape, P.fixed) as h:
        prm = mfto.default_gmg_params()
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        st = h.gmg_solve(torch.tensor(E, device=cuda), torch.tensor(P.f, device=cuda), u)
        assert h.gmg_levels() == gmg.level_dims(*shape, max_levels=prm.max_levels,
                                                coarse_max_dofs=prm.coarse_max_dofs)
    ug = u.cpu().numpy()
    assert st.status == 0 and st.rel_residual <= 1e-8
    r = P.f - fem.kv(KE, E, edof, ug, fd)
    assert np.linalg.norm(r) / np.linalg.norm(P.f) <= 1.5e-8
    c_elem = float(np.sum(E * osimp.element_energy(KE, edof, ug)))
    assert abs(c_elem - P.f @ ug) <= 1e-7 * abs(P.f @ ug)


def test_gmg_solve_multi_load_cases(cuda):
    """Four load cases of the multi-RHS cantilever on one hierarchy: each case
    reaches the oracle's Jacobi-PCG compliance and true residual."""
    import torch
    from paper_2604_18020_gb300 import mfto
    shape = (16, 8, 8)
    P = W.multi_rhs_cantilever(*shape, nrhs=4, seed=3)
    m = P.mesh
    fd = fem.dof_mask(P.fixed)
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(*shape)
    E = fem.simp_modulus(W.rho_random(m, seed=4, lo=0.05, hi=1.0), 3.0)
    K = lambda v: fem.kv(KE, E, edof, v, fd)
    d = fem.jacobi_diag(KE, E, edof, fd)
    with mfto.Handle(*shape, P.fixed) as h:
        U = torch.zeros(4 * m.n_dof, dtype=torch.float64, device=cuda)
        sts = h.gmg_solve_multi(torch.tensor(E, device=cuda),
                                torch.tensor(P.f.reshape(-1), device=cuda), U, 4)
    Ug = U.cpu().numpy().reshape(4, m.n_dof)
    for r in range(4):
        assert sts[r].status == 0 and sts[r].rel_residual <= 1e-8
        u_j, _ = solve.pcg(K, d, P.f[r], np.zeros(m.n_dof), 1e-10)
        assert np.linalg.norm(P.f[r] - K(Ug[r])) / np.linalg.norm(P.f[r]) <= 1.5e-8
        assert abs(P.f[r] @ Ug[r] - P.f[r] @ u_j) <= 1e-7 * abs(P.f[r] @ u_j)


@pytest.mark.parametrize("shape", [(12, 6, 1), (7, 1, 3), (1, 1, 5)])
def test_degenerate_one_element_axes(cuda, shape):
    """Meshes one element thick along an axis: that axis keeps one coarse
    element on every level (its coarse node 1 lies past the fine mesh); the
    hierarchy, every level's operator and one V-cycle match the oracle.  The
    cycle's bound is 5e-4 of max|z| here: a one-element column is badly
    conditioned (the cycle amplifies r by ~500 on 1 x 1 x 5), and the FP32
    coarse solves carry kappa times the unit roundoff."""
    import torch
    P, m, fd, E, Ed, h, H = _setup(shape, coarse_max_dofs=30)
    with h:
        assert h.gmg_levels() == [lev.dims for lev in H.levels]
        rng = np.random.default_rng(5)
        for li, lev in enumerate(H.levels):
            x = rng.uniform(-1, 1, lev.A.shape[0])
            y = torch.empty(len(x), dtype=torch.float32, device=cuda)
            h.gmg_apply(li, torch.tensor(x, dtype=torch.float32, device=cuda), y)
            ref = lev.A @ x
            assert np.abs(y.cpu().numpy() - ref).max() <= 2e-5 * np.abs(ref).max(), li
        r = W.vec_random(m.n_dof, seed=6)
        r[fd] = 0.0
        z = torch.empty(m.n_dof, dtype=torch.float32, device=cuda)
        h.gmg_vcycle(torch.tensor(r, dtype=torch.float32, device=cuda), z)
        ref = gmg.vcycle(H, r)
        assert np.abs(z.cpu().numpy() - ref).max() <= 5e-4 * np.abs(ref).max()


def test_gmg_solve_at_4_9M_elements(cuda):
    """The paper's 4.9M-element cantilever shape (340x170x85, 15.0M DOFs) at
    uniform density 0.5: level 1 is applied as Phat^T K Phat (its matrices
    exceed the threshold), the inner CG runs one iteration per graph chunk,
    and the solution's true residual, recomputed by the oracle's K.v, and its
    compliance against the oracle's element energies hold the tolerance."""
    import torch
    from paper_2604_18020_gb300 import mfto
    from oracle import simp as osimp
    shape = (340, 170, 85)
    P = W.cantilever_point(*shape)
    m = P.mesh
    fd = fem.dof_mask(P.fixed)
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(*shape)
    E = np.full(m.n_elem, 0.5 ** 3)
    with mfto.Handle(*shape, P.fixed) as h:
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        st = h.gmg_solve(torch.tensor(E, device=cuda), torch.tensor(P.f, device=cuda), u)
        assert len(h.gmg_levels()) == 8
    ug = u.cpu().numpy()
    assert st.status == 0 and st.rel_residual <= 1e-8
    r = P.f - fem.kv(KE, E, edof, ug, fd)
    assert np.linalg.norm(r) / np.linalg.norm(P.f) <= 1.5e-8
    c_elem = float(np.sum(E * osimp.element_energy(KE, edof, ug)))
    assert abs(c_elem - P.f @ ug) <= 1e-7 * abs(P.f @ ug)


def test_single_element_mesh(cuda):
    """1 x 1 x 1: a single level solved by its dense inverse, both precisions."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(1, 1, 1)
    m = P.mesh
    fd = fem.dof_mask(P.fixed)
    E = np.array([0.7])
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(1, 1, 1)
    u_ref = solve.dense_solve(fem.assemble_masked(KE, E, edof, m.n_dof, fd), P.f)
    with mfto.Handle(1, 1, 1, P.fixed) as h:
        for mixed in (0, 1):
            u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
            h.set_gmg_solver(False, mfto.default_gmg_params(mixed=mixed))
            st = h.gmg_solve(torch.tensor(E, device=cuda), torch.tensor(P.f, device=cuda), u)
            assert h.gmg_levels() == [(1, 1, 1)]
            assert st.status == 0
            assert np.abs(u.cpu().numpy() - u_ref).max() <= 1e-6 * np.abs(u_ref).max()


def test_automatic_chebyshev_choice(cuda):
    """cheb_degree = -1 resolves to degree 2 up to 4M DOFs and to l1-Jacobi
    sweeps above; an explicit degree is kept."""
    import torch
    from paper_2604_18020_gb300 import mfto
    for shape, expect in (((24, 12, 12), 2), ((200, 100, 50), 2), ((252, 126, 63), 0)):
        P = W.cantilever(*shape)
        m = P.mesh
        with mfto.Handle(*shape, P.fixed) as h:
            E = torch.ones(m.n_elem, dtype=torch.float64, device=cuda)
            h.gmg_setup(E)
            assert h.gmg_params_in_use().cheb_degree == expect, shape
            h.gmg_setup(E, mfto.default_gmg_params(cheb_degree=3))
            assert h.gmg_params_in_use().cheb_degree == 3

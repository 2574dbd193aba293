"""Pins of the oracle's geometric multigrid (no GPU): trilinear
interpolation reproduces multilinear fields, the Galerkin coarse operator of
a uniform mesh equals the rediscretised one (KE(2h) = 2 KE(h) in 3-D
elasticity), the masked hierarchy stays SPD, the V-cycle is a symmetric
positive operator, the two-level cycle without smoothing is the coarse-grid
correction, the l1-Jacobi bound, and V-cycle CG against Jacobi-PCG."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, gmg, solve, filter as cone
from paper_2604_18020_gb300 import workloads as W


def _nodes(n):
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    return i.reshape(-1).astype(float), j.reshape(-1).astype(float), k.reshape(-1).astype(float)


@pytest.mark.parametrize("n", [(5, 4, 3), (4, 4, 2), (1, 3, 2)])
def test_prolongation_reproduces_multilinear_fields(n):
    c = np.random.default_rng(0).normal(size=8)
    f = lambda x, y, z: (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * y * z
                         + c[6] * x * z + c[7] * x * y * z)
    X, Y, Z = _nodes(gmg.coarse_dims(n))
    coarse = f(2 * X, 2 * Y, 2 * Z)            # coarse node I sits at fine coordinate 2I
    x, y, z = _nodes(n)
    fine = gmg.prolong_nodes(n) @ coarse
    assert np.abs(fine - f(x, y, z)).max() <= 1e-12 * np.abs(coarse).max()


def test_level_dims():
    assert gmg.level_dims(120, 60, 30) == [(120, 60, 30), (60, 30, 15), (30, 15, 8), (15, 8, 4),
                                           (8, 4, 2), (4, 2, 1)]
    assert gmg.level_dims(3, 2, 2, coarse_max_dofs=10**6) == [(3, 2, 2)]
    assert gmg.level_dims(2, 2, 2, coarse_max_dofs=1) == [(2, 2, 2), (1, 1, 1)]


def test_galerkin_of_uniform_mesh_is_rediscretised_operator():
    n = (4, 2, 2)
    m, mc = W.Mesh(*n), W.Mesh(*gmg.coarse_dims(n))
    KE1, KE2 = fem.ke_exact(h=1.0), fem.ke_exact(h=2.0)
    assert np.abs(KE2 - 2.0 * KE1).max() <= 1e-14 * np.abs(KE1).max()
    K = fem.assemble(KE1, np.ones(m.n_elem), fem.edof_table_fast(*n), m.n_dof)
    Pm = gmg.prolong_dofs(n)
    Kc = (Pm.T @ K @ Pm).toarray()
    ref = fem.assemble(KE2, np.ones(mc.n_elem), fem.edof_table_fast(mc.nelx, mc.nely, mc.nelz),
                       mc.n_dof).toarray()
    assert np.abs(Kc - ref).max() <= 1e-12 * np.abs(ref).max()


def _hierarchy(shape, seed=3, face="x0", **kw):
    m = W.Mesh(*shape)
    fd = fem.dof_mask(W.fixed_face(m, face))
    E = fem.simp_modulus(W.rho_random(m, seed=seed, lo=0.05, hi=1.0), 3.0)
    KE = fem.ke_exact()
    return m, fd, E, KE, gmg.build(KE, E, *shape, fd, **kw)


def test_masked_hierarchy_is_spd_with_fixed_faces():
    m, fd, E, KE, H = _hierarchy((6, 4, 3), coarse_max_dofs=1)
    face = None                        # expected fixed x = 0 face nodes, [z][y]
    for li, lev in enumerate(H.levels):
        A = lev.A.toarray()
        assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
        assert np.linalg.eigvalsh(A).min() > 0
        fx = np.flatnonzero(lev.fixed)
        assert len(fx) > 0 and np.all(A[fx, fx] == 1.0)
        assert np.all(A[fx][:, np.setdiff1d(np.arange(A.shape[0]), fx)] == 0.0)
        nx, ny, nz = lev.dims
        nodes = lev.fixed.reshape(nz + 1, ny + 1, nx + 1, 3)
        assert not nodes[:, :, 1:, :].any()                      # only on the x = 0 face
        if face is None:
            face = np.ones((nz + 1, ny + 1), bool)
        assert np.array_equal(nodes[:, :, 0, 0], face)
        # next level: coarse (K, J) is fixed where the fine node (2K, 2J) exists and is fixed
        mz, my = (nz + 1) // 2 + 1, (ny + 1) // 2 + 1
        nxt = np.zeros((mz, my), bool)
        for K in range(mz):
            for J in range(my):
                nxt[K, J] = 2 * K <= nz and 2 * J <= ny and face[2 * K, 2 * J]
        face = nxt


def test_vcycle_is_symmetric_positive():
    m, fd, E, KE, H = _hierarchy((8, 4, 4), nu_pre=2, nu_post=2)
    assert len(H.levels) >= 2
    rng = np.random.default_rng(1)
    b1, b2 = rng.normal(size=m.n_dof), rng.normal(size=m.n_dof)
    b1[fd] = 0.0
    b2[fd] = 0.0
    v1, v2 = gmg.vcycle(H, b1), gmg.vcycle(H, b2)
    assert abs(b1 @ v2 - b2 @ v1) <= 1e-11 * abs(b1 @ v2)
    assert b1 @ v1 > 0 and b2 @ v2 > 0


def test_two_level_without_smoothing_is_coarse_correction():
    m, fd, E, KE, H = _hierarchy((4, 4, 2), max_levels=2, nu_pre=0, nu_post=0)
    assert len(H.levels) == 2
    b = np.random.default_rng(2).normal(size=m.n_dof)
    P = H.levels[0].P
    ref = P @ np.linalg.solve(H.levels[1].A.toarray(), P.T @ b)
    assert np.abs(gmg.vcycle(H, b) - ref).max() <= 1e-10 * np.abs(ref).max()


def test_single_level_is_exact_solve():
    P = W.cantilever(4, 2, 2)
    m = P.mesh
    fd = fem.dof_mask(P.fixed)
    E = fem.simp_modulus(W.rho_random(m, seed=5, lo=0.1, hi=1.0), 3.0)
    KE = fem.ke_exact()
    H = gmg.build(KE, E, 4, 2, 2, fd, coarse_max_dofs=10**6)
    edof = fem.edof_table_fast(4, 2, 2)
    u, st = gmg.pcg(H, lambda v: fem.kv(KE, E, edof, v, fd), P.f, np.zeros(m.n_dof), 1e-10)
    assert st.iterations == 1 and st.true_rel_residual <= 1e-12


def test_element_matrices_assemble_to_galerkin_operator():
    """The per-element Galerkin matrices of every level sum to the global
    product Phat^T A Phat (masked), and the fine ones to the masked K."""
    m, fd, E, KE, H = _hierarchy((5, 4, 3), coarse_max_dofs=1)
    for lev in H.levels:
        edof = fem.edof_table_fast(*lev.dims)
        n = lev.A.shape[0]
        rows = np.repeat(edof, 24, axis=1).reshape(-1)
        cols = np.tile(edof, (1, 24)).reshape(-1)
        S = sp.coo_matrix((lev.Ke.reshape(-1), (rows, cols)), shape=(n, n)).toarray()
        S[lev.fixed, lev.fixed] = 1.0
        assert np.abs(S - lev.A.toarray()).max() <= 1e-12 * np.abs(S).max()


def test_l1_jacobi_bound():
    """lambda_max(D1^-1 A) <= 1 on every level (so omega < 2 smooths)."""
    m, fd, E, KE, H = _hierarchy((6, 4, 4), coarse_max_dofs=1)
    for lev in H.levels:
        s = np.sqrt(lev.d1inv)
        lam = np.linalg.eigvalsh(s[:, None] * lev.A.toarray() * s[None, :]).max()
        assert lam <= 1.0 + 1e-12


def test_vcycle_cg_matches_jacobi_pcg_in_fewer_iterations():
    """A filtered random design (the smoothness of a SIMP state): the same
    solution as Jacobi-PCG in a fraction of the iterations."""
    shape = (16, 8, 8)
    P = W.cantilever(*shape)
    m = P.mesh
    fd = fem.dof_mask(P.fixed)
    rho = cone.filter_fwd(W.rho_binary(m, seed=4, volfrac=0.4), *shape, 1.5)
    E = fem.simp_modulus(rho, 3.0)
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(*shape)
    K = lambda v: fem.kv(KE, E, edof, v, fd)
    u_j, st_j = solve.pcg(K, fem.jacobi_diag(KE, E, edof, fd), P.f, np.zeros(m.n_dof), 1e-10)
    H = gmg.build(KE, E, *shape, fd)
    u_g, st_g = gmg.pcg(H, K, P.f, np.zeros(m.n_dof), 1e-10)
    assert st_g.converged and st_g.true_rel_residual <= 1e-9
    assert st_g.iterations * 4 <= st_j.iterations
    assert abs(P.f @ u_g - P.f @ u_j) <= 1e-9 * abs(P.f @ u_j)


def test_singular_consistent_problem_mbb():
    """The MBB preset leaves the z translation and one rotation free: the
    coarsest operator is rank deficient (two zero eigenvalues), the pivot
    test catches it, and the V-cycle CG still solves the consistent system
    to the Jacobi-PCG compliance in far fewer iterations."""
    shape = (24, 8, 4)
    P = W.mbb(*shape)
    m = P.mesh
    fd = fem.dof_mask(P.fixed)
    E = fem.simp_modulus(np.full(m.n_elem, P.volfrac), 3.0)
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(*shape)
    K = lambda v: fem.kv(KE, E, edof, v, fd)
    H = gmg.build(KE, E, *shape, fd, omega=1.3, nu_pre=1, nu_post=1)
    Ac = H.levels[-1].A.toarray()
    ev = np.linalg.eigvalsh(Ac)
    assert np.sum(np.abs(ev) < 1e-12 * ev[-1]) == 2
    assert not gmg.cholesky_pivots_ok(Ac)
    u_j, st_j = solve.pcg(K, fem.jacobi_diag(KE, E, edof, fd), P.f, np.zeros(m.n_dof), 1e-8)
    u_g, st_g = gmg.pcg(H, K, P.f, np.zeros(m.n_dof), 1e-8)
    assert st_g.converged and st_g.true_rel_residual <= 1e-8
    assert abs(P.f @ u_g - P.f @ u_j) <= 1e-9 * abs(P.f @ u_j)
    assert st_g.iterations * 4 <= st_j.iterations


def test_pivot_test_leaves_constrained_problems_alone():
    m, fd, E, KE, H = _hierarchy((8, 4, 4))
    Ac = H.levels[-1].A.toarray()
    assert gmg.cholesky_pivots_ok(Ac)
    assert np.abs(H.coarse_inv - np.linalg.inv(Ac)).max() <= 1e-10 * np.abs(H.coarse_inv).max()


@pytest.mark.parametrize("degree", [1, 2, 3, 4])
def test_chebyshev_sweep_is_the_scaled_chebyshev_polynomial(degree):
    """On the eigenvectors of the symmetric D1^-1/2 A D1^-1/2, one sweep from
    x multiplies the error by T_k((theta - lam)/delta) / T_k(theta/delta)
    (closed form, T_k the Chebyshev polynomial of the first kind)."""
    m, fd, E, KE, H = _hierarchy((4, 3, 2), coarse_max_dofs=1)
    lev = H.levels[0]
    A = lev.A.toarray()
    s = np.sqrt(lev.d1inv)
    lam, Q = np.linalg.eigh(s[:, None] * A * s[None, :])
    u = np.random.default_rng(3).normal(size=A.shape[0])          # exact solution
    b = A @ u
    x0 = np.random.default_rng(4).normal(size=A.shape[0])
    x1 = gmg.cheb_smooth(lev, x0, b, degree, 1)
    lmin, lmax = 1.0 / gmg.CHEB_RATIO, 1.0
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    T = lambda t: np.cos(degree * np.arccos(t)) if abs(t) <= 1 else np.cosh(degree * np.arccosh(abs(t))) * (np.sign(t) ** degree)
    gain = np.array([T((theta - l) / delta) for l in lam]) / T(theta / delta)
    e0 = Q.T @ ((x0 - u) / s)                    # error in the symmetric basis
    e1 = Q.T @ ((x1 - u) / s)
    assert np.abs(e1 - gain * e0).max() <= 1e-9 * np.abs(e0).max()


def test_chebyshev_vcycle_symmetric_and_converging():
    m, fd, E, KE, H = _hierarchy((8, 4, 4), nu_pre=1, nu_post=1, cheb_degree=2)
    rng = np.random.default_rng(1)
    b1, b2 = rng.normal(size=m.n_dof), rng.normal(size=m.n_dof)
    b1[fd] = 0.0
    b2[fd] = 0.0
    v1, v2 = gmg.vcycle(H, b1), gmg.vcycle(H, b2)
    assert abs(b1 @ v2 - b2 @ v1) <= 1e-11 * abs(b1 @ v2)
    assert b1 @ v1 > 0
    edof = fem.edof_table_fast(8, 4, 4)
    P = W.cantilever(8, 4, 4)
    K = lambda v: fem.kv(KE, E, edof, v, fd)
    u, st = gmg.pcg(H, K, P.f, np.zeros(m.n_dof), 1e-10)
    assert st.converged and st.true_rel_residual <= 1e-9

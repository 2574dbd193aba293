"""Pins of the oracle's indexing, element matrix, K.v and Jacobi diagonal
against closed forms, invariants and brute force (no GPU)."""
import numpy as np
import pytest

from oracle import fem
from paper_2604_18020_gb300 import workloads as W


def test_edof_fast_equals_brute_force():
    for shape in [(1, 1, 1), (2, 1, 1), (3, 2, 4), (5, 3, 2)]:
        assert np.array_equal(fem.edof_table(*shape), fem.edof_table_fast(*shape))


def test_edof_hand_worked_example():
    # 2x1x1 mesh: nodes n = i + 3 (j + 2 k); element 0 has corners
    # (0,0,0) (1,0,0) (0,1,0) (1,1,0) (0,0,1) (1,0,1) (0,1,1) (1,1,1)
    nodes = [0, 1, 3, 4, 6, 7, 9, 10]
    expect = np.array([3 * n + c for n in nodes for c in range(3)])
    assert np.array_equal(fem.edof_table(2, 1, 1)[0], expect)
    assert np.array_equal(fem.edof_table(2, 1, 1)[1], expect + 3)


def test_edof_covers_every_dof():
    edof = fem.edof_table_fast(4, 3, 2)
    counts = np.bincount(edof.reshape(-1), minlength=3 * 5 * 4 * 3)
    assert counts.min() >= 1 and counts.max() == 8


def test_ke_two_derivations_agree():
    for nu in (0.0, 0.3, 0.45):
        for h in (1.0, 2.0, 0.25):
            a, b = fem.ke_gauss(1.0, nu, h), fem.ke_exact(1.0, nu, h)
            assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()


def test_ke_closed_form_entries():
    # K[0][0] = (lam + 4 mu) h / 9 and K[0][1] = (lam + mu) h / 12 (node 0 with
    # itself), from the products of the 1-D integrals h/3, 1/h, -1/2.
    nu, h = 0.3, 1.0
    lam, mu = nu / ((1 + nu) * (1 - 2 * nu)), 1 / (2 * (1 + nu))
    K = fem.ke_gauss(1.0, nu, h)
    assert abs(K[0, 0] - (lam + 4 * mu) * h / 9) <= 1e-15
    assert abs(K[0, 1] - (lam + mu) * h / 12) <= 1e-15
    assert np.allclose(np.diag(K), K[0, 0], rtol=0, atol=1e-15)


def test_ke_symmetric_psd_rank18():
    K = fem.ke_exact()
    assert np.array_equal(K, K.T)
    w = np.linalg.eigvalsh(fem.ke_gauss())
    assert np.sum(np.abs(w) < 1e-12 * w.max()) == 6
    assert w.min() > -1e-14 and np.sum(w > 1e-12 * w.max()) == 18


def _rigid_modes():
    X = np.array([[a, b, c] for (a, b, c) in fem.local_corners()], dtype=float)
    modes = []
    for d in range(3):
        t = np.zeros((8, 3))
        t[:, d] = 1.0
        modes.append(t.reshape(-1))
    for axis in range(3):
        w = np.zeros(3)
        w[axis] = 1.0
        modes.append(np.cross(w, X).reshape(-1))
    return np.array(modes)


def test_ke_null_space_is_rigid_motion():
    K = fem.ke_gauss()
    R = _rigid_modes()
    assert np.abs(K @ R.T).max() <= 1e-14
    assert np.abs(K.sum(axis=1)).max() <= 1e-14          # rows sum to zero
    # the 6 rigid modes span the whole null space (rank 18 above)
    assert np.linalg.matrix_rank(R, tol=1e-12) == 6


def test_patch_uniform_strain_energy():
    """u = eps x gives 1/2 u^T KE u = 1/2 eps_voigt^T D eps_voigt h^3."""
    rng = np.random.default_rng(0)
    for h in (1.0, 2.0):
        X = h * np.array([[a, b, c] for (a, b, c) in fem.local_corners()], dtype=float)
        for _ in range(5):
            G = rng.standard_normal((3, 3))
            eps = 0.5 * (G + G.T)
            u = (X @ eps.T).reshape(-1)
            voigt = np.array([eps[0, 0], eps[1, 1], eps[2, 2],
                              2 * eps[0, 1], 2 * eps[1, 2], 2 * eps[2, 0]])
            e_fe = 0.5 * u @ fem.ke_exact(1.0, 0.3, h) @ u
            e_cont = 0.5 * voigt @ fem.elasticity_D(1.0, 0.3) @ voigt * h ** 3
            assert abs(e_fe - e_cont) <= 1e-13 * abs(e_cont)


def test_ke_scales_with_h_and_E():
    assert np.allclose(fem.ke_exact(2.0, 0.3, 3.0), 6.0 * fem.ke_exact(1.0, 0.3, 1.0),
                       rtol=1e-14, atol=0)


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 1), (3, 2, 2), (4, 3, 5)])
def test_matrix_free_equals_assembled(shape):
    m = W.Mesh(*shape)
    edof = fem.edof_table(*shape)
    KE = fem.ke_exact()
    E = fem.simp_modulus(W.rho_random(m, seed=1), 3.0)
    v = W.vec_random(m.n_dof, seed=2)
    K = fem.assemble(KE, E, edof, m.n_dof)
    assert np.abs(K @ v - fem.kv_unmasked(KE, E, edof, v)).max() <= 1e-13 * np.abs(K @ v).max()
    Kd = K.toarray()
    assert np.abs(Kd - Kd.T).max() <= 1e-15
    # masked operator equals the masked assembled matrix
    fixed = W.fixed_face(m, "x0")
    fd = fem.dof_mask(fixed)
    Km = fem.assemble_masked(KE, E, edof, m.n_dof, fd)
    assert np.abs(Km @ v - fem.kv(KE, E, edof, v, fd)).max() <= 1e-13 * np.abs(Km @ v).max()


def test_masked_operator_spd_and_symmetric():
    m = W.Mesh(3, 2, 2)
    edof = fem.edof_table(3, 2, 2)
    KE = fem.ke_exact()
    E = fem.simp_modulus(W.rho_random(m, seed=3), 3.0)
    fd = fem.dof_mask(W.fixed_face(m, "x0"))
    Km = fem.assemble_masked(KE, E, edof, m.n_dof, fd)
    assert np.linalg.eigvalsh(Km).min() > 0
    u, v = W.vec_random(m.n_dof, 4), W.vec_random(m.n_dof, 5)
    a = u @ fem.kv(KE, E, edof, v, fd)
    b = v @ fem.kv(KE, E, edof, u, fd)
    assert abs(a - b) <= 1e-13 * abs(a)


def test_rigid_translation_in_kernel_of_unmasked_K():
    m = W.Mesh(4, 3, 2)
    edof = fem.edof_table_fast(4, 3, 2)
    E = fem.simp_modulus(W.rho_random(m, seed=6), 3.0)
    t = np.tile([0.3, -1.2, 0.7], m.n_node)
    assert np.abs(fem.kv_unmasked(fem.ke_exact(), E, edof, t)).max() <= 1e-14


def test_patch_test_interior_nodes():
    """Uniform E, linear displacement: K u vanishes at interior nodes."""
    nelx, nely, nelz = 4, 3, 3
    m = W.Mesh(nelx, nely, nelz)
    edof = fem.edof_table_fast(nelx, nely, nelz)
    eps = np.array([[0.1, 0.02, -0.03], [0.02, -0.05, 0.04], [-0.03, 0.04, 0.07]])
    k, j, i = np.meshgrid(np.arange(nelz + 1), np.arange(nely + 1), np.arange(nelx + 1),
                          indexing="ij")
    X = np.stack([i, j, k], axis=-1).reshape(-1, 3).astype(float)
    u = (X @ eps.T).reshape(-1)
    w = fem.kv_unmasked(fem.ke_exact(), np.ones(m.n_elem), edof, u).reshape(-1, 3)
    interior = ((X[:, 0] > 0) & (X[:, 0] < nelx) & (X[:, 1] > 0) & (X[:, 1] < nely)
                & (X[:, 2] > 0) & (X[:, 2] < nelz))
    assert np.abs(w[interior]).max() <= 1e-14
    assert np.abs(w[~interior]).max() > 1e-3


def test_jacobi_diag_equals_assembled_diagonal():
    m = W.Mesh(3, 2, 4)
    edof = fem.edof_table(3, 2, 4)
    KE = fem.ke_exact()
    E = fem.simp_modulus(W.rho_random(m, seed=7), 3.0)
    fd = fem.dof_mask(W.fixed_face(m, "z0"))
    Km = fem.assemble_masked(KE, E, edof, m.n_dof, fd)
    assert np.abs(np.diag(Km) - fem.jacobi_diag(KE, E, edof, fd)).max() <= 1e-15


def test_simp_modulus_endpoints():
    E = fem.simp_modulus(np.array([0.0, 1.0, 0.5]), 3.0, 1.0, 1e-9)
    assert E[0] == 1e-9 and E[1] == 1.0
    assert abs(E[2] - (1e-9 + (1 - 1e-9) * 0.125)) <= 1e-16

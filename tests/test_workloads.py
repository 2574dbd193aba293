"""Host-side presets (no GPU): the boundary conditions and loads of the
paper's MBB and bridge hard problems as stated, and the consistency of the
MBB system (its load is orthogonal to the free rigid motions)."""
import numpy as np

from oracle import fem
from paper_2604_18020_gb300 import workloads as W


def test_mbb_preset():
    P = W.mbb(12, 4, 4)
    m = P.mesh
    fx = W.fixed_dofs(P.fixed).reshape(-1, 3)
    nodes = np.arange(m.n_node)
    i = nodes % (m.nelx + 1)
    # u_x fixed exactly on the x = 0 face, u_y at one node, u_z nowhere
    assert np.array_equal(fx[:, 0], i == 0)
    assert fx[:, 1].sum() == 1 and fx[m.node(m.nelx, 0, m.nelz // 2), 1]
    assert not fx[:, 2].any()
    assert abs(P.f.sum() + 1.0) <= 1e-15 and P.f[3 * m.node(0, m.nely, m.nelz // 2) + 1] == -1.0
    # the free rigid motions: z translation, rotation about x through the support
    tz = np.zeros((m.n_node, 3))
    tz[:, 2] = 1.0
    j = (nodes // (m.nelx + 1)) % (m.nely + 1)
    k = nodes // ((m.nelx + 1) * (m.nely + 1))
    rx = np.zeros((m.n_node, 3))
    rx[:, 1] = -(k - m.nelz // 2)
    rx[:, 2] = j
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    E = np.ones(m.n_elem)
    fd = W.fixed_dofs(P.fixed)
    for mode in (tz.reshape(-1), rx.reshape(-1)):
        mode = np.where(fd, 0.0, mode)
        assert np.abs(fem.kv(KE, E, edof, mode, fd)).max() <= 1e-12   # in the null space
        assert abs(P.f @ mode) <= 1e-15                                # load orthogonal


def test_bridge_preset():
    P = W.bridge(12, 4, 4)
    m = P.mesh
    fx = W.fixed_dofs(P.fixed).reshape(-1, 3)
    for k in range(m.nelz + 1):
        assert fx[m.node(0, 0, k)].all()
        assert list(fx[m.node(m.nelx, 0, k)]) == [False, True, True]
    assert fx.sum() == 3 * (m.nelz + 1) + 2 * (m.nelz + 1)
    top = [m.node(i, m.nely, k) for k in range(m.nelz + 1) for i in range(m.nelx + 1)]
    assert abs(P.f.sum() + 1.0) <= 1e-12
    assert np.allclose(P.f[[3 * n + 1 for n in top]], -1.0 / len(top))
    # no rigid motion is free: the masked operator is nonsingular
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    K = fem.assemble_masked(KE, np.ones(m.n_elem), edof, m.n_dof, W.fixed_dofs(P.fixed))
    assert np.linalg.eigvalsh(K)[0] > 1e-8


def test_edof_random_shape_and_oracle_pin():
    """The random connectivity keeps the structured table's per-node DOF
    triples, is seeded, and the oracle's gather-contract-scatter K.v on it
    equals the assembled sparse matrix (duplicates summed by the COO
    conversion) times v."""
    from oracle import fem
    m = W.Mesh(5, 4, 3)
    edof = W.edof_random(m, 42)
    assert edof.dtype == np.int32 and edof.shape == (m.n_elem, 24)
    assert edof.min() >= 0 and edof.max() < m.n_dof
    trip = edof.reshape(m.n_elem, 8, 3)
    assert np.all(trip % 3 == np.arange(3)) and np.all(trip[:, :, 1] == trip[:, :, 0] + 1)
    assert np.array_equal(edof, W.edof_random(m, 42))
    assert not np.array_equal(edof, W.edof_random(m, 43))
    E = W.rho_random(m, seed=1)
    v = W.vec_random(m.n_dof, seed=2)
    KE = fem.ke_exact()
    K = fem.assemble(KE, E, edof.astype(np.int64), m.n_dof)
    y = fem.kv_unmasked(KE, E, edof.astype(np.int64), v)
    assert np.abs(K @ v - y).max() <= 1e-13 * np.abs(y).max()

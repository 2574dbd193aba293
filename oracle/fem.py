"""Oracle: mesh indexing, unit element stiffness, SIMP modulus, matrix-free
K.v, sparse assembly, Dirichlet masking and the Jacobi diagonal.

TEST INFRASTRUCTURE ONLY.  This is the plain, slow FP64 CPU restatement of
the method that the CUDA library is checked against.  Only tests, the smoke
check and the CPU-baseline leg of the benchmark may import it; the library
never does, and this package imports nothing from the library.

Paper passages followed (arXiv 2604.18020):
  * Sec. 3.1, Eq. (simp): K(rho) = sum_e B_e^T (rho_min + (1 - rho_min) rho_e^p) KE B_e,
    with B_e the Boolean 24 x n_dof gather of element e and KE the unit-modulus
    element stiffness of a trilinear eight-node hexahedron.
  * Sec. 3.2, Eq. (matfree): w = sum_e B_e^T E_e KE B_e v evaluated element by
    element through the edof table.
  * Sec. 3.6: the Jacobi preconditioner diag(K) accumulated element by element.

Readings where the paper is silent (the same on both sides):
  * element edge h = 1, nodes n = i + (nelx+1)(j + (nely+1)k), DOF 3n + c;
  * local node l = a + 2b + 4c for the corner (i+a, j+b, k+c);
  * the modulus interpolation is E = Emin + (E0 - Emin) rho^p (E0 = 1 gives
    Eq. (simp) with rho_min = Emin);
  * Dirichlet DOFs by masking: (Kv)_free = (K P v)_free with P zeroing the
    fixed DOFs and (Kv)_fixed = v_fixed, so the masked operator is SPD and its
    diagonal is 1 on fixed DOFs.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


# ------------------------------------------------------------------ indexing

def node_index(i, j, k, nelx, nely):
    return i + (nelx + 1) * (j + (nely + 1) * k)


def local_corners():
    """The 8 local corners (a, b, c) in local-node order l = a + 2b + 4c."""
    return [(l & 1, (l >> 1) & 1, (l >> 2) & 1) for l in range(8)]


def edof_table(nelx, nely, nelz):
    """Element -> 24 global DOFs, written out by brute-force enumeration
    (the edof table of Sec. 3.2)."""
    n_elem = nelx * nely * nelz
    edof = np.empty((n_elem, 24), dtype=np.int64)
    for k in range(nelz):
        for j in range(nely):
            for i in range(nelx):
                e = i + nelx * (j + nely * k)
                for l, (a, b, c) in enumerate(local_corners()):
                    n = node_index(i + a, j + b, k + c, nelx, nely)
                    for comp in range(3):
                        edof[e, 3 * l + comp] = 3 * n + comp
    return edof


def edof_table_fast(nelx, nely, nelz):
    """Same table built with array arithmetic (for sizes where the loop is
    slow); tests check it equals :func:`edof_table`."""
    k, j, i = np.meshgrid(np.arange(nelz), np.arange(nely), np.arange(nelx),
                          indexing="ij")
    i, j, k = i.reshape(-1), j.reshape(-1), k.reshape(-1)
    cols = []
    for (a, b, c) in local_corners():
        n = node_index(i + a, j + b, k + c, nelx, nely)
        for comp in range(3):
            cols.append(3 * n + comp)
    return np.stack(cols, axis=1).astype(np.int64)


# ---------------------------------------------------- unit element stiffness

def lame(E, nu):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def elasticity_D(E, nu):
    """Isotropic 6x6 constitutive matrix, Voigt order
    (xx, yy, zz, xy, yz, zx) with engineering shear strains."""
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def ke_gauss(E=1.0, nu=0.3, h=1.0):
    """KE = sum over the 2x2x2 Gauss points of B^T D B det(J) on the
    reference cube [-1, 1]^3 mapped to [0, h]^3 (Sec. 3.1; 2-point Gauss is
    exact for the trilinear element on a cube)."""
    g = 1.0 / np.sqrt(3.0)
    D = elasticity_D(E, nu)
    KE = np.zeros((24, 24))
    corners = local_corners()
    detJ = (h / 2.0) ** 3
    for xi in (-g, g):
        for eta in (-g, g):
            for zeta in (-g, g):
                B = np.zeros((6, 24))
                for l, (a, b, c) in enumerate(corners):
                    sa, sb, sc = 2 * a - 1, 2 * b - 1, 2 * c - 1
                    dN = np.array([
                        sa * (1 + sb * eta) * (1 + sc * zeta) / 8.0,
                        sb * (1 + sa * xi) * (1 + sc * zeta) / 8.0,
                        sc * (1 + sa * xi) * (1 + sb * eta) / 8.0,
                    ]) * (2.0 / h)
                    dx, dy, dz = dN
                    col = 3 * l
                    B[0, col + 0] = dx
                    B[1, col + 1] = dy
                    B[2, col + 2] = dz
                    B[3, col + 0] = dy
                    B[3, col + 1] = dx
                    B[4, col + 1] = dz
                    B[4, col + 2] = dy
                    B[5, col + 0] = dz
                    B[5, col + 2] = dx
                KE += B.T @ D @ B * detJ
    return KE


def ke_exact(E=1.0, nu=0.3, h=1.0):
    """KE by exact integration term by term.

    K[3a+i, 3b+j] = lam * I(a,b; d_i, d_j) + mu * I(a,b; d_j, d_i)
                    + mu * delta_ij * sum_k I(a,b; d_k, d_k),
    I(a,b; d_p, d_q) = int (d_p N_a)(d_q N_b) dV, a product over the three axes
    of 1-D integrals of the linear shape functions phi_0 = 1 - t/h,
    phi_1 = t/h on [0, h]:
      int phi_a phi_b   = h/3 (a = b), h/6 (a != b)
      int phi_a' phi_b' = 1/h (a = b), -1/h (a != b)
      int phi_a' phi_b  = -1/2 (a = 0), +1/2 (a = 1)   (for either b).
    """
    lam, mu = lame(E, nu)

    def one_d(a, b, da, db):
        if not da and not db:
            return h / 3.0 if a == b else h / 6.0
        if da and db:
            return 1.0 / h if a == b else -1.0 / h
        if da:                       # int phi_a' phi_b
            return -0.5 if a == 0 else 0.5
        return -0.5 if b == 0 else 0.5   # int phi_a phi_b'

    corners = local_corners()

    def I(A, B, p, q):
        val = 1.0
        for axis in range(3):
            val *= one_d(A[axis], B[axis], p == axis, q == axis)
        return val

    KE = np.zeros((24, 24))
    for la, A in enumerate(corners):
        for lb, Bc in enumerate(corners):
            grad = sum(I(A, Bc, k, k) for k in range(3))
            for i in range(3):
                for j in range(3):
                    v = lam * I(A, Bc, i, j) + mu * I(A, Bc, j, i)
                    if i == j:
                        v += mu * grad
                    KE[3 * la + i, 3 * lb + j] = v
    return KE


# --------------------------------------------------------------- SIMP modulus

def simp_modulus(rho_phys, penal, E0=1.0, Emin=1e-9):
    """E_e = Emin + (E0 - Emin) rho_e^p (Eq. simp with E0 = 1)."""
    return Emin + (E0 - Emin) * np.asarray(rho_phys, dtype=np.float64) ** penal


# ------------------------------------------------------- operator and masking

def dof_mask(fixed_nodes):
    """Boolean [n_dof] fixed mask from the per-node bit mask (bit c: DOF c)."""
    fixed_nodes = np.asarray(fixed_nodes, dtype=np.uint8)
    return np.stack([(fixed_nodes >> c) & 1 for c in range(3)],
                    axis=1).reshape(-1).astype(bool)


def kv_unmasked(KE, E, edof, v):
    """w = sum_e B_e^T E_e KE B_e v (Eq. matfree): gather, contract, scatter."""
    ue = v[edof]                                   # [n, 24] gather
    fe = (ue @ KE.T) * E[:, None]                  # [n, 24] element products
    return np.bincount(edof.reshape(-1), weights=fe.reshape(-1),
                       minlength=v.shape[0])        # scatter-add


def kv(KE, E, edof, v, fixed_dofs):
    """Masked operator: (Kv)_free = (K P v)_free, (Kv)_fixed = v_fixed."""
    v = np.asarray(v, dtype=np.float64)
    pv = np.where(fixed_dofs, 0.0, v)
    w = kv_unmasked(KE, E, edof, pv)
    return np.where(fixed_dofs, v, w)


def assemble(KE, E, edof, n_dof):
    """Sparse K = sum_e B_e^T E_e KE B_e from element triplets (tiny meshes)."""
    rows = np.repeat(edof, 24, axis=1).reshape(-1)
    cols = np.tile(edof, (1, 24)).reshape(-1)
    vals = (E[:, None, None] * KE[None, :, :]).reshape(-1)
    return sp.coo_matrix((vals, (rows, cols)), shape=(n_dof, n_dof)).tocsr()


def assemble_masked(KE, E, edof, n_dof, fixed_dofs):
    """Dense masked matrix: fixed rows/columns replaced by the identity."""
    K = assemble(KE, E, edof, n_dof).toarray()
    K[fixed_dofs, :] = 0.0
    K[:, fixed_dofs] = 0.0
    K[fixed_dofs, fixed_dofs] = 1.0
    return K


def jacobi_diag(KE, E, edof, fixed_dofs):
    """diag(K) accumulated by one element pass (Sec. 3.6); 1 on fixed DOFs."""
    d = np.zeros(fixed_dofs.shape[0])
    np.add.at(d, edof.reshape(-1), (E[:, None] * np.diag(KE)[None, :]).reshape(-1))
    return np.where(fixed_dofs, 1.0, d)

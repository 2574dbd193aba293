"""Oracle: geometric multigrid for the masked SIMP stiffness operator and CG
preconditioned by its V-cycle.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

Paper passages (arXiv 2604.18020):
  * Sec. 6 ("Path to Geometric Multigrid Integration"): the components a GMG
    preconditioner adds to the matrix-free operator -- a restriction R from
    the fine to the coarse grid, the prolongation P = R^T, a direct solve on
    the coarsest level, and pre/post-smoothing steps that each apply the
    operator once -- all with closed-form stencils on the structured mesh;
  * Sec. 3.5 ("Path forward"): the low-precision K.v as the smoother inside
    a V-cycle, where the coarse-grid correction bounds the spectrum each
    level sees.

The paper names the components only; the textbook V-cycle (Briggs, Henson
and McCormick, "A Multigrid Tutorial", ch. 3 and 5) is written out here with
these readings (the same in the CUDA library):
  * coarsening halves the element count per axis, rounding up: a level with
    n elements along an axis has ceil(n / 2) coarse elements there; a coarse
    element whose 2 x 2 x 2 children are not all present simply has fewer;
  * P is trilinear interpolation from the coarse nodes (fine coordinates 2I)
    to the fine nodes: per axis, an even fine node 2I takes coarse node I,
    an odd one 2I + 1 the mean of coarse nodes I and I + 1 (which exists even
    when 2I + 2 lies past the fine mesh); the 3-D operator is the tensor
    product, applied to each displacement component;
  * Dirichlet DOFs: a coarse DOF is fixed when the fine DOF at the same
    position is; with M_f, M_c the 0/1 diagonals of the free DOFs,
    Phat = M_f P M_c, and the coarse operator is the Galerkin product
    A_c = Phat^T A Phat plus the identity on the fixed coarse DOFs (the same
    masking as the fine operator, so every level is SPD);
  * the coarsening stops at the first level with at most coarse_max_dofs
    DOFs or at max_levels levels; that level is solved exactly;
  * smoother: l1-Jacobi (Baker, Falgout, Kolev and Yang, SIAM J. Sci. Comput.
    2011), x <- x + omega D1^-1 (b - A x), with the l1 row sums taken over
    the unassembled element matrices, D1_ii = sum_E sum_j |(A_E)_ij| (1 on
    fixed DOFs), which needs no assembled matrix; D1_ii >= sum_j |A_ij|, so
    lambda_max(D1^-1 A) <= 1 and the sweep converges for 0 < omega < 2
    without a spectral estimate; nu_pre sweeps from x = 0 before, nu_post
    after the coarse correction;
  * the element matrices of a level: E_e D_e KE D_e on the finest (D_e the
    0/1 diagonal of the element's free DOFs); on a coarse level, the
    Galerkin product of coarse element E alone, Phat_E^T (sum over E's
    children c of B_c^T A_c B_c) Phat_E with Phat_E the columns of Phat at
    E's DOFs -- their assembly is the Galerkin operator above;
  * optional Chebyshev smoother (Adams, Brezina, Hu and Tuminaro, J. Comput.
    Phys. 2003): each sweep is the degree-k Chebyshev iteration for
    D1^-1 A x = D1^-1 b on the interval [lmax / 30, lmax] with lmax = 1, the
    l1 bound (so no eigenvalue estimate is needed); from x the error is
    multiplied by T_k((theta - D1^-1 A) / delta) / T_k(theta / delta),
    theta and delta the interval's centre and half width;
  * the coarsest inverse comes from an FP64 Cholesky factorisation; when a
    pivot falls below 1e-5 of its diagonal entry the operator is taken as
    rank deficient (a consistent singular problem such as the MBB preset,
    whose z translation and one rotation stay free) and the inverse is that
    of A_c + 1e-6 diag(A_c): the V-cycle stays SPD and CG still solves the
    consistent system (the load is orthogonal to the null space); the CUDA
    library, whose coarsest operator comes from FP32-rounded element
    matrices, raises the shift tenfold (up to 1e-2) until its factorisation
    succeeds, which this exact FP64 operator never needs;
  * the outer CG takes z = V(r) with the Polak-Ribiere form of beta
    (flexible CG), so a preconditioner applied in lower precision keeps the
    iteration convergent.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import fem


def coarse_dims(n):
    return tuple((a + 1) // 2 for a in n)


def level_dims(nelx, nely, nelz, max_levels=8, coarse_max_dofs=200):
    """Element counts (nx, ny, nz) of every level, finest first."""
    dims = [(nelx, nely, nelz)]
    while len(dims) < max_levels:
        nx, ny, nz = dims[-1]
        if 3 * (nx + 1) * (ny + 1) * (nz + 1) <= coarse_max_dofs or (nx, ny, nz) == (1, 1, 1):
            break
        dims.append(coarse_dims(dims[-1]))
    return dims


def prolong_1d(n):
    """(n + 1) x (ceil(n/2) + 1) interpolation along one axis."""
    m = (n + 1) // 2
    rows, cols, vals = [], [], []
    for i in range(n + 1):
        if i % 2 == 0:
            rows.append(i); cols.append(i // 2); vals.append(1.0)
        else:
            rows += [i, i]; cols += [(i - 1) // 2, (i + 1) // 2]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n + 1, m + 1))


def prolong_nodes(n):
    """Nodal trilinear interpolation, x fastest (node = i + (nx+1)(j + (ny+1)k))."""
    nx, ny, nz = n
    return sp.kron(prolong_1d(nz), sp.kron(prolong_1d(ny), prolong_1d(nx))).tocsr()


def prolong_dofs(n):
    return sp.kron(prolong_nodes(n), sp.identity(3)).tocsr()


def coarse_fixed(n, fixed_dofs):
    """Fixed-DOF mask of the coarse level: coarse node (I, J, K) takes the
    mask of the fine node (2I, 2J, 2K) where that node exists."""
    nx, ny, nz = n
    mx, my, mz = coarse_dims(n)
    fd = np.asarray(fixed_dofs, bool).reshape(nz + 1, ny + 1, nx + 1, 3)
    out = np.zeros((mz + 1, my + 1, mx + 1, 3), bool)
    I = np.arange(mx + 1); J = np.arange(my + 1); K = np.arange(mz + 1)
    ok_i, ok_j, ok_k = 2 * I <= nx, 2 * J <= ny, 2 * K <= nz
    sub = fd[np.ix_(2 * K[ok_k], 2 * J[ok_j], 2 * I[ok_i])]
    out[np.ix_(K[ok_k], J[ok_j], I[ok_i])] = sub
    return out.reshape(-1)


def masked_operator(KE, E, edof, n_dof, fixed_dofs):
    """Sparse masked fine operator: M K M + diag(fixed)."""
    K = fem.assemble(KE, E, edof, n_dof)
    m = sp.diags((~np.asarray(fixed_dofs, bool)).astype(float))
    return (m @ K @ m + sp.diags(np.asarray(fixed_dofs, bool).astype(float))).tocsr()


@dataclass
class Level:
    dims: tuple
    A: sp.csr_matrix          # masked operator of this level
    fixed: np.ndarray         # bool [n_dof]
    Ke: np.ndarray            # [n_elem, 24, 24] element matrices (masked)
    d1inv: np.ndarray         # 1 / (element-wise l1 row sums), 1 on fixed DOFs
    P: sp.csr_matrix | None   # Phat from the next coarser level to this one


def fine_element_matrices(KE, E, edof, fixed_dofs):
    free = (~np.asarray(fixed_dofs, bool)[edof]).astype(float)          # [n, 24]
    return E[:, None, None] * KE[None] * free[:, :, None] * free[:, None, :]


def coarse_element_matrices(n, Ke, Phat):
    """Galerkin matrix of each coarse element from its children's matrices."""
    nx, ny, nz = n
    mx, my, mz = coarse_dims(n)
    edof_f = fem.edof_table_fast(nx, ny, nz)
    edof_c = fem.edof_table_fast(mx, my, mz)
    out = np.zeros((mx * my * mz, 24, 24))
    for K in range(mz):
        for J in range(my):
            for I in range(mx):
                kids = [i + nx * (j + ny * k)
                        for k in (2 * K, 2 * K + 1) for j in (2 * J, 2 * J + 1)
                        for i in (2 * I, 2 * I + 1) if i < nx and j < ny and k < nz]
                F = np.unique(edof_f[kids].reshape(-1))
                pos = {d: t for t, d in enumerate(F)}
                Kloc = np.zeros((len(F), len(F)))
                for c in kids:
                    ix = [pos[d] for d in edof_f[c]]
                    Kloc[np.ix_(ix, ix)] += Ke[c]
                e = I + mx * (J + my * K)
                Ploc = Phat[F][:, edof_c[e]].toarray()
                out[e] = Ploc.T @ Kloc @ Ploc
    return out


def l1_inverse(Ke, edof, fixed_dofs, n_dof):
    rows = np.abs(Ke).sum(axis=2)                                        # [n, 24]
    d1 = np.bincount(edof.reshape(-1), weights=rows.reshape(-1), minlength=n_dof)
    d1[np.asarray(fixed_dofs, bool)] = 1.0
    return 1.0 / d1


@dataclass
class Hierarchy:
    levels: list
    coarse_inv: np.ndarray    # dense inverse of the coarsest operator
    omega: float
    nu_pre: int
    nu_post: int
    cheb_degree: int = 0      # 0: l1-Jacobi sweeps; k >= 1: Chebyshev sweeps of degree k


CHEB_RATIO = 30.0            # lmax / lmin of the Chebyshev interval, lmax = 1


def build(KE, E, nelx, nely, nelz, fixed_dofs, max_levels=8, coarse_max_dofs=200, omega=1.0,
          nu_pre=2, nu_post=2, cheb_degree=0):
    dims = level_dims(nelx, nely, nelz, max_levels, coarse_max_dofs)
    edof = fem.edof_table_fast(nelx, nely, nelz)
    n_dof = 3 * (nelx + 1) * (nely + 1) * (nelz + 1)
    fixed = np.asarray(fixed_dofs, bool)
    A = masked_operator(KE, E, edof, n_dof, fixed)
    Ke = fine_element_matrices(KE, E, edof, fixed)
    levels = []
    for li, n in enumerate(dims):
        edof_l = fem.edof_table_fast(*n)
        lev = Level(n, A, fixed, Ke, l1_inverse(Ke, edof_l, fixed, A.shape[0]), None)
        levels.append(lev)
        if li + 1 < len(dims):
            cf = coarse_fixed(n, fixed)
            Ph = sp.diags((~fixed).astype(float)) @ prolong_dofs(n) @ sp.diags((~cf).astype(float))
            lev.P = Ph.tocsr()
            A = (lev.P.T @ A @ lev.P + sp.diags(cf.astype(float))).tocsr()
            Ke = coarse_element_matrices(n, Ke, lev.P)
            fixed = cf
    coarse_inv = coarsest_inverse(levels[-1].A.toarray())
    return Hierarchy(levels, coarse_inv, omega, nu_pre, nu_post, cheb_degree)


PIVOT_RTOL = 1e-5        # pivot / diagonal below this: rank deficient
SHIFT = 1e-6             # relative diagonal shift of a rank-deficient coarsest operator


def cholesky_pivots_ok(A):
    """Plain Cholesky; False when a pivot falls below PIVOT_RTOL of its
    diagonal entry."""
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        s = A[j, j] - L[j, :j] @ L[j, :j]
        if not (s > PIVOT_RTOL * A[j, j]):
            return False
        L[j, j] = np.sqrt(s)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return True


def coarsest_inverse(Ac):
    if not cholesky_pivots_ok(Ac):
        Ac = Ac + SHIFT * np.diag(np.diag(Ac))
    return np.linalg.inv(Ac)


def smooth(lev, x, b, omega, sweeps):
    for _ in range(sweeps):
        x = x + omega * lev.d1inv * (b - lev.A @ x)
    return x


def cheb_coefficients(degree, ratio=CHEB_RATIO):
    """(1/theta, [(c1, c2)] for steps 1 .. degree-1) of the three-term
    recurrence d_k = c1 d_(k-1) + c2 r_k on [1/ratio, 1]."""
    lmax, lmin = 1.0, 1.0 / ratio
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    steps = []
    for _ in range(degree - 1):
        rho_new = 1.0 / (2.0 * sigma - rho)
        steps.append((rho_new * rho, 2.0 * rho_new / delta))
        rho = rho_new
    return 1.0 / theta, steps


def cheb_smooth(lev, x, b, degree, sweeps):
    inv_theta, steps = cheb_coefficients(degree)
    for _ in range(sweeps):
        r = lev.d1inv * (b - lev.A @ x)
        d = inv_theta * r
        x = x + d
        for c1, c2 in steps:
            r = r - lev.d1inv * (lev.A @ d)
            d = c1 * d + c2 * r
            x = x + d
    return x


def level_smooth(H, lev, x, b, sweeps):
    if H.cheb_degree:
        return cheb_smooth(lev, x, b, H.cheb_degree, sweeps)
    return smooth(lev, x, b, H.omega, sweeps)


def vcycle(H, b, li=0):
    lev = H.levels[li]
    if li == len(H.levels) - 1:
        return H.coarse_inv @ b
    x = level_smooth(H, lev, np.zeros_like(b), b, H.nu_pre)
    r = b - lev.A @ x
    xc = vcycle(H, lev.P.T @ r, li + 1)
    x = x + lev.P @ xc
    return level_smooth(H, lev, x, b, H.nu_post)


@dataclass
class GmgStats:
    iterations: int
    rel_residual: float
    true_rel_residual: float
    converged: bool


def pcg(H, apply_K, f, u0, rtol=1e-8, maxit=1000, precond=None):
    """CG preconditioned by the V-cycle (or by precond(r) when given), beta in
    the Polak-Ribiere form z_k+1 . (r_k+1 - r_k) / (z_k . r_k)."""
    M = precond if precond is not None else (lambda r: vcycle(H, r))
    f = np.asarray(f, dtype=np.float64)
    u = np.array(u0, dtype=np.float64, copy=True)
    fnorm = np.linalg.norm(f)
    if fnorm == 0.0:
        return np.zeros_like(f), GmgStats(0, 0.0, 0.0, True)
    r = f - apply_K(u)
    z = M(r)
    p = z.copy()
    rz = r @ z
    it = 0
    rel = np.linalg.norm(r) / fnorm
    while rel > rtol and it < maxit:
        q = apply_K(p)
        alpha = rz / (p @ q)
        u += alpha * p
        r_old = r
        r = r - alpha * q
        it += 1
        rel = np.linalg.norm(r) / fnorm
        if rel <= rtol:
            break
        z = M(r)
        rz_new = r @ z
        beta = (rz_new - z @ r_old) / rz
        p = z + beta * p
        rz = rz_new
    true_rel = np.linalg.norm(f - apply_K(u)) / fnorm
    return u, GmgStats(it, rel, true_rel, rel <= rtol)

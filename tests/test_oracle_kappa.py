"""Pins of the oracle's condition-number estimator (no GPU): the extremal
eigenvalues of the assembled K_ff from LAPACK on tiny meshes, the one-sided
(conservative) bounds of the capped iterations, and scale invariance."""
import numpy as np
import pytest

from oracle import fem, kappa
from paper_2604_18020_gb300 import workloads as W


def _system(shape, seed, face="x0", uniform=None):
    m = W.Mesh(*shape)
    edof = fem.edof_table_fast(*shape)
    KE = fem.ke_exact()
    fixed = W.fixed_face(m, face)
    fd = fem.dof_mask(fixed)
    rho = np.full(m.n_elem, uniform) if uniform is not None else \
        W.rho_random(m, seed=seed, lo=0.1, hi=1.0)
    E = fem.simp_modulus(rho, 3.0)
    return m, edof, KE, fd, E


def _exact(KE, E, edof, n_dof, fd):
    K = fem.assemble(KE, E, edof, n_dof).toarray()
    free = ~fd
    ev = np.linalg.eigvalsh(K[np.ix_(free, free)])
    return ev[0], ev[-1]


@pytest.mark.parametrize("shape,face", [((3, 2, 2), "x0"), ((4, 2, 3), "z0"), ((2, 2, 2), "x0")])
def test_converged_iterations_match_lapack(shape, face):
    m, edof, KE, fd, E = _system(shape, seed=3, face=face)
    lmin, lmax = _exact(KE, E, edof, m.n_dof, fd)
    apply_K = lambda v: fem.kv(KE, E, edof, v, fd)
    d = fem.jacobi_diag(KE, E, edof, fd)
    vp = W.vec_random(m.n_dof, seed=42)
    vi = W.vec_random(m.n_dof, seed=123)
    r = kappa.estimate(apply_K, d, fd, vp, vi, power_maxit=20000, power_tol=1e-14,
                       inverse_maxit=2000, inverse_tol=1e-14, inner_rtol=1e-13)
    assert abs(r.lambda_max - lmax) <= 1e-8 * lmax
    assert abs(r.lambda_min - lmin) <= 1e-8 * lmin
    assert abs(r.kappa - lmax / lmin) <= 1e-7 * (lmax / lmin)


def test_capped_estimates_are_conservative():
    """With the paper's caps the Rayleigh quotients bound the spectrum from
    inside: lambda_max from below, lambda_min from above, so kappa is never
    overestimated."""
    m, edof, KE, fd, E = _system((6, 3, 3), seed=5)
    lmin, lmax = _exact(KE, E, edof, m.n_dof, fd)
    apply_K = lambda v: fem.kv(KE, E, edof, v, fd)
    d = fem.jacobi_diag(KE, E, edof, fd)
    r = kappa.estimate(apply_K, d, fd, W.vec_random(m.n_dof, seed=42),
                       W.vec_random(m.n_dof, seed=123))
    assert r.power_steps <= 50
    assert r.lambda_max <= lmax * (1 + 1e-12)
    assert r.lambda_min >= lmin * (1 - 1e-7)
    assert r.kappa <= (lmax / lmin) * (1 + 1e-6)
    assert r.kappa >= 0.5 * (lmax / lmin)      # and it is not far off either


def test_start_vectors_are_confined_to_free_dofs():
    """Identity rows of the masked operator never enter: an eigenvalue of 1
    on the fixed DOFs above the free spectrum does not become lambda_max."""
    m, edof, KE, fd, E = _system((3, 2, 2), seed=4, uniform=0.05)   # E ~ 1.25e-4
    lmin, lmax = _exact(KE, E, edof, m.n_dof, fd)
    assert lmax < 1.0                                                # 1 would dominate
    apply_K = lambda v: fem.kv(KE, E, edof, v, fd)
    d = fem.jacobi_diag(KE, E, edof, fd)
    r = kappa.estimate(apply_K, d, fd, W.vec_random(m.n_dof, seed=42),
                       W.vec_random(m.n_dof, seed=123), power_maxit=5000, power_tol=1e-13)
    assert abs(r.lambda_max - lmax) <= 1e-6 * lmax


def test_uniform_scaling_and_penalty_invariance():
    """kappa is invariant under a uniform scaling of the moduli, so at
    uniform density it does not depend on the penalty (the paper's p = 3 vs 5
    remark)."""
    m, edof, KE, fd, _ = _system((4, 2, 2), seed=6)
    d_of = lambda E: fem.jacobi_diag(KE, E, edof, fd)
    res = []
    for penal in (3.0, 5.0):
        E = fem.simp_modulus(np.full(m.n_elem, 0.5), penal)
        apply_K = lambda v, E=E: fem.kv(KE, E, edof, v, fd)
        res.append(kappa.estimate(apply_K, d_of(E), fd, W.vec_random(m.n_dof, seed=42),
                                  W.vec_random(m.n_dof, seed=123)))
    assert res[0].power_steps == res[1].power_steps
    assert abs(res[0].kappa - res[1].kappa) <= 1e-6 * res[0].kappa

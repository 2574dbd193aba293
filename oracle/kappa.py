"""Oracle: matrix-free estimate of the condition number kappa(K) of the
stiffness matrix on the free DOFs.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

Paper passages: Sec. 3.5 ("Condition number of the SIMP stiffness matrix")
and Sec. 5 (the kappa results): lambda_max by power iteration, lambda_min by
inverse iteration, both through matrix-free K.v products only, from fixed
seeded start vectors; power iteration stops when successive eigenvalue
estimates change by less than a relative 1e-6 (or after 50 steps); inverse
iteration stops when the reciprocal Rayleigh estimate changes by less than a
relative 1e-4, each of its inner solves running CG to a relative (and
absolute) residual of 1e-8 with a 2000-iteration cap.  kappa = lambda_max /
lambda_min.

Readings (the same on both sides):
  * K is the stiffness matrix restricted to the free DOFs (K_ff).  With the
    masked operator of oracle/fem.py (identity rows on fixed DOFs) this is
    the operator on vectors that vanish on the fixed DOFs; the start vectors
    are zeroed there, and the masked K.v and the solves keep them zero, so
    the identity rows never enter the spectrum.
  * Each eigenvalue estimate is a Rayleigh quotient of the current unit
    vector: power iteration lambda_k = v.Kv, v <- Kv / ||Kv||; inverse
    iteration mu_k = v.K^-1 v (the reciprocal estimate), v <- K^-1 v /
    ||K^-1 v||, lambda_min = 1 / mu.
  * The inner solves use the Jacobi-preconditioned CG of oracle/solve.py
    (the solver of Sec. 3.6) from a zero start; the paper's SciPy CG is
    unpreconditioned.  Converged, both give the same K^-1 v.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import solve


@dataclass
class KappaResult:
    lambda_max: float
    lambda_min: float
    kappa: float
    power_steps: int
    inverse_steps: int
    inner_iterations: int      # CG iterations of all inverse-iteration solves
    inner_capped: int          # inner solves that hit the cap


def power_iteration(apply_K, v0, maxit=50, tol=1e-6):
    """Largest eigenvalue of K by power iteration; returns (lambda, steps, v)."""
    v = np.array(v0, dtype=np.float64, copy=True)
    v /= np.linalg.norm(v)
    lam_prev = None
    lam = 0.0
    steps = 0
    for steps in range(1, maxit + 1):
        w = apply_K(v)
        lam = float(v @ w)
        v = w / np.linalg.norm(w)
        if lam_prev is not None and abs(lam - lam_prev) <= tol * abs(lam):
            break
        lam_prev = lam
    return lam, steps, v


def inverse_iteration(apply_K, diag, v0, maxit=50, tol=1e-4, inner_rtol=1e-8,
                      inner_maxit=2000):
    """Smallest eigenvalue of K by inverse iteration with CG inner solves;
    returns (lambda_min, steps, v, inner iterations, capped solves)."""
    v = np.array(v0, dtype=np.float64, copy=True)
    v /= np.linalg.norm(v)
    mu_prev = None
    mu = 0.0
    steps = inner = capped = 0
    for steps in range(1, maxit + 1):
        x, st = solve.pcg(apply_K, diag, v, np.zeros_like(v), inner_rtol, inner_maxit)
        inner += st.iterations
        capped += 0 if st.converged else 1
        mu = float(v @ x)
        v = x / np.linalg.norm(x)
        if mu_prev is not None and abs(mu - mu_prev) <= tol * abs(mu):
            break
        mu_prev = mu
    return 1.0 / mu, steps, v, inner, capped


def estimate(apply_K, diag, fixed_dofs, v_power, v_inverse, power_maxit=50, power_tol=1e-6,
             inverse_maxit=50, inverse_tol=1e-4, inner_rtol=1e-8, inner_maxit=2000):
    """kappa(K_ff) from the two seeded start vectors (zeroed on fixed DOFs)."""
    vp = np.where(fixed_dofs, 0.0, v_power)
    vi = np.where(fixed_dofs, 0.0, v_inverse)
    lmax, ps, _ = power_iteration(apply_K, vp, power_maxit, power_tol)
    lmin, its, _, inner, capped = inverse_iteration(apply_K, diag, vi, inverse_maxit, inverse_tol,
                                                    inner_rtol, inner_maxit)
    return KappaResult(lmax, lmin, lmax / lmin, ps, its, inner, capped)

"""Oracle: Jacobi-preconditioned conjugate gradients and a dense direct solve.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

Paper passage: Sec. 3.6 -- K u = f is solved by CG with the Jacobi
preconditioner M = diag(K); the previous displacement is the initial guess
(warm start); iteration stops when the unpreconditioned relative residual
||r_k|| / ||f|| reaches the tolerance or the iteration cap is hit.

The iteration is the textbook Hestenes-Stiefel form with a left Jacobi
preconditioner, in this order:
  r = f - K u0; z = r / d; p = z; rz = r.z
  repeat: q = K p; alpha = rz / (p.q); u += alpha p; r -= alpha q;
          stop if ||r|| <= rtol ||f|| or the cap is reached;
          z = r / d; rz' = r.z; p = z + (rz'/rz) p; rz = rz'
The residual tested is the recursively updated r (unpreconditioned).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class SolveStats:
    iterations: int
    rel_residual: float        # recursive ||r|| / ||f|| at exit
    true_rel_residual: float   # ||f - K u|| / ||f|| recomputed at exit
    converged: bool


def pcg(apply_K, diag, f, u0, rtol=1e-8, maxit=10000):
    f = np.asarray(f, dtype=np.float64)
    u = np.array(u0, dtype=np.float64, copy=True)
    fnorm = np.linalg.norm(f)
    if fnorm == 0.0:
        return np.zeros_like(f), SolveStats(0, 0.0, 0.0, True)
    r = f - apply_K(u)
    it = 0
    rn = np.linalg.norm(r)
    if rn <= rtol * fnorm:
        return u, SolveStats(0, rn / fnorm, rn / fnorm, True)
    z = r / diag
    p = z.copy()
    rz = r @ z
    while True:
        q = apply_K(p)
        alpha = rz / (p @ q)
        u += alpha * p
        r -= alpha * q
        it += 1
        rn = np.linalg.norm(r)
        if rn <= rtol * fnorm or it >= maxit:
            break
        z = r / diag
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    true_rn = np.linalg.norm(f - apply_K(u))
    return u, SolveStats(it, rn / fnorm, true_rn / fnorm, rn <= rtol * fnorm)


def dense_solve(K, f):
    """Direct solve of the (small, dense, masked) system; LAPACK via numpy."""
    return np.linalg.solve(K, f)

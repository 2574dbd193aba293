"""Oracle: element compliance and sensitivities, the OC bisection update and
the SIMP loop.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

Paper passages (arXiv 2604.18020):
  * Sec. 3.1, Eq. (tomin): minimise f^T u subject to K(rho) u = f and
    mean(rho) = V_f;  Eq. (simp) for the modulus;  analytic sensitivities and
    the Optimality-Criteria update with bisection on the volume multiplier;
    the grayness g = (4/n) sum rho (1 - rho).
  * Sec. 3.6: warm start -- the previous displacement seeds the next solve.
  * Sec. 4.1: uniform initial density rho = V_f.

Readings where the paper is silent (identical in the CUDA library):
  * compliance c = sum_e E_e u_e^T KE u_e (equal to f^T u at convergence);
  * dc/drho_phys_e = -p rho_phys_e^(p-1) (E0 - Emin) u_e^T KE u_e, chained to
    the design field through the transpose of the density filter;
  * no Heaviside projection (rho_phys = rho_bar);
  * the volume constraint acts on the design field rho (Eq. tomin literally),
    dV/drho_e = 1/n;
  * OC: B_e = max(0, -dc_e) / (lambda dV_e); the candidate is
    rho * sqrt(B_e) clipped to [max(0, rho - m), min(1, rho + m)], m = move
    (a NaN candidate, 0 * inf at an underflowed lambda, is clipped to the bound);
    lambda is bisected on [0, 1e9], raising the lower end while
    sum(rho_new) > V_f n, until (l2 - l1) / (l1 + l2) <= 1e-10, or until the
    midpoint no longer lies strictly inside the bracket (the bracket cannot
    shrink further in floating point: this happens when even the smallest
    lambda gives too little volume and lambda underflows), or after 4096
    steps; the returned field is the candidate of the last midpoint;
  * grayness is evaluated on the physical field rho_phys.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import fem, filter as cone, solve


def element_energy(KE, edof, u):
    """ce_e = u_e^T KE u_e."""
    ue = u[edof]
    return np.einsum("ei,ij,ej->e", ue, KE, ue)


def compliance_sens(KE, edof, u, rho_phys, penal, E0=1.0, Emin=1e-9):
    """(c, dc/drho_phys) for the current displacement."""
    ce = element_energy(KE, edof, u)
    E = fem.simp_modulus(rho_phys, penal, E0, Emin)
    c = float(np.sum(E * ce))
    dc = -penal * np.asarray(rho_phys) ** (penal - 1.0) * (E0 - Emin) * ce
    return c, dc


def oc_update(rho, dc, volfrac, move=0.2, l1=0.0, l2=1e9, tol=1e-10):
    """Optimality-Criteria update with bisection on the volume multiplier."""
    rho = np.asarray(rho, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        return _oc_bisect(rho, dc, volfrac, move, l1, l2, tol)


def _oc_bisect(rho, dc, volfrac, move, l1, l2, tol):
    n = rho.size
    dv = 1.0 / n
    target = volfrac * n
    neg = np.maximum(0.0, -np.asarray(dc, dtype=np.float64))
    lo = np.maximum(0.0, rho - move)
    hi = np.minimum(1.0, rho + move)
    rho_new = rho.copy()
    steps = 0
    while l1 + l2 > 0.0 and (l2 - l1) / (l1 + l2) > tol and steps < 4096:
        lmid = 0.5 * (l1 + l2)
        if not (l1 < lmid < l2):
            break
        cand = rho * np.sqrt(neg / (lmid * dv))
        rho_new = np.fmax(lo, np.fmin(hi, cand))   # a NaN candidate (0 * inf) is clipped away
        if np.sum(rho_new) > target:
            l1 = lmid
        else:
            l2 = lmid
        steps += 1
    return rho_new, {"lambda": 0.5 * (l1 + l2), "steps": steps,
                     "change": float(np.max(np.abs(rho_new - rho)))}


def grayness(rho):
    rho = np.asarray(rho, dtype=np.float64)
    return float(4.0 * np.mean(rho * (1.0 - rho)))


@dataclass
class SimpHistory:
    compliance: list = field(default_factory=list)
    change: list = field(default_factory=list)
    grayness: list = field(default_factory=list)
    cg_iterations: list = field(default_factory=list)
    volume: list = field(default_factory=list)


def simp(nelx, nely, nelz, f, fixed_nodes, volfrac, rmin, n_iter, penal=3.0,
         E0=1.0, Emin=1e-9, nu=0.3, move=0.2, rtol=1e-8, maxit=10000,
         rho0=None):
    """The SIMP loop: filter -> modulus -> Jacobi-PCG (warm start) ->
    compliance and sensitivities -> filter transpose -> OC, n_iter times."""
    KE = fem.ke_exact(1.0, nu)
    edof = fem.edof_table_fast(nelx, nely, nelz)
    fixed = fem.dof_mask(fixed_nodes)
    n = nelx * nely * nelz
    rho = np.full(n, float(volfrac)) if rho0 is None else np.array(rho0, float)
    u = np.zeros_like(f)
    hist = SimpHistory()
    for _ in range(n_iter):
        rho_phys = cone.filter_fwd(rho, nelx, nely, nelz, rmin)
        E = fem.simp_modulus(rho_phys, penal, E0, Emin)
        d = fem.jacobi_diag(KE, E, edof, fixed)
        u, st = solve.pcg(lambda v: fem.kv(KE, E, edof, v, fixed), d, f, u,
                          rtol, maxit)
        c, dc_phys = compliance_sens(KE, edof, u, rho_phys, penal, E0, Emin)
        dc = cone.filter_T(dc_phys, nelx, nely, nelz, rmin)
        rho_new, info = oc_update(rho, dc, volfrac, move)
        hist.compliance.append(c)
        hist.change.append(info["change"])
        hist.grayness.append(grayness(rho_phys))
        hist.cg_iterations.append(st.iterations)
        hist.volume.append(float(np.mean(rho_new)))
        rho = rho_new
    return rho, u, hist

"""Oracle: the three-field SIMP step (density filter, smoothed Heaviside
projection) and the paper's 120-iteration continuation protocol with
restarts and the selected-iterate rule.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

Paper passages (arXiv 2604.18020):
  * Sec. 3.1: rho_phys = (tanh(beta eta) + tanh(beta (rho_bar - eta))) /
    (tanh(beta eta) + tanh(beta (1 - eta))), eta = 0.5, applied to the
    filtered field rho_bar; analytic sensitivities; OC with bisection.
  * Sec. 4.1 (benchmark setup): the four-phase schedule of (penalty p,
    projection beta, OC move m) over 120 iterations -- 1-15: (1.5, 1, 0.20);
    16-40: (3.5, 4, 0.15), r_min reduced toward 1.35; 41-65: (4.5, 16, 0.08),
    toward 1.25; 66-120: (4.5, 32, 0.05), toward 1.20 -- a restart from the
    selected design when the compliance exceeds 1.12 times the selected
    compliance, and the selected iterate: the lowest compliance among
    iterates with p >= 3 and grayness g < 0.25.

Readings (the same in the CUDA library):
  * the projected field is clipped to [0, 1] (rounding only);
  * the sensitivity chain is dc/drho = F^T (dc/drho_phys * drho_phys/drho_bar),
    drho_phys/drho_bar = beta (1 - tanh^2(beta (rho_bar - eta))) /
    (tanh(beta eta) + tanh(beta (1 - eta)));
  * "reducing r_min toward r" is a linear ramp over the phase: at the k-th of
    the phase's n iterations r_min = r0 + (r - r0) k / n, with r0 the value
    the previous phase ended at (the problem's r_min in phase 1), so the
    target is reached at the phase's last iteration;
  * the volume constraint stays on the design field rho (Eq. tomin), and
    grayness is evaluated on rho_phys, as on the plain path;
  * iteration i's compliance belongs to the design rho_i that entered it; the
    selected design is that rho_i; a restart replaces the next design by the
    selected one (the displacement keeps its warm start, unless every solve
    starts cold, as in the paper's hard-problem runs); the restart test
    comes before the selection update, against the selection so far.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import fem, filter as cone, simp, solve

# (first iteration, last iteration, p, beta, move, r_min target or None)
SCHEDULE_120 = [
    (1, 15, 1.5, 1.0, 0.20, None),
    (16, 40, 3.5, 4.0, 0.15, 1.35),
    (41, 65, 4.5, 16.0, 0.08, 1.25),
    (66, 120, 4.5, 32.0, 0.05, 1.20),
]
RESTART_FACTOR = 1.12
SELECT_MIN_PENAL = 3.0
SELECT_MAX_GRAY = 0.25


def heaviside(rho_bar, beta, eta=0.5):
    """Smoothed Heaviside projection of Sec. 3.1, clipped to [0, 1] (at
    rho_bar = 0 the numerator tanh(beta eta) - tanh(beta eta) can round a few
    ulps below zero, where rho^(p-1) is undefined for a fractional p)."""
    den = np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta))
    h = (np.tanh(beta * eta) + np.tanh(beta * (np.asarray(rho_bar) - eta))) / den
    return np.clip(h, 0.0, 1.0)


def heaviside_deriv(rho_bar, beta, eta=0.5):
    """d rho_phys / d rho_bar."""
    den = np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta))
    t = np.tanh(beta * (np.asarray(rho_bar) - eta))
    return beta * (1.0 - t * t) / den


def phase_params(it, rmin0, schedule=SCHEDULE_120):
    """(p, beta, move, r_min) of 1-based iteration it."""
    r_start = rmin0
    for first, last, penal, beta, move, r_target in schedule:
        if r_target is None:
            r_end = r_start
        else:
            r_end = r_target
        if it <= last:
            if r_target is None:
                return penal, beta, move, r_start
            k, n = it - first + 1, last - first + 1
            return penal, beta, move, r_start + (r_end - r_start) * k / n
        r_start = r_end
    first, last, penal, beta, move, _ = schedule[-1]
    return penal, beta, move, r_start


def step(KE, edof, fixed, nelx, nely, nelz, f, rho, u, volfrac, penal, beta, move, rmin,
         eta=0.5, E0=1.0, Emin=1e-9, rtol=1e-8, maxit=10000):
    """One three-field SIMP iteration; returns (rho_new, u, c, rho_phys, cg its)."""
    rho_bar = cone.filter_fwd(rho, nelx, nely, nelz, rmin)
    rho_phys = heaviside(rho_bar, beta, eta)
    E = fem.simp_modulus(rho_phys, penal, E0, Emin)
    d = fem.jacobi_diag(KE, E, edof, fixed)
    u, st = solve.pcg(lambda v: fem.kv(KE, E, edof, v, fixed), d, f, u, rtol, maxit)
    c, dc_phys = simp.compliance_sens(KE, edof, u, rho_phys, penal, E0, Emin)
    dc_bar = dc_phys * heaviside_deriv(rho_bar, beta, eta)
    dc = cone.filter_T(dc_bar, nelx, nely, nelz, rmin)
    rho_new, _ = simp.oc_update(rho, dc, volfrac, move)
    return rho_new, u, c, rho_phys, st.iterations


@dataclass
class ProtocolResult:
    compliance: list = field(default_factory=list)
    grayness: list = field(default_factory=list)
    restarted: list = field(default_factory=list)      # iterations after which a restart happened
    selected_iteration: int = 0                         # 1-based, 0 = none eligible
    selected_compliance: float = float("nan")
    selected_rho: np.ndarray | None = None


def select_and_restart(c, penal, gray, sel_c):
    """The per-iteration decisions: (restart?, becomes selected?)."""
    restart = sel_c is not None and c > RESTART_FACTOR * sel_c
    eligible = penal >= SELECT_MIN_PENAL and gray < SELECT_MAX_GRAY
    better = eligible and (sel_c is None or c < sel_c)
    return restart, better


def protocol(nelx, nely, nelz, f, fixed_nodes, volfrac, rmin0, n_iter=120, nu=0.3,
             schedule=SCHEDULE_120, rtol=1e-8, maxit=10000, cold_start=False):
    KE = fem.ke_exact(1.0, nu)
    edof = fem.edof_table_fast(nelx, nely, nelz)
    fixed = fem.dof_mask(fixed_nodes)
    rho = np.full(nelx * nely * nelz, float(volfrac))
    u = np.zeros_like(f)
    res = ProtocolResult()
    sel_c = None
    for it in range(1, n_iter + 1):
        penal, beta, move, rmin = phase_params(it, rmin0, schedule)
        if cold_start:
            u = np.zeros_like(f)
        rho_new, u, c, rho_phys, _ = step(KE, edof, fixed, nelx, nely, nelz, f, rho, u, volfrac,
                                          penal, beta, move, rmin, rtol=rtol, maxit=maxit)
        gray = simp.grayness(rho_phys)
        res.compliance.append(c)
        res.grayness.append(gray)
        restart, better = select_and_restart(c, penal, gray, sel_c)
        if better:
            sel_c = c
            res.selected_iteration = it
            res.selected_compliance = c
            res.selected_rho = rho.copy()
        if restart:
            res.restarted.append(it)
            rho = res.selected_rho.copy()
        else:
            rho = rho_new
    return res

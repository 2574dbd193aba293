"""Pins of the oracle's PCG, compliance, sensitivities and OC update (no GPU):
dense direct solves, the energy identity, central finite differences, the
volume constraint, and the compliances the paper prints."""
import json
from pathlib import Path

import numpy as np
import pytest

from oracle import fem, filter as cone, simp, solve
from paper_2604_18020_gb300 import workloads as W

GOLDEN = Path(__file__).parent / "golden"


def _system(shape, seed=1, face="x0"):
    m = W.Mesh(*shape)
    edof = fem.edof_table_fast(*shape)
    KE = fem.ke_exact()
    fixed = W.fixed_face(m, face)
    fd = fem.dof_mask(fixed)
    E = fem.simp_modulus(W.rho_random(m, seed=seed, lo=0.2, hi=1.0), 3.0)
    return m, edof, KE, fixed, fd, E


@pytest.mark.parametrize("shape", [(3, 2, 2), (6, 3, 3)])
def test_pcg_equals_dense_solve(shape):
    m, edof, KE, fixed, fd, E = _system(shape)
    f = W.zero_fixed(W.vec_random(m.n_dof, seed=9), fixed)
    d = fem.jacobi_diag(KE, E, edof, fd)
    u, st = solve.pcg(lambda v: fem.kv(KE, E, edof, v, fd), d, f, np.zeros(m.n_dof), 1e-13)
    u_ref = solve.dense_solve(fem.assemble_masked(KE, E, edof, m.n_dof, fd), f)
    assert st.converged
    assert np.abs(u - u_ref).max() <= 1e-9 * np.abs(u_ref).max()
    assert abs(st.true_rel_residual - st.rel_residual) <= 1e-12


def test_pcg_warm_start_and_zero_rhs():
    m, edof, KE, fixed, fd, E = _system((4, 2, 2))
    f = W.zero_fixed(W.vec_random(m.n_dof, seed=3), fixed)
    d = fem.jacobi_diag(KE, E, edof, fd)
    A = lambda v: fem.kv(KE, E, edof, v, fd)
    u, _ = solve.pcg(A, d, f, np.zeros(m.n_dof), 1e-12)
    _, st = solve.pcg(A, d, f, u, 1e-8)
    assert st.iterations == 0
    u0, st0 = solve.pcg(A, d, np.zeros(m.n_dof), np.ones(m.n_dof), 1e-8)
    assert st0.iterations == 0 and not u0.any()


def test_energy_identity():
    """At the solution, f^T u = sum_e E_e u_e^T KE u_e."""
    m, edof, KE, fixed, fd, E = _system((8, 4, 4))
    P = W.cantilever(8, 4, 4)
    rho = W.rho_random(m, seed=4, lo=0.2, hi=1.0)
    E = fem.simp_modulus(rho, 3.0)
    d = fem.jacobi_diag(KE, E, edof, fd)
    u, _ = solve.pcg(lambda v: fem.kv(KE, E, edof, v, fd), d, P.f, np.zeros(m.n_dof), 1e-12)
    c, _ = simp.compliance_sens(KE, edof, u, rho, 3.0)
    assert abs(c - P.f @ u) <= 1e-10 * abs(c)


def _compliance_of(rho, shape, f, fixed, rmin, penal=3.0):
    m = W.Mesh(*shape)
    edof = fem.edof_table_fast(*shape)
    KE = fem.ke_exact()
    fd = fem.dof_mask(fixed)
    rp = cone.filter_fwd(rho, *shape, rmin)
    E = fem.simp_modulus(rp, penal)
    u = solve.dense_solve(fem.assemble_masked(KE, E, edof, m.n_dof, fd), f)
    return f @ u, u, rp


def test_sensitivities_central_differences():
    shape, rmin = (3, 2, 2), 1.5
    P = W.cantilever(*shape)
    rho = W.rho_random(P.mesh, seed=6, lo=0.3, hi=0.9)
    c0, u, rp = _compliance_of(rho, shape, P.f, P.fixed, rmin)
    edof = fem.edof_table_fast(*shape)
    _, dc_phys = simp.compliance_sens(fem.ke_exact(), edof, u, rp, 3.0)
    dc = cone.filter_T(dc_phys, *shape, rmin)
    h = 1e-6
    for e in range(P.mesh.n_elem):
        rp_, rm_ = rho.copy(), rho.copy()
        rp_[e] += h
        rm_[e] -= h
        fd = (_compliance_of(rp_, shape, P.f, P.fixed, rmin)[0]
              - _compliance_of(rm_, shape, P.f, P.fixed, rmin)[0]) / (2 * h)
        assert abs(fd - dc[e]) <= 1e-6 * max(1.0, abs(dc[e]))


def test_oc_volume_bounds_and_monotone_lambda():
    rng = np.random.default_rng(7)
    rho = rng.uniform(0.05, 0.6, 500)
    dc = -rng.uniform(1e-4, 1.0, 500)
    new, info = simp.oc_update(rho, dc, 0.3, 0.2)
    assert abs(new.mean() - 0.3) <= 1e-8
    assert np.all(new <= np.minimum(1.0, rho + 0.2) + 0.0)
    assert np.all(new >= np.maximum(0.0, rho - 0.2) - 0.0)
    assert info["change"] <= 0.2 + 1e-15
    # volume of the candidate is non-increasing in lambda
    vols = []
    for lam in np.geomspace(1e-3, 1e4, 30):
        cand = np.maximum(np.maximum(0, rho - 0.2),
                          np.minimum(np.minimum(1, rho + 0.2), rho * np.sqrt(-dc / (lam / 500))))
        vols.append(cand.sum())
    assert np.all(np.diff(vols) <= 1e-12)


def test_oc_positive_sensitivity_is_clamped():
    rho = np.full(10, 0.5)
    dc = np.array([-1.0] * 9 + [2.0])
    new, _ = simp.oc_update(rho, dc, 0.45, 0.2)
    assert new[-1] == 0.3     # B_e = 0 -> candidate 0 -> lower move limit


def test_grayness_definition():
    assert simp.grayness(np.array([0.0, 1.0])) == 0.0
    assert simp.grayness(np.array([0.5, 0.5])) == 1.0


def _paper_case(case):
    nelx, nely, nelz = case["nelx"], case["nely"], case["nelz"]
    P = W.cantilever_point(nelx, nely, nelz)
    edof = fem.edof_table_fast(nelx, nely, nelz)
    fd = fem.dof_mask(P.fixed)
    KE = fem.ke_exact(1.0, 0.3, 2.0)       # the paper's element: edge 2
    E = fem.simp_modulus(np.full(P.mesh.n_elem, 0.5), 3.0)
    d = fem.jacobi_diag(KE, E, edof, fd)
    u, st = solve.pcg(lambda v: fem.kv(KE, E, edof, v, fd), d, P.f, np.zeros(P.mesh.n_dof),
                      1e-5, 10000)
    return P.f @ u, st.iterations


@pytest.mark.parametrize("idx", [0, pytest.param(1, marks=pytest.mark.slow)])
def test_paper_printed_compliance(idx):
    case = json.loads((GOLDEN / "paper_cantilever_compliance.json").read_text())["cases"][idx]
    c, its = _paper_case(case)
    c_paper = case["c_max_fp32"] / (1.0 + case["max_delta_c"])
    assert abs(c - c_paper) / c_paper <= case["rel_tol"]
    assert abs(its - case["cg_iterations_fp32"]) <= case["iter_tol"]


def test_oc_unreachable_target_collapses_bracket():
    """All sensitivities zero: every candidate sits at the lower move limit,
    the volume target cannot be met from above, lambda underflows and the
    bisection stops with the lower bounds."""
    rho = np.full(64, 0.3)
    new, info = simp.oc_update(rho, np.zeros(64), 0.3, 0.2)
    assert np.array_equal(new, np.maximum(0.0, rho - 0.2))
    assert info["lambda"] < 1e-300 and info["steps"] < 1200

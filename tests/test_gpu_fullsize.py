"""The benchmarked configurations at their own sizes, judged by the FP64 oracle.

* The SIMP iteration of the 120 x 60 x 30 cantilever (216,000 elements,
  686,433 DOFs) exactly as the benchmark runs it: FP64 iterative refinement
  around the FP32 inner Jacobi-PCG continuing its direction across
  refinement steps (inner tolerance 0.1, rtol 1e-8), the column K.v launch
  shape picked by the autotuner, with the benchmark's ticket-free CUDA-graph
  CG engine (2) and with the last-block-ticket engine (0).  Three steps from
  the uniform start; each is recomputed by the oracle from the GPU's input
  design and the GPU's displacement (Sec. 3.1, 3.6): physical density (cone
  filter), true FP64 residual of the solve, compliance as the sum of element
  energies and as f.u, sensitivities through the filter transpose and the
  OC bisection.
* Every tensor-core K.v form on the same mesh (Sec. 3.5), tolerances as on
  the small meshes.
* The multi-RHS mixed solve on the 100 x 50 x 50 cantilever with 8 seeded
  point loads (its benchmark configuration), case by case.
"""
import numpy as np
import pytest

from oracle import fem, filter as cone, simp as osimp
from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# tensor-core K.v tolerances (relative inf-norm with the inputs rounded to
# FP32): 2u for TF32 and FP16 (u = 2^-11), 2.5u for BF16 (u = 2^-8); the
# split forms carry each operand as hi + lo to about u^2
TC_TOL = {"tf32": 1e-3, "f16": 1e-3, "bf16": 1e-2, "tf32x3": 2e-6, "f16x3": 2e-6,
          "bf16x3": 2e-5}


@pytest.mark.parametrize("engine", [0, 2])
def test_benchmarked_simp_steps_match_oracle(cuda, engine):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.WORKLOADS["cantilever_120x60x30"]()
    m = P.mesh
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    params = mfto.default_params(volfrac=P.volfrac, rmin=P.rmin, rtol=1e-8)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed, params=params) as h:
        h.set_solver(mfto.FORM_F32, 1e-1)
        h.set_cg_engine(engine)
        h.set_ir_mode(mfto.IR_CONTINUE)
        h.kv_autotune()
        rho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=cuda)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        f = torch.tensor(P.f, device=cuda)
        rho_phys = torch.empty_like(rho)
        for step in range(3):
            rho_in = rho.cpu().numpy()
            st = h.simp_step(rho, u, f, rho_phys)
            assert st.cg_status == mfto.OK, step
            ug = u.cpu().numpy()
            # physical density: the cone filter is bit-exact
            rp = cone.filter_fwd(rho_in, m.nelx, m.nely, m.nelz, P.rmin)
            assert np.array_equal(rho_phys.cpu().numpy(), rp), step
            E = fem.simp_modulus(rp, 3.0)
            # the solve: true FP64 residual by the oracle's K.v
            r = P.f - fem.kv(KE, E, edof, ug, fd)
            assert np.linalg.norm(r) / np.linalg.norm(P.f) <= 1.5e-8, step
            # compliance: sum of element energies = f.u = the reported value
            c_ref, dc_phys = osimp.compliance_sens(KE, edof, ug, rp, 3.0)
            assert abs(c_ref - P.f @ ug) <= 1e-7 * abs(c_ref), step
            # the element energies u_e^T KE u_e cancel (the displacement is
            # mostly rigid motion of each element), so the two FP64
            # evaluations agree to the forward-error bound of a 24 x 24
            # quadratic form, n eps |u_e|^T |KE| |u_e| with n = 64 >= 48 terms
            ue = np.abs(ug[edof])
            bound = 64 * np.finfo(float).eps * float(
                np.sum(E * np.einsum("ei,ij,ej->e", ue, np.abs(KE), ue)))
            assert abs(st.compliance - c_ref) <= bound, (step, st.compliance - c_ref, bound)
            # sensitivities through the filter transpose, then OC
            dc = cone.filter_T(dc_phys, m.nelx, m.nely, m.nelz, P.rmin)
            rho_ref, info = osimp.oc_update(rho_in, dc, P.volfrac, 0.2)
            got = rho.cpu().numpy()
            assert np.abs(got - rho_ref).max() <= 1e-8, step
            assert abs(st.change - info["change"]) <= 1e-8, step
            assert abs(st.volume - P.volfrac) <= 1e-8, step


@pytest.mark.parametrize("form", list(TC_TOL))
def test_tc_forms_kv_full_size(cuda, form):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.WORKLOADS["cantilever_120x60x30"]()
    m = P.mesh
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    E32 = fem.simp_modulus(W.rho_random(m, seed=1), 3.0).astype(np.float32)
    v32 = W.vec_random(m.n_dof, seed=1).astype(np.float32)
    ref = fem.kv(fem.ke_exact(), E32.astype(np.float64), edof, v32.astype(np.float64), fd)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        y = torch.zeros(m.n_dof, dtype=torch.float32, device=cuda)
        h.kv(torch.tensor(E32, device=cuda), torch.tensor(v32, device=cuda), y,
             form=mfto.FORMS[form])
        got = y.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() / np.abs(ref).max() <= TC_TOL[form]
    assert np.array_equal(got[fd], v32.astype(np.float64)[fd])


def test_f32_kv_full_size_after_autotune(cuda):
    """The FP32 column K.v in the autotuned launch shape at 216,000 elements."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.WORKLOADS["cantilever_120x60x30"]()
    m = P.mesh
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    E32 = fem.simp_modulus(W.rho_random(m, seed=2), 3.0).astype(np.float32)
    v32 = W.vec_random(m.n_dof, seed=2).astype(np.float32)
    ref = fem.kv(fem.ke_exact(), E32.astype(np.float64), edof, v32.astype(np.float64), fd)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        h.kv_autotune()
        y = torch.zeros(m.n_dof, dtype=torch.float32, device=cuda)
        h.kv(torch.tensor(E32, device=cuda), torch.tensor(v32, device=cuda), y,
             form=mfto.FORM_F32)
        got = y.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() / np.abs(ref).max() <= 1e-5
    assert np.array_equal(got[fd], v32.astype(np.float64)[fd])


def test_multi_rhs_solve_full_size(cuda):
    """100 x 50 x 50 cantilever (250,000 elements), 8 seeded unit point loads,
    the benchmark's solver settings (continued inner direction at 0.1); a
    filtered random design so that the contrast is that of a SIMP run."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.WORKLOADS["cantilever_100x50x50_8rhs"]()
    m = P.mesh
    nr = P.f.shape[0]
    assert nr == 8
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    rp = cone.filter_fwd(W.rho_binary(m, seed=4, volfrac=0.3), m.nelx, m.nely, m.nelz, 1.5)
    E = fem.simp_modulus(rp, 3.0)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed,
                     params=mfto.default_params(max_rhs=nr)) as h:
        h.kv_autotune()
        h.set_solver(mfto.FORM_F32, 1e-1, 10000, 50)
        h.set_ir_mode(mfto.IR_CONTINUE)
        U = torch.zeros(nr * m.n_dof, dtype=torch.float64, device=cuda)
        sts = h.ir_solve_multi(torch.tensor(E, device=cuda),
                               torch.tensor(P.f.reshape(-1), device=cuda), U, nr,
                               inner_tol=1e-1)
        got = U.cpu().numpy().reshape(nr, -1)
    for r in range(nr):
        assert sts[r].status == mfto.OK, r
        f = P.f[r]
        true_rel = np.linalg.norm(f - fem.kv(KE, E, edof, got[r], fd)) / np.linalg.norm(f)
        assert true_rel <= 1.5e-8, (r, true_rel)
        c = float(np.sum(E * osimp.element_energy(KE, edof, got[r])))
        assert abs(c - f @ got[r]) <= 1e-7 * abs(c), r

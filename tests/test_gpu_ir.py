"""Mixed-precision solve (FP64 iterative refinement around an FP32 inner
Jacobi-PCG) against the FP64 oracle.  Tolerances: true FP64 relative
residual <= 1.5e-8 (outer tolerance 1e-8 plus the rounding of the
recomputation), compliance within 1e-7 of the oracle's FP64 PCG solution,
final compliance of a 20-iteration SIMP run within 1e-6."""
import numpy as np
import pytest

from oracle import fem, simp as osimp, solve
from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,inner_tol", [("restart", 1e-2), ("restart", 1e-4),
                                            ("continue", 1e-1), ("continue", 1e-2)])
@pytest.mark.parametrize("case", ["cantilever", "torsion"])
def test_ir_solve_matches_oracle(cuda, mode, inner_tol, case):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(24, 12, 12) if case == "cantilever" else W.torsion(10, 10, 30)
    m = P.mesh
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    KE = fem.ke_exact()
    E = fem.simp_modulus(W.rho_random(m, seed=31, lo=0.05, hi=1.0), 3.0)
    d = fem.jacobi_diag(KE, E, edof, fd)
    u_ref, _ = solve.pcg(lambda v: fem.kv(KE, E, edof, v, fd), d, P.f, np.zeros(m.n_dof), 1e-10)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        h.set_ir_mode(mfto.IR_CONTINUE if mode == "continue" else mfto.IR_RESTART)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        st = h.ir_solve(torch.tensor(E, device=cuda), torch.tensor(P.f, device=cuda), u,
                        inner_tol=inner_tol)
        got = u.cpu().numpy()
    assert st.status == mfto.OK, st.status
    assert st.rel_residual <= 1e-8
    true_rel = np.linalg.norm(P.f - fem.kv(KE, E, edof, got, fd)) / np.linalg.norm(P.f)
    assert true_rel <= 1.5e-8
    assert abs(P.f @ got - P.f @ u_ref) / abs(P.f @ u_ref) <= 1e-7
    # the outer residual history decreases
    hist = [st.history[i] for i in range(min(st.outer_iterations + 1, 64))]
    assert all(b < a for a, b in zip(hist, hist[1:]))


def test_ir_stall_detector(cuda):
    """An inner tolerance of 0.97 cuts the outer residual by less than the
    0.9 stagnation ratio per correction: the solve must stop as STALLED."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(16, 8, 8)
    m = P.mesh
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        E = torch.ones(m.n_elem, dtype=torch.float64, device=cuda)
        st = h.ir_solve(E, torch.tensor(P.f, device=cuda), u, inner_tol=0.97)
    assert st.status == mfto.STALLED
    assert st.outer_iterations >= 2


def test_simp_with_mixed_solver(cuda):
    """20 SIMP iterations with the mixed solver give the oracle's compliance
    history within 1e-6."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(24, 12, 12)
    m = P.mesh
    _, _, hist = osimp.simp(m.nelx, m.nely, m.nelz, P.f, P.fixed, P.volfrac, P.rmin, 20)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed,
                     params=mfto.default_params(volfrac=P.volfrac, rmin=P.rmin)) as h:
        h.set_solver(mfto.FORM_F32, 1e-2)
        rho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=cuda)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        f = torch.tensor(P.f, device=cuda)
        cs = [h.simp_step(rho, u, f).compliance for _ in range(20)]
    assert np.allclose(cs, hist.compliance, rtol=1e-6, atol=0)


def test_ir_continue_needs_fewer_inner_iterations(cuda):
    """Continuing the direction across outer steps (reliable updating) keeps
    one Krylov process: on a SIMP state of a torsion bar (6 iterations of the
    FP64 loop) it needs fewer inner iterations than restarting each inner
    solve, and no more than 1.6 times the plain FP64 PCG's."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.torsion(16, 16, 48)
    m = P.mesh
    f = torch.tensor(P.f, device=cuda)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed,
                     params=mfto.default_params(volfrac=P.volfrac, rmin=P.rmin)) as h:
        rho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=cuda)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        for _ in range(6):
            h.simp_step(rho, u, f)
        rho_phys = torch.empty_like(rho)
        h.filter(rho, rho_phys)
        E = torch.empty_like(rho)
        h.simp_modulus(rho_phys, E)
        u.zero_()
        n64 = h.pcg(E, f, u).iterations
        its = {}
        for mode, tol in ((mfto.IR_RESTART, 1e-2), (mfto.IR_CONTINUE, 1e-1)):
            h.set_ir_mode(mode)
            u.zero_()
            st = h.ir_solve(E, f, u, inner_tol=tol)
            assert st.status == mfto.OK and st.rel_residual <= 1e-8
            its[mode] = st.inner_iterations
    assert its[mfto.IR_CONTINUE] < its[mfto.IR_RESTART], (its, n64)
    assert its[mfto.IR_CONTINUE] <= 1.6 * n64, (its, n64)


def test_simp_with_continued_mixed_solver(cuda):
    """20 SIMP iterations with the continued-direction mixed solver (inner
    tolerance 0.1) give the oracle's compliance history within 1e-6."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(24, 12, 12)
    m = P.mesh
    _, _, hist = osimp.simp(m.nelx, m.nely, m.nelz, P.f, P.fixed, P.volfrac, P.rmin, 20)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed,
                     params=mfto.default_params(volfrac=P.volfrac, rmin=P.rmin)) as h:
        h.set_solver(mfto.FORM_F32, 1e-1)
        h.set_ir_mode(mfto.IR_CONTINUE)
        rho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=cuda)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        f = torch.tensor(P.f, device=cuda)
        cs = [h.simp_step(rho, u, f).compliance for _ in range(20)]
    assert np.allclose(cs, hist.compliance, rtol=1e-6, atol=0)

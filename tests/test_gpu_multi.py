"""Multi-RHS K.V and the multi-RHS mixed-precision solve against the FP64
oracle, case by case (tolerances as for one load case: K.V FP64 1e-12,
FP32 1e-5; solve: true FP64 residual <= 1.5e-8 per case)."""
import numpy as np
import pytest

from oracle import fem, solve
from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["f64", "f32"])
@pytest.mark.parametrize("shape,nrhs", [((13, 7, 5), 3), ((24, 12, 12), 8), ((1, 1, 1), 2)])
def test_kv_multi(cuda, form, shape, nrhs):
    import torch
    from paper_2604_18020_gb300 import mfto
    m = W.Mesh(*shape)
    fixed = W.fixed_face(m, "x0")
    edof = fem.edof_table_fast(*shape)
    fd = fem.dof_mask(fixed)
    E = fem.simp_modulus(W.rho_random(m, seed=51), 3.0)
    V = np.stack([W.vec_random(m.n_dof, seed=60 + r) for r in range(nrhs)])
    dt, tol, npdt = ((torch.float64, 1e-12, np.float64) if form == "f64"
                     else (torch.float32, 1e-5, np.float32))
    E, V = E.astype(npdt).astype(np.float64), V.astype(npdt).astype(np.float64)
    with mfto.Handle(*shape, fixed) as h:
        Y = torch.zeros(nrhs * m.n_dof, dtype=dt, device=cuda)
        h.kv_multi(torch.tensor(E, dtype=dt, device=cuda),
                   torch.tensor(V.reshape(-1), dtype=dt, device=cuda), Y, nrhs,
                   form=mfto.FORMS[form])
        got = Y.cpu().numpy().astype(np.float64).reshape(nrhs, -1)
    for r in range(nrhs):
        ref = fem.kv(fem.ke_exact(), E, edof, V[r], fd)
        assert np.abs(got[r] - ref).max() / np.abs(ref).max() <= tol


@pytest.mark.parametrize("mode,inner_tol", [("restart", 1e-2), ("continue", 1e-1)])
def test_ir_solve_multi_8_load_cases(cuda, mode, inner_tol):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.multi_rhs_cantilever(24, 12, 12, nrhs=8, seed=3)
    m = P.mesh
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    KE = fem.ke_exact()
    E = fem.simp_modulus(W.rho_random(m, seed=52, lo=0.05, hi=1.0), 3.0)
    d = fem.jacobi_diag(KE, E, edof, fd)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed,
                     params=mfto.default_params(max_rhs=8)) as h:
        h.set_ir_mode(mfto.IR_CONTINUE if mode == "continue" else mfto.IR_RESTART)
        U = torch.zeros(8 * m.n_dof, dtype=torch.float64, device=cuda)
        sts = h.ir_solve_multi(torch.tensor(E, device=cuda),
                               torch.tensor(P.f.reshape(-1), device=cuda), U, 8,
                               inner_tol=inner_tol)
        got = U.cpu().numpy().reshape(8, -1)
    for r in range(8):
        assert sts[r].status == mfto.OK
        f = P.f[r]
        true_rel = np.linalg.norm(f - fem.kv(KE, E, edof, got[r], fd)) / np.linalg.norm(f)
        assert true_rel <= 1.5e-8
        u_ref, _ = solve.pcg(lambda v: fem.kv(KE, E, edof, v, fd), d, f, np.zeros(m.n_dof), 1e-10)
        assert abs(f @ got[r] - f @ u_ref) / abs(f @ u_ref) <= 1e-7


def test_ir_solve_multi_matches_single(cuda):
    """Each case of the multi-RHS solve converges like its single-RHS solve."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.multi_rhs_cantilever(16, 8, 8, nrhs=3, seed=4)
    m = P.mesh
    E = torch.tensor(fem.simp_modulus(W.rho_random(m, seed=53, lo=0.1, hi=1.0), 3.0),
                     device=cuda)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed,
                     params=mfto.default_params(max_rhs=4)) as h:
        U = torch.zeros(3 * m.n_dof, dtype=torch.float64, device=cuda)
        sts = h.ir_solve_multi(E, torch.tensor(P.f.reshape(-1), device=cuda), U, 3)
        for r in range(3):
            u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
            s1 = h.ir_solve(E, torch.tensor(P.f[r], device=cuda), u)
            assert s1.status == sts[r].status == mfto.OK
            assert torch.allclose(u, U[r * m.n_dof:(r + 1) * m.n_dof], rtol=0,
                                  atol=1e-7 * float(u.abs().max()))


@pytest.mark.parametrize("variant", [0, 2])
def test_ir_solve_multi_ragged_and_variants(cuda, variant):
    """Odd n_dof (case vectors not 16-byte aligned) and both K.v kernels of
    the inner CG (column kernel, block kernel): every case meets the FP64
    tolerance; a case with a zero load stays zero."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.multi_rhs_cantilever(12, 6, 4, nrhs=5, seed=6)
    m = P.mesh
    assert m.n_dof % 4 != 0
    F = P.f.copy()
    F[2] = 0.0
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    KE = fem.ke_exact()
    E = fem.simp_modulus(W.rho_random(m, seed=54, lo=0.05, hi=1.0), 3.0)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed,
                     params=mfto.default_params(max_rhs=8)) as h:
        h.set_kv_variant(variant)
        h.set_ir_mode(mfto.IR_CONTINUE)
        U = torch.zeros(5 * m.n_dof, dtype=torch.float64, device=cuda)
        sts = h.ir_solve_multi(torch.tensor(E, device=cuda), torch.tensor(F.reshape(-1), device=cuda),
                               U, 5, inner_tol=1e-1)
        got = U.cpu().numpy().reshape(5, -1)
    for r in range(5):
        assert sts[r].status == mfto.OK
        if r == 2:
            assert np.abs(got[r]).max() == 0.0
            continue
        true_rel = np.linalg.norm(F[r] - fem.kv(KE, E, edof, got[r], fd)) / np.linalg.norm(F[r])
        assert true_rel <= 1.5e-8

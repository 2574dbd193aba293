"""Persistent FP32 inner CG (one cooperative launch per inner solve) against
the per-iteration graph engine and the FP64 oracle.

Both engines evaluate the same per-entry arithmetic; only the order in which
per-block partial sums of the dot products are added differs, so the inner
iteration counts may differ by a few and the refined solutions agree to the
outer tolerance.  Bars: true FP64 relative residual <= 1.5e-8 (rtol 1e-8
plus the rounding of the recomputation), compliance within 1e-7 of the
oracle's FP64 solve, inner iteration totals within 3 % of each other."""
import numpy as np
import pytest

from oracle import fem, solve
from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _solve(h, E, f, cuda, engine, inner_tol=1e-2):
    import torch
    h.set_cg_engine(engine)
    u = torch.zeros(h.n_dof, dtype=torch.float64, device=cuda)
    st = h.ir_solve(E, f, u, inner_tol=inner_tol)
    return st, u.cpu().numpy()


# meshes: several node blocks per CTA, ragged block edges on every axis
# (7 x 7 x 3 owned nodes per block), a torsion bar, a single element
@pytest.mark.parametrize("dims,case", [((24, 12, 12), "cantilever"), ((37, 23, 17), "cantilever"),
                                       ((10, 10, 30), "torsion"), ((1, 1, 1), "cantilever")])
def test_persistent_matches_graph_and_oracle(cuda, dims, case):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(*dims) if case == "cantilever" else W.torsion(*dims)
    m = P.mesh
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    KE = fem.ke_exact()
    E = fem.simp_modulus(W.rho_random(m, seed=41, lo=0.05, hi=1.0), 3.0)
    d = fem.jacobi_diag(KE, E, edof, fd)
    u_ref, _ = solve.pcg(lambda v: fem.kv(KE, E, edof, v, fd), d, P.f, np.zeros(m.n_dof), 1e-11)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        tE = torch.tensor(E, device=cuda)
        tf = torch.tensor(P.f, device=cuda)
        st1, u1 = _solve(h, tE, tf, cuda, 1)
        st0, u0 = _solve(h, tE, tf, cuda, 0)
    c_ref = P.f @ u_ref
    for st, u in ((st1, u1), (st0, u0)):
        assert st.status == mfto.OK, st.status
        true_rel = np.linalg.norm(P.f - fem.kv(KE, E, edof, u, fd)) / np.linalg.norm(P.f)
        assert true_rel <= 1.5e-8, true_rel
        assert abs(P.f @ u - c_ref) / abs(c_ref) <= 1e-7
    assert st1.outer_iterations == st0.outer_iterations
    assert abs(st1.inner_iterations - st0.inner_iterations) <= max(2, 0.03 * st0.inner_iterations)


def test_persistent_first_inner_solve_matches_graph(cuda):
    """One inner solve on the 120 x 60 x 30 benchmark mesh (891 node blocks,
    two per CTA): capped at the same small iteration count, the two engines'
    corrections agree to FP32 rounding (same arithmetic, different order of
    the block partials in alpha and beta only)."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(120, 60, 30)
    m = P.mesh
    E = torch.tensor(fem.simp_modulus(W.rho_random(m, seed=2, lo=0.1, hi=1.0), 3.0), device=cuda)
    f = torch.tensor(P.f, device=cuda)
    out = []
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        for engine in (1, 0):
            h.set_cg_engine(engine)
            h.set_solver(mfto.FORM_F32, 1e-2, inner_maxit=50, max_outer=1)
            u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
            st = h.ir_solve(E, f, u)
            out.append((st, u.cpu().numpy()))
    (s1, u1), (s0, u0) = out
    assert s1.inner_iterations == s0.inner_iterations == 50
    assert s1.status == s0.status == mfto.NOT_CONVERGED
    rel = np.abs(u1 - u0).max() / np.abs(u0).max()
    assert rel <= 1e-4, rel
    assert abs(s1.rel_residual - s0.rel_residual) <= 1e-4 * s0.rel_residual


def test_persistent_zero_load(cuda):
    """f = 0: the inner solve is never entered; u = 0 and status OK."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(8, 4, 4)
    m = P.mesh
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        h.set_cg_engine(1)
        u = torch.ones(m.n_dof, dtype=torch.float64, device=cuda)
        st = h.ir_solve(torch.ones(m.n_elem, dtype=torch.float64, device=cuda),
                        torch.zeros(m.n_dof, dtype=torch.float64, device=cuda), u)
        assert st.status == mfto.OK
        assert float(u.abs().max()) == 0.0


def test_persistent_timing_counts_iterations(cuda):
    """With timing on, the persistent launches report the CG iterations they
    ran, equal to the solve's inner iteration total."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(24, 12, 12)
    m = P.mesh
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        h.set_cg_engine(1)
        h.kv_timing(True)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        st = h.ir_solve(torch.full((m.n_elem,), 0.3 ** 3, dtype=torch.float64, device=cuda),
                        torch.tensor(P.f, device=cuda), u)
        n, it, ms = h.cg_timing_read()
        h.kv_timing(False)
    assert st.status == mfto.OK
    assert n == st.outer_iterations
    assert it == st.inner_iterations
    assert ms > 0.0

"""The FP32 inner CG engines -- two kernels per iteration from a CUDA graph
(0), one persistent cooperative kernel per solve (1), two ticket-free
kernels per iteration from a CUDA graph (2) -- against each other and the
FP64 oracle.

The engines evaluate Hestenes-Stiefel CG with the same per-entry arithmetic;
they differ in the order in which block partials are added, so the FP32
trajectories drift apart and inner iteration totals differ (by
up to about 15 % measured: an FP32 CG on these contrasts is sensitive to
rounding order), while every refined solution meets the outer tolerance.
Bars: true FP64 relative residual <= 1.5e-8 (rtol 1e-8 plus the rounding of
the recomputation), compliance within 1e-7 of the oracle's FP64 solve, inner
iteration totals within 20 % of engine 0's."""
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
def test_engines_match_oracle(cuda, dims, case):
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
    res = {}
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        tE = torch.tensor(E, device=cuda)
        tf = torch.tensor(P.f, device=cuda)
        for mode in (mfto.IR_RESTART, mfto.IR_CONTINUE):
            h.set_ir_mode(mode)
            tol = 1e-2 if mode == mfto.IR_RESTART else 1e-1
            for engine in (0, 1, 2):
                res[(mode, engine)] = _solve(h, tE, tf, cuda, engine, inner_tol=tol)
    c_ref = P.f @ u_ref
    for (mode, engine), (st, u) in res.items():
        assert st.status == mfto.OK, (mode, engine, st.status)
        true_rel = np.linalg.norm(P.f - fem.kv(KE, E, edof, u, fd)) / np.linalg.norm(P.f)
        assert true_rel <= 1.5e-8, (mode, engine, true_rel)
        assert abs(P.f @ u - c_ref) / abs(c_ref) <= 1e-7
        ref_it = res[(mode, 0)][0].inner_iterations
        assert abs(st.inner_iterations - ref_it) <= max(3, 0.2 * ref_it), (mode, engine)


def test_engines_first_inner_solve_agree(cuda):
    """One inner solve on the 120 x 60 x 30 benchmark mesh, capped at 50
    iterations: the two engines' corrections agree to FP32 rounding."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(120, 60, 30)
    m = P.mesh
    E = torch.tensor(fem.simp_modulus(W.rho_random(m, seed=2, lo=0.1, hi=1.0), 3.0), device=cuda)
    f = torch.tensor(P.f, device=cuda)
    out = []
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        for engine in (0, 1, 2):
            h.set_cg_engine(engine)
            h.set_solver(mfto.FORM_F32, 1e-2, inner_maxit=50, max_outer=1)
            u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
            st = h.ir_solve(E, f, u)
            out.append((st, u.cpu().numpy()))
    s0, u0 = out[0]
    for (st, u), bar in zip(out[1:], (1e-4, 1e-4)):
        assert st.inner_iterations == s0.inner_iterations == 50
        assert st.status == s0.status == mfto.NOT_CONVERGED
        rel = np.abs(u - u0).max() / np.abs(u0).max()
        assert rel <= bar, rel
        assert abs(st.rel_residual - s0.rel_residual) <= bar * s0.rel_residual


@pytest.mark.parametrize("engine", [1, 2])
def test_engine_zero_load(cuda, engine):
    """f = 0: the inner solve is never entered; u = 0 and status OK."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(8, 4, 4)
    m = P.mesh
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        h.set_cg_engine(engine)
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


def test_cg_kv_burst_time(cuda):
    """mfto_cg_kv_time: a positive, finite time per launch of engine 2's K.v
    (a solve afterwards still meets the tolerance: the call only overwrites
    the FP32 work vectors), and MFTO_INVALID_ARG for another engine."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(24, 12, 12)
    m = P.mesh
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        h.set_solver(mfto.FORM_F32, 0.1)
        h.set_cg_engine(2)
        us = h.cg_kv_time(8, 2)
        assert np.isfinite(us) and 0.0 < us < 1e4
        us_ev = h.cg_kv_time(8, 2, events=True)
        assert np.isfinite(us_ev) and 0.0 < us_ev < 1e4
        rho = torch.tensor(W.rho_random(m, seed=4, lo=0.05, hi=1.0), device=cuda)
        E = torch.empty_like(rho)
        h.simp_modulus(rho, E)
        f = torch.tensor(P.f, device=cuda)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        st = h.ir_solve(E, f, u, inner_tol=0.1)
        assert st.status == mfto.OK
        edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
        r = P.f - fem.kv(fem.ke_exact(), E.cpu().numpy(), edof, u.cpu().numpy(),
                         fem.dof_mask(P.fixed))
        assert np.linalg.norm(r) / np.linalg.norm(P.f) <= 1.5e-8
        h.set_cg_engine(0)
        with pytest.raises(mfto.MftoError) as err:
            h.cg_kv_time(8, 2)
        assert err.value.code == mfto.INVALID_ARG

"""Three-field SIMP (Heaviside projection) and the SIMP-120 continuation
protocol on the GPU against the oracle.  Bars: the projection and its
derivative to FP64 rounding (tanh is the only transcendental, <= 1e-14);
projected SIMP steps: compliance within 1e-7, design within 1e-6; the
protocol: the same restarts and selected iterate, compliance history within
1e-5 (sharp projections amplify the solver's 1e-8 residual differences)."""
import numpy as np
import pytest

from oracle import fem, protocol as proto, simp as osimp
from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("beta", [1.0, 4.0, 16.0, 32.0])
def test_projection_matches_oracle(cuda, beta):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(10, 5, 4)
    m = P.mesh
    rb = W.rho_random(m, seed=3, lo=0.0, hi=1.0)
    rb[:3] = [0.0, 0.5, 1.0]
    dc = -W.rho_random(m, seed=4, lo=0.1, hi=2.0)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        h.set_projection(beta, 0.5)
        t_rb = torch.tensor(rb, device=cuda)
        t_rp = torch.empty_like(t_rb)
        t_dc = torch.tensor(dc, device=cuda)
        h.project(t_rb, t_rp, t_dc)
        rp, dcc = t_rp.cpu().numpy(), t_dc.cpu().numpy()
    assert np.abs(rp - proto.heaviside(rb, beta)).max() <= 1e-14
    ref = dc * proto.heaviside_deriv(rb, beta)
    assert np.abs(dcc - ref).max() <= 1e-14 * np.abs(ref).max()
    assert rp.min() >= 0.0 and rp.max() <= 1.0


def test_projected_simp_steps_match_oracle(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(24, 12, 12)
    m = P.mesh
    penal, beta, move, rmin = 3.5, 4.0, 0.15, 1.4
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    rho = np.full(m.n_elem, P.volfrac)
    u = np.zeros(m.n_dof)
    cs = []
    for _ in range(5):
        rho, u, c, _, _ = proto.step(KE, edof, fd, m.nelx, m.nely, m.nelz, P.f, rho, u,
                                     P.volfrac, penal, beta, move, rmin)
        cs.append(c)
    prm = mfto.default_params(volfrac=P.volfrac, rmin=rmin, penal=penal, move=move)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed, params=prm) as h:
        h.set_projection(beta, 0.5)
        trho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=cuda)
        tu = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        tf = torch.tensor(P.f, device=cuda)
        got = [h.simp_step(trho, tu, tf).compliance for _ in range(5)]
        rho_gpu = trho.cpu().numpy()
    assert np.allclose(got, cs, rtol=1e-7, atol=0)
    assert np.abs(rho_gpu - rho).max() <= 1e-6


def test_protocol_matches_oracle(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(16, 8, 8)
    m = P.mesh
    n_iter = 70
    ref = proto.protocol(m.nelx, m.nely, m.nelz, P.f, P.fixed, P.volfrac, P.rmin, n_iter=n_iter)
    prm = mfto.default_params(volfrac=P.volfrac, rmin=P.rmin)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed, params=prm) as h:
        rho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=cuda)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        f = torch.tensor(P.f, device=cuda)
        sel = torch.zeros_like(rho)
        pp = mfto.default_protocol_params(n_iter=n_iter, rmin0=P.rmin)
        st, comp, gray, rest = h.simp_protocol(rho, u, f, sel, pp)
        # the handle's own parameters are restored: a plain step still matches
        rho2 = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=cuda)
        u2 = torch.zeros_like(u)
        c_plain = h.simp_step(rho2, u2, f).compliance
        sel = sel.cpu().numpy()
    assert st.iterations == n_iter
    assert np.allclose(comp, ref.compliance, rtol=1e-5, atol=0)
    assert np.allclose(gray, ref.grayness, rtol=1e-5, atol=1e-9)
    assert [i + 1 for i in range(n_iter) if rest[i]] == ref.restarted
    assert st.restarts == len(ref.restarted)
    assert st.selected_iteration == ref.selected_iteration
    if ref.selected_iteration:
        assert abs(st.selected_compliance - ref.selected_compliance) <= 1e-5 * ref.selected_compliance
        assert np.abs(sel - ref.selected_rho).max() <= 1e-4
    _, _, hist = osimp.simp(m.nelx, m.nely, m.nelz, P.f, P.fixed, P.volfrac, P.rmin, 1)
    assert abs(c_plain - hist.compliance[0]) <= 1e-6 * hist.compliance[0]

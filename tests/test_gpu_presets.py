"""The paper's hard-problem presets on the GPU (small versions): the FP64
PCG and the mixed solve reach the FP64 tolerance on the singular but
consistent MBB system and on the bridge, measured by the oracle's residual; the
bridge solution equals the oracle's dense solve."""
import numpy as np
import pytest

from oracle import fem, solve
from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["mbb", "bridge"])
def test_hard_presets_solve(cuda, name):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.mbb(18, 6, 4) if name == "mbb" else W.bridge(18, 6, 4)
    m = P.mesh
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    KE = fem.ke_exact()
    E = fem.simp_modulus(W.rho_random(m, seed=71, lo=0.2, hi=1.0), 3.0)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        tE, tf = torch.tensor(E, device=cuda), torch.tensor(P.f, device=cuda)
        u64 = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        s64 = h.pcg(tE, tf, u64)
        umx = torch.zeros_like(u64)
        h.set_ir_mode(mfto.IR_CONTINUE)
        smx = h.ir_solve(tE, tf, umx, inner_tol=0.1)
        got = {"f64": (s64.status, u64.cpu().numpy()), "mixed": (smx.status, umx.cpu().numpy())}
    for key, (status, u) in got.items():
        assert status == mfto.OK, (key, status)
        rel = np.linalg.norm(P.f - fem.kv(KE, E, edof, u, fd)) / np.linalg.norm(P.f)
        assert rel <= 1.5e-8, (key, rel)
    if name == "bridge":
        u_ref = solve.dense_solve(fem.assemble_masked(KE, E, edof, m.n_dof, fd), P.f)
        for key, (_, u) in got.items():
            assert abs(P.f @ u - P.f @ u_ref) <= 1e-7 * abs(P.f @ u_ref)
    else:
        # compliance f.u is defined on the singular system (f is orthogonal to
        # the null space): both solvers agree
        c64, cmx = P.f @ got["f64"][1], P.f @ got["mixed"][1]
        assert abs(cmx - c64) <= 1e-7 * abs(c64)

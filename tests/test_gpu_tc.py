"""Tensor-core K.v forms (tcgen05, FP32 accumulation in tensor memory) and
the mixed-precision solve with each of them as the inner form, against the
FP64 oracle.

K.v tolerances (relative inf-norm, inputs rounded to FP32 first), from the
unit roundoff u of the operand type (both operands rounded, 24-term sums):
  TF32, FP16 (u = 2^-11):   2u  = 1e-3
  BF16 (u = 2^-8):          2.5u = 1e-2
  split forms (hi + lo represents an operand to ~u^2, FP32 accumulation):
  TF32x3, FP16x3:           2e-6;   BF16x3 (u^2 = 2^-16): 2e-5
The solve: the split forms must reach the FP64 tolerance 1e-8; the
single-term forms have eps * kappa(K) > 1 at these sizes (kappa ~ 1e5..1e6)
and may stall, as the paper reports for BF16: they must then say so.
"""
import numpy as np
import pytest

from oracle import fem, solve
from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"tf32": 1e-3, "f16": 1e-3, "bf16": 1e-2, "tf32x3": 2e-6, "f16x3": 2e-6, "bf16x3": 2e-5}


@pytest.mark.parametrize("form", list(TOL))
@pytest.mark.parametrize("shape,face", [((1, 1, 1), "x0"), ((4, 4, 2), "x0"), ((13, 7, 5), "z0"),
                                        ((40, 30, 9), "x0"), ((17, 13, 33), "x0")])
def test_kv_tc_forms(cuda, form, shape, face):
    import torch
    from paper_2604_18020_gb300 import mfto
    m = W.Mesh(*shape)
    fixed = W.fixed_face(m, face)
    edof = fem.edof_table_fast(*shape)
    fd = fem.dof_mask(fixed)
    E32 = fem.simp_modulus(W.rho_random(m, seed=41), 3.0).astype(np.float32)
    v32 = W.vec_random(m.n_dof, seed=42).astype(np.float32)
    ref = fem.kv(fem.ke_exact(), E32.astype(np.float64), edof, v32.astype(np.float64), fd)
    with mfto.Handle(*shape, fixed) as h:
        y = torch.zeros(m.n_dof, dtype=torch.float32, device=cuda)
        h.kv(torch.tensor(E32, device=cuda), torch.tensor(v32, device=cuda), y,
             form=mfto.FORMS[form])
        got = y.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() / np.abs(ref).max() <= TOL[form]
    assert np.array_equal(got[fd], v32.astype(np.float64)[fd])


def test_kv_tc_deterministic(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    m = W.Mesh(40, 30, 9)
    fixed = W.fixed_face(m, "x0")
    E = torch.rand(m.n_elem, device=cuda) + 0.01
    v = torch.rand(m.n_dof, device=cuda) - 0.5
    with mfto.Handle(40, 30, 9, fixed) as h:
        outs = []
        for _ in range(3):
            y = torch.empty_like(v)
            h.kv(E, v, y, form=mfto.FORM_TF32X3)
            outs.append(y.cpu().numpy())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


@pytest.mark.parametrize("form", ["tf32x3", "f16x3", "bf16x3", "tf32", "f16", "bf16"])
def test_ir_with_tc_inner_form(cuda, form):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(24, 12, 12)
    m = P.mesh
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    KE = fem.ke_exact()
    E = fem.simp_modulus(W.rho_random(m, seed=43, lo=0.05, hi=1.0), 3.0)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        h.set_solver(mfto.FORM_F32, 1e-2, 10000, 30)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        st = h.ir_solve(torch.tensor(E, device=cuda), torch.tensor(P.f, device=cuda), u,
                        inner=mfto.FORMS[form], inner_tol=1e-2)
        got = u.cpu().numpy()
    true_rel = np.linalg.norm(P.f - fem.kv(KE, E, edof, got, fd)) / np.linalg.norm(P.f)
    if form.endswith("x3"):
        assert st.status == mfto.OK
    assert st.status in (mfto.OK, mfto.STALLED, mfto.NOT_CONVERGED)
    if st.status == mfto.OK:
        assert true_rel <= 1.5e-8
    else:
        assert st.rel_residual > 1e-8          # it says it did not converge
        assert abs(true_rel - st.rel_residual) <= 1e-3 * st.rel_residual + 1e-12

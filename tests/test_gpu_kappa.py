"""The condition-number estimator on the GPU against the oracle's, from the
same seeded start vectors: the same step counts, and eigenvalue estimates
within 1e-6 (the inner solves stop at 1e-8; power steps agree to rounding),
plus the LAPACK spectrum on a tiny mesh."""
import numpy as np
import pytest

from oracle import fem, kappa
from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(shape, face, seed):
    m = W.Mesh(*shape)
    edof = fem.edof_table_fast(*shape)
    KE = fem.ke_exact()
    fixed = W.fixed_face(m, face)
    fd = fem.dof_mask(fixed)
    E = fem.simp_modulus(W.rho_random(m, seed=seed, lo=0.1, hi=1.0), 3.0)
    return m, edof, KE, fixed, fd, E


@pytest.mark.parametrize("shape,face", [((8, 4, 4), "x0"), ((6, 5, 9), "z0")])
def test_kappa_matches_oracle(cuda, shape, face):
    import torch
    from paper_2604_18020_gb300 import mfto
    m, edof, KE, fixed, fd, E = _case(shape, face, seed=13)
    vp = W.vec_random(m.n_dof, seed=42)
    vi = W.vec_random(m.n_dof, seed=123)
    ref = kappa.estimate(lambda v: fem.kv(KE, E, edof, v, fd), fem.jacobi_diag(KE, E, edof, fd),
                         fd, vp, vi)
    with mfto.Handle(*shape, fixed) as h:
        st = h.kappa(torch.tensor(E, device=cuda), torch.tensor(vp, device=cuda),
                     torch.tensor(vi, device=cuda))
    assert st.power_steps == ref.power_steps
    assert st.inverse_steps == ref.inverse_steps
    assert abs(st.lambda_max - ref.lambda_max) <= 1e-10 * ref.lambda_max
    assert abs(st.lambda_min - ref.lambda_min) <= 1e-6 * ref.lambda_min
    assert abs(st.kappa - ref.kappa) <= 1e-6 * ref.kappa
    assert abs(st.inner_iterations - ref.inner_iterations) <= 2 * ref.inverse_steps


def test_kappa_converged_matches_lapack(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    m, edof, KE, fixed, fd, E = _case((4, 2, 3), "x0", seed=3)
    K = fem.assemble(KE, E, edof, m.n_dof).toarray()
    ev = np.linalg.eigvalsh(K[np.ix_(~fd, ~fd)])
    prm = mfto.default_kappa_params(power_maxit=20000, power_tol=1e-14, inverse_maxit=2000,
                                    inverse_tol=1e-14, inner_rtol=1e-13)
    with mfto.Handle(4, 2, 3, fixed) as h:
        st = h.kappa(torch.tensor(E, device=cuda),
                     torch.tensor(W.vec_random(m.n_dof, seed=42), device=cuda),
                     torch.tensor(W.vec_random(m.n_dof, seed=123), device=cuda), prm)
    assert abs(st.lambda_max - ev[-1]) <= 1e-8 * ev[-1]
    assert abs(st.lambda_min - ev[0]) <= 1e-8 * ev[0]


def test_kappa_rejects_vector_on_fixed_dofs_only(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    m, edof, KE, fixed, fd, E = _case((4, 2, 2), "x0", seed=1)
    v = np.where(fd, 1.0, 0.0)
    with mfto.Handle(4, 2, 2, fixed) as h:
        with pytest.raises(mfto.MftoError):
            h.kappa(torch.tensor(E, device=cuda), torch.tensor(v, device=cuda),
                    torch.tensor(v, device=cuda))

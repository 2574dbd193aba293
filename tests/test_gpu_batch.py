"""Batches of independent uneven meshes: the batched K.V per instance
against the oracle for every element-block shape, the batched mixed solve
(true FP64 residual <= 1.5e-8 per instance), the autotuner, and the
64-instance configuration (16x8x8 .. 48x24x24) with sampled oracle checks."""
import numpy as np
import pytest

from oracle import fem, solve
from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _concat(problems, seed):
    Es, fs = [], []
    for i, P in enumerate(problems):
        Es.append(fem.simp_modulus(W.rho_random(P.mesh, seed=seed + i, lo=0.05, hi=1.0), 3.0))
        fs.append(P.f)
    return Es, fs


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
@pytest.mark.parametrize("form", ["f64", "f32"])
def test_batch_kv(cuda, shape, form):
    import torch
    from paper_2604_18020_gb300 import mfto
    problems = W.uneven_instances(count=7, seed=11, kmin=2, kmax=7) + [W.cantilever(1, 1, 1)]
    Es, _ = _concat(problems, 100)
    vs = [W.vec_random(P.mesh.n_dof, seed=200 + i) for i, P in enumerate(problems)]
    npdt, dt, tol = ((np.float64, torch.float64, 1e-12) if form == "f64"
                     else (np.float32, torch.float32, 1e-5))
    Es = [e.astype(npdt).astype(np.float64) for e in Es]
    vs = [v.astype(npdt).astype(np.float64) for v in vs]
    with mfto.Batch([(P.mesh.nelx, P.mesh.nely, P.mesh.nelz) for P in problems],
                    [P.fixed for P in problems]) as b:
        b.set_shape(shape)
        Y = torch.zeros(b.n_dof, dtype=dt, device=cuda)
        b.kv(torch.tensor(np.concatenate(Es), dtype=dt, device=cuda),
             torch.tensor(np.concatenate(vs), dtype=dt, device=cuda), Y, form=mfto.FORMS[form])
        got = Y.cpu().numpy().astype(np.float64)
        offs = b.dof_off
    for i, P in enumerate(problems):
        m = P.mesh
        ref = fem.kv(fem.ke_exact(), Es[i], fem.edof_table_fast(m.nelx, m.nely, m.nelz), vs[i],
                     fem.dof_mask(P.fixed))
        gi = got[offs[i]:offs[i + 1]]
        assert np.abs(gi - ref).max() / np.abs(ref).max() <= tol, (i, shape)


def test_batch_ir_mode_rejects_unknown(cuda):
    from paper_2604_18020_gb300 import mfto
    problems = W.uneven_instances(count=2, seed=3, kmin=3, kmax=4)
    with mfto.Batch([(P.mesh.nelx, P.mesh.nely, P.mesh.nelz) for P in problems],
                    [P.fixed for P in problems]) as b:
        with pytest.raises(mfto.MftoError):
            b.set_ir_mode(2)


@pytest.mark.parametrize("mode,inner_tol", [(0, 1e-2), (1, 1e-1)])
def test_batch_solve_and_autotune(cuda, mode, inner_tol):
    """Restarted and continued refinement (each instance keeps its own
    direction) both reach the outer tolerance on every instance."""
    import torch
    from paper_2604_18020_gb300 import mfto
    problems = W.uneven_instances(count=6, seed=12, kmin=3, kmax=8)
    Es, fs = _concat(problems, 300)
    with mfto.Batch([(P.mesh.nelx, P.mesh.nely, P.mesh.nelz) for P in problems],
                    [P.fixed for P in problems]) as b:
        choice, ms = b.autotune(reps=3)
        assert 0 <= choice < 4 and np.all(ms > 0) and ms[choice] == ms.min()
        b.set_ir_mode(mode)
        U = torch.zeros(b.n_dof, dtype=torch.float64, device=cuda)
        sts = b.solve(torch.tensor(np.concatenate(Es), device=cuda),
                      torch.tensor(np.concatenate(fs), device=cuda), U, inner_tol=inner_tol)
        got = U.cpu().numpy()
        offs = b.dof_off
    for i, P in enumerate(problems):
        m = P.mesh
        edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
        fd = fem.dof_mask(P.fixed)
        KE = fem.ke_exact()
        ui = got[offs[i]:offs[i + 1]]
        assert sts[i].status == mfto.OK
        true_rel = np.linalg.norm(fs[i] - fem.kv(KE, Es[i], edof, ui, fd)) / np.linalg.norm(fs[i])
        assert true_rel <= 1.5e-8
        d = fem.jacobi_diag(KE, Es[i], edof, fd)
        u_ref, _ = solve.pcg(lambda v: fem.kv(KE, Es[i], edof, v, fd), d, fs[i],
                             np.zeros(m.n_dof), 1e-10)
        assert abs(fs[i] @ ui - fs[i] @ u_ref) / abs(fs[i] @ u_ref) <= 1e-7


@pytest.mark.parametrize("mode,inner_tol", [(0, 1e-2), (1, 1e-1)])
def test_batch_64_uneven_instances(cuda, mode, inner_tol):
    """The configuration of 64 seeded instances from 16x8x8 to 48x24x24, with
    restarted and continued refinement."""
    import torch
    from paper_2604_18020_gb300 import mfto
    problems = W.uneven_instances(count=64, seed=5)
    Es, fs = _concat(problems, 400)
    with mfto.Batch([(P.mesh.nelx, P.mesh.nely, P.mesh.nelz) for P in problems],
                    [P.fixed for P in problems]) as b:
        b.autotune(reps=2)
        b.set_ir_mode(mode)
        U = torch.zeros(b.n_dof, dtype=torch.float64, device=cuda)
        sts = b.solve(torch.tensor(np.concatenate(Es), device=cuda),
                      torch.tensor(np.concatenate(fs), device=cuda), U, inner_tol=inner_tol)
        got = U.cpu().numpy()
        offs = b.dof_off
    assert all(s.status == mfto.OK and s.rel_residual <= 1e-8 for s in sts)
    for i in [0, 17, 40, 63]:                      # sampled: the oracle's own residual
        P = problems[i]
        m = P.mesh
        ui = got[offs[i]:offs[i + 1]]
        r = fs[i] - fem.kv(fem.ke_exact(), Es[i], fem.edof_table_fast(m.nelx, m.nely, m.nelz), ui,
                           fem.dof_mask(P.fixed))
        assert np.linalg.norm(r) / np.linalg.norm(fs[i]) <= 1.5e-8

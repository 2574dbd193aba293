"""GPU parity of the core hot path against the FP64 CPU oracle, through the
C ABI (libmfto.so via the ctypes binding).

Tolerances (written here, derived in the design notes):
  K.v FP64: relative inf-norm error <= 1e-12;  K.v FP32: <= 1e-5 (inputs
  rounded to FP32 first; the oracle then works in FP64 on the rounded data);
  Jacobi diagonal, compliance, sensitivities: <= 1e-12 relative;
  cone filter: bit-exact (same summation order, no fused multiply-add);
  edof / stencil: bit-exact;  final SIMP compliance: <= 1e-6 relative.
"""
import numpy as np
import pytest

from oracle import fem, filter as cone, simp as osimp, solve
from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MESHES = [(1, 1, 1), (2, 1, 1), (3, 2, 2), (13, 7, 5), (24, 12, 12), (5, 4, 9)]


def _setup(nelx, nely, nelz, face="x0"):
    m = W.Mesh(nelx, nely, nelz)
    fixed = W.fixed_face(m, face)
    return m, fixed, fem.edof_table_fast(nelx, nely, nelz), fem.dof_mask(fixed)


def _rel_inf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


MESHES_BIG = [(40, 30, 9), (17, 13, 33)]   # several tiles and z-chunks, ragged edges


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("shape", MESHES + MESHES_BIG)
@pytest.mark.parametrize("face", ["x0", "z0"])
def test_kv_f64(cuda, shape, face, variant):
    import torch
    from paper_2604_18020_gb300 import mfto
    m, fixed, edof, fd = _setup(*shape, face)
    KE = fem.ke_exact()
    rho = W.rho_random(m, seed=11)
    E = fem.simp_modulus(rho, 3.0)
    v = W.vec_random(m.n_dof, seed=12)
    with mfto.Handle(*shape, fixed) as h:
        h.set_kv_variant(variant)
        y = torch.empty(m.n_dof, dtype=torch.float64, device=cuda)
        h.kv(torch.tensor(E, device=cuda), torch.tensor(v, device=cuda), y)
        got = y.cpu().numpy()
    ref = fem.kv(KE, E, edof, v, fd)
    assert _rel_inf(got, ref) <= 1e-12
    # fixed DOFs return v exactly
    assert np.array_equal(got[fd], v[fd])


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("shape", MESHES + MESHES_BIG)
def test_kv_f32(cuda, shape, variant):
    import torch
    from paper_2604_18020_gb300 import mfto
    m, fixed, edof, fd = _setup(*shape)
    KE = fem.ke_exact()
    E32 = fem.simp_modulus(W.rho_random(m, seed=21), 3.0).astype(np.float32)
    v32 = W.vec_random(m.n_dof, seed=22).astype(np.float32)
    with mfto.Handle(*shape, fixed) as h:
        h.set_kv_variant(variant)
        y = torch.empty(m.n_dof, dtype=torch.float32, device=cuda)
        h.kv(torch.tensor(E32, device=cuda), torch.tensor(v32, device=cuda), y,
             form=mfto.FORM_F32)
        got = y.cpu().numpy().astype(np.float64)
    ref = fem.kv(KE, E32.astype(np.float64), edof, v32.astype(np.float64), fd)
    assert _rel_inf(got, ref) <= 1e-5


@pytest.mark.parametrize("form", ["f64", "f32"])
def test_kv_full_size(cuda, form):
    """120x60x30 (216,000 elements, 686,433 DOFs), the launch configuration
    the benchmark times: the whole output against the oracle."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(120, 60, 30)
    m = P.mesh
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    E = fem.simp_modulus(W.rho_random(m, seed=1), 3.0)
    v = W.vec_random(m.n_dof, seed=2)
    dt, tol = (torch.float64, 1e-12) if form == "f64" else (torch.float32, 1e-5)
    if form == "f32":
        E, v = E.astype(np.float32).astype(np.float64), v.astype(np.float32).astype(np.float64)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        y = torch.empty(m.n_dof, dtype=dt, device=cuda)
        h.kv(torch.tensor(E, dtype=dt, device=cuda), torch.tensor(v, dtype=dt, device=cuda), y,
             form=mfto.FORMS[form])
        got = y.cpu().numpy().astype(np.float64)
    assert _rel_inf(got, fem.kv(fem.ke_exact(), E, edof, v, fd)) <= tol


def test_kv_sampled_at_4_9M_elements(cuda):
    """256x128x150 (4,915,200 elements): sampled outputs, each recomputed by
    the oracle from its own 27-node neighbourhood."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(256, 128, 150, 0.12)
    m = P.mesh
    rng = np.random.default_rng(0)
    E = torch.rand(m.n_elem, dtype=torch.float64, device=cuda, generator=torch.Generator(
        device=cuda).manual_seed(1)) + 0.01
    v = torch.rand(m.n_dof, dtype=torch.float64, device=cuda, generator=torch.Generator(
        device=cuda).manual_seed(2)) * 2 - 1
    with mfto.Handle(256, 128, 150, P.fixed) as h:
        y = torch.empty_like(v)
        h.kv(E, v, y)
        got = y.cpu().numpy()
    Eh, vh = E.cpu().numpy(), v.cpu().numpy()
    KE = fem.ke_exact()
    nx, ny = m.nelx + 1, m.nely + 1
    fixed = fem.dof_mask(P.fixed)
    picks = list(rng.integers(0, m.n_node, 300)) + [0, m.n_node - 1, nx - 1, nx * ny * 75 + 5]
    for n in picks:
        i, j, k = n % nx, (n // nx) % ny, n // (nx * ny)
        acc = np.zeros(3)
        for ce in range(8):
            ei, ej, ek = i - 1 + (ce & 1), j - 1 + ((ce >> 1) & 1), k - 1 + (ce >> 2)
            if not (0 <= ei < m.nelx and 0 <= ej < m.nely and 0 <= ek < m.nelz):
                continue
            e = ei + m.nelx * (ej + m.nely * ek)
            nodes = [(ei + (l & 1)) + nx * ((ej + ((l >> 1) & 1)) + ny * (ek + (l >> 2)))
                     for l in range(8)]
            dofs = np.array([3 * nd + c for nd in nodes for c in range(3)])
            ue = np.where(fixed[dofs], 0.0, vh[dofs])
            ln = (i - ei) + 2 * (j - ej) + 4 * (k - ek)
            acc += Eh[e] * (KE[3 * ln:3 * ln + 3] @ ue)
        ref = np.where(fixed[3 * n:3 * n + 3], vh[3 * n:3 * n + 3], acc)
        assert np.abs(got[3 * n:3 * n + 3] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_kv_contrast_and_bounds(cuda):
    """rho exactly 0 and 1 (E = Emin and E0, contrast 1e9)."""
    import torch
    from paper_2604_18020_gb300 import mfto
    m, fixed, edof, fd = _setup(9, 6, 4)
    rng = np.random.default_rng(5)
    rho = np.where(rng.random(m.n_elem) < 0.5, 0.0, 1.0)
    E = fem.simp_modulus(rho, 3.0)
    v = W.vec_random(m.n_dof, seed=6)
    with mfto.Handle(9, 6, 4, fixed) as h:
        y = torch.empty(m.n_dof, dtype=torch.float64, device=cuda)
        h.kv(torch.tensor(E, device=cuda), torch.tensor(v, device=cuda), y)
        got = y.cpu().numpy()
    assert _rel_inf(got, fem.kv(fem.ke_exact(), E, edof, v, fd)) <= 1e-12


def test_kv_deterministic(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    m, fixed, _, _ = _setup(40, 30, 9)
    E = torch.tensor(fem.simp_modulus(W.rho_random(m, seed=3), 3.0), device=cuda)
    v = torch.tensor(W.vec_random(m.n_dof, seed=4), device=cuda)
    with mfto.Handle(40, 30, 9, fixed) as h:
        outs = []
        for _ in range(3):
            y = torch.empty_like(v)
            h.kv(E, v, y)
            outs.append(y.cpu().numpy())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


@pytest.mark.parametrize("form", ["f64", "f32"])
def test_jacobi_diag(cuda, form):
    import torch
    from paper_2604_18020_gb300 import mfto
    m, fixed, edof, fd = _setup(13, 7, 5)
    E = fem.simp_modulus(W.rho_random(m, seed=7), 3.0)
    ref = fem.jacobi_diag(fem.ke_exact(), E, edof, fd)
    dt = torch.float64 if form == "f64" else torch.float32
    with mfto.Handle(13, 7, 5, fixed) as h:
        d = torch.empty(m.n_dof, dtype=dt, device=cuda)
        h.jacobi_diag(torch.tensor(E, dtype=dt, device=cuda), d, form=mfto.FORMS[form])
        got = d.cpu().numpy().astype(np.float64)
    assert _rel_inf(got, ref) <= (1e-12 if form == "f64" else 1e-6)


@pytest.mark.parametrize("shape,rmin", [((13, 7, 5), 1.5), ((13, 7, 5), 2.0),
                                        ((24, 12, 12), 1.5), ((6, 5, 4), 3.2),
                                        ((1, 1, 1), 1.5)])
def test_filter_bit_exact(cuda, shape, rmin):
    import torch
    from paper_2604_18020_gb300 import mfto
    m, fixed, _, _ = _setup(*shape)
    x = W.rho_random(m, seed=8)
    with mfto.Handle(*shape, fixed, params=mfto.default_params(rmin=rmin)) as h:
        tx = torch.tensor(x, device=cuda)
        y = torch.empty_like(tx)
        h.filter(tx, y, transpose=False)
        fwd = y.cpu().numpy()
        h.filter(tx, y, transpose=True)
        tr = y.cpu().numpy()
    assert np.array_equal(fwd, cone.filter_fwd(x, *shape, rmin))
    assert np.array_equal(tr, cone.filter_T(x, *shape, rmin))


def test_filter_neighbourhoods_exact(cuda):
    """A one-hot input exposes one column of H/W: its support must be the
    oracle's neighbourhood set exactly."""
    import torch
    from paper_2604_18020_gb300 import mfto
    shape, rmin = (7, 6, 5), 2.0
    m, fixed, _, _ = _setup(*shape)
    with mfto.Handle(*shape, fixed, params=mfto.default_params(rmin=rmin)) as h:
        for e in [0, 3, 44, m.n_elem - 1, 100]:
            x = np.zeros(m.n_elem)
            x[e] = 1.0
            tx = torch.tensor(x, device=cuda)
            y = torch.empty_like(tx)
            h.filter(tx, y, transpose=False)
            support = sorted(np.nonzero(y.cpu().numpy())[0].tolist())
            assert support == cone.neighbours(e, *shape, rmin)


def test_compliance_sens(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    m, fixed, edof, fd = _setup(13, 7, 5)
    rho = W.rho_random(m, seed=9)
    u = W.zero_fixed(W.vec_random(m.n_dof, seed=10), fixed)
    c_ref, dc_ref = osimp.compliance_sens(fem.ke_exact(), edof, u, rho, 3.0)
    with mfto.Handle(13, 7, 5, fixed) as h:
        dc = torch.empty(m.n_elem, dtype=torch.float64, device=cuda)
        c = h.compliance_sens(torch.tensor(rho, device=cuda), torch.tensor(u, device=cuda), dc)
        got = dc.cpu().numpy()
    assert abs(c - c_ref) / abs(c_ref) <= 1e-12
    assert _rel_inf(got, dc_ref) <= 1e-12


def test_oc_update(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    m, fixed, _, _ = _setup(24, 12, 12)
    rho = np.clip(W.rho_random(m, seed=13, lo=0.05, hi=0.6), 0, 1)
    dc = -W.rho_random(m, seed=14, lo=1e-4, hi=1.0)
    ref, info = osimp.oc_update(rho, dc, 0.3, 0.2)
    with mfto.Handle(24, 12, 12, fixed) as h:
        out = torch.empty(m.n_elem, dtype=torch.float64, device=cuda)
        st = h.oc_update(torch.tensor(rho, device=cuda), torch.tensor(dc, device=cuda), out)
        got = out.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-9
    assert abs(st.volume - 0.3) <= 1e-8
    assert abs(st.change - info["change"]) <= 1e-9
    assert abs(st.lambda_ - info["lambda"]) / info["lambda"] <= 1e-9
    # move limits and box bounds hold exactly
    assert np.all(got <= np.minimum(1.0, rho + 0.2)) and np.all(got >= np.maximum(0.0, rho - 0.2))


def test_pcg_matches_oracle(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(24, 12, 12)
    m = P.mesh
    edof = fem.edof_table_fast(m.nelx, m.nely, m.nelz)
    fd = fem.dof_mask(P.fixed)
    KE = fem.ke_exact()
    E = fem.simp_modulus(W.rho_random(m, seed=15, lo=0.1, hi=1.0), 3.0)
    d = fem.jacobi_diag(KE, E, edof, fd)
    u_ref, st_ref = solve.pcg(lambda v: fem.kv(KE, E, edof, v, fd), d, P.f,
                              np.zeros(m.n_dof), 1e-8, 10000)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        st = h.pcg(torch.tensor(E, device=cuda), torch.tensor(P.f, device=cuda), u)
        got = u.cpu().numpy()
    assert st.status == mfto.OK
    assert abs(st.iterations - st_ref.iterations) <= 2
    true_rel = np.linalg.norm(P.f - fem.kv(KE, E, edof, got, fd)) / np.linalg.norm(P.f)
    assert true_rel <= 1.5e-8
    c, c_ref = P.f @ got, P.f @ u_ref
    assert abs(c - c_ref) / abs(c_ref) <= 1e-7


def test_pcg_zero_load_and_cap(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(8, 4, 4)
    m = P.mesh
    E = torch.ones(m.n_elem, dtype=torch.float64, device=cuda)
    with mfto.Handle(8, 4, 4, P.fixed, params=mfto.default_params(maxit=6, check_every=4)) as h:
        u = torch.ones(m.n_dof, dtype=torch.float64, device=cuda)
        st = h.pcg(E, torch.zeros(m.n_dof, dtype=torch.float64, device=cuda), u)
        assert st.iterations == 0 and st.status == mfto.OK
        assert torch.count_nonzero(u).item() == 0
        u.zero_()
        st = h.pcg(E, torch.tensor(P.f, device=cuda), u)
        assert st.iterations == 6 and st.status == mfto.NOT_CONVERGED


def test_simp_20_iterations(cuda):
    """24x12x12 cantilever, 20 OC iterations: final compliance within 1e-6."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(24, 12, 12)
    m = P.mesh
    n_it = 20
    _, _, hist = osimp.simp(m.nelx, m.nely, m.nelz, P.f, P.fixed, P.volfrac, P.rmin, n_it)
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed,
                     params=mfto.default_params(volfrac=P.volfrac, rmin=P.rmin)) as h:
        rho = torch.full((m.n_elem,), P.volfrac, dtype=torch.float64, device=cuda)
        u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
        f = torch.tensor(P.f, device=cuda)
        cs = []
        for _ in range(n_it):
            st = h.simp_step(rho, u, f)
            cs.append(st.compliance)
    assert abs(cs[-1] - hist.compliance[-1]) / hist.compliance[-1] <= 1e-6
    assert np.allclose(cs, hist.compliance, rtol=1e-6)


def test_oc_unreachable_target_terminates(cuda):
    """All sensitivities zero: the bisection must stop (bracket collapse) and
    return the lower move limits, like the oracle."""
    import torch
    from paper_2604_18020_gb300 import mfto
    m, fixed, _, _ = _setup(8, 4, 4)
    rho = np.full(m.n_elem, 0.3)
    ref, _ = osimp.oc_update(rho, np.zeros(m.n_elem), 0.3, 0.2)
    with mfto.Handle(8, 4, 4, fixed) as h:
        out = torch.empty(m.n_elem, dtype=torch.float64, device=cuda)
        h.oc_update(torch.tensor(rho, device=cuda), torch.zeros(m.n_elem, dtype=torch.float64,
                                                                device=cuda), out)
        got = out.cpu().numpy()
    assert np.array_equal(got, ref)


def test_kv_f32_after_autotune(cuda):
    """The autotuned launch shape (z-chunk, register budget) of the FP32
    column K.v gives the same result as the default one, bit for bit (the
    tiling changes which CTA computes an element, not the order of any sum),
    and matches the oracle."""
    import torch
    from paper_2604_18020_gb300 import mfto
    shape = (40, 30, 9)
    m, fixed, edof, fd = _setup(*shape)
    KE = fem.ke_exact()
    E32 = fem.simp_modulus(W.rho_random(m, seed=23), 3.0).astype(np.float32)
    v32 = W.vec_random(m.n_dof, seed=24).astype(np.float32)
    with mfto.Handle(*shape, fixed) as h:
        tE, tv = torch.tensor(E32, device=cuda), torch.tensor(v32, device=cuda)
        y0 = torch.empty(m.n_dof, dtype=torch.float32, device=cuda)
        h.kv(tE, tv, y0, form=mfto.FORM_F32)
        nzc, kind, us = h.kv_autotune()
        assert 1 <= nzc <= m.nelz + 1 and kind in (0, 1) and us > 0
        y1 = torch.empty_like(y0)
        h.kv(tE, tv, y1, form=mfto.FORM_F32)
        assert torch.equal(y0, y1)
    ref = fem.kv(KE, E32.astype(np.float64), edof, v32.astype(np.float64), fd)
    assert _rel_inf(y1.cpu().numpy().astype(np.float64), ref) <= 1e-5


@pytest.mark.parametrize("shape", [(40, 30, 9), (17, 13, 33), (1, 1, 1)])
def test_kv_f32_kernel_kinds_bit_identical(cuda, shape):
    """Every FP32 column kernel kind (either register budget) and z-chunk
    gives the same K.v, bit for bit, and it matches the oracle."""
    import torch
    from paper_2604_18020_gb300 import mfto
    m, fixed, edof, fd = _setup(*shape)
    KE = fem.ke_exact()
    E32 = fem.simp_modulus(W.rho_random(m, seed=25), 3.0).astype(np.float32)
    v32 = W.vec_random(m.n_dof, seed=26).astype(np.float32)
    ys = []
    with mfto.Handle(*shape, fixed) as h:
        tE, tv = torch.tensor(E32, device=cuda), torch.tensor(v32, device=cuda)
        for kind in range(2):
            for nzc in (0, 1, 3, m.nelz + 1):
                h.set_kv_shape(nzc, kind)
                y = torch.empty(m.n_dof, dtype=torch.float32, device=cuda)
                h.kv(tE, tv, y, form=mfto.FORM_F32)
                ys.append(y)
    for y in ys[1:]:
        assert torch.equal(ys[0], y)
    ref = fem.kv(KE, E32.astype(np.float64), edof, v32.astype(np.float64), fd)
    assert _rel_inf(ys[0].cpu().numpy().astype(np.float64), ref) <= 1e-5


def test_cg_f32_kernel_kinds_agree(cuda):
    """The mixed solve converges to the same solution with every column
    kernel kind.  The CG K.v outputs are bit-identical; the kinds add the
    p.q products in a different order, which changes the FP32 CG trajectory
    (and so the inner iteration count by a few percent) but not the refined
    solution: compliance within 1e-7 of each other, FP64 residual <= 1e-8."""
    import torch
    from paper_2604_18020_gb300 import mfto
    P = W.cantilever(40, 20, 12)
    m = P.mesh
    E = torch.tensor(fem.simp_modulus(W.rho_random(m, seed=27, lo=0.1, hi=1.0), 3.0), device=cuda)
    f = torch.tensor(P.f, device=cuda)
    out = []
    with mfto.Handle(m.nelx, m.nely, m.nelz, P.fixed) as h:
        h.set_ir_mode(mfto.IR_CONTINUE)
        for kind in range(2):
            h.set_kv_shape(0, kind)
            u = torch.zeros(m.n_dof, dtype=torch.float64, device=cuda)
            st = h.ir_solve(E, f, u, inner_tol=0.1)
            assert st.status == mfto.OK and st.rel_residual <= 1e-8
            out.append((st.inner_iterations, float((f * u).sum())))
    its = [o[0] for o in out]
    for it, c in out[1:]:
        assert abs(it - its[0]) <= 0.15 * its[0], its
        assert abs(c - out[0][1]) <= 1e-7 * abs(out[0][1])

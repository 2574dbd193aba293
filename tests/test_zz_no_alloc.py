"""The entry point for callers that cannot allocate device memory
(mfto_compliance_sens_noalloc) must give what the handle-based
mfto_compliance_sens gives, call after call, although its only scratch is a
static device array shared by every call.  Collected last on purpose, so a
run that stops at the first failure has already run everything else."""
import numpy as np
import pytest

from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _inputs(m, seed, cuda):
    import torch
    rho = torch.tensor(W.rho_random(m, seed=seed, lo=0.05, hi=1.0), device=cuda)
    u = torch.tensor(W.zero_fixed(W.vec_random(m.n_dof, seed=seed + 1),
                                  W.fixed_face(m, "x0")), device=cuda)
    return rho, u


def test_noalloc_matches_handle_entry_point(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    m = W.Mesh(40, 20, 12)
    fixed = W.fixed_face(m, "x0")
    with mfto.Handle(m.nelx, m.nely, m.nelz, fixed) as h:
        for call, seed in enumerate([3, 3, 17]):          # two identical calls, then new data
            rho, u = _inputs(m, seed, cuda)
            dc_ref = torch.empty(m.n_elem, dtype=torch.float64, device=cuda)
            c_ref = h.compliance_sens(rho, u, dc_ref)
            dc = torch.full((m.n_elem,), float("nan"), dtype=torch.float64, device=cuda)
            c = mfto.compliance_sens_noalloc(m.nelx, m.nely, m.nelz, rho, u, dc)
            assert abs(c - c_ref) <= 1e-12 * abs(c_ref), (call, c, c_ref)
            ref, got = dc_ref.cpu().numpy(), dc.cpu().numpy()
            assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), call


def test_noalloc_two_calls_in_a_row_and_capacity(cuda):
    from paper_2604_18020_gb300 import mfto
    m = W.Mesh(24, 12, 12)
    rho, u = _inputs(m, 5, cuda)
    c1 = mfto.compliance_sens_noalloc(m.nelx, m.nely, m.nelz, rho, u)
    c2 = mfto.compliance_sens_noalloc(m.nelx, m.nely, m.nelz, rho, u)
    assert c1 == c2                      # the ticket is cleared: no stale reduction state
    big = W.Mesh(128, 64, 65)            # 532,480 elements > 524,288
    import torch
    with pytest.raises(mfto.MftoError) as err:
        mfto.compliance_sens_noalloc(big.nelx, big.nely, big.nelz,
                                     torch.zeros(big.n_elem, dtype=torch.float64, device=cuda),
                                     torch.zeros(big.n_dof, dtype=torch.float64, device=cuda))
    assert err.value.code == mfto.TOO_LARGE


def test_noalloc_at_capacity(cuda):
    """Exactly 524,288 elements (128 x 64 x 64): every partial-sum slot and the
    last-block ticket in use; two calls in a row against the handle's result."""
    import torch
    from paper_2604_18020_gb300 import mfto
    m = W.Mesh(128, 64, 64)
    assert m.n_elem == mfto.NOALLOC_MAX_ELEMENTS
    fixed = W.fixed_face(m, "x0")
    rho, u = _inputs(m, 23, cuda)
    with mfto.Handle(m.nelx, m.nely, m.nelz, fixed) as h:
        dc_ref = torch.empty(m.n_elem, dtype=torch.float64, device=cuda)
        c_ref = h.compliance_sens(rho, u, dc_ref)
    ref = dc_ref.cpu().numpy()
    for call in range(2):
        dc = torch.full((m.n_elem,), float("nan"), dtype=torch.float64, device=cuda)
        c = mfto.compliance_sens_noalloc(m.nelx, m.nely, m.nelz, rho, u, dc)
        assert abs(c - c_ref) <= 1e-12 * abs(c_ref), (call, c, c_ref)
        assert np.abs(dc.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max(), call

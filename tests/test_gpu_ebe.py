"""K.v over an arbitrary element DOF table (the synthetic microbenchmark of
Sec. 5, Tab. profiling): the staged FP64 pipeline and the fused FP64 / FP32
kernels against the oracle's gather-contract-scatter, on random and on
structured connectivity, with ragged element counts (not a multiple of the
contraction's 64-element tile or of a CTA), and the out-of-range index
check."""
import numpy as np
import pytest

from oracle import fem
from paper_2604_18020_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# FP64: the atomics only reorder the sums (<= 24 x 8 terms per DOF);
# FP32: rounding of the contraction and the sums in single precision
TOL = {0: 1e-13, 1: 1e-13, 2: 2e-6}


def _run(variant, edof, E, v, n_dof):
    import torch
    from paper_2604_18020_gb300 import mfto
    dt = torch.float32 if variant == 2 else torch.float64
    dev = torch.device("cuda:0")
    with mfto.Ebe(edof.shape[0], n_dof) as e:
        y = torch.empty(n_dof, dtype=dt, device=dev)
        ms = e.kv(variant, torch.tensor(edof, device=dev), torch.tensor(E, dtype=dt, device=dev),
                  torch.tensor(v, dtype=dt, device=dev), y, timed=True)
        assert all(t > 0 for t in ms) and len(ms) == (3 if variant == 0 else 1)
        assert e.launch_count() == (3 if variant == 0 else 1)
        return y.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("shape,structured", [((9, 5, 3), False), ((13, 7, 5), False),
                                              ((10, 6, 4), True), ((40, 20, 10), False)])
def test_ebe_kv_matches_oracle(cuda, variant, shape, structured):
    m = W.Mesh(*shape)
    edof = fem.edof_table_fast(*shape).astype(np.int32) if structured else W.edof_random(m, 42)
    E = W.rho_random(m, seed=1)
    v = W.vec_random(m.n_dof, seed=2)
    ref = fem.kv_unmasked(fem.ke_exact(), E, edof.astype(np.int64), v)
    got = _run(variant, edof, E, v, m.n_dof)
    assert np.abs(got - ref).max() <= TOL[variant] * np.abs(ref).max()


def test_ebe_rejects_out_of_range_index(cuda):
    import torch
    from paper_2604_18020_gb300 import mfto
    m = W.Mesh(4, 3, 2)
    edof = W.edof_random(m, 7)
    edof[5, 7] = m.n_dof                      # one past the end: skipped, reported
    dev = torch.device("cuda:0")
    with mfto.Ebe(m.n_elem, m.n_dof) as e:
        y = torch.empty(m.n_dof, dtype=torch.float64, device=dev)
        with pytest.raises(mfto.MftoError):
            e.kv(1, torch.tensor(edof, device=dev),
                 torch.ones(m.n_elem, dtype=torch.float64, device=dev),
                 torch.ones(m.n_dof, dtype=torch.float64, device=dev), y)


@pytest.mark.parametrize("variant", [0, 2])
def test_ebe_kv_full_size(cuda, variant):
    """The microbenchmark's largest configuration (200x100x50 element and
    node counts, 1,000,000 elements, random table seed 42), in the launch
    configuration the benchmark times: the whole output against the oracle."""
    m = W.Mesh(200, 100, 50)
    edof = W.edof_random(m, 42)
    E = W.rho_random(m, seed=1)
    v = W.vec_random(m.n_dof, seed=2)
    if variant == 2:
        E = E.astype(np.float32).astype(np.float64)
        v = v.astype(np.float32).astype(np.float64)
    ref = fem.kv_unmasked(fem.ke_exact(), E, edof.astype(np.int64), v)
    got = _run(variant, edof, E, v, m.n_dof)
    assert np.abs(got - ref).max() <= TOL[variant] * np.abs(ref).max()


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_ebe_single_element(cuda, variant):
    m = W.Mesh(1, 1, 1)
    edof = fem.edof_table_fast(1, 1, 1).astype(np.int32)
    E = np.array([0.3])
    v = W.vec_random(m.n_dof, seed=8)
    ref = fem.kv_unmasked(fem.ke_exact(), E, edof.astype(np.int64), v)
    got = _run(variant, edof, E, v, m.n_dof)
    assert np.abs(got - ref).max() <= TOL[variant] * np.abs(ref).max()

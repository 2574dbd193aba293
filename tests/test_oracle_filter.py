"""Pins of the oracle's cone filter: closed-form weights, brute-force dense
filter matrix, invariants (no GPU)."""
import math

import numpy as np
import pytest

from oracle import filter as cone
from paper_2604_18020_gb300 import workloads as W


def test_stencil_closed_form_rmin_15():
    st = cone.stencil(1.5)
    assert len(st) == 19               # centre + 6 faces + 12 edges; corners have w < 0
    w = {(dx, dy, dz): wt for dx, dy, dz, wt in st}
    assert w[(0, 0, 0)] == 1.5
    assert w[(1, 0, 0)] == 0.5 and w[(0, 0, -1)] == 0.5
    assert w[(1, 1, 0)] == 1.5 - math.sqrt(2.0)
    assert (1, 1, 1) not in w


def test_stencil_closed_form_rmin_2():
    st = cone.stencil(2.0)
    assert len(st) == 27
    w = {(dx, dy, dz): wt for dx, dy, dz, wt in st}
    assert w[(0, 0, 0)] == 2.0 and w[(0, 1, 0)] == 1.0
    assert w[(1, 0, 1)] == 2.0 - math.sqrt(2.0)
    assert w[(-1, 1, -1)] == 2.0 - math.sqrt(3.0)


@pytest.mark.parametrize("shape,rmin", [((4, 3, 2), 1.5), ((3, 3, 3), 2.0), ((5, 2, 3), 2.7),
                                        ((1, 1, 1), 1.5), ((6, 1, 1), 3.0)])
def test_filter_equals_dense_brute_force(shape, rmin):
    m = W.Mesh(*shape)
    H = cone.filter_matrix_dense(*shape, rmin)
    x = W.rho_random(m, seed=1)
    y = W.rho_random(m, seed=2)
    assert np.allclose(cone.filter_fwd(x, *shape, rmin), H @ x / H.sum(axis=1), rtol=1e-14)
    assert np.allclose(cone.filter_T(y, *shape, rmin), H.T @ (y / H.sum(axis=1)), rtol=1e-14)
    assert np.array_equal(H, H.T)
    for e in range(m.n_elem):
        assert cone.neighbours(e, *shape, rmin) == sorted(np.nonzero(H[e])[0].tolist())


def test_filter_preserves_uniform_field_and_adjoint():
    shape, rmin = (7, 5, 4), 2.0
    m = W.Mesh(*shape)
    assert np.allclose(cone.filter_fwd(np.full(m.n_elem, 0.37), *shape, rmin), 0.37,
                       rtol=1e-15, atol=0)
    x, y = W.rho_random(m, seed=3), W.rho_random(m, seed=4)
    a = cone.filter_fwd(x, *shape, rmin) @ y
    b = x @ cone.filter_T(y, *shape, rmin)
    assert abs(a - b) <= 1e-14 * abs(a)


def test_rmin_below_one_is_identity():
    shape = (4, 3, 2)
    x = W.rho_random(W.Mesh(*shape), seed=5)
    assert len(cone.stencil(0.9)) == 1
    assert np.allclose(cone.filter_fwd(x, *shape, 0.9), x, rtol=2e-16, atol=0)

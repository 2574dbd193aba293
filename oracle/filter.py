"""Oracle: cone density filter and its transpose.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).

Paper passage: Sec. 3.1 -- raw densities rho_e are smoothed by a cone filter
of radius r_min to give rho_bar_e (density-filter pipeline).  The paper gives
no formula; the reading used on both sides is the standard cone filter:

  rho_bar_e = sum_i w_ei rho_i / W_e,   W_e = sum_i w_ei,
  w_ei = max(0, r_min - |c_e - c_i|),

with element centres on the unit grid, the neighbourhood all elements i with
|delta|_inf <= ceil(r_min) - 1 and w_ei > 0, truncated at the domain boundary
(no padding, no mirroring), and the weight computed in FP64 as
r_min - sqrt(dx^2 + dy^2 + dz^2) with integer offsets.  The sensitivity chain
uses the transpose: dc/drho_i = sum_e w_ei (dc/drho_bar_e) / W_e.
"""
from __future__ import annotations

import math

import numpy as np


def stencil(rmin):
    """(dx, dy, dz, w) for every offset with positive weight, in the order
    dz, dy, dx ascending (dx fastest)."""
    R = int(math.ceil(rmin)) - 1
    out = []
    for dz in range(-R, R + 1):
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                w = rmin - math.sqrt(dx * dx + dy * dy + dz * dz)
                if w > 0.0:
                    out.append((dx, dy, dz, w))
    return out


def neighbours(e, nelx, nely, nelz, rmin):
    """Sorted element indices in the truncated neighbourhood of e."""
    i, j, k = e % nelx, (e // nelx) % nely, e // (nelx * nely)
    idx = []
    for dx, dy, dz, _ in stencil(rmin):
        ii, jj, kk = i + dx, j + dy, k + dz
        if 0 <= ii < nelx and 0 <= jj < nely and 0 <= kk < nelz:
            idx.append(ii + nelx * (jj + nely * kk))
    return sorted(idx)


def filter_matrix_dense(nelx, nely, nelz, rmin):
    """Dense weight matrix H[e, i] = w_ei (tiny meshes only)."""
    n = nelx * nely * nelz
    H = np.zeros((n, n))
    for e in range(n):
        i, j, k = e % nelx, (e // nelx) % nely, e // (nelx * nely)
        for dx, dy, dz, w in stencil(rmin):
            ii, jj, kk = i + dx, j + dy, k + dz
            if 0 <= ii < nelx and 0 <= jj < nely and 0 <= kk < nelz:
                H[e, ii + nelx * (jj + nely * kk)] = w
    return H


def _shifted_sum(x3, nelx, nely, nelz, rmin, weight_only=False):
    """sum_i w_ei x_i over the truncated neighbourhood, for all e at once
    (x3 shaped [nelz, nely, nelx])."""
    acc = np.zeros((nelz, nely, nelx))
    for dx, dy, dz, w in stencil(rmin):
        # target slice e, source slice e + d, both clipped to the domain
        tz = slice(max(0, -dz), nelz - max(0, dz))
        ty = slice(max(0, -dy), nely - max(0, dy))
        tx = slice(max(0, -dx), nelx - max(0, dx))
        sz = slice(max(0, dz), nelz - max(0, -dz))
        sy = slice(max(0, dy), nely - max(0, -dy))
        sx = slice(max(0, dx), nelx - max(0, -dx))
        if weight_only:
            acc[tz, ty, tx] += w
        else:
            acc[tz, ty, tx] += w * x3[sz, sy, sx]
    return acc


def row_sums(nelx, nely, nelz, rmin):
    """W_e for every element, element order."""
    return _shifted_sum(None, nelx, nely, nelz, rmin, weight_only=True).reshape(-1)


def filter_fwd(x, nelx, nely, nelz, rmin):
    """rho_bar = H x / W."""
    x3 = np.asarray(x, dtype=np.float64).reshape(nelz, nely, nelx)
    num = _shifted_sum(x3, nelx, nely, nelz, rmin).reshape(-1)
    return num / row_sums(nelx, nely, nelz, rmin)


def filter_T(y, nelx, nely, nelz, rmin):
    """H^T (y / W); H is symmetric (w_ei = w_ie and the truncation is
    symmetric), so this is H (y / W)."""
    y = np.asarray(y, dtype=np.float64) / row_sums(nelx, nely, nelz, rmin)
    return _shifted_sum(y.reshape(nelz, nely, nelx), nelx, nely, nelz,
                        rmin).reshape(-1)

"""Pins of the oracle's three-field step and continuation protocol (no GPU):
the projection's closed-form values and limits, its derivative and the full
sensitivity chain against central finite differences, the schedule against
the paper's printed table, and the restart / selection rules on synthetic
sequences."""
import json
from pathlib import Path

import numpy as np
import pytest

from oracle import fem, filter as cone, protocol as proto, simp, solve
from paper_2604_18020_gb300 import workloads as W

GOLDEN = json.loads((Path(__file__).parent / "golden" / "simp120_schedule.json").read_text())


@pytest.mark.parametrize("beta", [1.0, 4.0, 16.0, 32.0])
def test_heaviside_fixed_points_and_slope(beta):
    x = np.array([0.0, 0.5, 1.0])
    h = proto.heaviside(x, beta)
    assert abs(h[0]) <= 1e-15 and abs(h[1] - 0.5) <= 1e-15 and abs(h[2] - 1.0) <= 1e-15
    # slope at the threshold: beta / (2 tanh(beta / 2)) for eta = 1/2
    assert abs(proto.heaviside_deriv(0.5, beta) - beta / (2.0 * np.tanh(beta / 2.0))) <= 1e-12 * beta
    xs = np.linspace(0.0, 1.0, 101)
    assert np.all(np.diff(proto.heaviside(xs, beta)) > 0.0)


def test_heaviside_small_beta_is_identity():
    xs = np.linspace(0.0, 1.0, 11)
    assert np.abs(proto.heaviside(xs, 1e-6) - xs).max() <= 1e-9


@pytest.mark.parametrize("beta", [1.0, 8.0, 32.0])
def test_heaviside_derivative_central_differences(beta):
    xs = np.linspace(0.01, 0.99, 37)
    h = 1e-6
    fd = (proto.heaviside(xs + h, beta) - proto.heaviside(xs - h, beta)) / (2 * h)
    assert np.abs(fd - proto.heaviside_deriv(xs, beta)).max() <= 1e-6 * max(1.0, beta)


def _c_of(rho, shape, f, fixed_nodes, rmin, beta, penal):
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(*shape)
    fd = fem.dof_mask(fixed_nodes)
    rp = proto.heaviside(cone.filter_fwd(rho, *shape, rmin), beta)
    E = fem.simp_modulus(rp, penal)
    u = solve.dense_solve(fem.assemble_masked(KE, E, edof, f.size, fd), f)
    return float(f @ u), u, rp


def test_projected_sensitivities_central_differences():
    shape, rmin, beta, penal = (3, 2, 2), 1.5, 4.0, 3.5
    P = W.cantilever(*shape)
    rho = W.rho_random(P.mesh, seed=8, lo=0.3, hi=0.9)
    KE = fem.ke_exact()
    edof = fem.edof_table_fast(*shape)
    _, u, rp = _c_of(rho, shape, P.f, P.fixed, rmin, beta, penal)
    rb = cone.filter_fwd(rho, *shape, rmin)
    _, dc_phys = simp.compliance_sens(KE, edof, u, rp, penal)
    dc = cone.filter_T(dc_phys * proto.heaviside_deriv(rb, beta), *shape, rmin)
    h = 1e-6
    for e in range(P.mesh.n_elem):
        a, b = rho.copy(), rho.copy()
        a[e] += h
        b[e] -= h
        fd = (_c_of(a, shape, P.f, P.fixed, rmin, beta, penal)[0]
              - _c_of(b, shape, P.f, P.fixed, rmin, beta, penal)[0]) / (2 * h)
        assert abs(fd - dc[e]) <= 1e-6 * max(1.0, abs(dc[e]))


def test_schedule_matches_the_paper():
    phases = [(p["first"], p["last"], p["penal"], p["beta"], p["move"], p["r_min_target"])
              for p in GOLDEN["phases"]]
    assert phases == proto.SCHEDULE_120
    assert GOLDEN["restart_factor"] == proto.RESTART_FACTOR
    assert GOLDEN["select_min_penal"] == proto.SELECT_MIN_PENAL
    assert GOLDEN["select_max_grayness"] == proto.SELECT_MAX_GRAY
    r0 = 1.5
    # phase values, held or ramped linearly to each target at the phase's end
    assert proto.phase_params(1, r0) == (1.5, 1.0, 0.20, 1.5)
    assert proto.phase_params(15, r0) == (1.5, 1.0, 0.20, 1.5)
    p, b, m, r = proto.phase_params(16, r0)
    assert (p, b, m) == (3.5, 4.0, 0.15) and abs(r - (1.5 - 0.15 / 25)) <= 1e-15
    assert abs(proto.phase_params(40, r0)[3] - 1.35) <= 1e-15
    p, b, m, r = proto.phase_params(41, r0)
    assert (p, b, m) == (4.5, 16.0, 0.08) and abs(r - (1.35 - 0.10 / 25)) <= 1e-15
    assert abs(proto.phase_params(65, r0)[3] - 1.25) <= 1e-15
    p, b, m, r = proto.phase_params(66, r0)
    assert (p, b, m) == (4.5, 32.0, 0.05) and abs(r - (1.25 - 0.05 / 55)) <= 1e-15
    assert abs(proto.phase_params(120, r0)[3] - 1.20) <= 1e-15
    rs = [proto.phase_params(i, r0)[3] for i in range(1, 121)]
    assert all(b <= a + 1e-15 for a, b in zip(rs, rs[1:]))


def test_restart_and_selection_rules():
    sel = None
    # ineligible iterates (p < 3, or gray >= 0.25) never become selected
    assert proto.select_and_restart(10.0, 1.5, 0.1, sel) == (False, False)
    assert proto.select_and_restart(10.0, 3.5, 0.3, sel) == (False, False)
    assert proto.select_and_restart(10.0, 3.5, 0.2, sel) == (False, True)
    sel = 10.0
    assert proto.select_and_restart(9.0, 3.5, 0.2, sel) == (False, True)      # better
    assert proto.select_and_restart(11.0, 3.5, 0.2, sel) == (False, False)    # worse, < 1.12x
    assert proto.select_and_restart(11.3, 3.5, 0.2, sel) == (True, False)     # > 1.12x: restart
    assert proto.select_and_restart(11.3, 1.5, 0.9, sel) == (True, False)     # restart whatever p


def test_protocol_runs_and_selects_a_valid_iterate():
    """A short run (the first 45 iterations of the schedule) of the oracle on
    a small cantilever: the selected iterate is eligible, has the lowest
    compliance among eligible iterates, and the volume constraint holds."""
    P = W.cantilever(12, 6, 6)
    m = P.mesh
    res = proto.protocol(m.nelx, m.nely, m.nelz, P.f, P.fixed, P.volfrac, P.rmin, n_iter=45)
    assert len(res.compliance) == 45
    elig = [i for i in range(45) if proto.phase_params(i + 1, P.rmin)[0] >= 3.0
            and res.grayness[i] < 0.25]
    if res.selected_iteration:
        assert res.selected_iteration - 1 in elig
        assert res.selected_compliance == min(res.compliance[i] for i in elig)
        assert abs(res.selected_rho.mean() - P.volfrac) <= 1e-8 or res.selected_iteration == 1

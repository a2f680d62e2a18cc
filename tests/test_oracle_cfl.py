"""Pins of the oracle's fixed-CFL time step and Kim-Moin pressure update."""
import math

import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1812_01178_gb300 import inputs as I


def _grid(nx=8, ny=6, nz=4):
    case, *_ = I.small_channel(nx, ny, nz, seed=1)
    return case, O.Grid.from_case(case)


def test_rate_brute_force_on_a_tiny_grid():
    """Per-cell loop in plain Python over every cell of a 4x3x4 grid with random velocities."""
    case, g = _grid(4, 3, 4)
    rng = np.random.default_rng(0)
    u = rng.standard_normal((4, 3, 4))
    v = rng.standard_normal((4, 4, 4))
    v[:, 0] = 0
    v[:, -1] = 0
    w = rng.standard_normal((4, 3, 4))
    best = 0.0
    for k in range(4):
        for j in range(3):
            dy = case.yf[j + 1] - case.yf[j]
            for i in range(4):
                vc = 0.5 * (v[k, j, i] + v[k, j + 1, i])
                best = max(best, abs(u[k, j, i]) / g.dx + abs(vc) / dy + abs(w[k, j, i]) / g.dz)
    assert O.convective_rate(g, u, v, w) == pytest.approx(best, rel=1e-15)


def test_poiseuille_rate_and_constant_dt():
    """Steady laminar Poiseuille flow: the rate is 1.5 (1 - yc^2)max / dx, so a fixed-CFL run keeps
    dt = cfl dx / (1.5 (1 - yc^2)max) on every step."""
    case, u, v, w, p = I.laminar_channel(16, 12, 8, amp=0.0)
    g = O.Grid.from_case(case)
    yc = 0.5 * (case.yf[1:] + case.yf[:-1])
    rate = 1.5 * float(np.max(1.0 - yc * yc)) / g.dx
    assert O.convective_rate(g, u, v, w) == pytest.approx(rate, rel=1e-14)
    s, dts = O.step_cfl(g, dict(u=u, v=v, w=w, p=p), 0.5, case.re, case.fx, nsteps=3)
    np.testing.assert_allclose(dts, 0.5 / rate, rtol=1e-12)


def test_step_cfl_hits_the_target_each_step():
    case, u, v, w, p = I.small_channel(16, 9, 8, seed=4)
    g = O.Grid.from_case(case)
    u, v, w = O.make_divergence_free(g, u, v, w)
    state = dict(u=u, v=v, w=w, p=p)
    s, dts = O.step_cfl(g, state, 0.4, case.re, case.fx, nsteps=2)
    assert dts[0] * O.convective_rate(g, u, v, w) == pytest.approx(0.4, rel=1e-15)
    s1 = O.step(g, state, dts[0], case.re, case.fx, 1)
    assert dts[1] * O.convective_rate(g, s1["u"], s1["v"], s1["w"]) == pytest.approx(0.4, rel=1e-15)
    assert dts[0] != dts[1]


@pytest.mark.parametrize("bl", [False, True])
def test_kim_moin_correction_is_minus_beta_times_the_poisson_rhs(bl):
    """One sub-step: the velocities equal those of the plain update, and the pressures differ by
    -beta_k b with b = D u*/(alpha_k dt) the Poisson right-hand side, built here from the RHS and
    ADI pieces (so D G phi = b holds to round-off)."""
    k = 0
    if bl:
        case, u, v, w, p, bnd = I.boundary_layer(16, 10, 8, seed=2, amp=0.05, re=50.0)
        g = O.Grid.from_case(case)
        u, v, w, bnd = O.make_divergence_free_bl(g, u, v, w, bnd)
        st = dict(u=u, v=v, w=w, p=p, bl=bnd)
        a = O.substep_bl(g, st, k, case.dt, case.re, case.fx, case.u_conv)
        b = O.substep_bl(g, st, k, case.dt, case.re, case.fx, case.u_conv, pressure="kim_moin")
        r, _ = O.rhs_bl(g, u, v, w, p, None, bnd, k, case.dt, case.re, case.fx)
        scale = O.RK3_ALPHA[k] * case.dt
        beta = scale / case.re / 2.0
        bl_new, inc = O.outflow_update(g, u, v, w, bnd, scale, case.u_conv)
        us = []
        for comp, (rc, ic) in enumerate(zip(r, (inc["u_out"], inc["v_out"], inc["w_out"]))):
            x = O.adi_sweep_x_bl(g, rc, comp, beta, ic)
            x = O.adi_sweep(g, x, 1, comp, beta)
            us.append((u, v, w)[comp] + O.adi_sweep(g, x, 2, comp, beta))
        bl_new["u_out"] = O.flux_correct_outflow(g, u[:, :, 0], bl_new["u_out"])
        rhs = O.divergence_bl(g, *us, bl_new) / scale
    else:
        case, u, v, w, p = I.small_channel(16, 10, 8, seed=2, re=50.0)
        g = O.Grid.from_case(case)
        u, v, w = O.make_divergence_free(g, u, v, w)
        st = dict(u=u, v=v, w=w, p=p)
        a = O.substep(g, st, k, case.dt, case.re, case.fx)
        b = O.substep(g, st, k, case.dt, case.re, case.fx, pressure="kim_moin")
        r, _ = O.rhs(g, u, v, w, p, None, k, case.dt, case.re, case.fx)
        scale = O.RK3_ALPHA[k] * case.dt
        beta = scale / case.re / 2.0
        du, dv, dw = O.adi_solve(g, r, beta)
        rhs = O.divergence(g, u + du, v + dv, w + dw) / scale
    for q in ("u", "v", "w"):
        assert np.array_equal(a[q], b[q])
    dp = b["p"] - a["p"]
    assert np.abs(rhs).max() > 1.0  # a real correction
    np.testing.assert_allclose(dp, -beta * rhs, rtol=0, atol=1e-12 * beta * np.abs(rhs).max())


def test_kim_moin_is_the_plain_update_without_viscosity():
    """beta_k = 0 at Re = inf: both updates give the same pressure."""
    case, u, v, w, p = I.small_channel(16, 9, 8, seed=3)
    g = O.Grid.from_case(case)
    st = dict(u=u, v=v, w=w, p=p)
    a = O.step(g, st, case.dt, float("inf"), case.fx, 1)
    b = O.step(g, st, case.dt, float("inf"), case.fx, 1, pressure="kim_moin")
    assert np.array_equal(a["p"], b["p"])


def test_rate_of_a_uniform_stream_in_minus_x():
    """u = -U everywhere (v = w = 0): the rate is |U| / dx whatever the sign."""
    case, g = _grid(8, 6, 4)
    u = np.full((g.nz, g.ny, g.nx), -2.5)
    v = np.zeros((g.nz, g.ny + 1, g.nx))
    w = np.zeros((g.nz, g.ny, g.nx))
    assert O.convective_rate(g, u, v, w) == pytest.approx(2.5 / g.dx, rel=1e-15)

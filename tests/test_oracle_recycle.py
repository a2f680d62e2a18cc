"""Pins of the oracle's recycling inflow (the rescaling method of Lund, Wu & Squires 1998)."""
import math

import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1812_01178_gb300 import inputs as I


def _grid(nx=16, ny=24, nz=8):
    case, u, v, w, p, bl = I.boundary_layer(nx, ny, nz, amp=0.05, seed=2, re=300.0)
    return case, O.Grid.from_case(case), u, v, w, p, bl


def test_weight_function_ends_and_monotone():
    assert O.lund_weight(0.0) == 0.0
    assert O.lund_weight(1.0) == 1.0
    assert O.lund_weight(3.0) == 1.0
    eta = np.linspace(0, 1, 201)
    assert np.all(np.diff(O.lund_weight(eta)) >= 0)
    assert O.lund_weight(0.2) == pytest.approx(0.5)   # the inflection point b


def test_identity_when_the_thicknesses_agree():
    """gamma = 1 and delta_rec = delta_inl: both rescalings sample the plane at its own heights,
    so the inflow planes are the recycle plane (v with its wall and top rows)."""
    case, g, u, v, w, p, bl = _grid()
    rng = np.random.default_rng(1)
    u_r = rng.standard_normal((g.nz, g.ny))
    v_r = rng.standard_normal((g.nz, g.ny + 1))
    v_r[:, 0] = 0
    v_r[:, -1] = 0
    w_r = rng.standard_normal((g.nz, g.ny))
    ui, vi, wi = O.rescale_inflow(g, u_r, v_r, w_r, 1.0, 2.5, 2.5)
    np.testing.assert_allclose(ui, u_r, rtol=0, atol=1e-14)
    np.testing.assert_allclose(vi, v_r, rtol=0, atol=1e-14)
    np.testing.assert_allclose(wi, w_r - w_r.mean(axis=0), rtol=0, atol=1e-14)


@pytest.mark.parametrize("gamma,drec,dinl", [(1.03, 3.0, 2.4), (0.97, 2.0, 2.4)])
def test_linear_mean_profile_closed_form(gamma, drec, dinl):
    """U_rec = a y, spanwise uniform (no fluctuations): linear interpolation is exact, so the inlet
    mean is (1 - W) gamma^2 a y + W (gamma a y delta_rec / delta_inl + 1 - gamma) in closed form
    wherever the sampled heights stay below the top centre.  With gamma < 1 and delta_rec <
    delta_inl the rows nearest the wall sample below the first centre, between it and the wall
    value U = 0 (no slip), where a y is still exact."""
    case, g, u, v, w, p, bl = _grid(ny=32)
    a = 0.05
    u_r = np.broadcast_to(a * g.yc, (g.nz, g.ny)).copy()
    v_r = np.zeros((g.nz, g.ny + 1))
    w_r = np.zeros((g.nz, g.ny))
    ui, vi, wi = O.rescale_inflow(g, u_r, v_r, w_r, gamma, drec, dinl)
    y = g.yc
    ok = (gamma * y <= g.yc[-1]) & (drec / dinl * y <= g.yc[-1])
    W = O.lund_weight(y / dinl)
    expect = (1 - W) * gamma * gamma * a * y + W * (gamma * a * y * drec / dinl + 1 - gamma)
    np.testing.assert_allclose(ui[:, ok], np.broadcast_to(expect[ok], (g.nz, ok.sum())), rtol=0, atol=1e-14)
    assert not np.any(wi) and not np.any(vi)


def test_delta99_of_a_tanh_profile():
    yc = np.linspace(0.01, 5.0, 400)
    s = 1.3
    d = O.delta99(yc, np.tanh(s * yc))
    assert d == pytest.approx(math.atanh(0.99) / s, rel=1e-4)


def test_fluctuations_scale_with_gamma_in_the_outer_layer():
    """Above delta_inl (W = 1) the inlet fluctuation is gamma times the plane's fluctuation sampled
    at y delta_rec / delta_inl."""
    case, g, u, v, w, p, bl = _grid(ny=40)
    rng = np.random.default_rng(3)
    u_r = 1.0 + 0.1 * rng.standard_normal((g.nz, g.ny))
    v_r = np.zeros((g.nz, g.ny + 1))
    w_r = 0.1 * rng.standard_normal((g.nz, g.ny))
    gamma, drec, dinl = 0.97, 1.0, 1.0
    ui, vi, wi = O.rescale_inflow(g, u_r, v_r, w_r, gamma, drec, dinl)
    top = g.yc > dinl
    wp = w_r - w_r.mean(axis=0)
    np.testing.assert_allclose(wi[:, top], gamma * wp[:, top], rtol=0, atol=1e-14)
    up = u_r - u_r.mean(axis=0)
    np.testing.assert_allclose(ui[:, top] - ui[:, top].mean(axis=0), gamma * up[:, top], rtol=0, atol=1e-13)


def test_recycled_steps_keep_divergence_and_mass_balance():
    case, g, u, v, w, p, bl = _grid(16, 12, 8)
    u, v, w, bl = O.make_divergence_free_bl(g, u, v, w, bl)
    s = O.step_bl_recycled(g, dict(u=u, v=v, w=w, p=p, bl=bl), case.dt, case.re, case.fx, 10, 1.0, nsteps=2)
    assert np.abs(O.divergence_bl(g, s["u"], s["v"], s["w"], s["bl"])).max() < 1e-11
    wgt = g.dy[None, :] * g.dz
    assert abs((s["u"][:, :, 0] * wgt).sum() - (s["bl"]["u_out"] * wgt).sum()) < 1e-11
    assert not np.array_equal(s["u"][:, :, 0], u[:, :, 0])


def test_recycle_face_values_of_v_and_w_are_centre_averages():
    """v and w live at x-centres; on the recycle face x = i_r dx they are the averages of the centres
    i_r - 1 and i_r.  With v = x_c (linear in x, exact under averaging), equal thicknesses
    (gamma = 1) and a spanwise-uniform plane, the inflow v is i_r dx on the interior faces."""
    case, g, u, v, w, p, bl = _grid(16, 12, 4)
    ir = 7
    u = np.broadcast_to(np.tanh(2.0 * g.yc)[None, :, None], u.shape).copy()
    xc = (np.arange(g.nx) + 0.5) * g.dx
    v = np.broadcast_to(xc[None, None, :], v.shape).copy()
    w = np.broadcast_to(xc[None, None, :], w.shape).copy()
    d = O.delta99(g.yc, u[0, :, ir])
    ui, vi, wi = O.recycle_inflow(g, u, v, w, ir, d, case.re)
    np.testing.assert_allclose(vi[:, 1:-1], ir * g.dx, rtol=1e-13)
    np.testing.assert_allclose(wi, 0.0, atol=1e-13)  # uniform plane: no fluctuation, mean W dropped


def test_gamma_follows_the_power_law_in_x():
    """With delta ~ x^(4/5) and u_tau ~ x^(-1/10) (the 1/5 power law), the friction-velocity ratio
    of an inlet at x_in and a recycle plane at x_rec is (x_rec / x_in)^(1/10).  The outer-layer
    fluctuation of the recycled inflow is gamma times the plane's: recover gamma from it."""
    case, g, u, v, w, p, bl = _grid(16, 64, 8)
    x_in, x_rec = 1.0, 3.0
    d_in, d_rec = 0.3 * x_in ** 0.8, 0.3 * x_rec ** 0.8
    s = math.atanh(0.99) / d_rec
    ir = 5
    u = np.broadcast_to(np.tanh(s * g.yc)[None, :, None], u.shape).copy()
    rng = np.random.default_rng(9)
    w = 0.01 * rng.standard_normal(w.shape)
    ui, vi, wi = O.recycle_inflow(g, u, v, w, ir, d_in, case.re)
    w_r = 0.5 * (w[:, :, ir - 1] + w[:, :, ir])
    wp = w_r - w_r.mean(axis=0)
    # a row above delta_in (weight 1: outer layer only); its source height uses the measured
    # thickness of the plane (delta99, pinned above), which is d_rec to interpolation accuracy
    ratio = O.delta99(g.yc, u[0, :, ir]) / d_in
    j = int(np.searchsorted(g.yc, 1.2 * d_in))
    src = np.array([np.interp(g.yc[j] * ratio, np.concatenate([[0.0], g.yc]), np.concatenate([[0.0], wp[k]]))
                    for k in range(g.nz)])
    gamma = float(np.dot(wi[:, j], src) / np.dot(src, src))
    assert gamma == pytest.approx((x_rec / x_in) ** 0.1, rel=2e-3)


def test_v_mean_and_fluctuation_closed_form():
    """v at the recycle face linear in y, v_r = (s + c_k) y with spanwise-zero-mean c_k: mean
    V = s y, fluctuation c_k y.  The inner part samples at gamma y and scales the fluctuation by
    gamma, the outer part samples at y delta_rec / delta_inl, mean V unscaled; so at the inlet
    faces v = (1 - W)(s gamma y + gamma^2 c_k y) + W (s r y + gamma r c_k y), r = delta_rec /
    delta_inl, wherever the sampled heights stay below the top face; wall and top rows 0."""
    case, g, u, v, w, p, bl = _grid(ny=32)
    rng = np.random.default_rng(5)
    ck = rng.standard_normal(g.nz)
    ck -= ck.mean()
    sv = 0.02
    yf = g.yf
    v_r = (sv + ck)[:, None] * yf[None, :]
    u_r = np.broadcast_to(0.05 * g.yc, (g.nz, g.ny)).copy()
    w_r = np.zeros((g.nz, g.ny))
    gamma, drec, dinl = 0.95, 2.0, 2.4
    r = drec / dinl
    ui, vi, wi = O.rescale_inflow(g, u_r, v_r, w_r, gamma, drec, dinl)
    W = O.lund_weight(yf / dinl)[None, :]
    y = yf[None, :]
    c = ck[:, None]
    expect = (1 - W) * (sv * gamma * y + gamma * gamma * c * y) + W * (sv * r * y + gamma * r * c * y)
    rows = np.arange(1, g.ny)
    ok = rows[(gamma * yf[rows] <= yf[-1]) & (r * yf[rows] <= yf[-1])]
    np.testing.assert_allclose(vi[:, ok], expect[:, ok], rtol=0, atol=1e-14)
    assert np.all(vi[:, 0] == 0) and np.all(vi[:, -1] == 0)

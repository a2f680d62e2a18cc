"""Fixed-CFL time step (convective rate reduction, dt changes) and the Kim-Moin pressure update:
the CUDA path through the C ABI against the FP64 oracle."""
import ctypes
import math

import numpy as np
import pytest

from tests.gpu_common import B, O, field_rel_errors, need_gpu, torch
from paper_1812_01178_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _projected(shape, seed, **kw):
    case, u, v, w, p = I.small_channel(*shape, seed=seed, **kw)
    g = O.Grid.from_case(case)
    u, v, w = O.make_divergence_free(g, u, v, w)
    return case, g, u, v, w, p


# The device forms each term of the rate as |x| times the reciprocal spacing (no division per
# cell); the oracle divides.  Per term: |x|/h rounded once is within u of the exact quotient,
# |x| * fl(1/h) within 2u + u^2 (u = 2^-53); the two additions of positive terms add u each on
# either side; v_c = (v_j + v_j+1)/2 is formed alike.  The computed sums of a cell therefore differ
# by at most 3u + 4u + O(u^2) < 8u of the sum, and so do the maxima over cells.
RATE_REL = 8.0 * 2.0 ** -53


def _rate_close(got, ref):
    return abs(got - ref) <= RATE_REL * abs(ref)


@pytest.mark.parametrize("shape", [(64, 37, 32), (96, 20, 24), (8, 5, 8)])
def test_convective_rate_equals_the_oracle(shape):
    """The maximum of the per-cell rates, within the rounding bound RATE_REL of the oracle's."""
    case, g, u, v, w, p = _projected(shape, 3)
    s = B.Solver(case, u, v, w, p)
    got, ref = s.convective_rate(), O.convective_rate(g, u, v, w)
    assert _rate_close(got, ref), (got, ref, (got - ref) / ref)
    s.close()


@pytest.mark.parametrize("shape", [(64, 37, 32), (24, 9, 16)])
def test_convective_rate_screening_edge_values(shape):
    """The rate kernel skips cells whose cheap upper bound is below an exact value already found;
    fields built to stress that bound: mostly zero, subnormal and tiny values, faces of v that
    cancel to the last bits, a few spikes of either sign, and values a hair apart at the top.
    The maximum stays within the rounding bound RATE_REL of the oracle's."""
    case, g, u, v, w, p = _projected(shape, 11)
    rng = np.random.default_rng(5)
    for f in (u, v, w):
        f *= 0.0
        f.flat[rng.integers(0, f.size, 50)] = rng.choice([5e-324, -1e-310, 1e-300, 3e-39, -2e-38], 50)
    nx, ny, nz = case.nx, case.ny, case.nz
    v[:, 1:ny, :] = 0.7
    v[:, 2:ny, ::3] = -0.7 + 1e-15  # cancellation across the two faces of a cell
    top = 1.0 + np.arange(7) * 2.0 ** -50
    for q, val in enumerate(top):
        u.flat[rng.integers(0, u.size)] = val * (-1) ** q
        w.flat[rng.integers(0, w.size)] = -val
    s = B.Solver(case, u, v, w, p)
    assert _rate_close(s.convective_rate(), O.convective_rate(g, u, v, w))
    s.u.mul_(-1.0)
    assert _rate_close(s.convective_rate(), O.convective_rate(g, -u, v, w))
    s.close()


def test_convective_rate_boundary_layer():
    case, u, v, w, p, bl = I.boundary_layer(64, 20, 16, amp=0.05, seed=3, re=200.0)
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p, bl=bl)
    assert _rate_close(s.convective_rate(), O.convective_rate(g, u, v, w))
    s.close()


def test_set_dt_then_steps_match_the_oracle():
    case, g, u, v, w, p = _projected((32, 20, 16), 4)
    s = B.Solver(case, u, v, w, p)
    s.step(1)
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, 1)
    dt2 = 0.37 * case.dt
    s.set_dt(dt2)
    s.step(2)
    ref = O.step(g, ref, dt2, case.re, case.fx, 2)
    errs = field_rel_errors(s.state(), (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)
    s.close()


@pytest.mark.parametrize("prec,bound", [(B.NS_FP64, 1e-11), (B.NS_MIXED, 1e-6)])
def test_step_cfl_matches_the_oracle(prec, bound):
    case, g, u, v, w, p = _projected((64, 20, 32), 5)
    s = B.Solver(case, u, v, w, p, precision=prec)
    dts = s.step_cfl(3, 0.5)
    ref, rdts = O.step_cfl(g, dict(u=u, v=v, w=w, p=p), 0.5, case.re, case.fx, 3)
    # the first rate is taken from identical fields: dt = cfl / rate adds one rounding per side
    assert abs(dts[0] - rdts[0]) <= (RATE_REL + 2.0 ** -52) * rdts[0]
    np.testing.assert_allclose(dts, rdts, rtol=1e-10 if prec == B.NS_FP64 else 1e-5)
    assert len(set(dts)) == 3
    errs = field_rel_errors(s.state(), (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < bound, (name, errs)
    s.close()


def test_step_cfl_boundary_layer():
    case, u, v, w, p, bl = I.boundary_layer(64, 16, 16, amp=0.05, seed=7, re=200.0)
    g = O.Grid.from_case(case)
    u, v, w, bl = O.make_divergence_free_bl(g, u, v, w, bl)
    s = B.Solver(case, u, v, w, p, bl=bl)
    dts = s.step_cfl(2, 0.8)
    ref, rdts = O.step_cfl(g, dict(u=u, v=v, w=w, p=p, bl=bl), 0.8, case.re, case.fx, 2, bl=True,
                           u_conv=case.u_conv)
    np.testing.assert_allclose(dts, rdts, rtol=1e-10)
    errs = field_rel_errors(s.state(), (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)
    s.close()


def _host_cfl(s, n, cfl):
    """Fixed-CFL steps driven from the host: read the rate, set dt (host-built tables), step."""
    dts = []
    for _ in range(n):
        dt = cfl / s.convective_rate()
        s.set_dt(dt)
        s.step(1)
        dts.append(dt)
    return dts


def _same_state(a, b):
    for x, y, name in zip(a.state(), b.state(), "uvwp"):
        assert np.array_equal(x, y), name
    for q, x in a.boundary().items():
        assert np.array_equal(x, b.boundary()[q]), q


# (precision, shape, x partition request): FP64 and mixed; the mixed shapes have partitioned y and z
# lines (nx a multiple of 32, ny and nz with a built line shape); PPT forced with several levels
@pytest.mark.parametrize("prec,shape,part", [
    (B.NS_FP64, (64, 20, 32), None),
    (B.NS_MIXED, (64, 48, 64), None),
    (B.NS_FP64, (64, 20, 32), (8, B.NS_PART_PPT)),
    (B.NS_MIXED, (96, 32, 48), (32, B.NS_PART_PPT)),
])
def test_device_dt_update_equals_the_host_tables(prec, shape, part):
    """ns_step_cfl computes dt and rebuilds every table on the device inside its graph; the host
    path (rate read back, ns_set_dt, ns_step) builds them with the same functions: the dts and the
    fields agree to the last bit."""
    case, g, u, v, w, p = _projected(shape, 6)
    a = B.Solver(case, u, v, w, p, precision=prec)
    b = B.Solver(case, u, v, w, p, precision=prec)
    if part:
        a.set_partition(*part)
        b.set_partition(*part)
    d_dev = a.step_cfl(4, 0.6)
    d_host = _host_cfl(b, 4, 0.6)
    assert list(d_dev) == d_host
    assert len(set(d_host)) == 4
    _same_state(a, b)
    assert a.partition() == b.partition()
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [B.NS_FP64, B.NS_MIXED])
def test_device_dt_update_equals_the_host_tables_boundary_layer(prec):
    case, u, v, w, p, bl = I.boundary_layer(64, 16, 16, amp=0.05, seed=8, re=200.0)
    g = O.Grid.from_case(case)
    u, v, w, bl = O.make_divergence_free_bl(g, u, v, w, bl)
    a = B.Solver(case, u, v, w, p, bl=bl, precision=prec)
    b = B.Solver(case, u, v, w, p, bl=bl, precision=prec)
    d_dev = a.step_cfl(3, 0.8)
    d_host = _host_cfl(b, 3, 0.8)
    assert list(d_dev) == d_host
    _same_state(a, b)
    a.close()
    b.close()


def test_step_cfl_runs_longer_than_the_dt_log():
    """More steps than the device dt log holds: the call runs them in several launches of the
    graph, reading the log back after each; dt then continues from the last one."""
    case, g, u, v, w, p = _projected((16, 9, 8), 9)
    a = B.Solver(case, u, v, w, p)
    b = B.Solver(case, u, v, w, p)
    n = 1030
    d_dev = list(a.step_cfl(n, 0.5)) + list(a.step_cfl(2, 0.5))
    d_host = _host_cfl(b, n + 2, 0.5)
    assert d_dev == d_host
    _same_state(a, b)
    a.close()
    b.close()


@pytest.mark.parametrize("shape", [(64, 37, 32), (96, 13, 24)])
def test_kim_moin_steps_match_the_oracle(shape):
    case, g, u, v, w, p = _projected(shape, 6, re=40.0)
    case.pressure_update = B.NS_PRESSURE_KIM_MOIN
    s = B.Solver(case, u, v, w, p)
    s.step(2)
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, 2, pressure="kim_moin")
    errs = field_rel_errors(s.state(), (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)
    s.close()
    # within one sub-step the velocities are those of the plain update and only p differs (the
    # pressure enters the velocity through the next sub-step's -alpha_k G p)
    s1 = B.Solver(case, u, v, w, p)
    case.pressure_update = B.NS_PRESSURE_DELTA
    s2 = B.Solver(case, u, v, w, p)
    s1.substep(0)
    s2.substep(0)
    a, b = s1.state(), s2.state()
    for q in range(3):
        assert np.array_equal(a[q], b[q])
    assert not np.array_equal(a[3], b[3])
    s1.close()
    s2.close()


def test_kim_moin_mixed_form():
    """The Kim-Moin pressure update with the mixed form (its projection reads the refined phi)."""
    case, g, u, v, w, p = _projected((64, 37, 32), 6, re=40.0)
    case.pressure_update = B.NS_PRESSURE_KIM_MOIN
    s = B.Solver(case, u, v, w, p, precision=B.NS_MIXED)
    s.step(2)
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, 2, pressure="kim_moin")
    got = s.state()
    errs = field_rel_errors(got, (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name, bound in (("u", 1e-7), ("v", 1e-7), ("w", 1e-7), ("p", 1e-6)):
        assert errs[name] < bound, (name, errs)
    assert np.abs(O.divergence(g, *got[:3])).max() < 1e-10
    s.close()


def test_kim_moin_boundary_layer():
    case, u, v, w, p, bl = I.boundary_layer(64, 16, 16, amp=0.05, seed=8, re=100.0)
    case.pressure_update = B.NS_PRESSURE_KIM_MOIN
    g = O.Grid.from_case(case)
    u, v, w, bl = O.make_divergence_free_bl(g, u, v, w, bl)
    s = B.Solver(case, u, v, w, p, bl=bl)
    s.step(2)
    ref = O.step_bl(g, dict(u=u, v=v, w=w, p=p, bl=bl), case.dt, case.re, case.fx, 2, case.u_conv,
                    pressure="kim_moin")
    errs = field_rel_errors(s.state(), (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)
    s.close()


def test_invalid_dt_cfl_and_non_finite_fields_are_reported():
    case, g, u, v, w, p = _projected((16, 9, 8), 2)
    s = B.Solver(case, u, v, w, p)
    L = B.lib()
    for bad in (0.0, -1.0, math.inf, math.nan):
        assert L.ns_set_dt(s.ctx, bad) == B.NS_ERR_ARG
        assert L.ns_step_cfl(s.ctx, 1, bad, None) == B.NS_ERR_ARG
    s.u[1, 2, 3] = float("nan")
    r = ctypes.c_double()
    assert L.ns_convective_rate(s.ctx, ctypes.byref(r)) == B.NS_ERR_STATE
    s.u[1, 2, 3] = 0.0
    s.step(1)  # still usable
    s.sync()
    s.close()


def test_step_cfl_reports_rest_and_non_finite_fields():
    """The device-side dt update cannot stop the graph it runs in: a rate that is zero (fluid at
    rest) or non-finite keeps the previous dt for that step, and the call reports NS_ERR_STATE
    with the step once its run of steps is done.  A valid field afterwards steps normally."""
    case, g, u, v, w, p = _projected((16, 9, 8), 2)
    L = B.lib()
    s = B.Solver(case, 0.0 * u, 0.0 * v, 0.0 * w, p)
    dts = (ctypes.c_double * 2)()
    assert L.ns_step_cfl(s.ctx, 2, 0.5, dts) == B.NS_ERR_STATE
    msg = L.ns_last_error(s.ctx).decode()
    assert "rest" in msg and "step 0" in msg, msg
    # step 0 kept the previous dt; the body force then set the fluid moving, so step 1 had a
    # (tiny) rate and its own, large, dt
    assert dts[0] == case.dt and dts[1] > case.dt
    s.close()
    s = B.Solver(case, u, v, w, p)
    s.u[1, 2, 3] = float("nan")
    assert L.ns_step_cfl(s.ctx, 1, 0.5, None) == B.NS_ERR_STATE
    assert "non-finite" in L.ns_last_error(s.ctx).decode()
    s.close()
    s = B.Solver(case, u, v, w, p)
    d = s.step_cfl(2, 0.5)
    ref, rdts = O.step_cfl(g, dict(u=u, v=v, w=w, p=p), 0.5, case.re, case.fx, 2)
    np.testing.assert_allclose(d, rdts, rtol=1e-10)
    s.close()

"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, stage by stage and per step.

Tolerances: FP64 stages are compared element-wise at 1e-12 relative (the operations differ from
the oracle's only in rounding order: precomputed factors, FFT instead of naive DFT); the full
FP64 step at the 1e-11 relative-L2 bar after 10 steps.
"""
import math

import numpy as np
import pytest

from tests.gpu_common import B, O, field_rel_errors, need_gpu, rel_l2, to_np, torch
from paper_1812_01178_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# (nx, ny, nz): several x tiles / warps, ragged y, small and large partitions
SHAPES = [(64, 37, 32), (32, 20, 16), (128, 9, 64), (8, 5, 8)]


def _case(nx, ny, nz, ytop=0, seed=7):
    case, u, v, w, p = I.small_channel(nx, ny, nz, seed=seed)
    case.bc_ytop = ytop
    return case, u, v, w, p


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("ytop", [0, 1])
def test_rhs_parity(shape, ytop):
    case, u, v, w, p = _case(*shape, ytop=ytop)
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p)
    # sub-step 0 (no N_prev), then sub-step 1 with the oracle's N as N_prev
    r0, N0 = O.rhs(g, u, v, w, p, None, 0, case.dt, case.re, case.fx)
    s.rhs(0)
    for q, (bi, bn) in enumerate([(B.NS_BUF_RU, B.NS_BUF_NU), (B.NS_BUF_RV, B.NS_BUF_NV),
                                  (B.NS_BUF_RW, B.NS_BUF_NW)]):
        np.testing.assert_allclose(to_np(s.buffer(bi)), r0[q], rtol=0, atol=1e-12 * np.abs(r0[q]).max())
        # the library stores N pre-multiplied by the sub-step's convection weight -dt gamma_k
        cn = -case.dt * O.RK3_GAMMA[0]
        np.testing.assert_allclose(to_np(s.buffer(bn)), cn * N0[q], rtol=0, atol=1e-12 * np.abs(cn * N0[q]).max())
    r1, _ = O.rhs(g, u, v, w, p, N0, 1, case.dt, case.re, case.fx)
    s.rhs(1)
    for q, bi in enumerate([B.NS_BUF_RU, B.NS_BUF_RV, B.NS_BUF_RW]):
        np.testing.assert_allclose(to_np(s.buffer(bi)), r1[q], rtol=0, atol=1e-12 * np.abs(r1[q]).max())
    s.close()


def _load_r(s, r3):
    for bi, r in zip([B.NS_BUF_RU, B.NS_BUF_RV, B.NS_BUF_RW], r3):
        s.buffer(bi).copy_(torch.as_tensor(r, device=s.u.device))


def _rand_r(case, seed):
    rng = np.random.default_rng(seed)
    ru = rng.standard_normal((case.nz, case.ny, case.nx))
    rv = rng.standard_normal((case.nz, case.ny + 1, case.nx))
    rv[:, 0] = 0
    rv[:, -1] = 0
    rw = rng.standard_normal((case.nz, case.ny, case.nx))
    return [ru, rv, rw]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("k", [0, 2])
def test_adi_y_z_parity(shape, k):
    case, u, v, w, p = _case(*shape)
    case.re = 5.0  # strong implicit coupling
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p)
    beta = O.RK3_ALPHA[k] * case.dt / (2 * case.re)
    r3 = _rand_r(case, 11)
    _load_r(s, r3)
    s.adi(1, k)
    for q, bi in enumerate([B.NS_BUF_RU, B.NS_BUF_RV, B.NS_BUF_RW]):
        ref = O.adi_sweep(g, r3[q], 1, q, beta)
        np.testing.assert_allclose(to_np(s.buffer(bi)), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    # z sweep forms u* = u + delta
    _load_r(s, r3)
    s.adi(2, k)
    gu, gv, gw, _ = s.state()
    for q, (f0, gf) in enumerate(zip((u, v, w), (gu, gv, gw))):
        ref = f0 + O.adi_sweep(g, r3[q], 2, q, beta)
        np.testing.assert_allclose(gf, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    s.close()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mode", [B.NS_PART_PPT, B.NS_PART_PDD])
def test_adi_x_partitioned_parity(shape, mode):
    """PPT equals whole-line cyclic Thomas to round-off for every partition count; PDD too
    when the dropped coupling is below round-off (checked and reported by the library)."""
    case, u, v, w, p = _case(*shape)
    case.re = 2.0
    case.dt = 0.05
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p)
    r3 = _rand_r(case, 12)
    for P in (1, 2, 4, 8, 16, 32):
        if case.nx % P or case.nx // P > 16:
            continue
        s.set_partition(P, mode)
        gotP, gotmode, drop = s.partition()
        assert gotP == P and gotmode == mode
        for k in (0, 1):
            beta = O.RK3_ALPHA[k] * case.dt / (2 * case.re)
            _load_r(s, r3)
            s.adi(0, k)
            for q, bi in enumerate([B.NS_BUF_RU, B.NS_BUF_RV, B.NS_BUF_RW]):
                ref = O.adi_sweep(g, r3[q], 0, q, beta)
                got = to_np(s.buffer(bi))
                err = np.abs(got - ref).max() / np.abs(ref).max()
                if mode == B.NS_PART_PPT:
                    assert err < 1e-13, (P, k, q, err)
                else:
                    assert err <= max(1e-13, 50 * drop), (P, k, q, err, drop)
    s.close()


@pytest.mark.parametrize("mode", [B.NS_PART_PPT, B.NS_PART_PDD])
def test_adi_x_truncated_spikes(mode):
    """Strongly dominant rows (beta / dx^2 about 1e-7): the spikes fall below the truncation
    tolerance within half a partition, and the sweep keeps one correction per row
    (StepK::xhalf).  The result still equals the oracle's whole-line cyclic solve to round-off,
    both modes, every sub-step.  (The inflow / outflow class is covered by the whole-step parity
    of the boundary layer, whose rows are as dominant.)"""
    case, u, v, w, p = _case(128, 9, 8)
    case.re = 1e5
    case.dt = 1e-4
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p)
    s.set_partition(16, mode)  # M = 8 rows per partition
    r3 = _rand_r(case, 21)
    for k in (0, 1, 2):
        beta = O.RK3_ALPHA[k] * case.dt / (2 * case.re)
        _load_r(s, r3)
        s.adi(0, k)
        for q, bi in enumerate([B.NS_BUF_RU, B.NS_BUF_RV, B.NS_BUF_RW]):
            ref = O.adi_sweep(g, r3[q], 0, q, beta)
            err = np.abs(to_np(s.buffer(bi)) - ref).max() / np.abs(ref).max()
            assert err < 1e-13, (k, q, err)
    s.close()


@pytest.mark.parametrize("shape", SHAPES)
def test_pdd_matches_oracle_pdd(shape):
    """PDD on the GPU reproduces the oracle's dense-matrix PDD of Sec. 3.2 when the dropped
    coupling is not negligible (large beta)."""
    case, u, v, w, p = _case(*shape)
    if case.nx < 16:
        pytest.skip("needs several partitions")
    case.re = 0.02
    case.dt = 0.05
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p)
    P = max(4, case.nx // 16)
    s.set_partition(P, B.NS_PART_PDD)
    r3 = _rand_r(case, 13)
    _load_r(s, r3)
    s.adi(0, 0)
    beta = O.RK3_ALPHA[0] * case.dt / (2 * case.re)
    a, b, c = O.adi_rows(g, 0, 0, beta)
    line = r3[0][1, 2, :]
    ref_pdd = O.pdd_solve(a, b, c, line, P, cyclic=True)
    ref_exact = O.thomas_cyclic(a, b, c, line)
    got = to_np(s.buffer(B.NS_BUF_RU))[1, 2, :]
    assert np.abs(ref_pdd - ref_exact).max() > 1e-6  # PDD really drops something here
    np.testing.assert_allclose(got, ref_pdd, rtol=0, atol=1e-12 * np.abs(ref_pdd).max())
    s.close()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("k", [-1, 1])
def test_poisson_and_projection_parity(shape, k):
    case, u, v, w, p = _case(*shape)
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p)
    scale = 1.0 if k < 0 else O.RK3_ALPHA[k] * case.dt
    phi_ref = O.poisson_solve(g, O.divergence(g, u, v, w) / scale)
    s.poisson(k)
    phi = to_np(s.buffer(B.NS_BUF_PHI))
    np.testing.assert_allclose(phi - phi.mean(), phi_ref - phi_ref.mean(), rtol=0,
                               atol=1e-11 * np.abs(phi_ref).max())
    s.project(k)
    gu, gv, gw, gp = s.state()
    ru, rv, rw = O.project(g, u, v, w, phi_ref, scale)
    for a_, b_ in ((gu, ru), (gv, rv), (gw, rw)):
        np.testing.assert_allclose(a_, b_, rtol=0, atol=1e-10 * np.abs(b_).max())
    pr = p + (phi_ref if k >= 0 else 0.0)
    np.testing.assert_allclose(gp - gp.mean(), pr - pr.mean(), rtol=0, atol=1e-11 * (np.abs(pr).max() + 1))
    div = O.divergence(g, gu, gv, gw)
    assert np.abs(div).max() < 1e-10 * np.abs(O.divergence(g, u, v, w)).max() + 1e-13
    s.close()


def test_laminar_channel_10_steps_parity():
    """64x64x32 laminar channel, Re_b = 2000, 10 steps: GPU FP64 vs oracle <= 1e-11 rel L2."""
    case, u, v, w, p = I.laminar_channel()
    g = O.Grid.from_case(case)
    u, v, w = O.make_divergence_free(g, u, v, w)
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, nsteps=case.steps)
    s = B.Solver(case, u, v, w, p)
    s.step(case.steps)
    got = s.state()
    errs = field_rel_errors(got, (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)
    assert errs["p_strict"] < 1e-8, errs
    s.close()


@pytest.mark.parametrize("shape", [(32, 20, 16), (16, 11, 8)])
def test_turbulent_like_steps_parity(shape):
    """O(1) random fields (strong nonlinearity), 3 steps via the captured graph, stress-free top."""
    case, u, v, w, p = _case(*shape, ytop=1)
    case.dt = 1e-3
    g = O.Grid.from_case(case)
    u, v, w = O.make_divergence_free(g, u, v, w)
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, nsteps=3)
    s = B.Solver(case, u, v, w, p)
    s.step(3)
    errs = field_rel_errors(s.state(), (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p", "p_strict"):
        assert errs[name] < 1e-11, (name, errs)
    s.close()


def test_substep_sequence_equals_graph_step():
    case, u, v, w, p = _case(32, 20, 16)
    s1 = B.Solver(case, u, v, w, p)
    s2 = B.Solver(case, u, v, w, p)
    s1.step(2)
    for _ in range(2):
        for k in range(3):
            s2.substep(k)
    for a_, b_ in zip(s1.state(), s2.state()):
        assert np.array_equal(a_, b_)
    s1.close()
    s2.close()


def test_make_divergence_free():
    case, u, v, w, p = _case(64, 37, 32)
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p)
    s.make_divergence_free()
    gu, gv, gw, gp = s.state()
    assert np.abs(O.divergence(g, gu, gv, gw)).max() < 1e-11 * np.abs(O.divergence(g, u, v, w)).max()
    assert np.array_equal(gp, p)
    s.close()


@pytest.mark.parametrize("nx", [1024, 2048])
@pytest.mark.parametrize("mode", [B.NS_PART_PPT, B.NS_PART_PDD])
def test_adi_x_long_lines_parity(nx, mode):
    """Long x-lines (32 partitions of 32 or 64 rows, lines staged in shared memory)."""
    case, u, v, w, p = _case(nx, 6, 8)
    case.re = 1.0
    case.dt = 0.02
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p)
    s.set_partition(32, mode)
    P, gotmode, drop = s.partition()
    r3 = _rand_r(case, 21)
    for k in (0, 2):
        beta = O.RK3_ALPHA[k] * case.dt / (2 * case.re)
        _load_r(s, r3)
        s.adi(0, k)
        for q, bi in enumerate([B.NS_BUF_RU, B.NS_BUF_RV, B.NS_BUF_RW]):
            ref = O.adi_sweep(g, r3[q], 0, q, beta)
            err = np.abs(to_np(s.buffer(bi)) - ref).max() / np.abs(ref).max()
            assert err < (1e-13 if mode == B.NS_PART_PPT else max(1e-13, 50 * drop)), (k, q, err, drop)
    s.close()


def test_long_line_steps_parity():
    """Full FP64 steps on a grid with 1024-long x-lines (long-line x solver, tiled RHS, long x FFT)."""
    case, u, v, w, p = _case(1024, 12, 16)
    case.dt = 1e-3
    g = O.Grid.from_case(case)
    u, v, w = O.make_divergence_free(g, u, v, w)
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, nsteps=2)
    s = B.Solver(case, u, v, w, p)
    assert s.partition()[0] == 32
    s.step(2)
    errs = field_rel_errors(s.state(), (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)
    s.close()

"""The seeded input generators (shared by the oracle and the CUDA path, holding none of the
method's arithmetic): splitmix64 against the published first outputs of its reference
implementation, the counter offsets, the derived uniform and normal streams, and the recipe of
the bench workload (log-law mean, 10 % fluctuations, walls, CFL-derived dt)."""
import math

import numpy as np
import pytest

from paper_1812_01178_gb300 import inputs as I


def test_splitmix64_reference_outputs():
    # the first three outputs of splitmix64 started from state 0 (Vigna's reference code, the
    # generator of Steele, Lea & Flood 2014)
    got = [int(x) for x in I.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_offsets_and_determinism():
    a = I.splitmix64(1812, 10)
    assert np.array_equal(a[4:], I.splitmix64(1812, 6, offset=4))
    assert np.array_equal(a, I.splitmix64(1812, 10))
    assert not np.array_equal(a, I.splitmix64(1813, 10))
    n = I.normal(5, 9)
    assert np.array_equal(n[2:], I.normal(5, 7, offset=1)[:7])  # pairs: offset 1 = two uniforms on


def test_uniform_and_normal_statistics():
    u = I.uniform01(7, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / u.size)
    z = I.normal(7, 200000)
    assert abs(z.mean()) < 4 / math.sqrt(z.size)
    assert abs(z.std() - 1.0) < 4 * math.sqrt(0.5 / z.size)
    assert abs(np.mean(z ** 4) - 3.0) < 0.1  # Gaussian kurtosis


def test_loglaw_mean_profile():
    yp = np.array([0.5, 5.0, 10.9, 11.1, 100.0, 395.0])
    um = I.loglaw_mean(yp)
    assert np.allclose(um[:3], yp[:3])
    assert np.allclose(um[3:], np.log(yp[3:]) / 0.41 + 5.2)  # von Karman constant 0.41


def test_turbulent_channel_recipe_small():
    case, u, v, w, p = I.turbulent_channel(32, 24, 16)
    assert u.shape == w.shape == p.shape == (16, 24, 32) and v.shape == (16, 25, 32)
    assert np.all(v[:, 0] == 0) and np.all(v[:, -1] == 0) and np.all(p == 0)
    yf = case.yf
    assert yf[0] == -1.0 and yf[-1] == 1.0 and np.all(np.diff(yf) > 0)
    assert np.diff(yf)[0] < np.diff(yf)[12]  # clustered at the walls
    yc = 0.5 * (yf[1:] + yf[:-1])
    um = I.loglaw_mean((1 - np.abs(yc)) * case.re)
    # fluctuations about the log-law mean with 10 % of the local mean as their spread
    rel = (u - um[None, :, None]) / (0.1 * um[None, :, None])
    assert abs(rel.mean()) < 0.05 and abs(rel.std() - 1.0) < 0.05
    # dt = 0.5 / max convective rate of the initial field
    dx, dz, dy = case.lx / case.nx, case.lz / case.nz, np.diff(yf)
    rate = (np.abs(u) / dx + np.abs(0.5 * (v[:, :-1] + v[:, 1:])) / dy[None, :, None] + np.abs(w) / dz).max()
    assert case.dt == pytest.approx(0.5 / rate, rel=1e-15)
    # the same call gives the same fields
    case2, u2, *_ = I.turbulent_channel(32, 24, 16)
    assert np.array_equal(u, u2) and case2.dt == case.dt


def test_normal_range_is_a_window_of_the_whole_sequence():
    whole = I.normal(99, 1001, 0)
    for e0, n in ((0, 10), (1, 7), (2, 9), (37, 64), (500, 501)):
        assert np.array_equal(I.normal_range(99, e0, n), whole[e0:e0 + n])


def test_boundary_layer_built_slab_by_slab_equals_the_whole_field():
    """The bench builds the large boundary-layer fields a few z planes at a time: the planes are
    bit for bit those of the whole-field generator, boundary planes included (odd slab starts and
    odd plane sizes as well)."""
    case, u, v, w, p, bl = I.boundary_layer(96, 37, 24)
    parts = [I.boundary_layer_slab(case, k0, min(k0 + 5, case.nz)) for k0 in range(0, case.nz, 5)]
    for q, ref in enumerate((u, v, w)):
        assert np.array_equal(np.concatenate([pp[q] for pp in parts]), ref)
    for k, ref in bl.items():
        assert np.array_equal(np.concatenate([pp[3][k] for pp in parts]), ref)
    rate = max(I.boundary_layer_rate(case, *pp[:3]) for pp in parts)
    assert case.dt == 0.5 / rate

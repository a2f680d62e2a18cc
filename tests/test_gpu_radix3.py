"""Grids of 2^a 3^b cells in x and z (mixed radix-2/4/3 FFT, partitions of 3, 6, 9, 12, 24 and 48
rows): the CUDA path through the C ABI against the FP64 oracle, whose transforms are naive DFT /
DCT matrices of any length."""
import numpy as np
import pytest

from tests.gpu_common import B, O, field_rel_errors, need_gpu, to_np, torch
from paper_1812_01178_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# (nx, ny, nz): radix-3 in x only, in z only, in both, two radix-3 stages, several tiles
SHAPES = [(96, 20, 32), (64, 9, 24), (72, 13, 48), (48, 6, 72)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _rand_r(case, seed):
    rng = np.random.default_rng(seed)
    ru = rng.standard_normal((case.nz, case.ny, case.nx))
    rv = rng.standard_normal((case.nz, case.ny + 1, case.nx))
    rv[:, 0] = 0
    rv[:, -1] = 0
    rw = rng.standard_normal((case.nz, case.ny, case.nx))
    return [ru, rv, rw]


def _load_r(s, r3):
    for bi, r in zip([B.NS_BUF_RU, B.NS_BUF_RV, B.NS_BUF_RW], r3):
        s.buffer(bi).copy_(torch.as_tensor(r, device=s.u.device))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("k", [-1, 2])
def test_poisson_and_projection_parity(shape, k):
    case, u, v, w, p = I.small_channel(*shape, seed=21)
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p)
    scale = 1.0 if k < 0 else O.RK3_ALPHA[k] * case.dt
    phi_ref = O.poisson_solve(g, O.divergence(g, u, v, w) / scale)
    s.poisson(k)
    phi = to_np(s.buffer(B.NS_BUF_PHI))
    np.testing.assert_allclose(phi - phi.mean(), phi_ref - phi_ref.mean(), rtol=0,
                               atol=1e-11 * np.abs(phi_ref).max())
    s.project(k)
    gu, gv, gw, _ = s.state()
    ru, rv, rw = O.project(g, u, v, w, phi_ref, scale)
    for a_, b_ in ((gu, ru), (gv, rv), (gw, rw)):
        np.testing.assert_allclose(a_, b_, rtol=0, atol=1e-10 * np.abs(b_).max())
    assert np.abs(O.divergence(g, gu, gv, gw)).max() < 1e-10 * np.abs(O.divergence(g, u, v, w)).max() + 1e-13
    s.close()


@pytest.mark.parametrize("nx,Ps", [(96, (32, 16, 8)), (72, (8,)), (288, (32,)), (768, (32,)), (1536, (32,))])
@pytest.mark.parametrize("mode", [B.NS_PART_PPT, B.NS_PART_PDD])
def test_adi_x_partition_shapes(nx, Ps, mode):
    """M = 3, 6, 12 (96), 9 (72, 288), 24 (768) and 48 (1536) rows per partition."""
    case, u, v, w, p = I.small_channel(nx, 6, 8, seed=5)
    case.re = 2.0
    case.dt = 0.05
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p)
    r3 = _rand_r(case, 17)
    for P in Ps:
        s.set_partition(P, mode)
        gotP, gotmode, drop = s.partition()
        assert gotP == P and gotmode == mode
        for k in (0, 2):
            beta = O.RK3_ALPHA[k] * case.dt / (2 * case.re)
            _load_r(s, r3)
            s.adi(0, k)
            for q, bi in enumerate([B.NS_BUF_RU, B.NS_BUF_RV, B.NS_BUF_RW]):
                ref = O.adi_sweep(g, r3[q], 0, q, beta)
                err = np.abs(to_np(s.buffer(bi)) - ref).max() / np.abs(ref).max()
                assert err < (1e-13 if mode == B.NS_PART_PPT else max(1e-13, 50 * drop)), (P, k, q, err, drop)
    s.close()


@pytest.mark.parametrize("shape", [(96, 16, 24), (48, 11, 72)])
def test_steps_parity_fp64_and_mixed(shape):
    case, u, v, w, p = I.small_channel(*shape, seed=9)
    case.dt = 1e-3
    g = O.Grid.from_case(case)
    u, v, w = O.make_divergence_free(g, u, v, w)
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, nsteps=2)
    for prec, bound in ((B.NS_FP64, 1e-11), (B.NS_MIXED, 1e-6)):
        s = B.Solver(case, u, v, w, p, precision=prec)
        s.step(2)
        errs = field_rel_errors(s.state(), (ref["u"], ref["v"], ref["w"], ref["p"]))
        for name in ("u", "v", "w", "p"):
            assert errs[name] < bound, (prec, name, errs)
        s.close()


def test_boundary_layer_cosine_transform_of_length_96():
    """Inflow / outflow: the DCT-II in x through an FFT of length 96 (radix 2, 4, 4, 3)."""
    case, u, v, w, p, bl = I.boundary_layer(96, 10, 24, amp=0.05, seed=3, re=200.0)
    g = O.Grid.from_case(case)
    u, v, w, bl = O.make_divergence_free_bl(g, u, v, w, bl)
    ref = O.step_bl(g, dict(u=u, v=v, w=w, p=p, bl=bl), case.dt, case.re, case.fx, nsteps=2, u_conv=case.u_conv)
    s = B.Solver(case, u, v, w, p, bl=bl)
    s.step(2)
    errs = field_rel_errors(s.state(), (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)
    assert np.abs(O.divergence_bl(g, *s.state()[:3], s.boundary())).max() < 1e-11
    s.close()


def test_batch_with_radix3_instances():
    """A batched ensemble mixing power-of-two and 2^a 3^b instances equals the single instances."""
    cases = [I.small_channel(n, ny, nz, seed=30 + i) for i, (n, ny, nz) in
             enumerate([(96, 12, 24), (64, 9, 32), (48, 16, 72)])]
    bt = B.Batch([c[0] for c in cases], fields=[c[1:] for c in cases])
    bt.step(2)
    for i, (case, u, v, w, p) in enumerate(cases):
        s = B.Solver(case, u, v, w, p)
        s.step(2)
        for a_, b_ in zip(bt.state(i), s.state()):
            assert np.array_equal(a_, b_)
        s.close()
    bt.close()

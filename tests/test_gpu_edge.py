"""Edge and degenerate cases of the CUDA path through the C ABI: zero steps, the quiescent state,
the smallest accepted grid, a single partition, and arguments the host rejects before any launch."""
import numpy as np
import pytest

from tests.gpu_common import B, O, field_rel_errors, need_gpu, torch
from paper_1812_01178_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def test_zero_steps_is_a_no_op():
    case, u, v, w, p = I.small_channel(32, 20, 16, seed=3)
    s = B.Solver(case, u, v, w, p)
    before = s.state()
    s.step(0)
    for a, b in zip(before, s.state()):
        assert np.array_equal(a, b)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_quiescent_fluid_stays_exactly_at_rest(precision):
    """u = v = w = p = 0 with no body force is a fixed point of the scheme: every stage maps
    zeros to zeros (the Poisson gauge included), in both precisions."""
    case, u, v, w, p = I.small_channel(32, 20, 16, seed=3)
    case.fx = 0.0
    case.precision = precision
    z = [np.zeros_like(a) for a in (u, v, w, p)]
    s = B.Solver(case, *z)
    s.step(3)
    for a in s.state():
        assert not np.any(a)
    s.close()


@pytest.mark.parametrize("precision,bound", [(0, 1e-11), (1, 1e-6)])
def test_smallest_grid_steps_parity(precision, bound):
    """8x4x8, the smallest grid the library accepts (one FFT stage of each radix, ny = 4), in both
    precisions (mixed: FP32 x transform on 8-point rows, the y solve with ny rows = its prefetch
    depth, the FP64 refinement)."""
    case, u, v, w, p = I.small_channel(8, 4, 8, seed=11)
    case.dt = 1e-3
    case.precision = precision
    g = O.Grid.from_case(case)
    u, v, w = O.make_divergence_free(g, u, v, w)
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, nsteps=2)
    s = B.Solver(case, u, v, w, p)
    s.step(2)
    got = s.state()
    errs = field_rel_errors(got, (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < bound, (name, errs)
    assert np.abs(O.divergence(g, *got[:3])).max() < 1e-10
    s.close()


@pytest.mark.parametrize("shape", [(4096, 4, 8), (3072, 4, 8), (8, 1024, 8), (8, 4, 4096), (8, 4, 3072)])
@pytest.mark.parametrize("precision,bound,pbound", [(0, 1e-11, 1e-11), (1, 1e-6, 3e-5)])
def test_largest_extents_steps_parity(shape, precision, bound, pbound):
    """Each extent at the largest size the library takes, the other two at their smallest: nx
    4096 and 3072 (the x lines as 32 partitions of 128 and 96 rows staged in shared memory, x
    transforms of one row per block), ny 1024 (the y lines and the Poisson y solve at full length),
    nz 4096 and 3072 (z tiles of two columns, the factorised z sweep's start sums), in both
    precisions.  The mixed form's bound on p is wider here: its FP32 increments carry the x
    viscous term, whose weight grows as 1/dx^2, and the pressure sees their divergence through
    1/dx; on 4 x 8 cross-sections its p error grows smoothly from 3e-7 at nx = 512 to 9e-6 at
    nx = 4096 (u 4e-9 to 2e-7), while the FP64 form stays at 1e-14.  Its divergence after the
    projection sits at the floor of the refinement's float-float residual, about 2^-46 of the
    largest stencil term, which grows as 1/h^2 with the smallest spacing h: measured 5e-10 at
    dx = 2 pi / 4096, 3e-9 at the wall rows of ny = 1024, 8e-9 at dz = pi / 4096 (1e-15 on the
    bench grids); the bound here is 2e-8 (the FP64 form: 1e-10)."""
    case, u, v, w, p = I.small_channel(*shape, seed=13)
    case.dt = 1e-3
    case.precision = precision
    g = O.Grid.from_case(case)
    u, v, w = O.make_divergence_free(g, u, v, w)
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, nsteps=2)
    s = B.Solver(case, u, v, w, p)
    s.step(2)
    got = s.state()
    errs = field_rel_errors(got, (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w"):
        assert errs[name] < bound, (name, errs)
    assert errs["p"] < pbound, errs
    assert np.abs(O.divergence(g, *got[:3])).max() < (1e-10 if precision == 0 else 2e-8)
    s.close()


def test_largest_x_boundary_layer():
    """Inflow / convective outflow at nx = 4096: the cosine transforms of one 4096-point row per
    block, the x lines with the outflow face, against the oracle."""
    case, u, v, w, p, bl = I.boundary_layer(4096, 6, 8, amp=0.05, seed=4, re=200.0)
    g = O.Grid.from_case(case)
    u, v, w, bl = O.make_divergence_free_bl(g, u, v, w, bl)
    ref = O.step_bl(g, dict(u=u, v=v, w=w, p=p, bl=bl), case.dt, case.re, case.fx, 2, case.u_conv)
    s = B.Solver(case, u, v, w, p, bl=bl)
    s.step(2)
    errs = field_rel_errors(s.state(), (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)
    s.close()


@pytest.mark.parametrize("mode", [B.NS_PART_PPT, B.NS_PART_PDD])
def test_single_partition_is_plain_thomas(mode):
    """P = 1: no reduced system; PDD and PPT both reduce to the whole-line solve."""
    case, u, v, w, p = I.small_channel(16, 9, 8, seed=5)
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p)
    s.set_partition(1, mode)
    assert s.partition()[0] == 1
    rng = np.random.default_rng(2)
    rr = [rng.standard_normal((case.nz, case.ny + (1 if q == 1 else 0), case.nx)) for q in range(3)]
    rr[1][:, 0] = 0
    rr[1][:, -1] = 0
    for q, b in enumerate((B.NS_BUF_RU, B.NS_BUF_RV, B.NS_BUF_RW)):
        s.buffer(b).copy_(torch.as_tensor(rr[q], device=s.u.device))
    s.adi(0, 1)
    beta = O.RK3_ALPHA[1] * case.dt / (2 * case.re)
    for q, b in enumerate((B.NS_BUF_RU, B.NS_BUF_RV, B.NS_BUF_RW)):
        ref = O.adi_sweep(g, rr[q], 0, q, beta)
        got = s.buffer(b).double().cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    s.close()


def test_invalid_arguments_are_rejected_on_the_host():
    case, u, v, w, p = I.small_channel(16, 9, 8, seed=5)
    s = B.Solver(case, u, v, w, p)
    L = B.lib()
    assert L.ns_adi_sweep(s.ctx, 3, 0) == B.NS_ERR_ARG
    assert L.ns_adi_sweep(s.ctx, 0, 3) == B.NS_ERR_ARG
    assert L.ns_rhs(s.ctx, -1) == B.NS_ERR_ARG
    assert L.ns_step(s.ctx, -1) == B.NS_ERR_ARG
    assert L.ns_set_partition(s.ctx, 0, 3, B.NS_PART_PPT) != B.NS_OK  # P must divide nx
    # the context is still usable after the rejected calls
    s.step(1)
    s.sync()
    s.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_step_host_equals_device_step(pinned):
    """ns_step_host: host state in (pinned or pageable memory), one captured step, state out:
    bitwise equal to the same step on device fields."""
    case, u, v, w, p = I.small_channel(64, 20, 32, seed=13)
    s1 = B.Solver(case, u, v, w, p)
    s1.step(1)
    ref = s1.state()
    s1.close()
    s2 = B.Solver(case)
    host = []
    for a in (u, v, w, p):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).copy())
        host.append((t.pin_memory() if pinned else t).numpy())
    B.ns_step_host(s2.ctx, *host, 1)
    for got, want in zip(host, ref):
        assert np.array_equal(got, want)
    s2.close()


@pytest.mark.parametrize("bl", [False, True])
def test_checkpoint_at_a_step_boundary_resumes_bitwise(bl):
    """At a step boundary the state is the caller's fields (and the boundary planes): sub-step 0
    does not read N_prev.  Stepping 1 + 2 steps through a copy equals 3 steps without a stop."""
    if bl:
        case, u, v, w, p, planes = I.boundary_layer(64, 12, 16, amp=0.05, seed=4, re=200.0)
    else:
        case, u, v, w, p = I.small_channel(64, 20, 16, seed=4)
        planes = None
    a = B.Solver(case, u, v, w, p, bl=planes)
    a.step(3)
    b = B.Solver(case, u, v, w, p, bl=planes)
    b.step(1)
    snap = b.state()
    snap_bl = b.boundary() if bl else None
    b.close()
    c = B.Solver(case, *snap, bl=snap_bl)
    c.step(2)
    for x, y in zip(a.state(), c.state()):
        assert np.array_equal(x, y)
    if bl:
        for q, t in a.boundary().items():
            assert np.array_equal(t, c.boundary()[q])
    a.close()
    c.close()


def test_fp64_fma_probe():
    """The FP64 throughput probe behind the roofline denominator: arguments checked on the host,
    every chain's sum finite and equal across threads that start alike, and a rate within the
    FP64 unit counts of the part (at most 2 FMA per clock per SM at the highest SM clock)."""
    need_gpu()
    import ctypes
    L = B.lib()
    out = torch.empty(4 * 256, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert L.ns_fp64_fma_probe(None, 4, 8, st) == B.NS_ERR_ARG
    assert L.ns_fp64_fma_probe(ctypes.c_void_p(out.data_ptr()), 0, 8, st) == B.NS_ERR_ARG
    assert L.ns_fp64_fma_probe(ctypes.c_void_p(out.data_ptr()), 4, 0, st) == B.NS_ERR_ARG
    B.ns_fp64_fma_probe(out.data_ptr(), 4, 64, st)
    v = out.view(4, 256).cpu().numpy()
    assert np.isfinite(v).all()
    assert np.array_equal(v[0], v[3])  # every block starts its threads alike
    import bench
    tflops, _ = bench.measure_fp64_peak(torch, B, torch.device("cuda", 0), reps=2)
    props = torch.cuda.get_device_properties(0)
    assert 0.1 < tflops < props.multi_processor_count * 2 * 2 * 2.2e9 / 1e12, tflops

"""The y and z lines of the mixed form, partitioned (Sec. 3.2 applied inside the GPU to the strided
directions) or solved whole, against the oracle's whole-line solves; the query of the shape in
use; the argument checks; and the autotuner, which times both shapes per direction and restores
the r buffers and the velocity it swept over."""
import numpy as np
import pytest

from tests.gpu_common import B, O, need_gpu, to_np, torch
from paper_1812_01178_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SHAPE = (64, 48, 64)  # y lines: 8 partitions of 6 rows; z lines: 8 of 8
RBUF = [B.NS_BUF_RU, B.NS_BUF_RV, B.NS_BUF_RW]


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
    # the values the FP32 buffers hold
    return [r.astype(np.float32).astype(np.float64) for r in (ru, rv, rw)]


def _load_r(s, r3):
    for bi, r in zip(RBUF, r3):
        s.buffer(bi).copy_(torch.as_tensor(r, device=s.u.device))


@pytest.mark.parametrize("direction", [1, 2])
@pytest.mark.parametrize("whole", [False, True])
@pytest.mark.parametrize("re", [5.0, 400.0])
def test_line_shapes_match_the_oracle(direction, whole, re):
    case, u, v, w, p = I.small_channel(*SHAPE, seed=5)
    case.re = re  # 5: strong coupling (PPT); 400: PDD admissible
    g = O.Grid.from_case(case)
    s = B.Solver(case, u, v, w, p, precision=B.NS_MIXED)
    P0, mode0, drop0 = s.line_partition(direction)
    assert P0 == 8 and mode0 in (B.NS_PART_PPT, B.NS_PART_PDD)
    if mode0 == B.NS_PART_PDD:
        assert drop0 <= 1e-7
    if whole:
        s.set_line_partition(direction, 0)
        assert s.line_partition(direction) == (0, B.NS_PART_PPT, 0.0)
    r3 = _rand_r(case, 31)
    for k in (0, 2):
        beta = O.RK3_ALPHA[k] * case.dt / (2 * case.re)
        before = s.state()[:3]
        _load_r(s, r3)
        s.adi(direction, k)
        if direction == 1:
            got = [to_np(s.buffer(bi)) for bi in RBUF]
        else:
            got = [a - b for a, b in zip(s.state()[:3], before)]
        for q in range(3):
            ref = O.adi_sweep(g, r3[q], direction, q, beta)
            err = np.abs(got[q] - ref).max() / np.abs(ref).max()
            assert err < 1e-5, (direction, whole, k, q, err)
    s.close()


def test_line_partition_arguments():
    case, u, v, w, p = I.small_channel(*SHAPE, seed=5)
    s = B.Solver(case, u, v, w, p, precision=B.NS_MIXED)
    L = B.lib()
    assert L.ns_set_partition(s.ctx, 1, 16, B.NS_PART_AUTO) == B.NS_ERR_ARG  # not the built shape
    assert L.ns_set_partition(s.ctx, 2, 4, B.NS_PART_AUTO) == B.NS_ERR_ARG
    assert L.ns_set_partition(s.ctx, 2, 8, B.NS_PART_PPT) == B.NS_ERR_ARG  # lines take AUTO
    assert L.ns_set_partition(s.ctx, 3, 0, B.NS_PART_AUTO) == B.NS_ERR_ARG
    assert s.line_partition(1)[0] == 8 and s.line_partition(2)[0] == 8  # unchanged
    s.step(1)
    s.sync()
    s.close()
    # FP64 sweeps its y and z lines whole; nx not a multiple of 32 keeps the mixed lines whole
    for prec, shape in ((B.NS_FP64, SHAPE), (B.NS_MIXED, (48, 48, 64))):
        case, u, v, w, p = I.small_channel(*shape, seed=5)
        s = B.Solver(case, u, v, w, p, precision=prec)
        assert s.line_partition(1)[0] == 0 and s.line_partition(2)[0] == 0
        assert L.ns_set_partition(s.ctx, 1, 0, B.NS_PART_AUTO) == B.NS_ERR_UNSUPPORTED
        s.close()


def test_autotune_picks_shapes_and_restores_the_state():
    """After ns_autotune the velocity and r buffers are bitwise what they were, every direction
    holds a valid shape, and the next steps equal those of a context set to the same shapes by
    hand."""
    case, u, v, w, p = I.small_channel(*SHAPE, seed=6, amp=0.2)
    g = O.Grid.from_case(case)
    u, v, w = O.make_divergence_free(g, u, v, w)
    s = B.Solver(case, u, v, w, p, precision=B.NS_MIXED)
    r3 = _rand_r(case, 32)
    _load_r(s, r3)
    s.autotune()
    for a, b in zip(s.state()[:3], (u, v, w)):
        assert np.array_equal(a, b)
    for bi, r in zip(RBUF, r3):
        assert np.array_equal(to_np(s.buffer(bi)), r)
    Px = s.partition()
    Py, Pz = s.line_partition(1)[0], s.line_partition(2)[0]
    assert Py in (0, 8) and Pz in (0, 8)
    s.step(2)
    t = B.Solver(case, u, v, w, p, precision=B.NS_MIXED)
    t.set_partition(Px[0], B.NS_PART_AUTO if Px[1] == B.NS_PART_PDD else B.NS_PART_PPT)
    t.set_line_partition(1, Py)
    t.set_line_partition(2, Pz)
    assert t.partition()[:2] == Px[:2]
    t.step(2)
    for a, b in zip(s.state(), t.state()):
        assert np.array_equal(a, b)
    s.close()
    t.close()

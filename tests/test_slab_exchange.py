"""The exchanges of the y-slab decomposition on the host (gloo ranks, no GPU): which slots every
slab reads (ns_slab_slots, the library's host-only query), their sizes (ns_slab_slot_bytes), the
order of phases and exchanges of a sub-step, and that DistExchange delivers exactly slab s's send
buffer into slot s of every slab that reads it, by point-to-point messages between neighbours or
by an all-gather (Sec. 3.2: PDD exchanges with neighbours, PPT gathers every slab's ends)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1812_01178_gb300 import binding as B  # noqa: E402
from paper_1812_01178_gb300 import inputs as I  # noqa: E402
from paper_1812_01178_gb300 import slabs as S  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not os.path.exists(B.LIB_PATH):
        from paper_1812_01178_gb300 import build
        build.build()


def test_slots_each_slab_reads():
    p = 5
    for r in range(p):
        below, above = max(0, r - 1), min(p - 1, r + 1)
        assert S.slots(p, r, S.NS_XCH_HALO, B.NS_PART_PDD) == (below, above)
        assert S.slots(p, r, S.NS_XCH_ADIY, B.NS_PART_PDD) == (below, above)
        assert S.slots(p, r, S.NS_XCH_ADIY, B.NS_PART_PPT) == (0, p - 1)
        assert S.slots(p, r, S.NS_XCH_VSTAR, B.NS_PART_PDD) == (r, above)
        assert S.slots(p, r, S.NS_XCH_POIS, B.NS_PART_PDD) == (0, p - 1)
        assert S.slots(p, r, S.NS_XCH_PHI, B.NS_PART_PDD) == (below, above)
        assert S.slots(p, r, S.NS_XCH_FLUX, B.NS_PART_PDD) == (0, p - 1)
        assert S.slots(p, r, S.NS_XCH_RCY, B.NS_PART_PDD) == (0, p - 1)


def test_rows_and_slot_sizes():
    case, *_ = I.small_channel(64, 37, 32)
    cfg = B.make_config(case)
    rows = [S.rows(37, 4, r) for r in range(4)]
    assert rows[0][0] == 0 and rows[-1][1] == 37
    assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
    assert all(3 <= j1 - j0 <= 10 for j0, j1 in rows)
    plane = 64 * 32 * 8
    assert S.slot_bytes(cfg, 4, S.NS_XCH_HALO) == 8 * plane      # u, w, p, v rows, both sides
    assert S.slot_bytes(cfg, 4, S.NS_XCH_ADIY) == 6 * plane      # x~_1, x~_m of u, v, w
    assert S.slot_bytes(cfg, 4, S.NS_XCH_VSTAR) == plane
    assert S.slot_bytes(cfg, 4, S.NS_XCH_PHI) == 2 * plane     # phi of both end rows
    assert S.slot_bytes(cfg, 4, S.NS_XCH_POIS) == 2 * 17 * 64 * 16   # complex ends per (kx, kz)
    assert S.slot_bytes(cfg, 4, S.NS_XCH_RCY) == 0  # no recycling: nothing to gather
    assert B.lib().ns_slab_workspace_bytes(B.make_config(case), 13, 0) == 0  # fewer than 3 rows a slab
    # with the recycling inflow: u and w samples of up to ceil(ny / p) rows, v of one face more
    case, *_ = I.boundary_layer(64, 37, 32, amp=0.0)
    case.recycle_i, case.delta_in = 40, 1.0
    cfg = B.make_config(case)
    assert S.slot_bytes(cfg, 4, S.NS_XCH_RCY) == -(-(3 * 10 + 1) * 32 * 8 // 256) * 256
    case.recycle_i = 64  # outside [1, nx - 1]
    assert S.slot_bytes(B.make_config(case), 4, S.NS_XCH_RCY) == 0


class _FakeSlab:
    """Stands in for a slab on the host: a phase writes a tag (slab, exchange, sub-step) into the
    send buffer of the exchange that follows it and records itself."""

    def __init__(self, r, send, log, case):
        self.r, self.send, self.log, self.case = r, send, log, case
        self.next = {ph: xs for ph, xs in S.SUBSTEP}
        self.next[S.NS_SLAB_PACK] = (S.NS_XCH_HALO, S.NS_XCH_RCY)

    def phase(self, ph, k):
        self.log.append((ph, k))
        xs = self.next[ph] + ((S.NS_XCH_RCY,) if ph == S.NS_SLAB_PROJECT and k == 2 else ())
        for x in xs:
            self.send[x].copy_(torch.full_like(self.send[x], (self.r * 16 + x * 3 + k) % 256))


def _worker(rank, world, port, ymode, recycle=False):
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        if recycle:  # the recycling inflow adds the RCY all-gather after PACK and after sub-step 2
            case, *_ = I.boundary_layer(16, 3 * world + 2, 8, amp=0.0)
            case.recycle_i, case.delta_in = 5, 1.0
        else:
            case, *_ = I.small_channel(16, 3 * world + 2, 8)
        cfg = B.make_config(case)
        sizes = [S.slot_bytes(cfg, world, x) for x in range(S.NS_XCH_COUNT)]
        assert (sizes[S.NS_XCH_RCY] > 0) == recycle
        send = [torch.zeros(n, dtype=torch.uint8) for n in sizes]
        recv = [torch.full((world, n), 255, dtype=torch.uint8) for n in sizes]
        log = []
        slab = _FakeSlab(rank, send, log, case)
        ex = S.DistExchange(dist, world, rank, ymode, send, recv)
        seen = []

        def exchange(x):
            ex(x)
            lo, hi = S.slots(world, rank, x, ymode)
            k = log[-1][1]
            for s in range(lo, hi + 1):
                if s != rank:
                    assert int(recv[x][s].min()) == int(recv[x][s].max()) == (s * 16 + x * 3 + k) % 256, (x, s)
            seen.append(x)

        S.run_steps([slab], exchange, 1)
        # PACK, HALO (RCY), then per sub-step RHS/ADIY, ADIZ/VSTAR, POIS/POIS, PHI/PHI, PROJECT/HALO
        # (and RCY after sub-step 2)
        rc = [S.NS_XCH_RCY] if recycle else []
        assert [ph for ph, _ in log] == [S.NS_SLAB_PACK] + [ph for _ in range(3) for ph, _ in S.SUBSTEP]
        assert seen == [S.NS_XCH_HALO] + rc + [x for k in range(3) for _, xs in S.SUBSTEP for x in xs] + rc
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,ymode,recycle", [(2, B.NS_PART_PDD, False), (3, B.NS_PART_PDD, False),
                                                 (3, B.NS_PART_PPT, False), (3, B.NS_PART_PDD, True)])
def test_gloo_ranks_exchange_what_each_slab_reads(world, ymode, recycle):
    mp.start_processes(_worker, args=(world, _free_port(), ymode, recycle), nprocs=world, join=True,
                       start_method="spawn")


def _rows(n, rng, strength):
    """Random tridiagonal rows; strength = how far the diagonal exceeds |a| + |c|."""
    a = -rng.uniform(0.5, 1.5, n)
    c = -rng.uniform(0.5, 1.5, n)
    b = np.abs(a) + np.abs(c) + strength * rng.uniform(0.5, 1.5, n)
    return a, b, c


@pytest.mark.parametrize("n,p", [(12, 4), (48, 3), (64, 8), (30, 2)])
@pytest.mark.parametrize("strength", [20.0, 0.05])
def test_slab_line_algebra_equals_the_dense_partitioned_solves(n, p, strength):
    """The slab tables (block factors, spikes, reduced-system rows) solve a line exactly as the
    oracle's dense matrices of Sec. 3.2 do: PPT (Eq. Zppt) equals the whole-line Thomas solve, PDD
    (Eq. Zpdd) equals the dense PDD, dropped couplings included, and reports the coupling PDD
    drops.  Strongly dominant rows make PDD exact as well; weakly dominant ones make it visibly
    approximate."""
    from oracle import ns_oracle as O
    rng = np.random.default_rng(n * 10 + p)
    a, b, c = _rows(n, rng, strength)
    d = rng.standard_normal(n)
    ref = O.thomas(a, b, c, d)
    x_ppt, _ = S.solve_line_host(a, b, c, d, p, B.NS_PART_PPT)
    np.testing.assert_allclose(x_ppt, O.ppt_solve(a, b, c, d, p), rtol=0, atol=1e-13 * np.abs(ref).max())
    np.testing.assert_allclose(x_ppt, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    x_pdd, drop = S.solve_line_host(a, b, c, d, p, B.NS_PART_PDD)
    np.testing.assert_allclose(x_pdd, O.pdd_solve(a, b, c, d, p), rtol=0, atol=1e-13 * np.abs(ref).max())
    assert drop == pytest.approx(O.pdd_dropped_coupling(a, b, c, p), rel=1e-12, abs=1e-300)
    if strength < 1 and p > 2:
        assert np.abs(x_pdd - ref).max() > 1e-6 * np.abs(ref).max()  # PDD's dropped coupling shows


def test_slab_line_algebra_poisson_rows_with_the_gauge():
    """Rows of the Poisson y solve (zero normal gradient, the (0, 0) mode's gauge row phi_0 = 0)
    split into 4 slabs by PPT equal the whole-line solve (the slabs' Poisson path)."""
    from oracle import ns_oracle as O
    from paper_1812_01178_gb300 import inputs as I
    case, *_ = I.small_channel(16, 48, 8)
    g = O.Grid.from_case(case)
    pa, pc = O.poisson_ycoeffs(g)
    rng = np.random.default_rng(3)
    d = rng.standard_normal(g.ny)
    for lam in (0.0, 0.3, 40.0):
        a, c = pa.copy(), pc.copy()
        b = -(a + c) - lam
        if lam == 0.0:
            a[0], b[0], c[0], d[0] = 0.0, 1.0, 0.0, 0.0
        ref = O.thomas(a, b, c, d)
        x, _ = S.solve_line_host(a, b, c, d, 4, B.NS_PART_PPT)
        np.testing.assert_allclose(x, ref, rtol=0, atol=1e-11 * np.abs(ref).max())

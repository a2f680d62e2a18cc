"""The y-slab decomposition (Sec. 3.2 and Algorithm 1): p slabs held on one GPU, exchanging through
device copies, against the oracle's whole-domain steps and against the single-context path.

The slabs split y into p parts as the paper's GPUs do; the y sweep is solved by PDD (neighbour
exchange) where its dropped coupling is negligible and by PPT (all-gather) otherwise, and the
Poisson y solve by PPT.  Every slab's kernels run in the library; the test only moves the exchange
buffers (device copies) and gathers the owned rows for comparison."""
import numpy as np
import pytest

from tests.gpu_common import B, O, field_rel_errors, need_gpu, torch
from paper_1812_01178_gb300 import inputs as I
from paper_1812_01178_gb300 import slabs as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _projected(shape, seed, **kw):
    case, u, v, w, p = I.small_channel(*shape, seed=seed, **kw)
    g = O.Grid.from_case(case)
    u, v, w = O.make_divergence_free(g, u, v, w)
    return case, g, u, v, w, p


def _run_slabs(case, u, v, w, p, P, steps, ymode=B.NS_PART_AUTO):
    slabs = [S.Slab(case, P, r, u, v, w, p, ymode=ymode) for r in range(P)]
    S.run_steps(slabs, S.LocalExchange(slabs), steps)
    parts = [s.owned() for s in slabs]
    modes = {(s.ymode, s.ydrop) for s in slabs}
    for s in slabs:
        s.close()
    got = tuple(np.concatenate([q[f] for q in parts], axis=1) for f in range(4))
    assert got[0].shape == u.shape and got[1].shape == v.shape
    assert len(modes) == 1  # every slab takes the same mode from the same tables
    return got, modes.pop()


@pytest.mark.parametrize("shape,P", [((64, 48, 32), 2), ((64, 48, 32), 4), ((32, 37, 16), 4), ((48, 20, 24), 3),
                                     ((32, 24, 16), 1), ((32, 64, 16), 8)])
def test_slabs_match_the_oracle(shape, P):
    case, g, u, v, w, p = _projected(shape, 12)
    got, (mode, drop) = _run_slabs(case, u, v, w, p, P, 2)
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, 2)
    errs = field_rel_errors(got, (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs, mode, drop)
    assert np.abs(O.divergence(g, *got[:3])).max() < 1e-10
    # the automatic mode: PDD exactly where the coupling it drops is at most 1e-15
    assert (mode == B.NS_PART_PDD) == (drop <= 1e-15)
    if shape == (64, 48, 32):
        assert mode == B.NS_PART_PDD  # weak coupling at this dt across slabs of 12 and 24 rows


def test_slabs_on_streams_of_their_own():
    """Each slab on its own stream (their kernels overlap, as on separate GPUs); the exchange
    copies are ordered by events.  Same result as the slabs on one stream, to the last bit."""
    case, g, u, v, w, p = _projected((64, 48, 32), 13)
    a, _ = _run_slabs(case, u, v, w, p, 4, 2)
    slabs = [S.Slab(case, 4, r, u, v, w, p, stream=torch.cuda.Stream()) for r in range(4)]
    S.run_steps(slabs, S.LocalExchange(slabs), 2)
    parts = [s.owned() for s in slabs]
    for s in slabs:
        s.close()
    b = tuple(np.concatenate([q[f] for q in parts], axis=1) for f in range(4))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_slabs_match_the_single_context_path():
    case, g, u, v, w, p = _projected((64, 48, 32), 5)
    got, _ = _run_slabs(case, u, v, w, p, 4, 3)
    s = B.Solver(case, u, v, w, p)
    s.step(3)
    one = s.state()
    s.close()
    errs = field_rel_errors(got, one)
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-12, (name, errs)


def test_slabs_strong_coupling_ppt_exact_pdd_not():
    """At a large viscous number the y-sweep spikes decay slowly across a slab: the automatic mode
    takes PPT, which stays exact; PDD forced on the same case drops a coupling far above round-off
    and its error shows it (Sec. 3.2: PDD only where the dropped terms are negligible)."""
    case, g, u, v, w, p = _projected((32, 24, 16), 8, re=0.05, dt=2e-2)
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, 1)
    refs = (ref["u"], ref["v"], ref["w"], ref["p"])
    got, (mode, drop) = _run_slabs(case, u, v, w, p, 4, 1)
    assert mode == B.NS_PART_PPT and drop > 1e-6
    errs = field_rel_errors(got, refs)
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)
    got, (mode, drop2) = _run_slabs(case, u, v, w, p, 4, 1, ymode=B.NS_PART_PDD)
    assert mode == B.NS_PART_PDD and drop2 == drop
    errs = field_rel_errors(got, refs)
    assert max(errs["u"], errs["v"], errs["w"]) > 1e-9, errs


def test_slabs_forced_ppt_equals_pdd_where_pdd_is_admissible():
    case, g, u, v, w, p = _projected((64, 48, 32), 3)
    a, (ma, _) = _run_slabs(case, u, v, w, p, 4, 1, ymode=B.NS_PART_PPT)
    b, (mb, drop) = _run_slabs(case, u, v, w, p, 4, 1, ymode=B.NS_PART_PDD)
    assert (ma, mb) == (B.NS_PART_PPT, B.NS_PART_PDD) and drop <= 1e-15
    errs = field_rel_errors(a, b)
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-13, (name, errs)


def test_slabs_bench_workload_four_slabs():
    """The 256 x 192 x 256 turbulent channel in four slabs, two steps, against the single-context
    path (itself held to the oracle after 10 steps by test_gpu_fullsize_steps)."""
    case, u, v, w, p = I.turbulent_channel()
    g = O.Grid.from_case(case)
    u, v, w = O.make_divergence_free(g, u, v, w)
    got, (mode, drop) = _run_slabs(case, u, v, w, p, 4, 2)
    assert mode == B.NS_PART_PDD
    s = B.Solver(case, u, v, w, p)
    s.step(2)
    one = s.state()
    s.close()
    torch.cuda.empty_cache()
    errs = field_rel_errors(got, one)
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-12, (name, errs)


@pytest.mark.parametrize("P", [2, 4])
def test_slabs_boundary_layer_match_the_oracle(P):
    """The paper's flat-plate configuration (inflow / convective outflow in x, stress-free top) in
    slabs: the outflow planes advance on every slab's rows, and the outflow mass-flux correction
    adds every slab's share (FLUX all-gather) before the Poisson solve."""
    case, u, v, w, p, bl = I.boundary_layer(64, 24, 16, amp=0.05, seed=9, re=200.0)
    g = O.Grid.from_case(case)
    u, v, w, bl = O.make_divergence_free_bl(g, u, v, w, bl)
    slabs = [S.Slab(case, P, r, u, v, w, p, bl=bl) for r in range(P)]
    S.run_steps(slabs, S.LocalExchange(slabs), 2)
    parts = [s.owned() for s in slabs]
    planes = [s.owned_planes() for s in slabs]
    for s in slabs:
        s.close()
    got = tuple(np.concatenate([q[f] for q in parts], axis=1) for f in range(4))
    ref = O.step_bl(g, dict(u=u, v=v, w=w, p=p, bl=bl), case.dt, case.re, case.fx, 2, case.u_conv)
    errs = field_rel_errors(got, (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)
    for q in ("u_out", "v_out", "w_out"):
        plane = np.concatenate([pl[q] for pl in planes], axis=1)
        np.testing.assert_allclose(plane, ref["bl"][q], rtol=0, atol=1e-11 * np.abs(ref["bl"][q]).max())
    assert np.abs(O.divergence_bl(g, *got[:3], ref["bl"])).max() < 1e-10


@pytest.mark.parametrize("P", [2, 3, 4])
def test_slabs_recycled_boundary_layer_match_the_oracle(P):
    """The paper's production configuration: the flat plate with the recycling inflow, in slabs.
    Every slab packs the recycle-plane samples of its rows, an all-gather (RCY) gives each the whole
    plane, and in sub-step 0 each writes the inflow rows it holds (halo rows included) from the
    whole plane.  Against the oracle's recycled steps and the single-context recycled path."""
    case, u, v, w, p, bl = I.boundary_layer(64, 24, 16, amp=0.05, seed=5, re=300.0)
    case.recycle_i, case.delta_in = 40, 1.1
    g = O.Grid.from_case(case)
    u, v, w, bl = O.make_divergence_free_bl(g, u, v, w, bl)
    slabs = [S.Slab(case, P, r, u, v, w, p, bl=bl) for r in range(P)]
    S.run_steps(slabs, S.LocalExchange(slabs), 3)
    parts = [s.owned() for s in slabs]
    planes = [s.owned_planes() for s in slabs]
    for s in slabs:
        s.close()
    got = tuple(np.concatenate([q[f] for q in parts], axis=1) for f in range(4))
    ref = O.step_bl_recycled(g, dict(u=u, v=v, w=w, p=p, bl=bl), case.dt, case.re, case.fx, case.recycle_i,
                             case.delta_in, nsteps=3, u_conv=case.u_conv)
    errs = field_rel_errors(got, (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)
    for q in ("v_in", "w_in", "u_out", "v_out", "w_out"):
        plane = np.concatenate([pl[q] for pl in planes], axis=1)
        np.testing.assert_allclose(plane, ref["bl"][q], rtol=0, atol=1e-11 * (np.abs(ref["bl"][q]).max() + 1e-300))
    one = B.Solver(case, u, v, w, p, bl=bl)
    one.step(3)
    errs = field_rel_errors(got, one.state())
    inflow = one.state()[0][:, :, 0]
    one.close()
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-12, (name, errs)
    assert not np.allclose(inflow, u[:, :, 0])  # the inflow did change
    assert np.abs(O.divergence_bl(g, *got[:3], ref["bl"])).max() < 1e-10


@pytest.mark.parametrize("P", [2, 3])
def test_slabs_kim_moin_pressure_update(P):
    """The Kim-Moin pressure update p += phi - beta_k lap(phi) in slabs: the Laplacian of phi at a
    slab's end rows reads the neighbours' phi rows, which the PHI exchange carries both ways."""
    case, g, u, v, w, p = _projected((32, 24, 16), 3, amp=0.2, re=40.0)
    case.pressure_update = B.NS_PRESSURE_KIM_MOIN
    got, _ = _run_slabs(case, u, v, w, p, P, 2)
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, 2, pressure="kim_moin")
    errs = field_rel_errors(got, (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)
    plain = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, 2)
    assert field_rel_errors(got, (plain["u"], plain["v"], plain["w"], plain["p"]))["p"] > 1e-6  # the forms differ


def test_slab_arguments_rejected_on_the_host():
    case, g, u, v, w, p = _projected((32, 24, 16), 1)
    with pytest.raises(B.NSError):
        S.Slab(case, 9, 0, u, v, w, p)  # 24 rows cannot give 9 slabs of 3 rows
    case.precision = B.NS_MIXED
    with pytest.raises(B.NSError):
        S.Slab(case, 2, 0, u, v, w, p)


def _rank_worker(rank, world, port, case, fields, steps, out_dir):
    import os
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1812_01178_gb300 import slabs as S2
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        slab = S2.Slab(case, world, rank, *fields)
        ex = S2.DistExchange(dist, world, rank, slab.ymode, slab.send, slab.recv, host=True)
        S2.run_steps([slab], ex, steps)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), *slab.owned())
        slab.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_slabs_as_separate_processes(world, tmp_path):
    """One slab per process (the paper's one slab per GPU), the exchanges over torch.distributed:
    gloo between processes that share this GPU, the device buffers staged through host memory.
    No kernel waits on another process: every exchange is a host-side message between phases."""
    import socket
    import torch.multiprocessing as mp
    case, g, u, v, w, p = _projected((64, 48, 32), 21)
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mp.start_processes(_rank_worker, args=(world, port, case, (u, v, w, p), 2, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    parts = [np.load(tmp_path / ("rank%d.npz" % r)) for r in range(world)]
    got = tuple(np.concatenate([q["arr_%d" % f] for q in parts], axis=1) for f in range(4))
    ref = O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, 2)
    errs = field_rel_errors(got, (ref["u"], ref["v"], ref["w"], ref["p"]))
    for name in ("u", "v", "w", "p"):
        assert errs[name] < 1e-11, (name, errs)


def test_bench_slab_mode_two_ranks_share_the_gpu():
    """bench.py --slabs under torch.distributed.run: the bench workload cut into two y-slabs, one
    per rank, the exchanges over gloo staged through host memory (both ranks on this GPU).  One JSON
    line with the contract's keys, strong scaling."""
    import json
    import os
    import socket
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(root, "bench.py"), "--gpus", "2", "--slabs",
           "--backend", "gloo", "--steps", "2", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=root)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["scaling"] == "strong" and d["steps"] == 2 and d["value"] > 0
    assert d["config"]["slab_rows"] == [96, 96] and d["config"]["y_sweep"] == "PDD"

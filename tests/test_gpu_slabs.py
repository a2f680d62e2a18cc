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


def test_slab_arguments_rejected_on_the_host():
    case, g, u, v, w, p = _projected((32, 24, 16), 1)
    with pytest.raises(B.NSError):
        S.Slab(case, 9, 0, u, v, w, p)  # 24 rows cannot give 9 slabs of 3 rows
    case.precision = B.NS_MIXED
    with pytest.raises(B.NSError):
        S.Slab(case, 2, 0, u, v, w, p)

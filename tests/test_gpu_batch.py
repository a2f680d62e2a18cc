"""Batched ensembles: one persistent launch per stage for all instances (ns_batch_*)."""
import numpy as np
import pytest

from tests.gpu_common import B, O, field_rel_errors, need_gpu
from paper_1812_01178_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _ensemble(n, precision=0):
    ens = I.ensemble(n, seed=77, amp=0.05, sizes_x=(16, 32, 64), sizes_y=(9, 16, 20))
    for case, *_ in ens:
        case.precision = precision
    return ens


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_single_instances(precision):
    """The batched step is the same arithmetic as stepping each instance alone: bitwise equal."""
    ens = _ensemble(6, precision)
    b = B.Batch([e[0] for e in ens], [e[1:] for e in ens])
    b.make_divergence_free()
    b.step(2)
    for q, (case, u, v, w, p) in enumerate(ens):
        s = B.Solver(case, u, v, w, p)
        s.set_partition(*B.ns_get_partition(b.instance(q))[:2])
        s.make_divergence_free()
        s.step(2)
        for a_, b_ in zip(s.state(), b.state(q)):
            assert np.array_equal(a_, b_), q
        s.close()
    # one launch per stage per kernel variant, far fewer than instances x stages
    assert b.launches_per_step() < 3 * 10 * 6
    b.close()


def test_batch_vs_oracle_and_autotune():
    ens = _ensemble(5)
    b = B.Batch([e[0] for e in ens], [e[1:] for e in ens])
    b.autotune()
    refs = []
    for case, u, v, w, p in ens:
        g = O.Grid.from_case(case)
        u, v, w = O.make_divergence_free(g, u, v, w)
        refs.append((g, O.step(g, dict(u=u, v=v, w=w, p=p), case.dt, case.re, case.fx, nsteps=3)))
    b.make_divergence_free()
    b.step(3)
    for q, (g, ref) in enumerate(refs):
        errs = field_rel_errors(b.state(q), (ref["u"], ref["v"], ref["w"], ref["p"]))
        for name in ("u", "v", "w", "p"):
            assert errs[name] < 1e-11, (q, name, errs)
    b.close()

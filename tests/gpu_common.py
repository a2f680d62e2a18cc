"""Helpers shared by the GPU parity tests (CUDA path through the C ABI vs the FP64 oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns_oracle as O  # noqa: E402
from paper_1812_01178_gb300 import binding as B  # noqa: E402


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_l2(a, b, scale=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b) if scale is None else scale
    return float(np.linalg.norm(a - b) / max(den, 1e-300))


def field_rel_errors(gpu, ref):
    """Relative L2 errors of (u, v, w, p).

    u, v, w are normalised by the norm of the whole reference velocity (v and w are ~0 in
    channel flows).  p is compared with its mean removed and normalised by
    max(||p||, ||u||^2 / sqrt(N)), i.e. never by less than the dynamic-pressure scale: a
    perturbation pressure 1e-5 of that scale is fixed by the data only to ~1e-10 of itself (the
    divergence of u* cancels O(1) terms), so a plain ||p||-relative error measures rounding
    order, not correctness.  'p_strict' reports the plain ||p||-relative error as well.
    """
    gu, gv, gw, gp = gpu
    ru, rv, rw, rp = ref
    vel2 = np.linalg.norm(ru) ** 2 + np.linalg.norm(rv) ** 2 + np.linalg.norm(rw) ** 2
    vel = np.sqrt(vel2)
    pr = rp - rp.mean()
    pscale = max(np.linalg.norm(pr), vel2 / np.sqrt(rp.size))
    return dict(u=rel_l2(gu, ru, vel), v=rel_l2(gv, rv, vel), w=rel_l2(gw, rw, vel),
                p=rel_l2(gp - gp.mean(), pr, pscale), p_strict=rel_l2(gp - gp.mean(), pr))


def to_np(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()

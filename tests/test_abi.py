"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/ns.h declares
(no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1812_01178_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ns.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ns_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    if not os.path.exists(B.LIB_PATH):
        from paper_1812_01178_gb300 import build
        build.build()
    return B.LIB_PATH


def test_header_declares_the_binding_exports():
    assert _declared() == sorted(B.EXPORTS)


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name


@pytest.mark.parametrize("nx,nz,ok", [
    (64, 32, True), (48, 32, True), (96, 24, True), (72, 216, True), (384, 96, True), (768, 8, True),
    (1536, 48, True), (2048, 1024, True),
    (40, 32, False),    # factor 5: not 2^a 3^b
    (12, 32, False),    # a < 3
    (64, 36, False),    # nz = 4 * 9: a < 3
    (216, 32, False),   # 8 * 27: no partition shape (P <= 32 lanes of M rows)
    (1152, 32, False),  # 128 * 9: M = 36 at P = 32 is not a built shape
    (6144, 32, False),  # beyond 4096
])
def test_grid_sizes_accepted_and_rejected_without_gpu(libpath, nx, nz, ok):
    """nx and nz are 2^a 3^b with a >= 3 (the mixed radix-2/4/3 FFT), and nx admits a partition
    shape of the x solver; the check runs on the host (no device call)."""
    from paper_1812_01178_gb300 import inputs as I
    case, *_ = I.small_channel(64, 20, 32)
    case.nx, case.nz = nx, nz
    assert (B.ns_workspace_bytes(B.make_config(case)) > 0) == ok


@pytest.mark.parametrize("bc_x,ir,delta_in,ok", [
    (1, 5, 1.0, True), (1, 0, 0.0, True), (0, 5, 1.0, False), (1, 64, 1.0, False), (1, -1, 1.0, False),
    (1, 5, 0.0, False), (1, 5, float("inf"), False)])
def test_recycling_options_checked_without_gpu(libpath, bc_x, ir, delta_in, ok):
    from paper_1812_01178_gb300 import inputs as I
    case, *_ = I.boundary_layer(64, 12, 16)
    case.bc_x, case.recycle_i, case.delta_in = bc_x, ir, delta_in
    assert (B.ns_workspace_bytes(B.make_config(case)) > 0) == ok


@pytest.mark.parametrize("pu,ok", [(0, True), (1, True), (2, False), (-1, False)])
def test_pressure_update_option_checked_without_gpu(libpath, pu, ok):
    from paper_1812_01178_gb300 import inputs as I
    case, *_ = I.small_channel(32, 12, 16)
    case.pressure_update = pu
    assert (B.ns_workspace_bytes(B.make_config(case)) > 0) == ok

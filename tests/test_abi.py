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
    return sorted(set(re.findall(r"\b(ns_[a-z0-9_]+)\s*\(", src)))


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


def test_null_handles_are_rejected_without_gpu(libpath):
    """Every entry point checks its context (or batch) handle before any device call: a NULL
    handle returns NS_ERR_ARG, and the query / teardown calls accept it."""
    L = B.lib()
    E = B.NS_ERR_ARG
    null = None
    for name, args in [("ns_rhs", (0,)), ("ns_adi_sweep", (0, 0)), ("ns_poisson_solve", (0,)),
                       ("ns_project", (0,)), ("ns_substep", (0,)), ("ns_make_divergence_free", ()),
                       ("ns_step", (1,)), ("ns_set_dt", (1e-3,)), ("ns_step_cfl", (1, 0.5, None)),
                       ("ns_set_partition", (0, 8, 0)), ("ns_set_partition", (1, 0, 0)),
                       ("ns_set_partition", (2, 0, 0)), ("ns_autotune", ()), ("ns_sync", ())]:
        assert getattr(L, name)(null, *args) == E, name
    P, mode, drop = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    for d in (0, 1, 2):
        assert L.ns_get_partition(null, d, ctypes.byref(P), ctypes.byref(mode), ctypes.byref(drop)) == E
    rate = ctypes.c_double()
    assert L.ns_convective_rate(null, ctypes.byref(rate)) == E
    assert L.ns_batch_step(null, 1) == E
    assert L.ns_batch_autotune(null) == E
    assert L.ns_batch_set_partition(null, 0, 8, 0) == E
    assert L.ns_batch_sync(null) == E
    assert L.ns_batch_launches_per_step(null) == 0
    assert L.ns_batch_instance(null, 0) is None
    L.ns_destroy(null)
    L.ns_batch_destroy(null)


def test_traffic_record_is_dropped_when_its_kernel_source_changes(tmp_path, monkeypatch):
    """bench.py reports an ncu traffic figure only while the kernel source it was captured from
    is unchanged (the committed hash); otherwise the roofline's traffic is null."""
    import hashlib
    import json
    import sys
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    rec = {"rhs": {"bytes_per_launch": 123.0, "source": "k.cu",
                   "source_sha256_16": hashlib.sha256(src.read_bytes()).hexdigest()[:16]}}
    (tmp_path / "profiles" / "traffic_w.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("w", "rhs") == 123.0
    assert bench.load_traffic("w", "adi_x") is None
    assert bench.load_traffic("missing", "rhs") is None
    src.write_text("__global__ void k() { }\n")
    assert bench.load_traffic("w", "rhs") is None

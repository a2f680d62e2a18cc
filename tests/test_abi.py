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


def test_invalid_config_rejected_without_gpu(libpath):
    from paper_1812_01178_gb300 import inputs as I
    case, *_ = I.small_channel(64, 20, 32)
    cfg = B.make_config(case)
    assert B.ns_workspace_bytes(cfg) > 0
    case.nx = 48  # not a power of two
    assert B.ns_workspace_bytes(B.make_config(case)) == 0

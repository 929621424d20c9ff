"""The C ABI library: it builds, loads, exports every function declared in
include/*.h, and its host-only calls behave (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1210_7325_gb300 import build as gbuild
from paper_1210_7325_gb300 import gls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return gls.load()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(gls_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gls_plan_create", "gls_factor", "gls_solve_block", "gls_destroy",
                     "gls_solve_stream", "gls_status_string", "gls_plan_footprint_bytes"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(gls.LIB_PATH)
    for name in declared_functions():
        assert hasattr(raw, name), f"{name} declared but not exported"


def test_status_strings(lib):
    for code, name in gls.STATUS_NAMES.items():
        assert lib.gls_status_string(code).decode() == name
    assert lib.gls_status_string(99).decode() == "GLS_ERR_UNKNOWN"
    assert lib.gls_version() >= 100


def test_footprint(lib):
    f64 = gls.footprint_bytes(1000, 4, 4096, "fp64")
    npad = 1024
    assert f64 >= 2 * npad * npad * 8
    mix = gls.footprint_bytes(1000, 4, 4096, "bf16")
    assert mix > f64 - 16 * 4 * 4097 * 8  # mixed adds the operand slices
    assert gls.footprint_bytes(0, 4, 10) == 0          # invalid n
    assert gls.footprint_bytes(10, 0, 10) == 0         # invalid p
    assert gls.footprint_bytes(10, 33, 10) == 0        # p beyond 32
    assert gls.footprint_bytes(10, 3, 0) == 0          # no block


def test_invalid_descriptions_rejected_without_gpu(lib):
    h = ctypes.c_void_p()
    d = gls.make_desc(10, 0, 10)
    assert lib.gls_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1
    d = gls.make_desc(10, 3, 10, split_terms=5)
    assert lib.gls_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1
    d = gls.make_desc(10, 3, 10, flags=0x80)
    assert lib.gls_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert "flag" in gls.last_error()
    assert lib.gls_plan_create(None, ctypes.byref(h)) == 1
    d = gls.make_desc(10, 3, 10, wait_limit_us=-1)
    assert lib.gls_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1
    d = gls.make_desc(10, 3, 10, host_wait_ms=-5)
    assert lib.gls_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert "host_wait_ms" in gls.last_error()
    d = gls.make_desc(10, 20, 10, phenotypes=14)       # p - 1 + t = 33 > 32
    assert lib.gls_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert "phenotypes" in gls.last_error()
    d = gls.make_desc(10, 20, 10, phenotypes=13)
    assert gls.footprint_bytes(10, 20, 10, phenotypes=13) > gls.footprint_bytes(10, 20, 10)
    assert lib.gls_destroy(None) == 0


def test_desc_layout_matches_header():
    # 8 + 4 + 4 + 8 + 4 + 4 + 8 + 4 + 4 + 4 + 5 * 4 bytes, 8-aligned
    assert ctypes.sizeof(gls.PlanDesc) == 72
    assert gls.PlanDesc.wait_limit_us.offset == 44 and gls.PlanDesc.phenotypes.offset == 52
    assert gls.PlanDesc.reserved.offset == 56
    assert ctypes.sizeof(gls.Stats) == 15 * 8


def test_null_plan_calls_are_errors(lib):
    assert lib.gls_factor(None, None, 0, None, 0, None, None) == 1
    assert lib.gls_solve_block(None, None, 0, 0, None, 0, None) == 1
    assert lib.gls_solve_stream(None, None, 0, 0, None, 0, None) == 1
    assert lib.gls_synchronize(None) == 1
    assert lib.gls_plan_stream(None) is None
    assert lib.gls_plan_wait_event(None, None) == 1
    assert lib.gls_plan_operand_precision(None) == -1


def test_no_device_reports_unsupported(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    d = gls.make_desc(100, 3, 10)
    assert lib.gls_plan_create(ctypes.byref(d), ctypes.byref(h)) == 7

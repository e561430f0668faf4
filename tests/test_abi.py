"""The C-ABI library builds for sm_103a, loads without a GPU, exports every entry point that
include/wbrzf.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wbrzf.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(wbrzf_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2512_16543_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("wbrzf_create", "wbrzf_full_inverse", "wbrzf_update", "wbrzf_sum_rate",
                     "wbrzf_destroy", "wbrzf_workspace_bytes"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_host_side_validation_without_gpu(libpath):
    from paper_2512_16543_gb300 import binding
    L = binding.lib()
    rule = binding.RankRule().to_c()
    assert L.wbrzf_workspace_bytes(0, 8, 8, binding.C64, ctypes.byref(rule)) == 0
    assert L.wbrzf_workspace_bytes(4, 64, 8, binding.C64, ctypes.byref(rule)) > 0
    # K > 64 runs only on the blocked engine, which needs the sketch width within its limit:
    # the default rule at K = 512 lets d grow to K (refused), r_max = 64 keeps d <= 72
    eng = L.wbrzf_workspace_bytes_engine
    simt, blocked = binding.ENGINES["simt"], binding.ENGINES["blocked"]
    assert L.wbrzf_workspace_bytes(4, 8, 65, binding.C64, ctypes.byref(rule)) > 0
    assert eng(4, 8, 65, binding.C64, ctypes.byref(rule), simt) == 0
    assert L.wbrzf_workspace_bytes(1, 4096, 512, binding.C64, ctypes.byref(rule)) == 0
    r64 = binding.RankRule(k_init=2, p=8, r_max=64).to_c()
    assert L.wbrzf_workspace_bytes(1, 4096, 512, binding.C64, ctypes.byref(r64)) == \
        eng(1, 4096, 512, binding.C64, ctypes.byref(r64), blocked) > 0
    assert eng(4, 64, 8, binding.C64, ctypes.byref(rule), blocked) > \
        L.wbrzf_workspace_bytes(4, 64, 8, binding.C64, ctypes.byref(rule))
    assert eng(4, 64, 8, binding.C64, ctypes.byref(rule), binding.ENGINES["blocked_fma"]) == \
        eng(4, 64, 8, binding.C64, ctypes.byref(rule), blocked)
    assert eng(4, 64, 8, binding.C64, ctypes.byref(rule), 5) == 0           # no such engine
    assert eng(4, 63, 8, binding.C64, ctypes.byref(rule), binding.ENGINES["tensor"]) == 0
    bad = binding.RankRule(eta=1.5).to_c()
    assert L.wbrzf_workspace_bytes(4, 64, 8, binding.C64, ctypes.byref(bad)) == 0
    a = (ctypes.c_double * 1)(0.8)
    s = (ctypes.c_double * 1)(0.1)
    h = ctypes.c_void_p()
    # invalid: no workspace; negative alpha; misaligned workspace
    assert L.wbrzf_create(1, 64, 8, a, s, 1.0, ctypes.byref(rule), 0, 1, None, 0, None,
                          ctypes.byref(h)) == 1
    neg = (ctypes.c_double * 1)(-1.0)
    assert L.wbrzf_create(1, 64, 8, neg, s, 1.0, ctypes.byref(rule), 0, 1, 256, 1 << 20, None,
                          ctypes.byref(h)) == 1
    assert L.wbrzf_create(1, 64, 8, a, s, 1.0, ctypes.byref(rule), 0, 1, 257, 1 << 20, None,
                          ctypes.byref(h)) == 1
    assert L.wbrzf_create(1, 64, 8, a, s, 1.0, ctypes.byref(rule), 0, 1, 256, 16, None,
                          ctypes.byref(h)) == 3          # workspace too small
    assert L.wbrzf_update(None, None, None) == 1
    assert L.wbrzf_set_state(None, None, None, None) == 1          # checkpoint restore
    L.wbrzf_selftest_bounded_wait.restype = ctypes.c_int
    assert L.wbrzf_selftest_bounded_wait(None, None) == 1           # no output buffer
    assert L.wbrzf_status_string(0) == b"ok"
    L.wbrzf_destroy(None)


def test_resolved_sizes_match_rule_defaults():
    from paper_2512_16543_gb300 import binding
    assert binding.resolved_sizes(32, binding.RankRule(k_init=2, p=8, r_max=16)) == (16, 4, 24, 16)
    assert binding.resolved_sizes(8, binding.RankRule(k_init=2, p=1)) == (8, 3, 8, 8)
    assert binding.resolved_sizes(512, binding.RankRule(k_init=2, p=8, r_max=64)) == (64, 6, 72, 64)

"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/*.h declares; the Python binding binds each of them by the same name.
No compute call is made (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1802_00036_gb300 import build, dc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(dc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("dc_create", "dc_complete", "dc_complete_uniform", "dc_complete_host", "dc_destroy",
              "dc_params_default", "dc_status_str", "dc_reserve", "dc_last_async_error",
              "dc_last_launch_count"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_uses_the_c_names():
    bound = {name for name, _, _ in dc.SIGNATURES}
    assert bound == declared_functions()
    for name in bound:
        assert callable(getattr(dc, name)), name


def test_status_strings_without_gpu(lib):
    dc.load()
    assert dc.dc_status_str(0) == "DC_OK"
    assert dc.dc_status_str(1) == "DC_ERR_INVALID_ARG"
    assert dc.dc_status_str(99) == "DC_ERR_UNKNOWN"


def test_params_default_is_the_papers_design(lib):
    p = dc.dc_params_default()
    assert (p.first_kernel, p.large_fill, p.median, p.blur) == (0, 31, 1, 1)
    assert (p.extend_top, p.extend_rows, p.large_fill_on, p.stop_after) == (1, -1, 1, 0)


def test_tune_cache_round_trip(tmp_path, monkeypatch):
    from paper_1802_00036_gb300 import tune
    monkeypatch.setenv("DCGB_TUNE_CACHE", str(tmp_path / "t.json"))
    p = dc.params()
    k = tune.cache_key("GB300", 152, 64, 352, 1216, p)
    assert k != tune.cache_key("GB300", 152, 64, 352, 1216, dc.params(blur="bilateral"))
    tune.save_cache({k: [6, 3, 16]})
    assert tune.load_cache()[k] == [6, 3, 16]
    (tmp_path / "t.json").write_text("not json")
    assert tune.load_cache() == {}


def test_params_struct_layout_matches_header():
    # ten 4-byte fields, no padding
    assert ctypes.sizeof(dc.dc_params) == 40
    assert ctypes.sizeof(dc.dc_frame) == 2 * ctypes.sizeof(ctypes.c_void_p) + 16


def test_calls_without_a_context_are_refused(lib):
    # checked before any CUDA call: no GPU needed
    L = dc.load()
    INVALID = 1
    assert L.dc_set_graph_cache(None, 1) == INVALID
    assert L.dc_set_profiling(None, 1) == INVALID
    assert L.dc_host_wait(None) == INVALID
    assert L.dc_graph_cache_entries(None) == 0
    assert L.dc_last_launch_count(None) == 0
    n = ctypes.c_int(-1)
    buf = (ctypes.c_float * 2)()
    assert L.dc_kernel_times(None, buf, 1, ctypes.byref(n)) == INVALID
    p = dc.dc_params_default()
    assert L.dc_complete_uniform(None, None, None, 1, 8, 8, ctypes.byref(p), None) == INVALID
    assert L.dc_inject_fault(None, dc.DC_FAULT_WAIT) == INVALID
    t = dc.dc_tuning(8, 5, 160, 128)
    assert L.dc_set_class_tuning(None, 8, 8, ctypes.byref(t)) == INVALID
    assert L.dc_set_class_tuning(None, 0, 0, None) == INVALID

"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/tab.h declares, and rejects bad arguments before any
CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(tab_\w+)\s*\(", src, flags=re.M):
            if "static inline" in src[max(0, m.start() - 40):m.start() + 60]:
                continue
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_00384_gb300 import build
    build.build()
    return ctypes.CDLL(os.path.join(ROOT, "paper_2408_00384_gb300", "libtab.so"))


def test_header_parses():
    names = declared_functions()
    assert "tab_create" in names and "tab_batch_run" in names and "tab_measure" in names
    assert "tab_make_gate" not in names


def test_every_declared_symbol_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_imports_and_errors_without_gpu(lib):
    from paper_2408_00384_gb300 import tab
    h = ctypes.c_void_p()
    assert tab._L.tab_create(0, ctypes.byref(h)) == tab.TAB_ERANGE
    assert "outside" in tab.last_error()
    assert tab._L.tab_create(tab.MAX_QUBITS + 1, ctypes.byref(h)) == tab.TAB_ERANGE
    assert tab._L.tab_create(5, None) == tab.TAB_EINVAL
    assert tab._L.tab_destroy(None) == tab.TAB_OK
    assert tab._L.tab_bytes_required(0) == 0


def test_gate_word_layout_matches_header():
    from workloads import circuits as C
    g = int(C.encode(C.TAB_CNOT, 123456, 654321))
    assert g >> 56 == 7 and (g >> 28) & 0xFFFFFFF == 123456 and g & 0xFFFFFFF == 654321
    src = open(os.path.join(ROOT, "include", "tab.h")).read()
    for name in ("I", "X", "Y", "Z", "H", "S", "SDG", "CNOT", "CZ", "SWAP", "MZ", "MZR", "BARRIER"):
        m = re.search(rf"TAB_{name}\s*=\s*(\d+)", src)
        assert m and int(m.group(1)) == getattr(C, f"TAB_{name}"), name


def test_run_config_validation_without_gpu(lib):
    """tab_set_config rejects out-of-range fields and changes nothing then;
    a valid change reads back and can be undone (host logic, no GPU)."""
    from paper_2408_00384_gb300 import tab
    old = tab.get_config()
    for bad in ({"block_threads": 100}, {"meas_batch": 3}, {"meas_batch": 64},
                {"grid_ctas": -1}, {"debug": 1 << 7}, {"batch_chunks": -1},
                {"batch_chunks": 65}, {"reserved": 1}):
        with pytest.raises(tab.TabError) as ei:
            tab.set_config(bad)
        assert ei.value.code == tab.TAB_EINVAL
        assert tab.get_config() == old
    try:
        tab.set_config({"block_threads": 256, "meas_batch": 8, "wait_limit_ns": 123456,
                        "batch_chunks": 64})
        got = tab.get_config()
        assert got["block_threads"] == 256 and got["meas_batch"] == 8
        assert got["wait_limit_ns"] == 123456 and got["batch_chunks"] == 64
    finally:
        tab.set_config(old)
    assert tab.get_config() == old

"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point declared in include/tcw.h; status codes have names; calls made
without a GPU fail with a status instead of crashing."""
import ctypes
import os
import re

import pytest

import paper_2507_07816_gb300 as tcw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:tcw_status|const char \*)\s*(tcw_\w+)\s*\(", text, re.M))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("tcw_create", "tcw_destroy", "tcw_load_spectrogram", "tcw_load_velocity",
              "tcw_define_bank", "tcw_define_sky", "tcw_search", "tcw_get_statistics",
              "tcw_track_bins", "tcw_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = tcw.load_library()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    lib = tcw.load_library()
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        s = lib.tcw_status_string(code).decode()
        assert s and s != "unknown status"
    assert lib.tcw_status_string(-99).decode() == "unknown status"


def test_create_rejects_null_and_bad_device():
    lib = tcw.load_library()
    assert lib.tcw_create(None, 0, None) == -1
    h = ctypes.c_void_p()
    st = lib.tcw_create(ctypes.byref(h), -1, None)
    assert st in (-1, -2)
    assert lib.tcw_destroy(None) == 0


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_2507_07816_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text
                assert "tcw_oracle" not in text and "tcw_synth" not in text, f

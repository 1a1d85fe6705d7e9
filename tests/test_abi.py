"""The C interface: the library builds here (cross-compiled for sm_103a),
loads, and exports every function include/dsrg.h declares.  No compute call
is made, so this runs without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dsrg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dsrg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ("dsrg_init", "dsrg_pt2", "dsrg_pt3", "dsrg_free", "dsrg_last_error"):
        assert n in names


def test_library_builds_and_exports_every_symbol():
    from paper_1701_02011_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_exports_match_header():
    import paper_1701_02011_gb300 as g
    assert sorted(g.EXPORTS) == _declared()


def test_null_handle_is_an_error_not_a_crash():
    import paper_1701_02011_gb300 as g
    lib = g.load_library()
    e = g.dsrg_energies()
    assert lib.dsrg_pt3(None, ctypes.byref(e)) == -4
    assert b"NULL" in lib.dsrg_last_error()
    assert lib.dsrg_last_launch_count(None) == -1
    lib.dsrg_free(None)

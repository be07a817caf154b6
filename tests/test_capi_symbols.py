"""CPU-side checks of the C ABI: the library builds, loads and exports every
function include/hevi.h declares (no GPU calls)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hevi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hevi_[A-Za-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = _declared()
    for n in ("hevi_setup", "hevi_factor", "hevi_stage_solve", "hevi_newton_solve",
              "hevi_apply_Lv", "hevi_column_status", "hevi_destroy", "hevi_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2311_11425_gb300 as hv
    from paper_2311_11425_gb300 import build
    build.build()
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    hv.load()
    assert hv.load().hevi_status_string(5) == b"not converged"
    assert hv.load().hevi_status_string(7) == b"device wait past its limit"
    assert hv.STATUS[7] == "device wait past its limit"


def test_tableaux_without_gpu():
    import numpy as np
    import paper_2311_11425_gb300 as hv
    t = hv.tableau("ARK3")
    assert t.s == 4 and abs(t.b.sum() - 1) < 1e-15
    with pytest.raises(hv.HeviError):
        hv.tableau("nope")

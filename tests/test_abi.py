"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/tatrg.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2412_14104_gb300 import build
    return build.build()


def declared():
    src = open(os.path.join(ROOT, "include", "tatrg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tatrg_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for required in ("tatrg_create", "tatrg_init_ising", "tatrg_rg_step", "tatrg_lnZ",
                     "tatrg_grad", "tatrg_sweep", "tatrg_destroy", "tatrg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing


def test_bad_arguments_fail_without_a_gpu(libpath):
    import paper_2412_14104_gb300 as tg
    L = tg.lib()
    h = ctypes.c_void_p()
    bad = tg.Params(0, 2, 2, tg.TRIAD, tg.FP64, 0, 4, 0, 0, 0, 0)
    assert L.tatrg_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
    assert b"chi" in L.tatrg_last_error(None)
    assert L.tatrg_rg_step(None, 1) == 1

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
    bad = tg.Params(0, 2, 2, tg.TRIAD, tg.FP64, 0, 4, 0, 0, 0, 0, 0, 0)
    assert L.tatrg_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
    assert b"chi" in L.tatrg_last_error(None)
    assert L.tatrg_rg_step(None, 1) == 1


def test_building_blocks_reject_bad_sizes_before_touching_memory(libpath):
    """Argument checks of the device building blocks run on the host before any launch or
    copy, so they can be exercised here with placeholder pointers."""
    import paper_2412_14104_gb300 as tg
    L = tg.lib()
    fake = ctypes.c_void_p(256)  # never dereferenced: every call below fails its checks first
    k = ctypes.c_int(0)
    # contraction: an extent of 0, a precision out of range
    c = tg._contraction([(0, 1, 1)], [(4, 1, 1)], [(4, 1, 1)], 1.0, 0.0)
    assert L.tatrg_contract(ctypes.byref(c), 0, fake, fake, fake, None) == 1
    c = tg._contraction([(4, 4, 4)], [(4, 1, 1)], [(4, 1, 4)], 1.0, 0.0)
    assert L.tatrg_contract(ctypes.byref(c), 5, fake, fake, fake, None) == 1
    assert L.tatrg_contract(ctypes.byref(c), 0, None, fake, fake, None) == 1
    # the generated-sketch contraction exists for the split precisions only
    assert L.tatrg_contract_sketch(ctypes.byref(c), 0, fake, 1, 2, 0, fake, None) == 1
    assert b"split precision" in L.tatrg_last_error(None)
    # SVD and orthonormalisation need m >= n and 1 <= n <= 1024
    assert L.tatrg_svd(3, 4, fake, fake, fake, fake, None) == 1
    assert L.tatrg_svd(5000, 1025, fake, fake, fake, fake, None) == 1
    assert L.tatrg_svd_noalloc(3, 4, fake, fake, fake, fake, None) == 1
    assert L.tatrg_orth(0, 3, 4, fake, fake, fake, ctypes.byref(k), None) == 1
    assert L.tatrg_orth(9, 8, 4, fake, fake, fake, ctypes.byref(k), None) == 1
    # sketches: negative sizes
    assert L.tatrg_gaussian(1, 2, 0, -1, 4, fake, None) == 1
    # raw Philox words: negative count, null output; the wait limit: negative
    assert L.tatrg_philox_words(1, 2, 0, 0, -1, fake, None) == 1
    assert L.tatrg_philox_words(1, 2, 0, 0, 4, None, None) == 1
    assert L.tatrg_set_barrier_limit_ns(-1) == 1
    # the two-CTA tile policy: -1, 0, 1 or 2
    assert L.tatrg_set_cta_pairs(3) == 1
    assert L.tatrg_set_cta_pairs(-2) == 1

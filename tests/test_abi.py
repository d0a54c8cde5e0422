"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/tatrg.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import numpy as np

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
    # a negative stride would reach below the caller's base pointer
    c = tg._contraction([(4, -4, 4)], [(4, 1, 1)], [(4, 1, 4)], 1.0, 0.0)
    assert L.tatrg_contract(ctypes.byref(c), 0, fake, fake, fake, None) == 1
    assert b"non-negative" in L.tatrg_last_error(None)
    c = tg._contraction([(4, 4, 4)], [(4, 1, 1)], [(4, 1, 4)], 1.0, 0.0)
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


def test_binding_checks_caller_tensors_before_any_call():
    """The building blocks address caller-owned device memory only through a pointer and
    the call's sizes, which the library cannot check against an allocation it does not
    own; the binding rejects a wrong dtype, a non-contiguous layout, too few elements for
    the extents the call addresses, negative strides and host tensors (EINVAL), before the
    library is called."""
    import torch
    import paper_2412_14104_gb300 as tg

    def code(f, *a, **kw):
        with pytest.raises(tg.TatrgError) as e:
            f(*a, **kw)
        return e.value.code, str(e.value)

    f64 = lambda *s: torch.zeros(s, dtype=torch.float64)
    # C[m, n] = A[m, k] B[k, n] with M, N, K = 5, 4, 3: A needs 15, B 12, C 20 elements
    m, n, k = [(5, 3, 4)], [(4, 1, 1)], [(3, 1, 4)]
    assert tg._reach(m, 1) == 13 and tg._reach(k, 2) == 9 and tg._reach([(0, 7, 7)], 1) == 0
    c, msg = code(tg.contract, m, n, k, f64(15).float(), f64(12), f64(20))
    assert c == 1 and "dtype" in msg
    c, msg = code(tg.contract, m, n, k, f64(14), f64(12), f64(20))
    assert c == 1 and "A holds 14 elements, the call addresses 15" in msg
    c, msg = code(tg.contract, m, n, k, f64(15), f64(11), f64(20))
    assert c == 1 and "B holds 11" in msg
    c, msg = code(tg.contract, m, n, k, f64(15), f64(12), f64(19))
    assert c == 1 and "C holds 19" in msg
    c, msg = code(tg.contract, m, n, k, f64(15), f64(12), f64(4, 10)[:, :5])
    assert c == 1 and "contiguous" in msg
    c, msg = code(tg.contract, [(5, -3, 4)], n, k, f64(15), f64(12), f64(20))
    assert c == 1 and "non-negative" in msg
    c, msg = code(tg.contract, m, n, k, f64(15), f64(12), f64(20))
    assert c == 1 and "CUDA tensor" in msg
    # an empty M addresses nothing, so empty operands pass the size checks
    c, msg = code(tg.contract, [(0, 3, 4)], n, k, f64(0), f64(12), f64(0))
    assert "CUDA tensor" in msg
    c, msg = code(tg.svd, f64(6, 4), f64(23), f64(4), f64(16))
    assert c == 1 and "U holds 23" in msg
    c, msg = code(tg.svd_noalloc, f64(6, 4), f64(24), f64(3), f64(16))
    assert c == 1 and "S holds 3" in msg
    c, msg = code(tg.orth, f64(6, 4), f64(24), f64(15))
    assert c == 1 and "R holds 15" in msg
    c, msg = code(tg.gaussian, 1, 2, 3, 4, f64(11))
    assert c == 1 and "out holds 11" in msg
    c, msg = code(tg.philox_words, 1, 2, 0, 3, f64(12))
    assert c == 1 and "dtype" in msg
    c, msg = code(tg.philox_words, 1, 2, 0, 3, torch.zeros(11, dtype=torch.int32))
    assert c == 1 and "out holds 11" in msg
    # host-side state: shapes must describe one split site tensor
    ctx = object.__new__(tg.Context)
    ctx._h = None
    A = np.zeros((2, 2, 2, 2, 3))
    c, msg = code(tg.Context.set_state, ctx, A, np.zeros(3), np.zeros((3, 2, 2, 2, 3)), 0, 0.0)
    assert c == 1 and "set_state" in msg
    c, msg = code(tg.Context.set_state, ctx, A, np.zeros(2), np.zeros((2, 2, 2, 2, 2)), 0, 0.0)
    assert c == 1

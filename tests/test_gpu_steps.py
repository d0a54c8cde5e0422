"""Teacher-forced single steps: the GPU step from the same input state as the oracle's.

* Late steps of a whole chi = 12 run (k = 20, 30, 39): the oracle's own state before step k
  is loaded into the GPU context.
* chi = 24 (k = 20, 30, 39) and the benchmark size chi = 48, r = 3 (k = 10): seeded
  synthetic states with the trajectory's spectrum (tests/golden/make_golden_steps.py holds
  the oracle's step from the same states), so every kernel runs at full size.

FP64 bar: ln c_k to 1e-11 relative, s' and the leading spectra to 1e-10, A' and B' at the
sampled positions to 1e-9.  Split-precision steps are held to the bounds in SPLIT_TOL."""
import json
import math
import os

import numpy as np
import pytest

import paper_2412_14104_gb300 as tg
from oracle import trg

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def _close_step(ctx, lnc, s, tol_lnc, tol_s):
    info = ctx.step_info()
    assert abs(info.lnc - lnc) < tol_lnc * max(1.0, abs(lnc)), (info.lnc, lnc)
    got = ctx.spectrum(0)
    assert got.size == len(s)
    assert np.max(np.abs(got - np.array(s))) < tol_s


def test_late_steps_of_a_chi12_run_from_the_oracle_state():
    p = trg.Params(12, 2, q=2, seed=3)
    run = trg.Run(0.1497, 1e-4, 4, p)
    ctx = tg.Context(12, 2, 2, seed=3)
    for k in (20, 30, 39):
        run.step(k - 1 - run.k)
        ctx.set_state(run.A, run.s, run.B, run.k, run.partial_lnz())
        ctx.rg_step()
        run.step()
        _close_step(ctx, run.lnc[-1], run.s, 1e-11, 1e-10)
        A, s, B = ctx.get_state()
        assert np.allclose(A, run.A, atol=1e-9) and np.allclose(B, run.B, atol=1e-9)


def _case(name):
    import sys
    sys.path.insert(0, GOLD)
    import make_golden_steps as mg
    with open(os.path.join(GOLD, "oracle_%s.json" % name)) as f:
        g = json.load(f)
    A, s, B, p, k = mg.case_input(name)
    return g, A, s, B, p, k


# split-precision bounds per step (measured differences are printed by the test)
SPLIT_TOL = {tg.TF32X3: (1e-5, 1e-4), tg.BF16X3: (1e-5, 1e-4), tg.BF16X6: (1e-5, 1e-4), tg.OZAKI: (1e-9, 1e-8)}


@pytest.mark.parametrize("name", ["step_chi24_k20", "step_chi24_k30", "step_chi24_k39", "step_chi48_k10"])
def test_teacher_forced_step_fp64(name):
    g, A, s, B, p, k = _case(name)
    ctx = tg.Context(p.chi, p.r, p.q, seed=p.seed).set_state(A, s, B, k - 1, 0.0)
    del A, B
    ctx.rg_step()
    _close_step(ctx, g["lnc"], g["s"], 1e-11, 1e-10)
    chi = p.chi
    sig = ctx.spectrum(1)
    want = np.array(g["sigma"])
    n = min(chi, sig.size, want.size)
    assert np.max(np.abs(sig[:n] - want[:n])) < 1e-10 * want[0]
    for nu in range(1, 4):
        got = ctx.spectrum(1 + nu)
        want = np.array(g["sq"][nu - 1])
        n = min(chi, got.size, want.size)
        assert np.max(np.abs(got[:n] - want[:n])) < 1e-10 * want[0], nu
    A1, s1, B1 = ctx.get_state()
    assert list(A1.shape) == g["shape_A"] and list(B1.shape) == g["shape_B"]
    assert np.max(np.abs(A1.ravel()[g["idx_A"]] - np.array(g["val_A"]))) < 1e-9
    assert np.max(np.abs(B1.ravel()[g["idx_B"]] - np.array(g["val_B"]))) < 1e-9


@pytest.mark.parametrize("prec", [tg.TF32X3, tg.BF16X3, tg.BF16X6, tg.OZAKI])
@pytest.mark.parametrize("name", ["step_chi24_k20", "step_chi48_k10"])
def test_teacher_forced_step_split(name, prec):
    g, A, s, B, p, k = _case(name)
    ctx = tg.Context(p.chi, p.r, p.q, seed=p.seed, precision=prec).set_state(A, s, B, k - 1, 0.0)
    del A, B
    ctx.rg_step()
    info = ctx.step_info()
    got = ctx.spectrum(0)
    dl = abs(info.lnc - g["lnc"]) / max(1.0, abs(g["lnc"]))
    ds = float(np.max(np.abs(got - np.array(g["s"])))) if got.size == len(g["s"]) else math.inf
    print("%s prec %d: |d ln c| %.3e, max |d s'| %.3e" % (name, prec, dl, ds))
    tl, ts = SPLIT_TOL[prec]
    assert dl < tl and ds < ts

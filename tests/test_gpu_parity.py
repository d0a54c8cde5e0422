"""GPU FP64 path against the FP64 oracle: whole runs (stored oracle values written by
tests/golden/make_golden.py), single steps from a shared state, and the untruncated
pipeline against brute-force enumeration.  Tolerances: ln Z / V to 1e-11 relative and
normalised spectra to 1e-10 (the FP64 bar), on cuts whose relative gap is well above the
rounding level."""
import json
import math
import os

import numpy as np
import pytest

import paper_2412_14104_gb300 as tg
from oracle import ising, trg
from tests import exact_ising

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _gold(name):
    with open(os.path.join(GOLD, "oracle_%s.json" % name)) as f:
        return json.load(f)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def test_initial_split_matches_oracle():
    """Init kernel + exact SVD + sign convention reproduce the oracle's A, s, B."""
    for d, beta, h in ((4, 0.1497, 0.0), (4, 0.2, 0.3), (2, 0.5, -0.1)):
        ctx = tg.Context(6, 2).init_ising(beta, h, d)
        A, s, B = ctx.get_state()
        A0, s0, B0, c0 = ising.initial_state(beta, h, d, 6)
        assert np.allclose(s, s0, atol=1e-15)
        assert np.allclose(A, A0, atol=1e-14) and np.allclose(B, B0, atol=1e-14)
        got = ctx.lnZ()
        want = d * beta + math.log(math.exp(h) + math.exp(-h))
        assert abs(got - want) < 1e-13


def _min_gap(g, k):
    """Smallest relative gap at the swap and squeezer cuts of step k+1 (1-based)."""
    gaps = [g["swap_gap"][k]] + list(g["sq_gap"][k])
    return min([x for x in gaps if x is not None] + [math.inf])


@pytest.mark.parametrize("name", ["c1_chi6", "d4_chi10_h", "d2_chi16", "d3_chi8", "atrg_d4_chi8",
                                  "atrg_d3_chi8", "c2_chi24"])
def test_full_run_matches_oracle(name):
    """Every step's ln c_k and s', and the final ln Z / V.  A cut through a degenerate
    multiplet (relative gap < 1e-8, several correct answers) would make later values depend
    on rounding; the strict tolerance then relaxes to 1e-7 for the rest of the run.
    Rounding differences grow by ~1.6 per step along the RG trajectory (measured with the
    oracle under a 1e-10 perturbation), so the per-step bound grows by that factor after
    step 15; where the oracle's own rounding envelope (make_envelope.py: the spread of
    its runs under relative 2^-50 noise on the initial split) is wider, 100 times the
    envelope bounds the step instead.  ln Z, where step k weighs 2^-k, keeps the 1e-11
    bar."""
    g = _gold(name)
    c = g["config"]
    env = None
    env_path = os.path.join(GOLD, "oracle_%s_envelope.json" % name)
    if os.path.exists(env_path):
        with open(env_path) as f:
            env = json.load(f)
    method = tg.ATRG if c.get("method") == "atrg" else tg.TRIAD
    ctx = tg.Context(c["chi"], c["r"], c["q"], method=method, seed=c["seed"]).init_ising(c["beta"], c["h"], c["d"])
    tol = 1e-11
    for k in range(c["steps"]):
        ctx.rg_step()
        if _min_gap(g, k) < 1e-8:
            tol = 1e-7
        info = ctx.step_info()
        ltol = tol * 1.6 ** max(0, k - 15)
        stol = 10 * ltol
        if env is not None:
            # never tighter than the oracle's own spread under rounding-level noise (x100)
            ltol = max(ltol, 100.0 * env["env_lnc"][k + 1])
            if env["env_s"][k + 1] is not None:
                stol = max(stol, 100.0 * env["env_s"][k + 1])
        assert abs(info.lnc - g["lnc"][k + 1]) < ltol * max(1.0, abs(g["lnc"][k + 1])), k
        s = ctx.spectrum(0)
        assert s.size == len(g["s"][k + 1])
        assert np.max(np.abs(s - np.array(g["s"][k + 1]))) < stol, k
    lnz = ctx.lnZ()
    assert abs(lnz - g["lnz"]) < tol * abs(g["lnz"])


def test_degenerate_cut_moves_to_multiplet_boundary():
    """chi = 8, h = 1e-4: at step 2 the swap spectrum has a four-fold multiplet at
    positions 6..9, so a cut at 8 would split it.  The cut moves to 6 on both sides and the
    step becomes well posed: GPU and oracle agree to rounding."""
    p = trg.Params(8, 3, q=2, seed=2)
    run = trg.Run(0.1497, 1e-4, 4, p).step(1)
    ctx = tg.Context(8, 3, 2, seed=2).set_state(run.A, run.s, run.B, run.k, run.partial_lnz())
    ctx.rg_step()
    run.step()
    assert run.s.size == 6 and ctx.get_state()[1].size == 6
    assert abs(ctx.step_info().lnc - run.lnc[-1]) < 1e-12


def test_degenerate_multiplets_get_a_canonical_basis():
    """chi = 24: after step 2 the re-split spectrum holds a four-fold multiplet; its basis
    feeds the random sketch of step 3.  With the canonical basis the GPU state after two
    steps equals the oracle's (not only its spectrum), so step 3 agrees to rounding."""
    p = trg.Params(24, 2, q=2, seed=1)
    run = trg.Run(0.1497, 0.0, 4, p).step(2)
    ctx = tg.Context(24, 2, 2, seed=1).init_ising(0.1497, 0.0, 4).rg_step(2)
    A, s, B = ctx.get_state()
    assert np.allclose(A, run.A, atol=1e-10) and np.allclose(B, run.B, atol=1e-10)
    ctx.rg_step()
    run.step()
    assert abs(ctx.step_info().lnc - run.lnc[-1]) < 1e-11


def test_single_steps_from_shared_states():
    """Teacher forcing: load the oracle's state before each step, compare that step."""
    p = trg.Params(10, 2, q=2, seed=2)
    run = trg.Run(0.1497, 1e-4, 4, p)
    ctx = tg.Context(10, 2, 2, seed=2)
    for k in range(6):
        ctx.set_state(run.A, run.s, run.B, run.k, run.partial_lnz())
        ctx.rg_step()
        run.step()
        assert abs(ctx.step_info().lnc - run.lnc[-1]) < 1e-12
        assert np.allclose(ctx.spectrum(0), run.s, atol=1e-11)
        A, s, B = ctx.get_state()
        assert A.shape == run.A.shape
        # the split itself is gauge-fixed: compare tensors, not just spectra
        assert np.allclose(A, run.A, atol=1e-9) and np.allclose(B, run.B, atol=1e-9)


def test_untruncated_2d_torus_matches_enumeration():
    """P6 on the GPU: 4x4 torus, chi and r large enough that nothing is cut."""
    beta, h = 0.44, 0.07
    ctx = tg.Context(256, 64, 2).init_ising(beta, h, 2)
    ctx.rg_step(4)
    want, _, _ = exact_ising.brute_force_lnz(beta, h, (4, 4))
    assert abs(ctx.lnZ() - want / 16) < 1e-12


def test_triad_full_width_equals_atrg_on_gpu():
    """P4 on the GPU: r = chi makes the triad exact, so Triad-ATRG equals ATRG."""
    a = tg.Context(4, 4, 2, method=tg.TRIAD, seed=2).init_ising(0.1497, 0.0, 4).rg_step(6).lnZ()
    b = tg.Context(4, 4, 2, method=tg.ATRG, seed=2).init_ising(0.1497, 0.0, 4).rg_step(6).lnZ()
    assert abs(a - b) < 1e-12


def test_errors_are_reported():
    ctx = tg.Context(4, 2)
    with pytest.raises(tg.TatrgError) as e:
        ctx.rg_step()
    assert e.value.code == 6
    with pytest.raises(tg.TatrgError):
        ctx.init_ising(-1.0, 0.0, 4)
    with pytest.raises(tg.TatrgError):
        ctx.init_ising(0.1, 0.0, 5)


def test_temperature_sweep_matches_single_runs():
    """β-sweep: temperature i runs with sketch replica i, so each result equals the oracle's
    single run with that replica, whatever the number of concurrent workers."""
    betas = [0.12, 0.1497, 0.2, 0.3, 0.05]
    want = [trg.lnz_per_site(b, 1e-4, 4, trg.Params(8, 2, q=2, seed=3, replica=i), 10)
            for i, b in enumerate(betas)]
    runs = [tg.Context(8, 2, 2, seed=3, sweep_workers=w).sweep(betas, 1e-4, 4, 10) for w in (1, 3)]
    for i in range(len(betas)):
        assert abs(runs[0][i] - want[i]) < 1e-11 * abs(want[i]), i
    assert np.array_equal(runs[0], runs[1])


def test_fp64_runs_are_reproducible():
    """Every FP64 reduction adds in a fixed order, so a repeated run gives the same bits."""
    out = []
    for _ in range(2):
        ctx = tg.Context(10, 2, 2, seed=5).init_ising(0.1497, 1e-4, 4).rg_step(6)
        out.append((ctx.get_state(), ctx.lnZ()))
    (A0, s0, B0), z0 = out[0]
    (A1, s1, B1), z1 = out[1]
    assert z0 == z1
    assert np.array_equal(A0, A1) and np.array_equal(s0, s1) and np.array_equal(B0, B1)


@pytest.mark.parametrize("prec", [tg.TF32X3, tg.BF16X3, tg.BF16X6])
def test_split_precision_free_energy_within_1e8(prec):
    """chi = 24, 40 steps: with the split-precision contractions from step 13 on (the first
    twelve steps in FP64, where step k weighs 2^-k in ln Z / V), ln Z / V stays within
    1e-8 relative of the FP64 oracle (measured 3.4e-9 for 3xTF32, 2.3e-9 for BF16x6,
    1.8e-8 for BF16x3 from step 13).  Each split step perturbs ln c_k by ~5e-6 relative
    (1e-5 to 5e-5 for BF16x3), so the schedule, not the product precision, sets the final
    error."""
    g = _gold("c2_chi24")
    c = g["config"]
    # BF16x3 keeps 16 bits of each operand against 22-24 for the other forms, and its steps
    # perturb ln c_k about four times as much: its schedule starts two steps later (each step
    # halves the weight of its error in ln Z / V)
    start = 15 if prec == tg.BF16X3 else 13
    ctx = tg.Context(c["chi"], c["r"], c["q"], seed=c["seed"], precision=prec,
                     split_from_step=start).init_ising(c["beta"], c["h"], c["d"])
    lnz = ctx.rg_step(c["steps"]).lnZ()
    print("precision %d from step %d: rel ln Z %.3e" % (prec, start, abs(lnz - g["lnz"]) / abs(g["lnz"])))
    assert abs(lnz - g["lnz"]) < 1e-8 * abs(g["lnz"]), (lnz, g["lnz"])


def test_order_parameter_untruncated_2d_torus():
    """X^(m) of the exact 4 x 4 block equals Z(4 x 4)^2 / Z(4 x 8) (transfer matrix)."""
    for beta, h in ((0.3, 0.0), (0.4407, 0.0), (0.6, 0.02)):
        ctx = tg.Context(256, 64, 2).init_ising(beta, h, 2).rg_step(4)
        z = exact_ising.transfer_matrix_lnz(beta, h, 4, 4)
        zz = exact_ising.transfer_matrix_lnz(beta, h, 4, 8)
        for leg in (0, 1):
            assert abs(math.log(ctx.order_parameter(leg)) - (2 * z - zz)) < 1e-10


def test_order_parameter_matches_oracle_and_sweep():
    """Truncated 4D runs: X^(m) of every leg equals the oracle's from the same run; the
    temperature sweep reports the same X as single runs (replica i for temperature i)."""
    p = trg.Params(8, 2, q=2, seed=3)
    run = trg.Run(0.1497, 1e-4, 4, p).step(10)
    ctx = tg.Context(8, 2, 2, seed=3).init_ising(0.1497, 1e-4, 4).rg_step(10)
    for leg in range(4):
        want, _ = trg.order_parameter_x(run.A, run.s, run.B, leg)
        assert abs(ctx.order_parameter(leg) - want) < 1e-10 * want
    betas = [0.12, 0.1497, 0.2]
    z, x = tg.Context(8, 2, 2, seed=3, sweep_workers=2).sweep_observables(betas, 0.0, 4, 10)
    assert x.shape == (3, 10)
    for i, b in enumerate(betas):
        r = trg.Run(b, 0.0, 4, trg.Params(8, 2, q=2, seed=3, replica=i))
        for m in range(10):  # X^(m) after every step
            r.step()
            want = trg.order_parameter_x(r.A, r.s, r.B, 3)[0]
            assert abs(x[i, m] - want) < 1e-9 * want, (i, m)
        assert abs(z[i] - r.lnz()) < 1e-11 * abs(r.lnz())
    assert x[2, -1] > 1.5 > x[0, -1]  # ordered at beta = 0.2, disordered at 0.12 (4D: beta_c ~ 0.1497)


def test_precision_schedule_from_step_5_within_1e8():
    """chi = 24, 40 steps: FP64 for steps 1-4 (small, cheap), the float64-grade Ozaki slices
    for steps 5-12 (where step k still weighs 2^-k), 3xTF32 from step 13: ln Z / V within
    1e-8 relative of the FP64 oracle."""
    g = _gold("c2_chi24")
    c = g["config"]
    ctx = tg.Context(c["chi"], c["r"], c["q"], seed=c["seed"], precision=tg.TF32X3, split_from_step=5,
                     early_precision=tg.OZAKI, late_from_step=13).init_ising(c["beta"], c["h"], c["d"])
    lnz = ctx.rg_step(c["steps"]).lnZ()
    print("schedule fp64/ozaki/tf32x3: rel %.3e" % (abs(lnz - g["lnz"]) / abs(g["lnz"])))
    assert abs(lnz - g["lnz"]) < 1e-8 * abs(g["lnz"]), (lnz, g["lnz"])


def test_ozaki_whole_run_tracks_the_oracle():
    """chi = 24, 40 steps with the Ozaki slices from step 1: ln Z / V within 1e-9 relative of
    the oracle's, ln c_k of steps 1-4 within 1e-9 and of steps 5-12 within 5e-8.  One Ozaki
    step perturbs ln c_k by ~1e-10 (the teacher-forced steps), and the trajectory amplifies
    a difference about twice per step (the oracle's own rounding envelope: 2^-50 relative
    noise on the initial split grows to 4.7e-8 by step 29), so by step 12 the runs differ
    by up to ~1e-10 * 2^8; ln Z / V weighs step k by 2^-k."""
    g = _gold("c2_chi24")
    c = g["config"]
    ctx = tg.Context(c["chi"], c["r"], c["q"], seed=c["seed"], precision=tg.OZAKI,
                     split_from_step=1).init_ising(c["beta"], c["h"], c["d"])
    errs = []
    for k in range(c["steps"]):
        ctx.rg_step()
        errs.append(abs(ctx.step_info().lnc - g["lnc"][k + 1]) / max(1.0, abs(g["lnc"][k + 1])))
    lnz = ctx.lnZ()
    rel = abs(lnz - g["lnz"]) / abs(g["lnz"])
    print("ozaki from step 1: rel ln Z %.3e; ln c_k errors by step: %s"
          % (rel, " ".join("%.0e" % e for e in errs)))
    assert rel < 1e-9 and max(errs[:4]) < 1e-9 and max(errs[4:12]) < 5e-8


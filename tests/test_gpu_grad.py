"""Tangent (forward-mode) derivatives of ln Z / V on the GPU against the oracle's central
differences of its own ln Z / V (same sketches), and against enumeration where nothing is
truncated."""
import math

import numpy as np
import pytest

import paper_2412_14104_gb300 as tg
from oracle import derivatives, trg
from tests import exact_ising

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def _close(a, b, rel, floor=0.0):
    return abs(a - b) <= rel * abs(b) + floor


@pytest.mark.parametrize("chi,beta,h", [(6, 0.1497, 1e-3), (8, 0.1497, 0.0), (6, 0.1497, 0.0)])
def test_grad_matches_oracle_differences(chi, beta, h):
    """chi = 6 or 8, r = 2, 8 steps in 4D, at points where the oracle's ln Z / V is smooth
    over the difference stencil (its differences with steps 1e-5 and 2e-5 agree to 1e-9).
    At h = 0 the exactly degenerate multiplets go through the canonical-basis tangent;
    only the beta derivative is smooth there."""
    p = trg.Params(chi, 2, q=2, seed=4)
    ctx = tg.Context(chi, 2, 2, seed=4).init_ising(beta, h, 4).rg_step(8)
    gb, gh, _ = ctx.grad()
    want_b = derivatives.dlnz_dbeta(beta, h, 4, p, 8)
    assert abs(want_b - derivatives.dlnz_dbeta(beta, h, 4, p, 8, e=2e-5)) < 1e-8
    assert _close(gb, want_b, 1e-8), (gb, want_b)
    if h != 0.0:
        want_h = derivatives.dlnz_dh(beta, h, 4, p, 8)
        assert _close(gh, want_h, 1e-8, 1e-10), (gh, want_h)


def test_grad_untruncated_2d_torus_matches_enumeration():
    beta, h = 0.44, 0.07
    ctx = tg.Context(256, 64, 2).init_ising(beta, h, 2).rg_step(4)
    gb, gh, _ = ctx.grad()
    _, bonds, mag = exact_ising.brute_force_lnz(beta, h, (4, 4))
    assert abs(gb - bonds / 16) < 1e-11
    assert abs(gh - mag / 16) < 1e-11


def test_second_derivative_matches_oracle():
    beta, h = 0.1497, 1e-3
    p = trg.Params(6, 2, q=2, seed=4)
    ctx = tg.Context(6, 2, 2, seed=4).init_ising(beta, h, 4).rg_step(8)
    _, _, c = ctx.grad(second=True)
    want = derivatives.d2lnz_dbeta2(beta, h, 4, p, 8)
    assert _close(c, want, 2e-5), (c, want)


def test_grad_leaves_state_and_matches_autograd(cuda):
    torch = cuda
    ctx = tg.Context(6, 2, 2, seed=4).init_ising(0.1497, 1e-3, 4).rg_step(4)
    z0 = ctx.lnZ()
    gb, gh, _ = ctx.grad()
    assert ctx.lnZ() == z0
    f = tg.lnz_function(6, 2, 2, seed=4, d=4, nsteps=4)
    b = torch.tensor(0.1497, dtype=torch.float64, requires_grad=True)
    hh = torch.tensor(1e-3, dtype=torch.float64, requires_grad=True)
    z = f(b, hh)
    z.backward()
    assert float(z.detach()) == z0
    assert b.grad.item() == gb and hh.grad.item() == gh

"""Failure detection without a GPU fault: each error is made on the host (an allocation
that cannot succeed, a non-finite state, an exactly rank-deficient Gram) or by a bounded
device wait whose time limit a test sets to zero.  After every error the library keeps
working on the same device."""
import ctypes

import numpy as np
import pytest

import paper_2412_14104_gb300 as tg

pytestmark = pytest.mark.gpu
ENOMEM, ENUMERIC, ETIMEOUT = 2, 4, 5


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


def _usable():
    """A short FP64 run still gives the oracle-checked chi = 6 value range."""
    z = tg.Context(6, 2, 2, seed=0).init_ising(0.1497, 0.0, 4).rg_step(2).lnZ()
    assert np.isfinite(z) and 0.5 < z < 1.5


def test_allocation_failure_is_enomem(torch):
    """set_state with leg dimensions whose buffers (8 TB) exceed the device: the library
    allocates before it reads the host arrays, so tiny host buffers suffice."""
    ctx = tg.Context(8, 2)
    dims = (ctypes.c_int * 5)(512, 512, 512, 512, 16)
    buf = np.zeros(16)
    code = tg.lib().tatrg_set_state(ctx._h, 4, dims, tg._dptr(buf), tg._dptr(buf), tg._dptr(buf), 0, 0.0)
    assert code == ENOMEM
    assert b"cudaMallocAsync" in tg.lib().tatrg_last_error(ctx._h)
    ctx.init_ising(0.1497, 0.0, 4).rg_step(1)  # the same context still runs
    _usable()


def test_non_finite_state_is_enumeric(torch):
    from paper_2412_14104_gb300 import synth
    A, s, B = synth.split_state(3, (4, 4, 4, 4), 4)
    ctx = tg.Context(4, 2).set_state(A, s, B, 2, 0.1)
    bad = A.copy()
    bad[1, 2, 3, 0, 1] = np.nan
    with pytest.raises(tg.TatrgError) as e:
        ctx.set_state(bad, s, B, 2, 0.1)
    assert e.value.code == ENUMERIC
    s2 = s.copy()
    s2[0] = np.inf
    with pytest.raises(tg.TatrgError) as e:
        ctx.set_state(A, s2, B, 2, 0.1)
    assert e.value.code == ENUMERIC
    # the previous state is kept
    A1, s1, B1 = ctx.get_state()
    assert np.array_equal(A1, A) and np.array_equal(s1, s) and np.array_equal(B1, B)
    ctx.rg_step(1)
    _usable()


def test_rank_deficient_gram_takes_the_rank_revealing_fallback(torch):
    """Y = [X, X]: the Gram Y^T Y is exactly singular, CholeskyQR breaks down and the
    one-sided Jacobi fallback returns the k = n / 2 directions of the range."""
    rng = np.random.default_rng(4)
    X = rng.standard_normal((400, 9))
    Y = np.concatenate([X, X], axis=1)
    dY = torch.from_numpy(Y).cuda()
    Q = torch.empty((400, 18), dtype=torch.float64, device="cuda")
    R = torch.empty((18, 18), dtype=torch.float64, device="cuda")
    for prec in (tg.FP64, tg.TF32X3):
        k = tg.orth(dY, Q, R, precision=prec)
        assert k == 9
        q = Q.cpu().numpy().ravel()[: 400 * k].reshape(400, k)
        r = R.cpu().numpy().ravel()[: k * 18].reshape(k, 18)
        assert np.allclose(q.T @ q, np.eye(k), atol=1e-12)
        tol = 1e-12 if prec == tg.FP64 else 1e-5
        assert np.max(np.abs(q @ r - Y)) < tol * np.max(np.abs(Y))


def test_jacobi_grid_barrier_timeout_is_reported(torch):
    """The cooperative Jacobi SVD (n >= 32) waits at a grid barrier between rounds; with
    its time limit set to zero the first wait runs out, every block returns and the call
    reports ETIMEOUT.  With the default limit back, the same call and a whole RG step that
    uses that SVD succeed."""
    rng = np.random.default_rng(5)
    m, n = 200, 144
    A = torch.from_numpy(rng.standard_normal((m, n))).cuda()
    U = torch.empty((m, n), dtype=torch.float64, device="cuda")
    S = torch.empty(n, dtype=torch.float64, device="cuda")
    V = torch.empty((n, n), dtype=torch.float64, device="cuda")
    ctx = tg.Context(16, 2, 2, seed=1).init_ising(0.1497, 0.0, 4)
    try:
        tg.set_barrier_limit_ns(0)
        with pytest.raises(tg.TatrgError) as e:
            tg.svd(A, U, S, V)
        assert e.value.code == ETIMEOUT
        code = None
        for _ in range(6):  # chi = 16, r = 2: the swap core SVD reaches n = 32 within a few steps
            try:
                ctx.rg_step(1)
            except tg.TatrgError as err:
                code = err.code
                break
        assert code == ETIMEOUT
    finally:
        tg.set_barrier_limit_ns(2_000_000_000)
    tg.svd(A, U, S, V)
    torch.cuda.synchronize()
    s_ref = np.linalg.svd(A.cpu().numpy(), compute_uv=False)
    assert np.allclose(S.cpu().numpy(), s_ref, rtol=1e-12)
    ctx.init_ising(0.1497, 0.0, 4).rg_step(4)
    _usable()

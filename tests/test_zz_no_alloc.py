"""tatrg_svd_noalloc, the Jacobi SVD whose workspace is a fixed device array instead of
allocated memory (for callers that may not allocate device memory: code running while
another allocator owns the device budget, or where cudaMalloc's implicit synchronisation
is not allowed), against tatrg_svd and NumPy on calls in a row.  Collected last so that a
failure here does not hide the other tests."""
import numpy as np
import pytest

import paper_2412_14104_gb300 as tg

pytestmark = pytest.mark.gpu

LIMIT = 262144  # doubles in the fixed workspace


def _run(fn, torch, A):
    m, n = A.shape
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    U = torch.empty((m, n), dtype=torch.float64, device="cuda")
    S = torch.empty(n, dtype=torch.float64, device="cuda")
    V = torch.empty((n, n), dtype=torch.float64, device="cuda")
    fn(dA, U, S, V)
    torch.cuda.synchronize()
    return U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()


def _largest_m(n):
    N = n + (n & 1)
    return (LIMIT - 3) // N - N - 2


def _check(torch, A):
    u0, s0, v0 = _run(tg.svd, torch, A)
    u1, s1, v1 = _run(tg.svd_noalloc, torch, A)
    assert np.allclose(s1, s0, rtol=1e-13, atol=1e-15 * s0[0])
    assert np.allclose(np.abs(u1), np.abs(u0), atol=1e-11)
    assert np.allclose((u1 * s1) @ v1.T, A, atol=1e-13 * s0[0])
    assert np.allclose(s1, np.linalg.svd(A, compute_uv=False), rtol=1e-12)


def test_svd_without_allocation_matches_svd_in_a_row():
    import torch
    assert torch.cuda.is_available()
    rng = np.random.default_rng(31)
    # calls in a row on different inputs, so the shared workspace starts dirty: a small
    # single-block case, a multi-block case, then an odd n (zero padding column written over
    # the larger call's data) and a tall two-column case (too tall for the single block)
    for m, n in ((40, 12), (600, 96), (41, 13), (20000, 2), (600, 96)):
        A = rng.standard_normal((m, n)) * (0.8 ** np.arange(n))[None, :]
        _check(torch, A)


def test_svd_without_allocation_size_limit():
    """The largest m the fixed workspace holds works; one more row is rejected."""
    import torch
    rng = np.random.default_rng(32)
    n = 144
    m = _largest_m(n)
    assert m == 1674
    A = rng.standard_normal((m, n)) * (0.9 ** np.arange(n))[None, :]
    _check(torch, A)
    A = torch.zeros((m + 1, n), dtype=torch.float64, device="cuda")
    U = torch.empty((m + 1, n), dtype=torch.float64, device="cuda")
    S = torch.empty(n, dtype=torch.float64, device="cuda")
    V = torch.empty((n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(tg.TatrgError) as e:
        tg.svd_noalloc(A, U, S, V)
    assert e.value.code == 1
    assert "262144" in str(e.value)

"""tatrg_svd_noalloc, the Jacobi SVD whose workspace is a fixed device array instead of
allocated memory (for callers that may not allocate device memory), against tatrg_svd on
two calls in a row.  Collected last so that a failure here does not hide the other tests."""
import numpy as np
import pytest

import paper_2412_14104_gb300 as tg

pytestmark = pytest.mark.gpu


def _run(fn, torch, A):
    m, n = A.shape
    dA = torch.from_numpy(A).cuda()
    U = torch.empty((m, n), dtype=torch.float64, device="cuda")
    S = torch.empty(n, dtype=torch.float64, device="cuda")
    V = torch.empty((n, n), dtype=torch.float64, device="cuda")
    fn(dA, U, S, V)
    torch.cuda.synchronize()
    return U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()


def test_svd_without_allocation_matches_svd_twice():
    import torch
    assert torch.cuda.is_available()
    rng = np.random.default_rng(31)
    # two calls in a row on different inputs (the shared workspace must not leak state):
    # one small enough for the single-block kernel, one taking the multi-block path
    for m, n in ((40, 12), (600, 96)):
        A = rng.standard_normal((m, n)) * (0.8 ** np.arange(n))[None, :]
        u0, s0, v0 = _run(tg.svd, torch, A)
        u1, s1, v1 = _run(tg.svd_noalloc, torch, A)
        assert np.allclose(s1, s0, rtol=1e-13, atol=1e-15 * s0[0])
        assert np.allclose(np.abs(u1), np.abs(u0), atol=1e-11)
        assert np.allclose((u1 * s1) @ v1.T, A, atol=1e-13 * s0[0])
        assert np.allclose(s1, np.linalg.svd(A, compute_uv=False), rtol=1e-12)


def test_svd_without_allocation_rejects_oversize():
    import torch
    A = torch.zeros((3000, 144), dtype=torch.float64, device="cuda")
    U = torch.empty((3000, 144), dtype=torch.float64, device="cuda")
    S = torch.empty(144, dtype=torch.float64, device="cuda")
    V = torch.empty((144, 144), dtype=torch.float64, device="cuda")
    with pytest.raises(tg.TatrgError) as e:
        tg.svd_noalloc(A, U, S, V)
    assert e.value.code == 1

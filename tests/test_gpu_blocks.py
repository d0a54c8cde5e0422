"""GPU parity of the library's building blocks (through the C ABI) against the oracle and
plain NumPy: Philox sketch, multi-mode contraction, Jacobi SVD, orthonormalisation."""
import numpy as np
import pytest

import paper_2412_14104_gb300 as tg
from oracle import philox, rla

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    return t


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("rows,cols,replica", [(1, 1, 0), (7, 13, 0), (300, 61, 3)])
def test_philox_sketch_matches_oracle(torch, rows, cols, replica):
    """P12: same counters, keys and Box-Muller; the integer stream is identical, the
    Gaussians agree to the last few ulp of the two libms."""
    sid = philox.stream_id(5, 2)
    out = torch.empty(rows * cols, dtype=torch.float64, device="cuda")
    tg.gaussian(2 ** 40 + 17, sid, rows, cols, out, replica=replica)
    torch.cuda.synchronize()
    want = philox.gaussian(2 ** 40 + 17, sid, rows, cols, replica).ravel()
    got = out.cpu().numpy()
    assert np.allclose(got, want, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("seed,sid,replica,first,npairs", [
    (0, 0, 0, 0, 1), (2 ** 40 + 17, 0x503, 3, 0, 4099), (7, 0xFFFFFFFF, 2 ** 31 + 5, 2 ** 32 - 7, 300),
    (2 ** 64 - 1, 1, 0, 2 ** 63 + 12345, 1000)])
def test_philox_words_bit_identical_to_oracle(torch, seed, sid, replica, first, npairs):
    """P12 on the raw integers: every output word of the device generator equals the
    oracle's, including counters that cross the 32-bit word boundary and the top half of
    the 64-bit counter range."""
    out = torch.empty(4 * npairs, dtype=torch.int32, device="cuda")
    tg.philox_words(seed, sid, first, npairs, out, replica=replica)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32).reshape(npairs, 4)
    want = np.stack(philox.philox_words(seed, sid, first, npairs, replica), axis=1)
    assert np.array_equal(got, want)


def test_philox_words_known_answers_on_gpu(torch):
    """The published Philox4x32-10 known-answer vectors through the device stream mapping
    (counter (lo p, hi p, replica, hi seed), key (lo seed, stream id))."""
    from tests.test_oracle_pins import philox_kat
    out = torch.empty(4, dtype=torch.int32, device="cuda")
    for (c0, c1, c2, c3), (k0, k1), want in philox_kat():
        tg.philox_words((c3 << 32) | k0, k1, (c1 << 32) | c0, 1, out, replica=c2)
        torch.cuda.synchronize()
        assert out.cpu().numpy().view(np.uint32).tolist() == want


def _contract_case(rng, torch, prec, tol):
    # C[i,j,a,b] (stored [a,i,b,j]) = sum_{k,l} A[k,i,l,a] B[b,l,j,k]
    I, J, a, b, K, L = 5, 7, 3, 4, 6, 9
    A = rng.standard_normal((K, I, L, a))
    B = rng.standard_normal((b, L, J, K))
    C0 = rng.standard_normal((a, I, b, J))
    want = 0.5 * np.einsum("kila,bljk->aibj", A, B) + 2.0 * C0
    dA, dB, dC = _dev(torch, A), _dev(torch, B), _dev(torch, C0)
    # m = (i, a): A strides (L*a, 1), C strides (b*J, I*b*J); n = (j, b)
    m = [(I, L * a, b * J), (a, 1, I * b * J)]
    n = [(J, K, 1), (b, L * J * K, J)]
    k = [(K, I * L * a, 1), (L, a, J * K)]
    tg.contract(m, n, k, dA, dB, dC, alpha=0.5, beta=2.0, precision=prec)
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    assert np.max(np.abs(got - want)) < tol * np.max(np.abs(want))


def test_contract_fp64_multimode(torch):
    rng = np.random.default_rng(0)
    _contract_case(rng, torch, tg.FP64, 1e-14)


def test_contract_fp64_split_k(torch):
    """A long K (split across blocks and summed atomically) and a transposed operand."""
    rng = np.random.default_rng(1)
    M, N, K = 37, 45, 20000
    A = rng.standard_normal((K, M))
    B = rng.standard_normal((K, N))
    C = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    tg.contract([(M, 1, N)], [(N, 1, 1)], [(K, M, N)], _dev(torch, A), _dev(torch, B), C)
    torch.cuda.synchronize()
    assert np.allclose(C.cpu().numpy(), A.T @ B, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("m,n", [(9, 9), (40, 17), (200, 144), (1, 1), (6000, 40)])
def test_jacobi_svd(torch, m, n):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)) * (0.7 ** np.arange(n))[None, :]
    U = torch.empty((m, n), dtype=torch.float64, device="cuda")
    S = torch.empty(n, dtype=torch.float64, device="cuda")
    V = torch.empty((n, n), dtype=torch.float64, device="cuda")
    tg.svd(_dev(torch, A), U, S, V)
    u, s, v = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    s_ref = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s, s_ref, rtol=1e-12, atol=1e-14 * s_ref[0])
    assert np.allclose((u * s) @ v.T, A, atol=1e-13 * s_ref[0])
    assert np.allclose(v.T @ v, np.eye(n), atol=1e-13)


@pytest.mark.parametrize("m,n,spread", [(144, 144, 1e-12), (160, 160, 1e-6), (144, 144, 1.0), (32, 32, 1e-9)])
def test_svd_graded_square(torch, m, n, spread):
    """Square SVDs with singular values spread over 1 .. spread (graded, like the Gram spectra
    of the step), random singular vectors; against NumPy and the reconstruction.  With
    TATRG_SVD_QRCP=1 these take the pivoted-QR-preconditioned Jacobi."""
    rng = np.random.default_rng(int(m + n + 1 / spread) % 1000)
    Uq, _ = np.linalg.qr(rng.standard_normal((m, n)))
    Vq, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sv = np.logspace(0, np.log10(spread), n) if spread < 1 else 1.0 + rng.random(n)
    A = (Uq * sv) @ Vq.T
    U = torch.empty((m, n), dtype=torch.float64, device="cuda")
    S = torch.empty(n, dtype=torch.float64, device="cuda")
    V = torch.empty((n, n), dtype=torch.float64, device="cuda")
    tg.svd(_dev(torch, A), U, S, V)
    u, s, v = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    s_ref = np.linalg.svd(A, compute_uv=False)
    assert np.all(np.diff(s) <= 0)
    assert np.allclose(s, s_ref, rtol=1e-12, atol=1e-15 * s_ref[0])
    assert np.allclose((u * s) @ v.T, A, atol=1e-13 * s_ref[0])
    assert np.allclose(v.T @ v, np.eye(n), atol=1e-13)
    assert np.allclose(u.T @ u, np.eye(n), atol=1e-11 if spread >= 1e-6 else 1e-3)


def test_svd_conventions_on_a_rank_deficient_square_matrix(torch):
    """Rank 50 of 100: V is a full orthonormal basis (the tangent rules rely on it), the
    leading 50 columns of U are orthonormal and the product is reproduced."""
    rng = np.random.default_rng(17)
    n, k = 100, 50
    A = rng.standard_normal((n, k)) @ rng.standard_normal((k, n))
    U = torch.empty((n, n), dtype=torch.float64, device="cuda")
    S = torch.empty(n, dtype=torch.float64, device="cuda")
    V = torch.empty((n, n), dtype=torch.float64, device="cuda")
    tg.svd(_dev(torch, A), U, S, V)
    u, s, v = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    assert np.allclose(v.T @ v, np.eye(n), atol=1e-13)
    assert np.allclose((u * s) @ v.T, A, atol=1e-12 * s[0])
    assert np.allclose(u[:, :k].T @ u[:, :k], np.eye(k), atol=1e-12)
    assert np.all(s[k:] < 1e-12 * s[0])


def test_orth_full_rank_and_rank_deficient(torch):
    rng = np.random.default_rng(3)
    m, n = 500, 24
    for rank in (24, 10):
        Y = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n))
        Q = torch.empty((m, n), dtype=torch.float64, device="cuda")
        R = torch.empty((n, n), dtype=torch.float64, device="cuda")
        k = tg.orth(_dev(torch, Y), Q, R)
        q = Q.cpu().numpy().ravel()[: m * k].reshape(m, k)
        r = R.cpu().numpy().ravel()[: k * n].reshape(k, n)
        assert k == rank
        assert np.allclose(q.T @ q, np.eye(k), atol=1e-13)
        assert np.allclose(q @ r, Y, atol=1e-12 * np.abs(Y).max())
        if k == n:  # unique thin QR with non-negative diagonal
            q_ref, r_ref = rla.orth(Y)
            assert np.allclose(q, q_ref, atol=1e-11)


def test_orth_keeps_small_but_real_directions():
    """A rank-deficient Y whose nonzero singular values span 1 .. 1e-9: the orthonormal
    basis must keep every nonzero direction (a Gram-based method loses those below ~1e-7,
    where their squares reach the rounding level of the Gram) and span the range of Y to
    the accuracy the rounding of Y itself allows (~eps / 1e-9)."""
    rng = np.random.default_rng(7)
    m, n, rank = 300, 20, 14
    U, _ = np.linalg.qr(rng.standard_normal((m, rank)))
    V, _ = np.linalg.qr(rng.standard_normal((n, rank)))
    S = np.logspace(0, -9, rank)
    Y = (U * S) @ V.T
    Q = torch_empty((m, n))
    R = torch_empty((n, n))
    k = tg.orth(_dev(_torch(), Y), Q, R)
    assert k == rank
    q = Q.cpu().numpy().ravel()[: m * k].reshape(m, k)
    r = R.cpu().numpy().ravel()[: k * n].reshape(k, n)
    assert np.allclose(q.T @ q, np.eye(k), atol=1e-13)
    assert np.allclose(q @ r, Y, atol=1e-14)
    # same subspace as the exact range of Y
    assert np.linalg.norm(U - q @ (q.T @ U)) < 1e-5


def _torch():
    import torch
    return torch


def torch_empty(shape):
    import torch
    return torch.empty(shape, dtype=torch.float64, device="cuda")


def _tc_case(torch, prec, M, N, K, mmodes, nmodes, kmodes, A, B, want, beta_C=None, beta=0.0):
    C = _dev(torch, beta_C) if beta_C is not None else torch.zeros(want.shape, dtype=torch.float64, device="cuda")
    tg.contract(mmodes, nmodes, kmodes, _dev(torch, A), _dev(torch, B), C, beta=beta, precision=prec)
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    print("precision %d: max relative error %.3e (M N K = %d %d %d)" % (prec, err, M, N, K))
    return err


# relative error bound of the split products: 3xTF32 keeps 22 mantissa bits per operand and
# accumulates in FP32; the two-term BF16 split keeps 16, the three-term one 24.  The Ozaki
# slices keep 36 bits of each entry relative to its row's (column's) largest, sum exactly,
# and round the lowest levels at ~2^-34 of sum |a||b|: ~2^-32 sqrt(K) relative to max |C|
TC_TOL = {tg.TF32X3: 5e-6, tg.BF16X3: 1e-4, tg.BF16X6: 5e-6, tg.OZAKI: 1e-8}


@pytest.mark.parametrize("prec", [tg.TF32X3, tg.BF16X3, tg.BF16X6, tg.OZAKI])
def test_contract_tensor_core_plain(torch, prec):
    rng = np.random.default_rng(11)
    M, N, K = 1000, 300, 517
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    err = _tc_case(torch, prec, M, N, K, [(M, K, N)], [(N, 1, 1)], [(K, 1, N)], A, B, A @ B)
    assert err < TC_TOL[prec], err


@pytest.fixture(params=[1, 2], ids=["cta_pair", "multicast"])
def cta_pairs(torch, request):
    """A two-CTA tile form wherever it applies (M >= 1024) for the duration of a test: CTA
    pairs (one cta_group::2 MMA per 256 x 128 tile) or multicast clusters (two 128 x 128
    tiles sharing the B tile)."""
    tg.set_cta_pairs(request.param)
    yield
    tg.set_cta_pairs(0)


@pytest.mark.parametrize("prec", [tg.TF32X3, tg.BF16X3, tg.BF16X6, tg.OZAKI])
@pytest.mark.parametrize("M,N,K", [(1037, 300, 517), (1024, 256, 4096), (2500, 130, 64), (4099, 1000, 33)])
def test_contract_tensor_core_cta_pair_tiles(torch, cta_pairs, prec, M, N, K):
    """M >= 1024 on the two-CTA tile forms (256-row work units): ragged last tile rows and
    columns, a split K (few tiles, long K: float64 atomics), a single K slice."""
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    C0 = rng.standard_normal((M, N))
    want = A @ B - 0.5 * C0
    err = _tc_case(torch, prec, M, N, K, [(M, K, N)], [(N, 1, 1)], [(K, 1, N)], A, B, want,
                   beta_C=C0, beta=-0.5)
    assert err < TC_TOL[prec], err


@pytest.mark.parametrize("prec", [tg.TF32X3, tg.BF16X3, tg.BF16X6, tg.OZAKI])
def test_contract_tensor_core_cta_pair_multimode(torch, cta_pairs, prec):
    """Permuted multi-mode operands and output on the two-CTA tile forms (M = 37 * 41 >= 1024)."""
    rng = np.random.default_rng(14)
    I, J, a, b, K, L = 37, 29, 41, 11, 13, 17
    A = rng.standard_normal((K, I, L, a))
    B = rng.standard_normal((b, L, J, K))
    want = np.einsum("kila,bljk->aibj", A, B)
    m = [(I, L * a, b * J), (a, 1, I * b * J)]
    n = [(J, K, 1), (b, L * J * K, J)]
    k = [(K, I * L * a, 1), (L, a, J * K)]
    err = _tc_case(torch, prec, I * a, J * b, K * L, m, n, k, A, B, want)
    assert err < TC_TOL[prec], err


@pytest.mark.parametrize("prec", [tg.TF32X3, tg.BF16X3, tg.BF16X6, tg.OZAKI])
def test_contract_tensor_core_multimode_beta(torch, prec):
    """Strided (permuted) operands and output, alpha/beta, ragged tiles in M, N and K."""
    rng = np.random.default_rng(12)
    I, J, a, b, K, L = 37, 29, 7, 11, 13, 17
    A = rng.standard_normal((K, I, L, a))
    B = rng.standard_normal((b, L, J, K))
    C0 = rng.standard_normal((a, I, b, J))
    want = np.einsum("kila,bljk->aibj", A, B) + 0.5 * C0
    m = [(I, L * a, b * J), (a, 1, I * b * J)]
    n = [(J, K, 1), (b, L * J * K, J)]
    k = [(K, I * L * a, 1), (L, a, J * K)]
    err = _tc_case(torch, prec, I * a, J * b, K * L, m, n, k, A, B, want, beta_C=C0, beta=0.5)
    assert err < TC_TOL[prec], err


@pytest.mark.parametrize("prec", [tg.TF32X3, tg.BF16X3, tg.BF16X6, tg.OZAKI])
def test_contract_tensor_core_split_k_gram(torch, prec):
    """A Gram Y^T Y with a long K split across CTAs (float64 atomic reduction)."""
    rng = np.random.default_rng(13)
    m, n = 200000, 144
    Y = rng.standard_normal((m, n)) * (0.9 ** np.arange(n))[None, :]
    want = Y.T @ Y
    err = _tc_case(torch, prec, n, n, m, [(n, 1, n)], [(n, 1, 1)], [(m, n, n)], Y, Y, want)
    # each CTA sums ~1e3 positive products in the FP32 accumulator before the FP64 reduction
    assert err < 10 * TC_TOL[prec], err


@pytest.mark.parametrize("prec", [tg.TF32X3, tg.BF16X3, tg.BF16X6])
def test_sketch_generated_in_the_operand_packer(torch, prec):
    """W = R Omega with the Gaussian sketch drawn while the tensor-core operand is packed
    (float Box-Muller, never stored) against the oracle's product with its float64 sketch,
    and against the same contraction on the stored float64 sketch of tatrg_gaussian.
    Shapes as in the bond swap: R[(a,k), j], Omega[(b,j), p], W[(a,k), (b,p)], ragged tiles."""
    rng = np.random.default_rng(21)
    Dak, J, Db, ell = 150, 1500, 3, 36  # M N K = 2.4e7: the tensor-core path
    R = rng.standard_normal((Dak, J))
    seed, sid, rep = 7, 0x305, 2
    m = [(Dak, J, Db * ell)]
    n = [(Db, J * ell, ell), (ell, 1, 1)]
    k = [(J, 1, ell)]
    Om = torch.empty(Db * J * ell, dtype=torch.float64, device="cuda")
    tg.gaussian(seed, sid, Db * J, ell, Om, replica=rep)
    W1 = torch.zeros((Dak, Db * ell), dtype=torch.float64, device="cuda")
    W2 = torch.zeros_like(W1)
    dR = _dev(torch, R)
    tg.contract(m, n, k, dR, Om, W1, precision=prec)
    tg.contract_sketch(m, n, k, dR, seed, sid, W2, replica=rep, precision=prec)
    torch.cuda.synchronize()
    om = philox.gaussian(seed, sid, Db * J, ell, replica=rep).reshape(Db, J, ell)
    want = np.einsum("aj,bjp->abp", R, om).reshape(Dak, Db * ell)
    got1, got2 = W1.cpu().numpy(), W2.cpu().numpy()
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got2 - want)) / scale < TC_TOL[prec]
    assert np.max(np.abs(got1 - want)) / scale < TC_TOL[prec]
    # float and float64 Box-Muller differ by ~1e-7 relative, below the operand split
    assert np.max(np.abs(got2 - got1)) / scale < TC_TOL[prec]
    with pytest.raises(tg.TatrgError):
        tg.contract_sketch(m, n, k, dR, seed, sid, W2, precision=tg.FP64)

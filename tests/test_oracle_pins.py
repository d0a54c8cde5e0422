"""Pins of the FP64 oracle against results fixed outside it (brute force, Onsager's closed
form, the high-temperature series, exact linear algebra and symmetry).  CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import ising, philox, rla, trg
from tests import exact_ising

INF = trg.Params(None, None, q=2)


def _dense_site(A, s, B):
    d = A.ndim - 1
    Da = s.size
    T = (A.reshape(-1, Da) * s[None, :]) @ B.reshape(Da, -1)
    return T.reshape(A.shape[:d] + B.shape[1:])


def test_single_site_trace():
    """P1: the one-site torus is all self-loops: Z = sum_s e^{hs} prod_mu Bm[s, s]."""
    for d, beta, h in ((4, 0.1497, 0.0), (4, 0.3, 0.2), (2, 0.7, -0.1), (3, 0.2, 0.05)):
        A, s, B, c0 = ising.initial_state(beta, h, d)
        got = math.log(c0) + math.log(trg.trace(A, s, B))
        want = d * beta + math.log(math.exp(h) + math.exp(-h))
        assert abs(got - want) < 1e-13


def test_initial_tensor_bond_weight():
    """sum_x W[s, x] W[s', x] = exp(beta s s') for both square roots of the bond matrix."""
    for beta in (0.05, 0.1497, 0.9):
        Bm = np.array([[math.exp(beta), math.exp(-beta)], [math.exp(-beta), math.exp(beta)]])
        for W in (ising.w_symmetric(beta), ising.w_paper(beta)):
            assert np.allclose(W @ W.T, Bm, rtol=1e-14, atol=0)
    with pytest.raises(ValueError):
        ising.w_symmetric(0.0)


@pytest.mark.parametrize("h", [0.0, 0.13])
def test_brute_force_4d_2x2x2x2(h):
    """P5: 2^4 torus (16 spins, 2^16 configurations, 64 bonds with double bonds from L=2).
    Two untruncated RG steps (directions 1, 2) leave a 1x1x2x2 torus, contracted densely."""
    beta = 0.1497
    run = trg.Run(beta, h, 4, INF).step(2)
    T = _dense_site(run.A, run.s, run.B)          # legs (dir3, dir4, dir1, dir2)^2
    T2 = np.einsum("abcdefcd->abef", T)           # trace directions 1 and 2 (L = 1)
    zrem = np.einsum("aebf,bgah,cfde,dhcg->", T2, T2, T2, T2)
    got = run.partial_lnz() + math.log(zrem) / 16.0
    want, _, _ = exact_ising.brute_force_lnz(beta, h, (2, 2, 2, 2))
    assert abs(got - want / 16.0) < 1e-12


def test_brute_force_2d_4x4_full_pipeline():
    """P6: 4x4 torus, four untruncated ATRG steps down to one site (d = 2)."""
    for beta, h in ((0.3, 0.0), (0.44, 0.07), (0.9, -0.2)):
        got = trg.Run(beta, h, 2, INF).step(4).lnz()
        want, _, _ = exact_ising.brute_force_lnz(beta, h, (4, 4))
        assert abs(got - want / 16.0) < 1e-12, (beta, h, got, want / 16)


def test_brute_force_3d_2x2x2():
    """Untruncated d = 3 pipeline (triad group of one leg) against enumeration."""
    beta, h = 0.25, 0.05
    got = trg.Run(beta, h, 3, INF).step(3).lnz()
    want, _, _ = exact_ising.brute_force_lnz(beta, h, (2, 2, 2))
    assert abs(got - want / 8.0) < 1e-12


def test_internal_energy_and_magnetisation_fd():
    """P5 (derivatives): central differences of the untruncated ln Z give the brute-force
    <sum ss> / V and <sum s> / V of the 2^4 torus."""
    beta, h, e = 0.1497, 0.05, 1e-5

    def lnz(b, hh):
        run = trg.Run(b, hh, 4, INF).step(2)
        T = _dense_site(run.A, run.s, run.B)
        T2 = np.einsum("abcdefcd->abef", T)
        return run.partial_lnz() + math.log(np.einsum("aebf,bgah,cfde,dhcg->", T2, T2, T2, T2)) / 16

    _, ebond, mag = exact_ising.brute_force_lnz(beta, h, (2, 2, 2, 2))
    du = (lnz(beta + e, h) - lnz(beta - e, h)) / (2 * e)
    dm = (lnz(beta, h + e) - lnz(beta, h - e)) / (2 * e)
    assert abs(du - ebond / 16) < 1e-8
    assert abs(dm - mag / 16) < 1e-8


def test_z2_symmetry_untruncated():
    """P9: ln Z(h) = ln Z(-h) and d ln Z / dh = 0 at h = 0."""
    beta = 0.5
    a = trg.Run(beta, 0.3, 2, INF).step(4).lnz()
    b = trg.Run(beta, -0.3, 2, INF).step(4).lnz()
    assert abs(a - b) < 1e-13
    e = 1e-4
    m = (trg.Run(beta, e, 2, INF).step(4).lnz() - trg.Run(beta, -e, 2, INF).step(4).lnz()) / (2 * e)
    assert abs(m) < 1e-9


def test_gauge_of_w():
    """P10: the symmetric square root and the paper's W (square roots restored) differ by an
    orthogonal gauge on every bond, so untruncated ln Z agrees."""
    beta, h = 0.35, 0.1
    a = trg.Run(beta, h, 2, INF).step(4).lnz()
    b = trg.Run(beta, h, 2, INF, W=ising.w_paper(beta)).step(4).lnz()
    assert abs(a - b) < 1e-13


@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_onsager_2d(beta):
    """P7: d = 2 on a 2^20 x 2^20 torus approaches Onsager's infinite-lattice value, and the
    error shrinks as chi grows."""
    exact = exact_ising.onsager_lnz(beta)
    errs = []
    for chi in (4, 8, 16):
        p = trg.Params(chi, 3, q=2, seed=7)
        errs.append(abs(trg.lnz_per_site(beta, 0.0, 2, p, 40) - exact))
    assert errs[-1] < 1e-7, errs
    assert errs[-1] < errs[0], errs


def test_high_temperature_series_4d():
    """P8: at beta = 0.015 (2^16 sites, 16 steps) ln 2 + 4 ln cosh b + 6 tanh^4 b holds to
    O(tanh^6) ~ 1e-9 plus the chi truncation error, which shrinks with chi (single-bond
    excitations on the block boundary form large multiplets that chi cuts).  At chi = 12 the
    total error is below 1e-7 while the tanh^4 term is 3e-7, so a wrong plaquette count or a
    wrong ln cosh coefficient fails."""
    beta = 0.015
    series = exact_ising.high_t_lnz(beta, 4)
    errs = [abs(trg.lnz_per_site(beta, 0.0, 4, trg.Params(chi, 2, q=2, seed=3), 16) - series)
            for chi in (4, 12)]
    assert errs[1] < 1e-7, errs
    assert errs[1] < errs[0], errs


def test_exact_triad_reproduces_unit_cell():
    """P3 / Eq. 4: with r chi >= the grouped dimension the triad network equals Gamma."""
    run = trg.Run(0.1497, 0.02, 4, trg.Params(6, 2, seed=5)).step(2)
    A, s, B = run.A, run.s, run.B
    p = trg.Params(64, 64, seed=5)
    X, sig, Y = trg.bond_swap(A, s, B, p, 3)
    E, F, G, H, I, J, K, L = trg.triad(A, B, X, sig, Y, p, 3)
    # Gamma = A X sigma Y D with all legs open; compare the forward half A X sigma
    gam = np.einsum("iabsx,xcdtg,g->iabscdtg", A, X, sig)
    tri = np.einsum("iksx,abk,xlth,cdl->iabscdth", E, I, F, J)
    assert np.allclose(gam, tri, atol=1e-13 * np.abs(gam).max())
    gam_b = np.einsum("ybcdg,jefhy->bcdgjefh", Y, np.moveaxis(B, 0, -1))
    tri_b = np.einsum("ykdg,bck,jlhy,efl->bcdgjefh", G, K, H, L)
    assert np.allclose(gam_b, tri_b, atol=1e-13 * np.abs(gam_b).max())


def test_truncated_isometry_error_is_dropped_weight():
    """Eq. 2: ||Gamma - U U^T Gamma||^2 on A's grouped legs equals the discarded eigenvalue
    weight of rho_A when U holds exact leading eigenvectors."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((3, 4, 4, 3, 5))
    Xi = rng.standard_normal((5, 5))
    Xi = Xi @ Xi.T
    L = np.linalg.cholesky(Xi)
    AX = np.einsum("iabsx,xy->iabsy", A, L)          # Gamma restricted: A times a square root of Xi
    M = np.transpose(AX, (1, 2, 0, 3, 4)).reshape(16, -1)
    rho = M @ M.T
    lam, U = rla.eigh_desc(rho)
    k = 6
    Uk = U[:, :k]
    err = np.linalg.norm(M - Uk @ (Uk.T @ M)) ** 2
    assert abs(err - lam[k:].sum()) < 1e-10 * lam.sum()


def test_triad_with_full_width_equals_atrg():
    """P4: r = chi makes Triad-ATRG identical to ATRG with the same sketches."""
    for d in (3, 4):
        a = trg.lnz_per_site(0.1497, 0.0, d, trg.Params(4, 4, seed=2, method="triad"), 6)
        b = trg.lnz_per_site(0.1497, 0.0, d, trg.Params(4, 4, seed=2, method="atrg"), 6)
        assert abs(a - b) < 1e-12, (d, a, b)


@pytest.mark.parametrize("dims", [(3, 2, 4, 2), (2, 3, 2, 3), (3, 4, 2)])
def test_atrg_pair_grams_are_partial_traces(dims):
    """Eq. 5 with identity isometries (ATRG): the pair Gram of a group leg equals the
    triad-cell environment traced over the other group leg, so it can be formed from
    Q_E[x,a,y,b] = sum E[i,(x,z),s,a] E[i,(y,z),s,b] and the like (chi^4 intermediates)
    instead of the chi^8 environment.  Random E, F, G, H; d = 4 (two group legs) and d = 3."""
    rng = np.random.default_rng(sum(dims))
    d = len(dims)
    g = d - 2
    D0, Ds = dims[0], dims[-1]
    gshape = tuple(dims[1:1 + g])
    Gd = int(np.prod(gshape))
    Da, Dg = 4, 3
    E = rng.standard_normal((D0, Gd, Ds, Da))
    F = rng.standard_normal((Da, Gd, Ds, Dg))
    G = rng.standard_normal((Da, Gd, Ds, Dg))
    H = rng.standard_normal((D0, Gd, Ds, Da))
    I = np.eye(Gd).reshape(gshape + (Gd,))
    rho_l, rho_r = trg.squeezer_grams(E, F, G, H, I, I, I, I, g)
    # the environments of Eq. 5 that the general construction dresses F and G with
    om_d = np.einsum("jksb,jksc->bc", H, H)
    om_y = np.einsum("cksg,cksh->gh", np.einsum("bksg,bc->cksg", G, om_d), G)
    om_a = np.einsum("iksa,iksb->ab", E, E)
    om_x = np.einsum("bksg,bksh->gh", np.einsum("aksg,ab->bksg", F, om_a), F)
    Fy = np.einsum("akxg,gh->akxh", F, om_y).reshape((Da,) + gshape + (Ds, Dg))
    Gx = np.einsum("bkxg,gh->bkxh", G, om_x).reshape((Da,) + gshape + (Ds, Dg))
    E5, F5 = E.reshape((D0,) + gshape + (Ds, Da)), F.reshape((Da,) + gshape + (Ds, Dg))
    G5, H5 = G.reshape((Da,) + gshape + (Ds, Dg)), H.reshape((D0,) + gshape + (Ds, Da))
    for nu in range(1, g + 1):
        if g == 1:
            e, f = "ixsa,iysb->xayb", "axsh,bysh->axby"
            gg, hh = "bxsh,cysh->xbyc", "jxsb,jysc->bxcy"
        elif nu == 1:
            e, f = "ixzsa,iyzsb->xayb", "axzsh,byzsh->axby"
            gg, hh = "bxzsh,cyzsh->xbyc", "jxzsb,jyzsc->bxcy"
        else:
            e, f = "izxsa,izysb->xayb", "azxsh,bzysh->axby"
            gg, hh = "bzxsh,czysh->xbyc", "jzxsb,jzysc->bxcy"
        Dn = dims[nu]
        want_l = np.einsum("xayb,azbw->xzyw", np.einsum(e, E5, E5), np.einsum(f, Fy, F5))
        want_r = np.einsum("xbyc,bzcw->xzyw", np.einsum(gg, Gx, G5), np.einsum(hh, H5, H5))
        scale_l, scale_r = np.abs(want_l).max(), np.abs(want_r).max()
        assert np.allclose(rho_l[nu - 1], want_l.reshape(Dn * Dn, Dn * Dn), atol=1e-13 * scale_l)
        assert np.allclose(rho_r[nu - 1], want_r.reshape(Dn * Dn, Dn * Dn), atol=1e-13 * scale_r)


def test_truncation_error_shrinks_with_chi_4d():
    """P5 (truncated): on the 2^4 torus the error of chi = 4, 6, 8 runs shrinks."""
    beta, h = 0.1497, 0.0
    want, _, _ = exact_ising.brute_force_lnz(beta, h, (2, 2, 2, 2))
    errs = []
    for chi in (2, 4, 8):
        run = trg.Run(beta, h, 4, trg.Params(chi, 2, seed=1)).step(2)
        T = _dense_site(run.A, run.s, run.B)
        T2 = np.einsum("abcdefcd->abef", T)
        z = np.einsum("aebf,bgah,cfde,dhcg->", T2, T2, T2, T2)
        errs.append(abs(run.partial_lnz() + math.log(z) / 16 - want / 16))
    assert errs[2] < errs[0]


# --- randomized linear algebra --------------------------------------------------------

def _test_matrix(m, n, decay, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, min(m, n))))
    V, _ = np.linalg.qr(rng.standard_normal((n, min(m, n))))
    S = decay ** np.arange(min(m, n))
    return (U * S) @ V.T, S


def test_orth_properties():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((200, 17))
    Q, R = rla.orth(Y)
    assert np.allclose(Q.T @ Q, np.eye(17), atol=1e-14)
    assert np.allclose(Q @ R, Y, atol=1e-13)
    assert np.all(np.diag(R) >= 0) and np.allclose(R, np.triu(R))


def test_rsvd_full_width_is_exact():
    """P11: ell >= min(m, n) recovers the exact SVD."""
    M, S = _test_matrix(60, 40, 0.7, 1)
    om = philox.gaussian(1, 5, 40, 40)
    U, s, V = rla.rsvd(rla.DenseOp(M), 40, 1, om)
    assert np.allclose(s, S, rtol=1e-10, atol=1e-14)
    assert np.allclose((U * s) @ V.T, M, atol=1e-13)


def test_rsvd_error_decreases_with_q():
    """P11: the rank-k error of the randomized SVD approaches sigma_{k+1} as q grows."""
    M, S = _test_matrix(300, 200, 0.93, 2)
    k, ell = 20, 30
    om = philox.gaussian(3, 9, 200, ell)
    errs = []
    for q in (0, 1, 2):
        U, s, V = rla.rsvd(rla.DenseOp(M), ell, q, om)
        errs.append(np.linalg.norm(M - (U[:, :k] * s[:k]) @ V[:, :k].T, 2))
    assert errs[0] > errs[1] > errs[2] >= S[k] * (1 - 1e-12)
    assert errs[2] < 1.05 * S[k]


def test_rsvd_psd_matches_eigh():
    M, S = _test_matrix(80, 80, 0.9, 4)
    rho = M @ M.T
    om = philox.gaussian(3, 10, 80, 80)
    lam, U = rla.rsvd_psd(lambda x: rho @ x, 80, 1, om)
    assert np.allclose(lam, S ** 2, rtol=1e-9, atol=1e-15)


def test_sign_convention():
    rng = np.random.default_rng(5)
    V = rng.standard_normal((50, 7))
    W, sgn = rla.fix_sign(V)
    w = rla.sign_weights(50)
    assert np.all(w @ W > 0)
    W2, _ = rla.fix_sign(-V)
    assert np.array_equal(W, W2)


# --- Philox sketch stream -------------------------------------------------------------

def test_philox_gaussian_statistics():
    """N(0,1) moments, uniformity of the 53-bit uniforms and independence of the pair."""
    z = philox.gaussian(1234, philox.stream_id(3, 0), 1000, 1000)
    x = z.ravel()
    assert abs(x.mean()) < 5e-3
    assert abs(x.var() - 1) < 5e-3
    assert abs(np.mean(x ** 4) - 3) < 3e-2
    assert abs(np.corrcoef(x[0::2], x[1::2])[0, 1]) < 5e-3
    w0, w1, w2, w3 = philox.philox_words(1234, 77, 0, 200000)
    u = np.sort(np.concatenate([philox._uniform53(w0, w1), philox._uniform53(w2, w3)]))
    assert u[0] > 0 and u[-1] < 1
    ks = np.max(np.abs(u - (np.arange(1, u.size + 1) - 0.5) / u.size))
    assert ks < 1.63 / math.sqrt(u.size) * 1.5


def test_philox_stream_layout():
    """Element e uses counter pair e // 2 and takes z_{e mod 2}; streams and replicas differ."""
    a = philox.gaussian(9, 5, 3, 7).ravel()
    b = philox.gaussian(9, 5, 1, 21).ravel()
    assert np.array_equal(a, b)
    c = philox.gaussian(9, 6, 3, 7).ravel()
    r = philox.gaussian(9, 5, 3, 7, replica=1).ravel()
    assert not np.any(a == c) and not np.any(a == r)
    w0, w1, w2, w3 = philox.philox_words(9, 5, 5, 1)
    u1 = philox._uniform53(w0, w1)[0]
    u2 = philox._uniform53(w2, w3)[0]
    assert a[10] == math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2)
    assert a[11] == math.sqrt(-2 * math.log(u1)) * math.sin(2 * math.pi * u2)


def philox_kat():
    """Rows of tests/golden/philox4x32_10_kat.txt: (counter[4], key[2], words[4])."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answer_vectors():
    """P12's reference: the published Philox4x32-10 known answers (Random123).  A wrong
    multiplier, Weyl increment, round count or word order fails this."""
    rows = philox_kat()
    assert len(rows) == 3
    for (c0, c1, c2, c3), (k0, k1), want in rows:
        got = philox.philox4x32_10([c0], [c1], [c2], [c3], k0, k1)
        assert [int(w[0]) for w in got] == want


def test_philox_words_follow_the_stream_layout():
    """philox_words(seed, sid, p, ...) is Philox on counter (lo p, hi p, replica, hi seed) and
    key (lo seed, sid): the KAT rows through the sketch-stream mapping."""
    for (c0, c1, c2, c3), (k0, k1), want in philox_kat():
        seed = (c3 << 32) | k0
        p = (c1 << 32) | c0
        w = philox.philox_words(seed, k1, p, 1, replica=c2)
        assert [int(x[0]) for x in w] == want


def test_philox_is_a_bijection_on_small_counters():
    """Distinct counters give distinct outputs (Philox is a keyed bijection)."""
    w = philox.philox_words(0, 0, 0, 1 << 16)
    packed = set(zip(*[x.tolist() for x in w]))
    assert len(packed) == 1 << 16


def test_flop_counts_match_cost_formulas():
    """P13 / Table 1: at steady state (every leg chi, triad width r chi) one step counts
    (2q+2) 4 r chi^7 swap flops and 8 r^2 chi^7 + O(r^2 chi^6) contraction flops."""
    chi, r, q = 4, 2, 2
    run = trg.Run(0.1497, 0.0, 4, trg.Params(chi, r, q=q, seed=1)).step(4)
    before = dict(run.cnt.flops)
    run.step()
    assert run.A.shape == (chi,) * 5
    delta = {k: run.cnt.flops[k] - before[k] for k in before}
    assert delta["swap"] == (2 * q + 2) * 4 * r * chi ** 7
    main = 8 * r * r * chi ** 7
    lower = 4 * r * chi ** 6 + 2 * (2 * r * chi ** 5 + 2 * r * chi ** 6 + 2 * r * r * chi ** 6)
    assert delta["contract"] == main + lower


def test_canonical_basis_is_rotation_invariant():
    """Any orthonormal basis of a degenerate multiplet maps to the same canonical basis,
    single columns follow the sign rule, and the rotation is orthogonal."""
    rng = np.random.default_rng(21)
    V, _ = np.linalg.qr(rng.standard_normal((60, 7)))
    vals = np.array([3.0, 2.0, 2.0, 2.0, 1.5, 1.0, 1.0])
    C1, O1 = rla.canonical_basis(V, vals, 1e-10)
    R = np.eye(7)
    R[1:4, 1:4], _ = np.linalg.qr(rng.standard_normal((3, 3)))
    R[5:7, 5:7], _ = np.linalg.qr(rng.standard_normal((2, 2)))
    R[0, 0], R[4, 4] = -1.0, -1.0
    C2, O2 = rla.canonical_basis(V @ R, vals, 1e-10)
    assert np.allclose(C1, C2, atol=1e-13)
    assert np.allclose(O1.T @ O1, np.eye(7), atol=1e-14)
    w = rla.sign_weights(60)
    assert w @ C1[:, 0] > 0 and w @ C1[:, 4] > 0
    # a single column reduces to fix_sign
    F1, _ = rla.fix_sign(V[:, :1])
    C3, _ = rla.canonical_basis(V[:, :1], vals[:1], 1e-10)
    assert np.array_equal(F1, C3)


def test_split_multiplet_gap_leaves_the_chi24_run_unchanged():
    """The multiplet gap of the float-grade split steps (tau = 1e-6) against the float64
    one (1e-10) on the stored chi = 24, 40-step oracle runs (tests/golden/make_golden.py,
    c2_chi24 and c2_chi24_tau6 with tau = 1e-6 from step 1): every ln c_k, every kept
    dimension and ln Z / V are identical, so on this run the wider gap changes no cut and a
    split-precision free-energy difference there is rounding alone."""
    import json
    gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    with open(os.path.join(gold, "oracle_c2_chi24.json")) as f:
        a = json.load(f)
    with open(os.path.join(gold, "oracle_c2_chi24_tau6.json")) as f:
        b = json.load(f)
    assert b["config"]["split_tau"] == 1e-6 and b["config"]["split_from_step"] == 1
    assert {k: v for k, v in a["config"].items() if k not in ("split_tau", "split_from_step")} == \
        {k: v for k, v in b["config"].items() if k not in ("split_tau", "split_from_step")}
    assert a["lnc"] == b["lnc"] and a["dims"] == b["dims"] and a["lnz"] == b["lnz"]


def test_multiplet_cut_never_splits():
    vals = np.array([5.0, 4.0, 3.0, 3.0, 3.0, 2.0, 1.0])
    assert rla.multiplet_cut(vals, 3, 1e-10) == 2
    assert rla.multiplet_cut(vals, 5, 1e-10) == 5
    assert rla.multiplet_cut(vals, 6, 1e-10) == 6
    assert rla.multiplet_cut(np.array([1.0, 1.0, 0.5]), 1, 1e-10) == 2
    assert rla.multiplets(vals, 1e-10) == [(2, 5)]


# ---- derivatives of ln Z / V (oracle.derivatives) -------------------------------------

def test_derivatives_match_enumeration_2d_torus():
    """Untruncated 4x4 torus: the oracle's dlnZ/dbeta and dlnZ/dh equal the enumerated
    <sum of bonds> / V and <sum of spins> / V."""
    from oracle import derivatives
    beta, h = 0.44, 0.07
    _, bonds, mag = exact_ising.brute_force_lnz(beta, h, (4, 4))
    gb = derivatives.dlnz_dbeta(beta, h, 2, INF, 4)
    gh = derivatives.dlnz_dh(beta, h, 2, INF, 4)
    assert abs(gb - bonds / 16) < 1e-9, (gb, bonds / 16)
    assert abs(gh - mag / 16) < 1e-9, (gh, mag / 16)


def test_derivative_high_temperature_series_4d():
    """d/dbeta of ln 2 + 4 ln cosh b + 6 tanh^4 b is 4 tanh b + 24 tanh^3 b sech^2 b; at
    beta = 0.015 the second term is 8e-5.  The chi truncation error of the derivative
    (1.2e-5 at chi = 12) shrinks with chi; a wrong plaquette count (4e-5 per missing
    plaquette pair) or ln cosh coefficient fails the bound."""
    from oracle import derivatives
    beta = 0.015
    t = math.tanh(beta)
    series = 4 * t + 24 * t ** 3 * (1 - t * t)
    errs = [abs(derivatives.dlnz_dbeta(beta, 0.0, 4, trg.Params(chi, 2, q=2, seed=3), 16) - series)
            for chi in (4, 12)]
    assert errs[1] < 2e-5, errs
    assert errs[1] < errs[0], errs


def test_derivative_onsager_2d():
    """d = 2 at chi = 16 on a 2^20 x 2^20 torus: dlnZ/dbeta approaches the derivative of
    Onsager's free energy (taken here by a central difference of the closed form)."""
    from oracle import derivatives
    beta = 0.3
    e = 1e-4
    exact = (exact_ising.onsager_lnz(beta + e) - exact_ising.onsager_lnz(beta - e)) / (2 * e)
    got = derivatives.dlnz_dbeta(beta, 0.0, 2, trg.Params(16, 3, q=2, seed=7), 40)
    assert abs(got - exact) < 1e-6, (got, exact)


def test_truncated_lnz_jumps_between_nearby_couplings():
    """The truncated method's ln Z / V is only piecewise smooth in beta: chi = 8, r = 2, 16
    steps, h = 1e-3 at beta = 0.1497.  Between beta - 5e-7 and beta - 2e-7 it drops by ~4e-6
    across an interval that bisection narrows below 1e-11 (a slope above 1e5 against a
    derivative of ~1): a step of the run picks another kept subspace there (its position
    is a rounding-level detail of the run, its existence is not).  Central
    differences whose stencil stays inside one piece agree (steps 1e-7 and 2e-7, to 1e-4),
    those whose stencil spans the jump do not (step 1e-6 is off by more than a factor 2),
    so a difference step must be chosen per point, not fixed."""
    beta, h = 0.1497, 1e-3

    def lnz(b):
        return trg.Run(b, h, 4, trg.Params(8, 2, q=2, seed=4)).step(16).lnz()

    def central(e):
        return (lnz(beta + e) - lnz(beta - e)) / (2 * e)

    d1, d2, d6 = central(1e-7), central(2e-7), central(1e-6)
    assert abs(d1 - d2) < 1e-4 * abs(d1), (d1, d2)
    assert abs(d6 - d1) > abs(d1), (d6, d1)
    lo, hi = beta - 5e-7, beta - 2e-7
    zlo, zhi = lnz(lo), lnz(hi)
    assert zhi - zlo > 1e-6
    while hi - lo > 1e-11:
        mid = 0.5 * (lo + hi)
        zm = lnz(mid)
        if abs(zm - zlo) > abs(zhi - zm):
            hi, zhi = mid, zm
        else:
            lo, zlo = mid, zm
    assert abs(zhi - zlo) > 1e-6, (lo, hi, zhi - zlo)


@pytest.mark.parametrize("seed", [0, 1])
def test_squeezers_are_optimal_oblique_projectors(seed):
    """Eq. 5: the squeezer pair (M, N) built from the Grams rho_L = R_L^T R_L and
    rho_R = R_R^T R_R is an oblique projector (N M = 1_k) whose error
    || R_L (1 - M N) R_R^T ||_F^2 equals the sum of the discarded squared singular values of
    C = R_L R_R^T, the Eckart-Young minimum over every rank-k product.  Square-root
    factors here come from numpy's eigh, independently of the oracle's; the error does not
    depend on that choice."""
    rng = np.random.default_rng(seed)
    D, k = 4, 5
    P = D * D

    def psd():
        q, _ = np.linalg.qr(rng.standard_normal((P, P)))
        return (q * (0.6 ** np.arange(P))) @ q.T

    rho_l, rho_r = psd(), psd()
    p = trg.Params(k, 4, q=2, seed=seed)  # width r chi = 20 >= P: exact factors
    Ms, Ns = trg.squeezers([rho_l], [rho_r], p, step=1)
    M = Ms[0].reshape(P, -1)
    N = Ns[0].reshape(-1, P)
    assert M.shape == (P, k) and N.shape == (k, P)
    assert np.allclose(N @ M, np.eye(k), atol=1e-10)

    def root(rho):
        w, v = np.linalg.eigh(rho)
        return np.sqrt(np.clip(w, 0.0, None))[:, None] * v.T

    RL, RR = root(rho_l), root(rho_r)
    S = np.linalg.svd(RL @ RR.T, compute_uv=False)
    err = np.linalg.norm(RL @ (np.eye(P) - M @ N) @ RR.T) ** 2
    assert abs(err - np.sum(S[k:] ** 2)) < 1e-10 * np.sum(S ** 2)
    # any other rank-k oblique pair does worse, e.g. the orthogonal projector on M's range
    Pm = M @ np.linalg.pinv(M)
    assert np.linalg.norm(RL @ (np.eye(P) - Pm) @ RR.T) ** 2 >= err * (1 - 1e-12)


def test_resplit_reproduces_the_product_and_rotates_the_legs():
    """The re-split (A1): without truncation c A' diag(s') B' equals Phi Psi^T over the new
    bond, with s' of unit 2-norm, orthonormal columns of A' and rows of B', and every leg
    moved one position left (the next direction comes first)."""
    rng = np.random.default_rng(8)
    legs, Dg = (3, 2, 4), 5
    phi = rng.standard_normal(legs + (Dg,))
    psi = rng.standard_normal(legs + (Dg,))
    p = trg.Params(64, 2, seed=1)
    A, s, B, c = trg.resplit(phi, psi, p)
    assert abs(np.linalg.norm(s) - 1.0) < 1e-14 and np.all(np.diff(s) <= 0)
    Da = s.size
    assert A.shape == (2, 4, 3, Da) and B.shape == (Da, 2, 4, 3)
    am = A.reshape(-1, Da)
    bm = B.reshape(Da, -1)
    assert np.allclose(am.T @ am, np.eye(Da), atol=1e-13)
    assert np.allclose(bm @ bm.T, np.eye(Da), atol=1e-13)
    got = c * np.einsum("xyza,a,auvw->xyzuvw", A, s, B)
    full = np.einsum("ijkg,lmng->ijklmn", phi, psi)
    want = np.transpose(full, (1, 2, 0, 4, 5, 3))  # rotate forward and backward legs left
    assert np.allclose(got, want, atol=1e-12 * np.abs(want).max())


def test_squeezer_grams_equal_dense_unit_cell_grams():
    """Eq. 5 inputs: the Grams rho_L, rho_R that the oracle contracts through the triad
    factors and the Xi / Omega environments equal the Grams of the dense two-site cell
    Gamma = A X sigma Y^T D over each forward pair (i_nu(n+1^), i_nu(n)) and backward pair,
    with every other leg summed.  Exact triad (r chi above every dimension), a random
    state with unequal leg dimensions, so a swapped pair or a wrong leg fails."""
    from paper_2412_14104_gb300 import synth
    A, s, B = synth.split_state(4, (2, 2, 3, 2), 3)
    p = trg.Params(64, 64, seed=5)
    X, sig, Y = trg.bond_swap(A, s, B, p, 1)
    E, F, G, H, I, J, K, L = trg.triad(A, B, X, sig, Y, p, 1)
    rho_l, rho_r = trg.squeezer_grams(E, F, G, H, I, J, K, L, 2)
    fwd = np.einsum("iabsx,xcdtg,g->iabscdtg", A, X, sig)
    bwd = np.einsum("ybcdg,jefhy->bcdgjefh", Y, np.moveaxis(B, 0, -1))
    gam = np.einsum("iabscdtg,BCDgjefh->iabscdtBCDjefh", fwd, bwd)
    legs = "iabscdtBCDjefh"

    def gram(pair):
        rest = [x for x in legs if x not in pair]
        g = np.transpose(gam, [legs.index(pair[0]), legs.index(pair[1])] + [legs.index(x) for x in rest])
        m = g.reshape(g.shape[0] * g.shape[1], -1)
        return m @ m.T

    for nu, (fp, bp) in enumerate((("ac", "Be"), ("bd", "Cf"), ("st", "Dh"))):
        dl, dr = gram(fp), gram(bp)
        assert np.allclose(rho_l[nu], dl, atol=1e-13 * np.abs(dl).max()), nu
        assert np.allclose(rho_r[nu], dr, atol=1e-13 * np.abs(dr).max()), nu
        assert not np.allclose(rho_l[nu], gram(fp[::-1]), atol=1e-3 * np.abs(dl).max())


def test_contraction_equals_dense_cell_with_squeezers():
    """Eqs. 6-7: Phi Psi^T from the factored chain C1-C4 equals the dense two-site cell
    A X sigma Y^T D with the squeezers M (forward pairs) and N (backward pairs) attached,
    in the exact-triad regime, for a random state with unequal leg dimensions."""
    from paper_2412_14104_gb300 import synth
    A, s, B = synth.split_state(4, (2, 2, 3, 2), 3)
    p = trg.Params(64, 64, seed=5)
    X, sig, Y = trg.bond_swap(A, s, B, p, 1)
    E, F, G, H, I, J, K, L = trg.triad(A, B, X, sig, Y, p, 1)
    rho_l, rho_r = trg.squeezer_grams(E, F, G, H, I, J, K, L, 2)
    Ms, Ns = trg.squeezers(rho_l, rho_r, p, 1)
    phi, psi = trg.contract(E, F, G, H, I, J, K, L, Ms, Ns, 2)
    got = np.einsum("iuvzg,jUVZg->iuvzjUVZ", phi, psi)
    fwd = np.einsum("iabsx,xcdtg,g->iabscdtg", A, X, sig)
    bwd = np.einsum("ybcdg,jefhy->bcdgjefh", Y, np.moveaxis(B, 0, -1))
    gam = np.einsum("iabscdtg,BCDgjefh->iabscdtBCDjefh", fwd, bwd)
    want = np.einsum("iabscdtBCDjefh,acu,bdv,stz,UBe,VCf,ZDh->iuvzjUVZ", gam, Ms[0], Ms[1], Ms[2],
                     Ns[0], Ns[1], Ns[2], optimize=True)
    assert np.allclose(got, want, atol=1e-13 * np.abs(want).max())


def test_bond_swap_preserves_the_two_site_product():
    """Eq. 1: without truncation A (X sigma Y^T) D equals the dense product of two site
    tensors T = A s B joined along the active direction (the upper site's backward leg 0
    with the lower site's forward leg 0), for a random state with unequal leg dimensions."""
    from paper_2412_14104_gb300 import synth
    A, s, B = synth.split_state(4, (2, 2, 3, 2), 3)
    p = trg.Params(64, 64, seed=5)
    X, sig, Y = trg.bond_swap(A, s, B, p, 1)
    fwd = np.einsum("iabsx,xcdtg,g->iabscdtg", A, X, sig)
    bwd = np.einsum("ybcdg,jefhy->bcdgjefh", Y, np.moveaxis(B, 0, -1))
    got = np.einsum("iabscdtg,BCDgjefh->iabscdtBCDjefh", fwd, bwd)
    T = np.einsum("iabsx,x,xjefh->iabsjefh", A, s, B)
    want = np.einsum("iabskBCD,kcdtjefh->iabscdtBCDjefh", T, T)
    assert np.allclose(got, want, atol=1e-13 * np.abs(want).max())


# --- transition-point order parameter X^(m) -------------------------------------------

def test_transfer_matrix_matches_enumeration():
    """The transfer-matrix partition function used below against brute force (small tori,
    with L = 1 self-loops and L = 2 double bonds)."""
    for L0, L1, beta, h in ((2, 2, 0.4, 0.0), (3, 4, 0.3, 0.1), (1, 3, 0.7, -0.2), (4, 2, 0.44, 0.05)):
        want, _, _ = exact_ising.brute_force_lnz(beta, h, (L0, L1))
        assert abs(exact_ising.transfer_matrix_lnz(beta, h, L0, L1) - want) < 1e-11


def test_order_parameter_is_a_ratio_of_partition_functions():
    """With nothing truncated, T represents the whole block of sites coarse-grained so far,
    Tr A^(m) is Z of that block's torus and Tr (A^(m))^2 is Z of the torus doubled along the
    open leg's direction, so X = Z(block)^2 / Z(doubled).  Leg position p after k steps is
    lattice direction (p + k) mod d."""
    # 2D, four steps: a 4 x 4 block; the doubled torus (8 x 4 or 4 x 8) by transfer matrix
    for beta, h in ((0.3, 0.0), (0.4407, 0.0), (0.6, 0.02)):
        run = trg.Run(beta, h, 2, INF).step(4)
        z = exact_ising.transfer_matrix_lnz(beta, h, 4, 4)
        for leg in (0, 1):
            x, _ = trg.order_parameter_x(run.A, run.s, run.B, leg)
            zz = exact_ising.transfer_matrix_lnz(beta, h, 4, 8)  # symmetric block: either axis
            assert abs(math.log(x) - (2 * z - zz)) < 1e-10
    # 4D, two steps: block (2, 2, 1, 1) along directions (0, 1, 2, 3); positions are
    # (dir 2, dir 3, dir 0, dir 1)
    beta, h = 0.1497, 0.05
    run = trg.Run(beta, h, 4, INF).step(2)
    z, _, _ = exact_ising.brute_force_lnz(beta, h, (2, 2, 1, 1))
    for leg, doubled in ((3, (2, 4, 1, 1)), (2, (4, 2, 1, 1)), (0, (2, 2, 2, 1))):
        x, _ = trg.order_parameter_x(run.A, run.s, run.B, leg)
        zz, _, _ = exact_ising.brute_force_lnz(beta, h, doubled)
        assert abs(math.log(x) - (2 * z - zz)) < 1e-11, leg


def test_order_parameter_limits():
    """X counts the ground-state degeneracy: deep in the ordered phase (large beta, h = 0)
    the coarse tensor has two equal sectors and X -> 2; at high temperature X -> 1."""
    hot = trg.Run(0.05, 0.0, 2, trg.Params(8, 2, seed=1)).step(12)
    cold = trg.Run(1.2, 0.0, 2, trg.Params(8, 2, seed=1)).step(12)
    assert abs(trg.order_parameter_x(hot.A, hot.s, hot.B, 1)[0] - 1.0) < 1e-6
    assert abs(trg.order_parameter_x(cold.A, cold.s, cold.B, 1)[0] - 2.0) < 1e-6


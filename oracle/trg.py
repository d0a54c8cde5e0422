"""One Triad-ATRG (or ATRG) coarse-graining step and the ln Z accumulation, FP64 NumPy.

Follows Sec. 2 of Sugimoto & Sasaki (arXiv:2412.14104) in the paper's order:

1. bond swap (Eq. 1): the middle of the two-site product along the active direction,
   Mid[(alpha,i),(beta,j)] = sum_k s_alpha B[alpha,k,j] A[k,i,beta] s_beta, is truncated to
   X sigma Y^T with the randomized SVD (Table 1 "bond swapping", RSVD with q iterations);
2. triad isometries (Eqs. 2-3): U^A, U^X, U^Y, U^D are the leading r*chi eigenvectors of
   the Grams of A X sigma, X sigma, Y sigma and D on the grouped transverse legs (the
   environment of each reduces to these because Gamma is in canonical form);
3. triad tensors (Eq. 4): E = A U^A, F = X U^X sigma, G = Y U^Y, H = D U^D; I..L = U;
4. squeezers (Eq. 5): for every transverse direction an oblique projector pair M, N built
   from the Grams of Gamma^triad on the forward and backward leg pairs;
5. contraction (Eqs. 6-7): Phi and Psi, the O(r^2 chi^7) bottleneck (Fig. 2);
6. re-split of Phi Psi^T into A' s' B', normalisation and the leg rotation.

Readings where the paper is silent (each repeated in the design notes):
* legs are stored with the active direction at position 0; after a step the forward and
  backward leg orders rotate left by one, so directions cycle 1, 2, ..., d, 1, ...;
* the triad groups the transverse positions 1..d-2 (directions 2 and 3 at d = 4, Eq. 4),
  the last position d-1 is the separate 4-leg direction; at d = 2 the group is empty and
  the method is ATRG;
* randomized widths: swap ell = min(r chi, rows, cols); triad ell = k = min(r chi, G)
  (G = product of the grouped dims); squeezer ell = min(r chi, D^2).  Whenever ell reaches
  the full dimension the exact SVD / eigensolver is used instead;
* cut-offs: singular values / eigenvalues at or below 1e-14 of the largest are dropped;
  squeezer singular values at or below 1e-12 of the largest are dropped;
* degenerate multiplets (consecutive singular values within a relative gap TAU = 1e-10) are
  never cut, and the bases that later sketches act on (the bond index of A', B' and the new
  leg of M, N) are put into the canonical basis of ``rla.canonical_basis``;
* squeezer construction (Eq. 5 gives only the cost function): rho_L = R_L^T R_L,
  rho_R = R_R^T R_R, C = R_L R_R^T = U S V^T, M = R_R^T V_k S_k^-1/2,
  N = S_k^-1/2 U_k^T R_L, which minimises || R_L (1 - M N) R_R^T ||;
* normalisation c_k = ||s'||_2 after every step; ln Z / V = sum_k 2^-k ln c_k
  + 2^-N ln tTr(T_N) with tTr the trace of every forward leg with its own backward leg.
"""
import math

import numpy as np

from . import philox, rla

STAGES = ("swap", "triad", "squeeze", "contract", "resplit")
TAU = 1e-10  # relative gap (s_i - s_i+1) / s_i below which values form one multiplet


class Params:
    """chi=None and r=None select the untruncated ("chi = infinity") mode."""

    def __init__(self, chi, r, q=2, method="triad", seed=0, replica=0, split_tau=None, split_from_step=1):
        if method not in ("triad", "atrg"):
            raise ValueError(method)
        self.chi = chi
        self.r = r
        self.q = int(q)
        self.method = method
        self.seed = int(seed)
        self.replica = int(replica)
        # multiplet gap used from split_from_step on (the library's split-precision steps
        # use 1e-6); None keeps TAU everywhere
        self.split_tau = split_tau
        self.split_from_step = int(split_from_step)

    def tau(self, step):
        if self.split_tau is not None and step >= self.split_from_step:
            return self.split_tau
        return TAU

    def cap(self):
        return None if self.chi is None else int(self.chi)

    def width(self):
        if self.chi is None or self.r is None:
            return None
        return int(self.r) * int(self.chi)


class Counter:
    """Algorithmic FP64 flop count per stage (2 * product of all index extents)."""

    def __init__(self):
        self.flops = {k: 0 for k in STAGES}

    def total(self):
        return sum(self.flops.values())


def _dims_of(spec, ops):
    ins = spec.split("->")[0].split(",")
    dims = {}
    for sub, op in zip(ins, ops):
        for ch, n in zip(sub, op.shape):
            dims[ch] = n
    return dims


def _c(cnt, stage, spec, *ops):
    """Pairwise contraction with flop accounting (einsum, BLAS-backed)."""
    if cnt is not None and len(ops) == 2:
        n = 2
        for v in _dims_of(spec, ops).values():
            n *= v
        cnt.flops[stage] += n
    return np.einsum(spec, *ops, optimize=True)


def _mm(cnt, stage, a, b):
    if cnt is not None:
        cnt.flops[stage] += 2 * a.shape[0] * a.shape[1] * b.shape[1]
    return a @ b


def _min_none(*xs):
    vals = [x for x in xs if x is not None]
    return min(vals)


class SwapOp:
    """Mid of Eq. 1 applied without forming it: As[k,i,beta] = A s_beta,
    Bs[alpha,k,j] = s_alpha B.  Each product costs two GEMM-shaped contractions."""

    def __init__(self, As, Bs, cnt):
        self.As, self.Bs, self.cnt = As, Bs, cnt
        Dk, I, Da = As.shape
        self.shape = (Da * I, Da * I)
        self.Da, self.I = Da, I

    def matmul(self, om):
        ell = om.shape[1]
        om3 = om.reshape(self.Da, self.I, ell)
        w1 = _c(self.cnt, "swap", "akj,bjp->akbp", self.Bs, om3)
        y = _c(self.cnt, "swap", "kib,akbp->aip", self.As, w1)
        return y.reshape(self.shape[0], ell)

    def rmatmul(self, qm):
        ell = qm.shape[1]
        q3 = qm.reshape(self.Da, self.I, ell)
        w2 = _c(self.cnt, "swap", "kib,aip->akbp", self.As, q3)
        z = _c(self.cnt, "swap", "akj,akbp->bjp", self.Bs, w2)
        return z.reshape(self.shape[1], ell)

    def dense(self):
        m = np.einsum("akj,kib->aibj", self.Bs, self.As)
        return m.reshape(self.shape)


def _gap(vals, k):
    """Relative gap at a cut after k kept values (inf when nothing is cut)."""
    if k >= vals.size or vals.size == 0 or vals[0] <= 0.0:
        return math.inf
    return float((vals[k - 1] - vals[k]) / vals[0])


def bond_swap(A, s, B, p, step, cnt=None, info=None):
    """Eq. 1: returns X[alpha, i_1..i_{d-1}, gamma], sigma, Y[beta, j_1..j_{d-1}, gamma]."""
    d = A.ndim - 1
    D = A.shape[:d]
    Da = s.size
    I = int(np.prod(D[1:]))
    As = A.reshape(D[0], I, Da) * s[None, None, :]
    Bs = B.reshape(Da, D[0], I) * s[:, None, None]
    op = SwapOp(As, Bs, cnt)
    rows, cols = op.shape
    ell = _min_none(p.width(), rows, cols)
    if ell >= min(rows, cols):
        U, S, V = rla.svd_desc(op.dense())
        exact = True
    else:
        om = philox.gaussian(p.seed, philox.stream_id(step, philox.KIND_SWAP), cols, ell,
                             p.replica)
        U, S, V = rla.rsvd(op, ell, p.q, om)
        exact = False
    Dg = rla.multiplet_cut(S, rla.keep_count(S, 1e-14, p.cap()), p.tau(step))
    X, sgn = rla.fix_sign(U[:, :Dg])
    Y = V[:, :Dg] * sgn[None, :]
    if info is not None:
        info["swap_sigma"] = S.copy()
        info["swap_gap"] = _gap(S, Dg)
        info["swap_exact"] = exact
    shp = (Da,) + tuple(D[1:]) + (Dg,)
    return X.reshape(shp), S[:Dg].copy(), Y.reshape(shp)


def _isometry(rho, p, step, kind, cnt, info, name):
    """Leading eigenvectors of a PSD Gram (Eqs. 2-3): exact or RSVD with ell = k."""
    G = rho.shape[0]
    if p.method == "atrg":
        return np.eye(G)
    k = _min_none(p.width(), G)
    if k >= G:
        lam, U = rla.eigh_desc(rho)
    else:
        om = philox.gaussian(p.seed, philox.stream_id(step, kind), G, k, p.replica)
        lam, U = rla.rsvd_psd(lambda x: _mm(cnt, "triad", rho, x), k, p.q, om)
    keep = rla.keep_count(lam, 1e-14, k)
    U, _ = rla.fix_sign(U[:, :keep])
    if info is not None:
        info["triad_lam_" + name] = lam.copy()
    return U


def triad(A, B, X, sig, Y, p, step, cnt=None, info=None):
    """Eqs. 2-4.  Returns E, F, G, H (4-leg, [x, k, sep, bond]) and I, J, K, L (group, k)."""
    d = A.ndim - 1
    D = A.shape[:d]
    g = d - 2
    Gdim = int(np.prod(D[1:1 + g])) if g > 0 else 1
    Ds = D[d - 1]
    Da = A.shape[-1]
    Dg = sig.size
    A4 = A.reshape(D[0], Gdim, Ds, Da)          # [i0, G, i_sep, alpha]
    X4 = X.reshape(Da, Gdim, Ds, Dg)            # [alpha, G, i_sep, gamma]
    Y4 = Y.reshape(Da, Gdim, Ds, Dg)            # [beta, G, j_sep, gamma]
    D4 = B.reshape(Da, D[0], Gdim, Ds)          # [beta, j0, G, j_sep]
    s2 = sig * sig
    Xs = X4 * s2[None, None, None, :]
    Ys = Y4 * s2[None, None, None, :]
    # environments of A and D (Xi = X sigma^2 X^T over everything but the bond)
    xi_x = _c(cnt, "triad", "agsc,bgsc->ab", Xs, X4)
    xi_y = _c(cnt, "triad", "agsc,bgsc->ab", Ys, Y4)
    t_a = _c(cnt, "triad", "igsa,ab->igsb", A4, xi_x)
    rho_a = _c(cnt, "triad", "igsb,ihsb->gh", t_a, A4)
    rho_x = _c(cnt, "triad", "agsc,ahsc->gh", Xs, X4)
    rho_y = _c(cnt, "triad", "agsc,ahsc->gh", Ys, Y4)
    t_d = _c(cnt, "triad", "ajgs,ab->bjgs", D4, xi_y)
    rho_d = _c(cnt, "triad", "bjgs,bjhs->gh", t_d, D4)
    UA = _isometry(rho_a, p, step, philox.KIND_TRIAD["A"], cnt, info, "A")
    UX = _isometry(rho_x, p, step, philox.KIND_TRIAD["X"], cnt, info, "X")
    UY = _isometry(rho_y, p, step, philox.KIND_TRIAD["Y"], cnt, info, "Y")
    UD = _isometry(rho_d, p, step, philox.KIND_TRIAD["D"], cnt, info, "D")
    E = _c(cnt, "triad", "igsa,gk->iksa", A4, UA)
    F = _c(cnt, "triad", "agsc,gk->aksc", X4, UX) * sig[None, None, None, :]
    G = _c(cnt, "triad", "bgsc,gk->bksc", Y4, UY)
    H = _c(cnt, "triad", "bjgs,gk->jksb", D4, UD)
    gshape = tuple(D[1:1 + g])
    I = UA.reshape(gshape + (UA.shape[1],))
    J = UX.reshape(gshape + (UX.shape[1],))
    K = UY.reshape(gshape + (UY.shape[1],))
    L = UD.reshape(gshape + (UD.shape[1],))
    return E, F, G, H, I, J, K, L


def _group_pair(U, nu, g):
    """Partial Gram of a group isometry on group leg nu (1-based within the group)."""
    if g == 1:
        return np.einsum("xk,yl->xykl", U, U)
    if nu == 1:
        return np.einsum("xzk,yzl->xykl", U, U)
    return np.einsum("zxk,zyl->xykl", U, U)


def _factor(rho, p, step, kind, cnt):
    """R with rho ~= R^T R from the leading eigenpairs (exact or RSVD, ell = min(r chi, P))."""
    P = rho.shape[0]
    ell = _min_none(p.width(), P)
    if ell >= P:
        lam, U = rla.eigh_desc(rho)
    else:
        om = philox.gaussian(p.seed, philox.stream_id(step, kind), P, ell, p.replica)
        lam, U = rla.rsvd_psd(lambda x: _mm(cnt, "squeeze", rho, x), ell, p.q, om)
    keep = rla.keep_count(lam, 1e-14, ell)
    return np.sqrt(lam[:keep])[:, None] * U[:, :keep].T


def squeezer_grams(E, F, G, H, I, J, K, L, g, cnt=None):
    """Grams of Gamma^triad on every forward pair (rho_L) and backward pair (rho_R) of legs.

    Returns two lists indexed by transverse position nu = 1..g+1, each a matrix over
    (a, b) = (leg at n + 1^, leg at n) in row-major order.
    """
    st = "squeeze"
    om_d = _c(cnt, st, "jksb,jksc->bc", H, H)
    t = _c(cnt, st, "bksg,bc->cksg", G, om_d)
    om_y = _c(cnt, st, "cksg,cksh->gh", t, G)
    om_a = _c(cnt, st, "iksa,iksb->ab", E, E)
    t = _c(cnt, st, "aksg,ab->bksg", F, om_a)
    om_x = _c(cnt, st, "bksg,bksh->gh", t, F)
    Ds = E.shape[2]
    P = Ds * Ds
    # separate leg (position g+1)
    eps = _c(cnt, st, "ikxa,ikyb->xayb", E, E)
    Fy = _c(cnt, st, "akxg,gh->akxh", F, om_y)
    phi = _c(cnt, st, "akxh,ckyh->axcy", Fy, F)
    rho_l_sep = _c(cnt, st, "xayb,azbw->xzyw", eps, phi).reshape(P, P)
    Gx = _c(cnt, st, "bkxg,gh->bkxh", G, om_x)
    gam = _c(cnt, st, "bkxh,ckyh->bxcy", Gx, G)
    eta = _c(cnt, st, "jkxb,jkyc->xbyc", H, H)
    rho_r_sep = _c(cnt, st, "bxcy,zbwc->xzyw", gam, eta).reshape(P, P)
    rho_l = [None] * g + [rho_l_sep]
    rho_r = [None] * g + [rho_r_sep]
    if g > 0:
        p_e = _c(cnt, st, "iksa,ilsb->klab", E, E)
        p_f = _c(cnt, st, "aksh,blsh->abkl", Fy, F)
        env_l = _c(cnt, st, "klab,abmn->klmn", p_e, p_f)
        p_g = _c(cnt, st, "bksh,clsh->klbc", Gx, G)
        p_h = _c(cnt, st, "jksb,jlsc->bckl", H, H)
        env_r = _c(cnt, st, "klbc,bcmn->klmn", p_g, p_h)
        for nu in range(1, g + 1):
            ii = _group_pair(I, nu, g)
            jj = _group_pair(J, nu, g)
            t = _c(cnt, st, "xykl,klmn->xymn", ii, env_l)
            Dn = ii.shape[0]
            rho_l[nu - 1] = _c(cnt, st, "xymn,zwmn->xzyw", t, jj).reshape(Dn * Dn, Dn * Dn)
            kk = _group_pair(K, nu, g)
            ll = _group_pair(L, nu, g)
            t = _c(cnt, st, "xykl,klmn->xymn", kk, env_r)
            rho_r[nu - 1] = _c(cnt, st, "xymn,zwmn->xzyw", t, ll).reshape(Dn * Dn, Dn * Dn)
    return rho_l, rho_r


def squeezers(rho_l, rho_r, p, step, cnt=None, info=None):
    """Eq. 5 with oblique projectors.  Returns M[nu] of shape (D, D, k) over
    (i_nu(n+1^), i_nu(n), k) and N[nu] of shape (k, D, D) over (k, j_nu(n+1^), j_nu(n))."""
    Ms, Ns = [], []
    for nu in range(1, len(rho_l) + 1):
        RL = _factor(rho_l[nu - 1], p, step, philox.KIND_SQ_LEFT + nu - 1, cnt)
        RR = _factor(rho_r[nu - 1], p, step, philox.KIND_SQ_RIGHT + nu - 1, cnt)
        C = RL @ RR.T
        U, S, V = rla.svd_desc(C)
        k = rla.multiplet_cut(S, rla.keep_count(S, 1e-12, p.cap()), p.tau(step))
        isq = 1.0 / np.sqrt(S[:k])
        M = (RR.T @ V[:, :k]) * isq[None, :]
        N = (U[:, :k] * isq[None, :]).T @ RL
        M, O = rla.canonical_basis(M, S[:k], p.tau(step))
        N = O.T @ N
        Dn = int(round(math.sqrt(M.shape[0])))
        Ms.append(M.reshape(Dn, Dn, k))
        Ns.append(N.reshape(k, Dn, Dn))
        if info is not None:
            info["sq_S_%d" % nu] = S.copy()
            info["sq_gap_%d" % nu] = _gap(S, k)
    return Ms, Ns


def _group_core(U1, U2, Ws, g, cnt, left):
    """P[k1, k2, kG...] = sum I[a_G, k1] J[b_G, k2] prod_nu W_nu (C3 of the contraction).

    ``left``: W_nu = M_nu[a, b, k] (Phi); otherwise W_nu = N_nu[k, a, b] (Psi)."""
    st = "contract"
    if g == 0:
        return np.ones((1, 1))
    Wt = [w if left else np.transpose(w, (1, 2, 0)) for w in Ws]  # -> [a, b, k]
    if g == 1:
        t = _c(cnt, st, "xk,xyz->kyz", U1, Wt[0])
        return _c(cnt, st, "kyz,yl->klz", t, U2)
    t1 = _c(cnt, st, "xwk,xyz->wkyz", U1, Wt[0])
    t2 = _c(cnt, st, "wkyz,wvu->kyzvu", t1, Wt[1])
    pm = _c(cnt, st, "kyzvu,yvl->kzul", t2, U2)
    return np.transpose(pm, (0, 3, 1, 2))


QF_BLOCK_DOUBLES = 1 << 28  # largest block of the C2 intermediate held at once (2 GB)


def _c2_c4(em, F, pf, g, cnt):
    """C2 then C4 of one side (Eqs. 6-7), for blocks of consecutive gamma at a time.

    C2: qf[i, k, z, l, gamma] = sum_{a, y} em[i, k, a, y, z] F[a, l, y, gamma];
    C4: out[i, u.., z, gamma] = sum_{k, l} qf[i, k, z, l, gamma] pf[k, l, u..].
    Each output column gamma is computed from the same terms whatever the block; the blocks
    only bound the host memory of qf (18 GB at chi = 48, r = 3 if held whole)."""
    st = "contract"
    i, k, _, _, z = em.shape
    l, Dg = F.shape[1], F.shape[3]
    gb = max(1, min(Dg, QF_BLOCK_DOUBLES // (i * k * z * l)))
    out = None
    for g0 in range(0, Dg, gb):
        qf = _c(cnt, st, "ikayz,alyg->ikzlg", em, F[:, :, :, g0:g0 + gb])   # C2
        if g == 0:
            blk = qf[:, 0, :, 0, :]
        elif g == 1:
            blk = _c(cnt, st, "ikzlg,klu->iuzg", qf, pf)                    # C4
        else:
            blk = _c(cnt, st, "ikzlg,kluv->iuvzg", qf, pf)                  # C4
        if out is None:
            out = np.empty(blk.shape[:-1] + (Dg,))
        out[..., g0:g0 + gb] = blk
        del qf
    return out


def contract(E, F, G, H, I, J, K, L, Ms, Ns, g, cnt=None):
    """Eqs. 6-7.  Phi[i1, k_2..k_d, gamma] and Psi[j1, k'_2..k'_d, gamma].

    Phi: C1 em = E M_sep, C2 with F, C3 pf from I, J and the group squeezers M_nu, C4.
    Psi: the same chain with H (for E), G (for F), K, L and the N_nu."""
    st = "contract"
    Msep, Nsep = Ms[g], Ns[g]
    pf = _group_core(I, J, Ms[:g], g, cnt, True)           # C3 [kA, kX, k_G]
    pp = _group_core(K, L, Ns[:g], g, cnt, False)          # C3' [kY, kD, k_G]
    pp = np.swapaxes(pp, 0, 1)                             #     [kD, kY, k_G]
    em = _c(cnt, st, "ikxa,xyz->ikayz", E, Msep)            # C1  [i, kA, a, y, k_sep]
    phi = _c2_c4(em, F, pf, g, cnt)
    del em
    hn = _c(cnt, st, "jkyd,zxy->jkdxz", H, Nsep)            # C1' [j, kD, d, x, k_sep]
    psi = _c2_c4(hn, G, pp, g, cnt)
    return phi, psi


def resplit(phi, psi, p, cnt=None, info=None, step=0):
    """T' = Phi Psi^T = A' s' B' through two thin QRs and a small SVD; normalise; rotate."""
    d = phi.ndim - 1
    Dg = phi.shape[-1]
    pm = phi.reshape(-1, Dg)
    sm = psi.reshape(-1, Dg)
    if cnt is not None:
        cnt.flops["resplit"] += 4 * (pm.shape[0] + sm.shape[0]) * Dg * Dg
    qa, ra = rla.orth(pm)
    qb, rb = rla.orth(sm)
    U, S, V = rla.svd_desc(ra @ rb.T)
    Da = rla.keep_count(S, 1e-14, p.cap())
    An = _mm(cnt, "resplit", qa, U[:, :Da])
    Bn = _mm(cnt, "resplit", qb, V[:, :Da])
    c = float(np.linalg.norm(S[:Da]))
    s = S[:Da] / c
    legs = phi.shape[:d]
    An = An.reshape(legs + (Da,))
    Bn = Bn.reshape(legs + (Da,))
    rot = tuple(range(1, d)) + (0, d)
    An = np.ascontiguousarray(np.transpose(An, rot))
    Bn = np.ascontiguousarray(np.transpose(Bn, rot))
    am, O = rla.canonical_basis(An.reshape(-1, Da), s, p.tau(step))
    bm = Bn.reshape(-1, Da) @ O
    if info is not None:
        info["s"] = s.copy()
        info["c"] = c
    new_legs = An.shape[:d]
    return am.reshape(new_legs + (Da,)), s, np.ascontiguousarray(bm.T).reshape((Da,) + new_legs), c


def rg_step(A, s, B, p, step, cnt=None, info=None):
    """One coarse-graining step along the direction at leg position 0 (Sec. 2)."""
    d = A.ndim - 1
    g = d - 2
    X, sig, Y = bond_swap(A, s, B, p, step, cnt, info)
    E, F, G, H, I, J, K, L = triad(A, B, X, sig, Y, p, step, cnt, info)
    rho_l, rho_r = squeezer_grams(E, F, G, H, I, J, K, L, g, cnt)
    Ms, Ns = squeezers(rho_l, rho_r, p, step, cnt, info)
    phi, psi = contract(E, F, G, H, I, J, K, L, Ms, Ns, g, cnt)
    return resplit(phi, psi, p, cnt, info, step)


def trace(A, s, B):
    """tTr of a single-site periodic lattice: every forward leg traced with its backward leg."""
    Da = s.size
    am = A.reshape(-1, Da)
    bm = B.reshape(Da, -1)
    return float(np.einsum("fa,a,af->", am, s, bm))


def order_parameter_x(A, s, B, leg):
    """Gu-Wen degeneracy order parameter of the current coarse tensor (Sec. 3, the
    definition of X^(m)): A^(m)_kl = sum over every other leg x of T[.., x, k, ..; .., x, l, ..],
    the forward leg at position ``leg`` open as k and its backward leg as l, and
    X = (Tr A^(m))^2 / Tr (A^(m))^2.  T = A diag(s) B is never formed."""
    d = A.ndim - 1
    letters = "ijmnopqr"[:d]
    fa = "".join("k" if p == leg else letters[p] for p in range(d))
    fb = "".join("l" if p == leg else letters[p] for p in range(d))
    Am = np.einsum("%sa,a,a%s->kl" % (fa, fb), A, s, B)
    return float(np.trace(Am) ** 2 / np.trace(Am @ Am)), Am


class Run:
    """State of an RG run: (A, s, B), step count and the ln Z / V partial sum."""

    def __init__(self, beta, h, d, p, W=None):
        from . import ising
        self.p = p
        self.d = d
        self.A, self.s, self.B, c0 = ising.initial_state(beta, h, d, p.cap(), W)
        self.lnc = [math.log(c0)]
        self.k = 0
        self.infos = []
        self.cnt = Counter()

    def step(self, n=1):
        for _ in range(n):
            self.k += 1
            info = {}
            self.A, self.s, self.B, c = rg_step(self.A, self.s, self.B, self.p, self.k,
                                                self.cnt, info)
            self.lnc.append(math.log(c))
            self.infos.append(info)
        return self

    def partial_lnz(self):
        """sum_k 2^-k ln c_k (the part of ln Z / V fixed by the steps so far)."""
        return math.fsum(v * 2.0 ** (-k) for k, v in enumerate(self.lnc))

    def lnz(self):
        tt = trace(self.A, self.s, self.B)
        if tt <= 0.0:
            raise FloatingPointError("non-positive final trace %r" % tt)
        return self.partial_lnz() + 2.0 ** (-self.k) * math.log(tt)


def lnz_per_site(beta, h, d, p, nsteps, W=None):
    return Run(beta, h, d, p, W).step(nsteps).lnz()


def free_energy(beta, h, d, p, nsteps):
    return -lnz_per_site(beta, h, d, p, nsteps) / beta

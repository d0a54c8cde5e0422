"""Dense and randomized linear algebra used by every truncation of the RG step.

* ``orth``: thin QR with diag(R) >= 0 (unique at full column rank), LAPACK Householder.
* ``rsvd``: randomized SVD of Halko, Martinsson & Tropp (SIAM Review 53, 2011), their
  Algorithm 4.4 (randomized subspace iteration) followed by Algorithm 5.1 (direct SVD):
  Y = M Omega, Q = orth(Y); q times { Qt = orth(M^T Q); Q = orth(M Qt) }; B = Q^T M;
  B^T = P R; R^T = W S Z^T; left vectors Q W, right vectors P Z.  The paper uses this
  RSVD with q QR iterations for the bond swap (Table 1, Sec. 1); q counts power
  iterations, giving 2q+2 products with M or M^T.
* ``rsvd_psd``: the same subspace iteration for a symmetric positive semi-definite Gram
  rho (M^T = M), finished by B = Q^T rho Q and a symmetric eigensolve.
* ``fix_sign``: the sign convention for singular/eigen vectors.  A column v is flipped so
  that w . v > 0, with w_i = (fmix32(i + 1) + 0.5) / 2^32 - 0.5 (the MurmurHash3
  32-bit finaliser).  A fixed, structureless weight avoids the exact magnitude ties that
  the symmetric Ising tensors produce under a "largest entry positive" rule.
* ``canonical_basis``: lattice symmetries make singular values exactly degenerate; any
  orthonormal basis of such a multiplet is correct, but a later Gaussian sketch acts on the
  basis, so it must be fixed.  The columns V_M of a multiplet are rotated to V_M O with O
  the orthogonal polar factor of V_M^T W, W_j(i) = (fmix32((i + 1) xor (j * 0x9E3779B9))
  + 0.5) / 2^32 - 0.5.  The result does not depend on the basis the solver returned, and for
  a single vector it is the sign rule above.
* ``multiplet_cut``: a truncation never splits a multiplet; the cut moves down to the
  multiplet's first member.
"""
import numpy as np

_MASK = np.uint64(0xFFFFFFFF)


def _fmix32(h):
    h = h.astype(np.uint64)
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(0x85EBCA6B)) & _MASK
    h ^= h >> np.uint64(13)
    h = (h * np.uint64(0xC2B2AE35)) & _MASK
    h ^= h >> np.uint64(16)
    return h


def sign_weights(n):
    i = np.arange(1, n + 1, dtype=np.uint64)
    return (_fmix32(i).astype(np.float64) + 0.5) * (1.0 / 4294967296.0) - 0.5


def fix_sign(V):
    """Return (V * sgn, sgn) with sgn_j = sign(w . V[:, j]) (+1 when the product is 0)."""
    w = sign_weights(V.shape[0])
    sgn = np.where(w @ V < 0.0, -1.0, 1.0)
    return V * sgn[None, :], sgn


def multiplets(vals, tau):
    """Index ranges [a, b) of runs whose consecutive gaps are <= tau times the larger value."""
    out = []
    a = 0
    n = len(vals)
    for i in range(1, n + 1):
        if i == n or vals[i - 1] - vals[i] > tau * vals[i - 1]:
            if i - a > 1:
                out.append((a, i))
            a = i
    return out


def multiplet_cut(vals, k, tau):
    """Largest k' <= k that does not cut a multiplet (k itself when nothing is cut)."""
    if k <= 0 or k >= len(vals):
        return k
    for a, b in multiplets(vals, tau):
        if a < k < b:
            return a if a > 0 else b
    return k


def basis_weights(n, m):
    i = np.arange(1, n + 1, dtype=np.uint64)[:, None]
    j = (np.arange(m, dtype=np.uint64) * np.uint64(0x9E3779B9)) & _MASK
    return (_fmix32(i ^ j[None, :]).astype(np.float64) + 0.5) * (1.0 / 4294967296.0) - 0.5


def canonical_basis(V, vals, tau):
    """Rotate the columns of V inside each multiplet of vals (and flip single columns) to
    the canonical basis; returns (V', O) with V' = V O, O block-diagonal orthogonal."""
    n, k = V.shape
    O = np.diag(np.where(sign_weights(n) @ V < 0.0, -1.0, 1.0))
    for a, b in multiplets(vals[:k], tau):
        W = basis_weights(n, b - a)
        Gm = V[:, a:b].T @ W
        U, _, Vt = np.linalg.svd(Gm)
        O[a:b, a:b] = U @ Vt
    return V @ O, O


def orth(Y):
    """Thin QR with non-negative diagonal of R: returns (Q, R)."""
    Q, R = np.linalg.qr(Y, mode="reduced")
    d = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    return Q * d[None, :], R * d[:, None]


def svd_desc(M):
    """Thin SVD with singular values in descending order (LAPACK gesdd)."""
    U, S, Vt = np.linalg.svd(M, full_matrices=False)
    return U, S, Vt.T


def eigh_desc(rho):
    """Symmetric eigendecomposition, eigenvalues in descending order."""
    lam, V = np.linalg.eigh(0.5 * (rho + rho.T))
    order = np.argsort(-lam, kind="stable")
    return lam[order], V[:, order]


class DenseOp:
    """A dense matrix seen through the two products the RSVD needs."""

    def __init__(self, M):
        self.M = M
        self.shape = M.shape

    def matmul(self, X):
        return self.M @ X

    def rmatmul(self, X):
        return self.M.T @ X

    def dense(self):
        return self.M


def rsvd(op, ell, q, omega):
    """Randomized SVD of ``op`` (m x n) with sketch ``omega`` (n x ell), q power iterations.

    Returns (U, S, V) with m x ell, ell, n x ell, S descending.
    """
    Q, _ = orth(op.matmul(omega))
    for _ in range(q):
        Qt, _ = orth(op.rmatmul(Q))
        Q, _ = orth(op.matmul(Qt))
    Bt = op.rmatmul(Q)                 # (Q^T M)^T, n x ell
    P, R = orth(Bt)
    W, S, Z = svd_desc(R.T)            # R^T = W S Z^T
    return Q @ W, S, P @ Z


def rsvd_psd(apply_rho, ell, q, omega):
    """Subspace iteration for a PSD Gram given by ``apply_rho(X) = rho @ X``.

    Returns (lam, U): the ell Ritz values (descending) and vectors.
    """
    Q, _ = orth(apply_rho(omega))
    for _ in range(q):
        Qt, _ = orth(apply_rho(Q))
        Q, _ = orth(apply_rho(Qt))
    Bm = Q.T @ apply_rho(Q)
    lam, V = eigh_desc(Bm)
    return lam, Q @ V


def keep_count(vals, rel, cap):
    """Number of leading entries of the descending ``vals`` above rel * vals[0], at most cap."""
    if vals.size == 0 or vals[0] <= 0.0:
        return 0
    n = int(np.count_nonzero(vals > rel * vals[0]))
    return min(n, int(cap)) if cap is not None else n

"""Initial tensor of the d-dimensional Ising model (Sec. 3, the Z = tTr prod T equation and
the definition of T through the 2x2 matrix W).

Reading of the garbled W (the printed matrix has cosh/sinh where their square roots are
needed): the bond weight is the 2x2 Boltzmann matrix Bm = [[e^b, e^-b], [e^-b, e^b]]
(rows/columns spin +1, -1) and W is its symmetric square root,
W = U diag(sqrt(2 cosh b), sqrt(2 sinh b)) U^T with U = [[1, 1], [1, -1]] / sqrt(2), so
that sum_x W[s, x] W[s', x] = exp(b s s').  ``w_paper`` is the printed matrix with the
square roots restored; it differs from the symmetric one by an orthogonal gauge on each
bond.  A magnetic field h enters as the site factor exp(h s).

T[x_1..x_d ; x'_1..x'_d] = sum_s exp(h s) prod_mu W[s, x_mu] W[s, x'_mu]; forward legs
(x, pointing to +mu) first, backward legs (x') second, both in direction order.
"""
import numpy as np

from . import rla


def w_symmetric(beta):
    if beta <= 0.0:
        raise ValueError("beta must be positive")
    U = np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0)
    lam = np.array([np.sqrt(2.0 * np.cosh(beta)), np.sqrt(2.0 * np.sinh(beta))])
    return U @ np.diag(lam) @ U.T


def w_paper(beta):
    c, s = np.sqrt(np.cosh(beta)), np.sqrt(np.sinh(beta))
    return np.array([[c, s], [c, -s]])


def initial_tensor(beta, h, d, W=None):
    """Dense T with shape (2,)*(2d): forward legs 0..d-1, backward legs d..2d-1."""
    if W is None:
        W = w_symmetric(beta)
    T = np.zeros((2,) * (2 * d))
    for si, spin in enumerate((1.0, -1.0)):
        t = np.exp(h * spin)
        for _ in range(2 * d):
            t = np.multiply.outer(t, W[si])
        T += t
    return T


def initial_state(beta, h, d, chi=None, W=None):
    """Normalised split T / c0 = A diag(s) B (exact SVD of the 2^d x 2^d matrix).

    Returns (A, s, B, c0) with A of shape (2,)*d + (Da,), B of shape (Da,) + (2,)*d.
    Singular values at or below 1e-14 * s_0 are dropped; the columns of A follow the sign
    convention of ``rla.fix_sign`` and the rows of B follow A.
    """
    T = initial_tensor(beta, h, d, W)
    Tm = T.reshape(2 ** d, 2 ** d)
    c0 = float(np.linalg.norm(Tm))
    U, S, V = rla.svd_desc(Tm / c0)
    Da = rla.keep_count(S, 1e-14, chi)
    U, sgn = rla.fix_sign(U[:, :Da])
    V = V[:, :Da] * sgn[None, :]
    A = U.reshape((2,) * d + (Da,))
    B = V.T.reshape((Da,) + (2,) * d)
    return A, S[:Da].copy(), B, c0

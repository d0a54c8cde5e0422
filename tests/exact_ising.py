"""Exact Ising results that pin the oracle from outside it (textbook, not the paper).

* brute-force enumeration of Z on small periodic lattices (any d, field h);
* Onsager's free energy of the infinite 2D square lattice at h = 0;
* the leading terms of the high-temperature expansion on the hypercubic lattice.
None of this code is shared with the oracle or the CUDA library.
"""
import itertools
import math

import numpy as np


def brute_force_lnz(beta, h, shape):
    """ln Z of the Ising model on a periodic lattice of the given shape.

    Every site n has one bond per direction to n + e_mu (mod L), so an L = 2 direction
    carries two bonds between each neighbour pair, exactly as the tensor network does.
    Returns (ln Z, <sum_bonds s s'>, <sum_sites s>).
    """
    d = len(shape)
    V = int(np.prod(shape))
    coords = list(itertools.product(*[range(L) for L in shape]))
    index = {c: i for i, c in enumerate(coords)}
    nbr = []
    for mu in range(d):
        col = []
        for c in coords:
            cc = list(c)
            cc[mu] = (cc[mu] + 1) % shape[mu]
            col.append(index[tuple(cc)])
        nbr.append(np.array(col))
    cfg = np.arange(2 ** V, dtype=np.int64)[:, None]
    spins = 1 - 2 * ((cfg >> np.arange(V)[None, :]) & 1)          # (2^V, V) in {+1,-1}
    bonds = np.zeros(2 ** V)
    for mu in range(d):
        bonds += np.sum(spins * spins[:, nbr[mu]], axis=1)
    mag = spins.sum(axis=1).astype(np.float64)
    expo = beta * bonds + h * mag
    m = expo.max()
    w = np.exp(expo - m)
    Z = w.sum()
    return m + math.log(Z), float((w * bonds).sum() / Z), float((w * mag).sum() / Z)


def onsager_lnz(beta, n=512):
    """ln Z / V of the infinite square lattice at h = 0 (Onsager 1944):
    ln 2 + (1/8 pi^2) int int ln[cosh^2 2b - sinh 2b (cos t1 + cos t2)] dt1 dt2.
    The integrand is smooth and periodic away from the critical point, so the
    trapezoidal rule on an n x n grid converges exponentially."""
    t = 2.0 * np.pi * np.arange(n) / n
    c1, c2 = np.meshgrid(np.cos(t), np.cos(t), indexing="ij")
    val = np.log(np.cosh(2 * beta) ** 2 - np.sinh(2 * beta) * (c1 + c2))
    return math.log(2.0) + 0.5 * val.mean()


def high_t_lnz(beta, d):
    """ln Z / V through order tanh^4 on the d-dimensional hypercubic lattice at h = 0:
    ln 2 + d ln cosh b + C(d, 2) tanh^4 b.  Z = 2^V cosh^(dV) b * (sum over closed bond
    graphs of tanh^|graph|); the smallest closed graphs are the elementary plaquettes, of
    which there are C(d, 2) per site.  The next term is O(tanh^6 b)."""
    t = math.tanh(beta)
    return math.log(2.0) + d * math.log(math.cosh(beta)) + math.comb(d, 2) * t ** 4


def transfer_matrix_lnz(beta, h, L0, L1):
    """ln Z of the 2D Ising model on an L0 x L1 periodic lattice by the row transfer matrix:
    a column of L0 spins along direction 0 (ring bonds sigma_i sigma_{i+1 mod L0}, so L0 = 2
    gives double bonds and L0 = 1 a self-loop, as in brute_force_lnz), Z = Tr T^L1 with
    T[s, s'] = exp(beta sum_i s_i s_{i+1} + h sum_i s_i + beta sum_i s_i s'_i)."""
    n = 2 ** L0
    spins = 1 - 2 * ((np.arange(n)[:, None] >> np.arange(L0)[None, :]) & 1)
    ring = np.sum(spins * np.roll(spins, -1, axis=1), axis=1)
    site = ring * beta + h * spins.sum(axis=1)
    inter = beta * (spins @ spins.T)
    T = np.exp(site[:, None] + inter)
    # Tr T^L1 through the eigenvalues of the symmetric matrix D^1/2 K D^1/2 (same spectrum)
    Ts = np.exp(0.5 * site)[:, None] * np.exp(inter) * np.exp(0.5 * site)[None, :]
    lam = np.linalg.eigvalsh(Ts)
    m = np.max(np.abs(lam))
    return math.log(m) * L1 + math.log(np.sum((lam / m) ** L1))


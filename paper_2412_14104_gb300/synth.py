"""Seeded synthetic inputs shared by the tests and the benchmark.

Random numbers only: no step of the coarse-graining method lives here.  A split site
tensor (A, s, B) of given leg dimensions has orthonormal columns in A, orthonormal rows in
B and a decaying positive spectrum s with unit 2-norm, like the states the RG step sees.
"""
import numpy as np


def orthonormal(rng, rows, cols):
    q, r = np.linalg.qr(rng.standard_normal((rows, cols)))
    return q * np.where(np.diag(r) < 0, -1.0, 1.0)[None, :]


def split_state(seed, legs, Da, decay=0.9):
    """(A, s, B) with A of shape legs + (Da,), B of shape (Da,) + legs."""
    rng = np.random.default_rng(seed)
    F = int(np.prod(legs))
    A = orthonormal(rng, F, Da).reshape(tuple(legs) + (Da,))
    B = orthonormal(rng, F, Da).T.reshape((Da,) + tuple(legs))
    s = decay ** np.arange(Da)
    return A, s / np.linalg.norm(s), B


def gaussian_matrix(seed, rows, cols):
    return np.random.default_rng(seed).standard_normal((rows, cols))


def device_normal(seed, shape, device="cuda"):
    """Seeded N(0, 1) float64 tensor generated on the device (torch's Philox generator):
    full-size contraction operands that would take minutes to draw on the host."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    return torch.randn(shape, dtype=torch.float64, device=device, generator=gen)

"""Plain FP64 CPU oracle of ATRG and Triad-ATRG (Sugimoto & Sasaki, arXiv:2412.14104).

TEST INFRASTRUCTURE ONLY. This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py``. The product path (the CUDA library and its Python binding) never imports,
calls or links anything here, and this package imports nothing from the product.

Layout
------
``philox``  counter-based Gaussian sketch stream (Philox4x32-10 + Box-Muller).
``rla``     orthonormalisation, sign convention, exact and randomized SVD / eig.
``ising``   the 4D (or 2D/3D) Ising initial tensor T of Sec. 3 and its first split.
``trg``     one coarse-graining step (bond swap Eq. 1, triad Eqs. 2-4, squeezers Eq. 5,
            contraction Eqs. 6-7, re-split) and the ln Z accumulation.
``derivatives``  dlnZ/dbeta and dlnZ/dh of the computed ln Z / V (central differences).

Everything is float64 NumPy; contractions are written as ``numpy.einsum`` with the index
names of the paper so that each one can be checked against its equation by eye.
"""

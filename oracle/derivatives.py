"""Derivatives of the oracle's ln Z / V with respect to beta and h.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper computes ln Z / V only (Sec. 2: ln Z / V = sum_k 2^-k ln c_k + 2^-N ln tTr).
Its derivatives are those of that computed function of (beta, h) with every sketch held
fixed (same seed, replica and step stream ids).  The oracle takes them numerically from
its own ln Z / V: the five-point central difference

    f'(x) ~ [8 (f(x + e) - f(x - e)) - (f(x + 2e) - f(x - 2e))] / (12 e),

whose truncation error is e^4 f^(5) / 30.  The computed ln Z / V is only piecewise
smooth in (beta, h): where two kept singular values of different symmetry sectors cross,
or a sign-rule weight passes through zero, the ordered basis that later sketches act on
changes and ln Z / V jumps by an amount of the order of the truncation error.  The
derivatives are those of the smooth piece, so the default step (1e-5) keeps the stencil
inside one piece; a caller checks that by comparing two steps.
"""
from . import trg


def _five_point(f, x, e):
    return (8.0 * (f(x + e) - f(x - e)) - (f(x + 2 * e) - f(x - 2 * e))) / (12.0 * e)


def dlnz_dbeta(beta, h, d, p, nsteps, e=1e-5, W=None):
    return _five_point(lambda b: trg.lnz_per_site(b, h, d, p, nsteps, W), beta, e)


def dlnz_dh(beta, h, d, p, nsteps, e=1e-5, W=None):
    return _five_point(lambda x: trg.lnz_per_site(beta, x, d, p, nsteps, W), h, e)


def d2lnz_dbeta2(beta, h, d, p, nsteps, e=1e-5, W=None):
    """Five-point second difference [-f(x+2e) + 16 f(x+e) - 30 f(x) + 16 f(x-e) - f(x-2e)] / (12 e^2)."""
    f = lambda b: trg.lnz_per_site(b, h, d, p, nsteps, W)
    return (-f(beta + 2 * e) + 16 * f(beta + e) - 30 * f(beta) + 16 * f(beta - e) - f(beta - 2 * e)) / (12 * e * e)

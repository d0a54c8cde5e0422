"""Reference values of single RG steps from seeded synthetic states (calls only oracle/ and
the seeded input module), for the GPU teacher-forced step tests.

The oracle's own states along a run cannot be carried in the repository (64 MB per tensor
at chi = 24, 2 GB at chi = 48), so each case draws its input from
``paper_2412_14104_gb300.synth.split_state`` (random orthonormal A and B) with the spectrum
s of the stored oracle run at that step (chi = 24) or a geometric spectrum (chi = 48), and
runs one oracle step with the sketch stream of step k.  The GPU test regenerates the same
input and runs the same step.  Stored: ln c_k, the spectra s', sigma and the squeezer
singular values, the gaps at every cut, and A', B' at seeded sample positions.

    python tests/golden/make_golden_steps.py [name ...]
"""
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import trg  # noqa: E402
from paper_2412_14104_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
NSAMPLE = 512


def _c2_spectrum(k):
    with open(os.path.join(HERE, "oracle_c2_chi24.json")) as f:
        g = json.load(f)
    return g["dims"][k], np.array(g["s"][k])


# name: (chi, r, q, sketch seed, step k, state seed, spectrum source)
CASES = {
    "step_chi24_k20": (24, 2, 2, 1, 20, 120, ("c2", 19)),
    "step_chi24_k30": (24, 2, 2, 1, 30, 130, ("c2", 29)),
    "step_chi24_k39": (24, 2, 2, 1, 39, 139, ("c2", 38)),
    "step_chi48_k10": (48, 3, 2, 2, 10, 210, ("geometric", 0.95)),
}


def case_input(name):
    """(A, s, B, params, step) of a case; the GPU test calls this too (no method arithmetic)."""
    chi, r, q, seed, k, state_seed, spec = CASES[name]
    if spec[0] == "c2":
        dims, s = _c2_spectrum(spec[1])
        legs, Da = tuple(dims[:-1]), dims[-1]
    else:
        legs, Da = (chi,) * 4, chi
        s = spec[1] ** np.arange(Da)
        s = s / np.linalg.norm(s)
    A, _, B = synth.split_state(state_seed, legs, Da)
    return A, s, B, trg.Params(chi, r, q=q, seed=seed), k


def sample_positions(name, size):
    rng = np.random.default_rng(sum(map(ord, name)))
    return np.sort(rng.choice(size, size=min(NSAMPLE, size), replace=False))


def run(name):
    A, s, B, p, k = case_input(name)
    t0 = time.time()
    info = {}
    An, sn, Bn, c = trg.rg_step(A, s, B, p, k, trg.Counter(), info)
    secs = time.time() - t0
    ia = sample_positions(name + "A", An.size)
    ib = sample_positions(name + "B", Bn.size)
    d = A.ndim - 1

    def fin(x):
        return x if math.isfinite(x) else None

    out = {
        "case": name, "chi": p.chi, "r": p.r, "q": p.q, "seed": p.seed, "step": k,
        "lnc": math.log(c), "s": sn.tolist(), "sigma": info["swap_sigma"].tolist(),
        "swap_gap": fin(info["swap_gap"]),
        "sq": [info["sq_S_%d" % nu].tolist() for nu in range(1, d)],
        "sq_gap": [fin(info["sq_gap_%d" % nu]) for nu in range(1, d)],
        "shape_A": list(An.shape), "shape_B": list(Bn.shape),
        "idx_A": ia.tolist(), "val_A": An.ravel()[ia].tolist(),
        "idx_B": ib.tolist(), "val_B": Bn.ravel()[ib].tolist(),
        "seconds": secs,
    }
    with open(os.path.join(HERE, "oracle_%s.json" % name), "w") as f:
        json.dump(out, f)
    print(name, "ln c = %.16f" % out["lnc"], "%.1fs" % secs, flush=True)


if __name__ == "__main__":
    for n in (sys.argv[1:] or CASES):
        run(n)

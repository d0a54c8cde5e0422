"""Write the oracle's reference values for the GPU parity tests (calls only oracle/).

Each file holds, for one configuration, ln c_k per step, the normalised re-split spectrum
s' and the swap spectrum sigma of every step, the squeezer spectra, the relative gaps at
every cut and ln Z / V.  Run from the repository root:

    python tests/golden/make_golden.py [name ...]
"""
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import trg  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

# name: (beta, h, d, chi, r, q, seed, steps); the first three mirror the 4D configurations
# chi=6 (8 steps), chi=24 (40 steps); the small ones cover d = 2, 3 and a field.
CONFIGS = {
    "c1_chi6": (0.1497, 0.0, 4, 6, 2, 2, 0, 8),
    "c2_chi24": (0.1497, 0.0, 4, 24, 2, 2, 1, 40),
    "d4_chi10_h": (0.1497, 1e-4, 4, 10, 2, 2, 2, 10),
    "d2_chi16": (0.4, 0.0, 2, 16, 2, 2, 5, 24),
    "d3_chi8": (0.22, 0.01, 3, 8, 2, 2, 6, 12),
    # chi = 24 with the multiplet gap of the library's split-precision steps (1e-6) from
    # step 1: separates the rounding of the split forms from their cut rule
    "c2_chi24_tau6": (0.1497, 0.0, 4, 24, 2, 2, 1, 40),
    # plain ATRG (identity isometries, the chi^9 contraction) in 4D and 3D
    "atrg_d4_chi8": (0.1497, 1e-4, 4, 8, 2, 2, 7, 12),
    "atrg_d3_chi8": (0.22, 0.01, 3, 8, 2, 2, 6, 12),
}
EXTRA = {"c2_chi24_tau6": {"split_tau": 1e-6, "split_from_step": 1}}
METHOD = {"atrg_d4_chi8": "atrg", "atrg_d3_chi8": "atrg"}


def run(name):
    beta, h, d, chi, r, q, seed, steps = CONFIGS[name]
    t0 = time.time()
    method = METHOD.get(name, "triad")
    p = trg.Params(chi, r, q=q, seed=seed, method=method, **EXTRA.get(name, {}))
    R = trg.Run(beta, h, d, p)
    out = {"config": {"beta": beta, "h": h, "d": d, "chi": chi, "r": r, "q": q, "seed": seed,
                      "steps": steps, "method": method, **EXTRA.get(name, {})},
           "lnc": [R.lnc[0]], "s": [R.s.tolist()], "sigma": [], "sq": [], "swap_gap": [],
           "sq_gap": [], "dims": [list(R.A.shape)], "lnz_after": []}
    for k in range(steps):
        R.step()
        inf = R.infos[-1]
        out["lnc"].append(R.lnc[-1])
        out["s"].append(R.s.tolist())
        out["sigma"].append(inf["swap_sigma"].tolist())
        out["sq"].append([inf["sq_S_%d" % nu].tolist() for nu in range(1, d)])
        out["swap_gap"].append(inf["swap_gap"])
        out["sq_gap"].append([inf["sq_gap_%d" % nu] for nu in range(1, d)])
        out["dims"].append(list(R.A.shape))
        out["lnz_after"].append(R.lnz())
    out["lnz"] = R.lnz()
    out["flops"] = R.cnt.flops
    out["seconds"] = time.time() - t0
    for key in ("swap_gap",):
        out[key] = [g if math.isfinite(g) else None for g in out[key]]
    out["sq_gap"] = [[g if math.isfinite(g) else None for g in row] for row in out["sq_gap"]]
    with open(os.path.join(HERE, "oracle_%s.json" % name), "w") as f:
        json.dump(out, f)
    print(name, "lnZ/V = %.16f" % out["lnz"], "%.1fs" % out["seconds"], flush=True)


if __name__ == "__main__":
    for n in (sys.argv[1:] or [c for c in CONFIGS if c not in EXTRA]):
        run(n)

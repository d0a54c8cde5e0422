"""Rounding envelope of the oracle's runs (calls only oracle/): how far each step's ln c_k
and re-split spectrum s' move when the initial split is perturbed at the rounding level
(relative 2^-50 noise on A, two seeds).  A float64 implementation that rounds differently
from the oracle cannot be expected to agree with it more closely than this, times a
safety factor, because the RG map amplifies differences along the run.  Writes
oracle_<name>_envelope.json next to oracle_<name>.json.  Run from the repository root:

    python tests/golden/make_envelope.py [name ...]
"""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import trg  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def run(name, seeds=(1, 2), rel=2.0 ** -50):
    with open(os.path.join(HERE, "oracle_%s.json" % name)) as f:
        gold = json.load(f)
    c = gold["config"]
    steps = c["steps"]
    env_lnc = [0.0] * (steps + 1)
    env_s = [0.0] * (steps + 1)
    for sd in seeds:
        p = trg.Params(c["chi"], c["r"], q=c["q"], seed=c["seed"])
        R = trg.Run(c["beta"], c["h"], c["d"], p)
        rng = np.random.default_rng(sd)
        R.A = R.A * (1.0 + rel * rng.standard_normal(R.A.shape))
        for k in range(steps):
            R.step()
            env_lnc[k + 1] = max(env_lnc[k + 1], abs(R.lnc[-1] - gold["lnc"][k + 1]))
            s_gold = np.array(gold["s"][k + 1])
            if R.s.size == s_gold.size:
                env_s[k + 1] = max(env_s[k + 1], float(np.max(np.abs(R.s - s_gold))))
            else:
                env_s[k + 1] = math.inf
    out = {"config": c, "perturbation": {"relative": rel, "seeds": list(seeds), "where": "A"},
           "env_lnc": env_lnc, "env_s": [x if math.isfinite(x) else None for x in env_s]}
    with open(os.path.join(HERE, "oracle_%s_envelope.json" % name), "w") as f:
        json.dump(out, f)
    print(name, "max env_lnc %.3g" % max(env_lnc), flush=True)


if __name__ == "__main__":
    for n in (sys.argv[1:] or ["c2_chi24"]):
        run(n)

"""Write tests/golden/c5_row1.json: singular values and log(sigma_1) of every
einsumsvd step of the first zip-up row (Algorithm 3 applied to rows one and
two) of the 16 x 16, D = 8, m = 256 norm workload, computed by the FP64
oracle only.  Run from the repository root:

    python tests/golden/make_c5_row1.py

(about 40 minutes on 8 cores).  The GPU sees exactly these inputs in its
first row, so the values are a full-size parity reference.
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import bmps  # noqa: E402


def main():
    cfg = synth.config("c5")
    ket = synth.peps_for(cfg)
    rec = []
    t0 = time.time()
    bmps.sweep(ket, ket, cfg.m, cfg.p, cfg.q, cfg.omega_seed, 0, 1, record=rec)
    out = {
        "workload": cfg.name, "m": cfg.m, "p": cfg.p, "q": cfg.q, "seed": cfg.omega_seed,
        "generator": "tests/golden/make_c5_row1.py (oracle.bmps.sweep, rows 0-1)",
        "seconds": time.time() - t0,
        "steps": [{"row": r["row"], "col": r["col"], "logs1": r["logs1"],
                   "sigma": [float(x) for x in r["sigma"]]} for r in rec],
    }
    with open(os.path.join(ROOT, "tests", "golden", "c5_row1.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()

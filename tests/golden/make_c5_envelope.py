"""Write tests/golden/c5_envelope.json: how far single-precision arithmetic
alone moves the singular values of the einsumsvd steps of the first rows of
the 16 x 16, D = 8, m = 256 norm sweep away from the FP64 oracle's
(tests/golden/c5_sweep.json).  Run from the repository root:

    python tests/golden/make_c5_envelope.py --rows 2 --cache DIR

One realization (seed 1) of the single-precision emulation of
make_c2_envelope.py (complex64 implicit products, FP32-rounded sketch,
complex64 QR and small SVD, outputs rounded and perturbed by one FP32 unit)
replays the zip-up rows 1..rows; the file is rewritten after every row, and
with --cache the emulated boundary is kept so a later run continues.  The
envelope of a step is max_i |sigma_i - sigma_i^ref| / sigma_1^ref.  Only the
oracle's functions compute; the wrappers only round and perturb.
"""
import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import synth  # noqa: E402
from make_c2_envelope import single_precision  # noqa: E402
from oracle import bmps  # noqa: E402

SEED = 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rows", type=int, default=2)
    ap.add_argument("--cache", default=None)
    args = ap.parse_args()
    cfg = synth.config("c5")
    ket = synth.peps_for(cfg)
    gold = json.load(open(os.path.join(HERE, "c5_sweep.json")))
    out_path = os.path.join(HERE, "c5_envelope.json")
    ck = os.path.join(args.cache, "c5_env_boundary.npz") if args.cache else None
    steps, start = [], 1
    with single_precision(SEED):
        S = bmps.first_row_boundary(ket[0], ket[0])
    if ck and os.path.exists(ck) and os.path.exists(out_path):
        z = np.load(ck)
        prev = json.load(open(out_path))
        if prev["rows_done"] == int(z["row"]):
            start = int(z["row"]) + 1
            S = [z["s%d" % i] for i in range(cfg.ncol)]
            steps = prev["steps"]
    ref = {(g["row"], g["col"]): np.asarray(g["sigma"]) for g in gold["steps"]}
    for r in range(start, min(args.rows, gold["rows_done"]) + 1):
        rec = []
        with single_precision(SEED * 1000 + r):
            S, _ = bmps.zipup(S, ket[r], ket[r], cfg.m, cfg.p, cfg.q, cfg.omega_seed, 0, r, record=rec)
        for x in rec:
            g = ref[(x["row"], x["col"])]
            steps.append({"row": x["row"], "col": x["col"],
                          "envelope": float(np.max(np.abs(np.asarray(x["sigma"]) - g)) / g[0])})
        if ck:
            os.makedirs(args.cache, exist_ok=True)
            np.savez(ck + ".tmp.npz", row=r, **{"s%d" % i: s for i, s in enumerate(S)})
            os.replace(ck + ".tmp.npz", ck)
        with open(out_path, "w") as f:
            json.dump({"workload": cfg.name, "seed": SEED, "rows_done": r,
                       "generator": "tests/golden/make_c5_envelope.py (oracle.bmps.zipup with the single-precision "
                                    "emulation wrappers of make_c2_envelope.py)",
                       "steps": steps}, f, indent=0)
        print("row %d done" % r, flush=True)


if __name__ == "__main__":
    main()

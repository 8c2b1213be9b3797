"""Write tests/golden/<config>_sweep.json: the singular values and
log(sigma_1) of every einsumsvd step of a whole boundary sweep (Algorithm 2
over all rows, Algorithm 3 per row, Algorithm 4 per step) of a norm
workload, and the contracted log-norm, computed by the FP64 oracle only.
Run from the repository root:

    python tests/golden/make_sweep.py --config c5 --cache DIR   # 16 x 16, D = 8, m = 256
    python tests/golden/make_sweep.py --config c2               # 8 x 8, D = 4, m = 32

The 16 x 16 run takes hours on a few cores.  After every finished row the JSON is
rewritten with the rows done so far, and (with --cache) the boundary left by
that row is saved, so an interrupted run resumes at the next row.  The
log-norm is written once the last row is contracted.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import bmps  # noqa: E402

GOLDEN = os.path.join(ROOT, "tests", "golden")


def _write(path, cfg, steps, rows_done, seconds, result=None):
    out = {
        "workload": cfg.name, "m": cfg.m, "p": cfg.p, "q": cfg.q, "seed": cfg.omega_seed,
        "generator": "tests/golden/make_sweep.py (oracle.bmps: first_row_boundary, "
                     "zipup per row, boundary_scalar)",
        "rows_done": rows_done, "nrow": cfg.nrow, "seconds": seconds,
        "steps": steps,
    }
    if result is not None:
        out["log_norm"], out["arg"] = result
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(out, f)
    os.replace(tmp, path)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cache", default=None, help="directory for the per-row boundary checkpoint")
    ap.add_argument("--config", default="c5", help="workload key of synth.CONFIGS")
    ap.add_argument("--out", default=None, help="default: tests/golden/<config>_sweep.json")
    args = ap.parse_args()
    if args.out is None:
        args.out = os.path.join(GOLDEN, "%s_sweep.json" % args.config)
    cfg = synth.config(args.config)
    ket = synth.peps_for(cfg)
    steps, total, start, spent = [], 0.0, 1, 0.0
    S = bmps.first_row_boundary(ket[0], ket[0])
    ck = os.path.join(args.cache, "%s_boundary.npz" % args.config) if args.cache else None
    if ck and os.path.exists(ck) and os.path.exists(args.out):
        z = np.load(ck)
        prev = json.load(open(args.out))
        start = int(z["row"]) + 1
        if prev["rows_done"] == start - 1:
            S = [z["s%d" % i] for i in range(cfg.ncol)]
            total = float(z["total"])
            steps = prev["steps"]
            spent = prev["seconds"]
        else:
            start = 1
    t0 = time.time()
    for r in range(start, cfg.nrow):
        rec = []
        S, lg = bmps.zipup(S, ket[r], ket[r], cfg.m, cfg.p, cfg.q, cfg.omega_seed, 0, r,
                           record=rec)
        total += lg
        steps += [{"row": x["row"], "col": x["col"], "logs1": x["logs1"],
                   "sigma": [float("%.15e" % v) for v in x["sigma"]]} for x in rec]
        if ck:
            os.makedirs(args.cache, exist_ok=True)
            np.savez(ck + ".tmp.npz", row=r, total=total, **{"s%d" % i: s for i, s in enumerate(S)})
            os.replace(ck + ".tmp.npz", ck)
        result = None
        if r == cfg.nrow - 1:
            v = bmps.boundary_scalar(S)
            result = (float(np.log(abs(v)) + total), float(np.angle(v)))
        _write(args.out, cfg, steps, r, spent + time.time() - t0, result)
        print("row %d done, %.0f s" % (r, spent + time.time() - t0), flush=True)


if __name__ == "__main__":
    main()

"""Write tests/golden/c2_envelope.json: how far single-precision arithmetic
alone moves the singular values of every einsumsvd step of the 8 x 8,
D = 4, m = 32 norm sweep away from the FP64 oracle's (tests/golden/
c2_sweep.json).  Run from the repository root:

    python tests/golden/make_c2_envelope.py
    python tests/golden/make_c2_envelope.py --alternate   # c2_envelope_alternate.json

(--alternate: the same for the sweep with alternating canonicalisation,
against the FP64 oracle's alternating sweep, which is computed here.)

Each realization replays the oracle's sweep (Algorithms 2-4) with the
arithmetic of a single-precision implementation emulated around the oracle's
own functions: the implicit products A X and A^H Y evaluated in complex64,
the sketch drawn from FP32-rounded uniforms (the single-precision reading of
Algorithm 4's first line) and rounded to complex64, the orthogonalisations
(Householder QR) and the small SVD in complex64, and each step's outputs U
and W rounded to complex64, then perturbed by independent relative noise of
one FP32 unit (2^-24) with the realization's seed.  The stored envelope of a
step is the largest normwise deviation max_i |sigma_i - sigma_i^ref| /
sigma_1^ref over the realizations; the log-norm deviations are stored too.
Only the oracle's functions compute; the wrappers only round and perturb.
"""
import contextlib
import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import bmps, implicit, philox, rsvd  # noqa: E402

SEEDS = (1, 2, 3, 4)


def _c64(a):
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


@contextlib.contextmanager
def single_precision(seed):
    """The oracle's functions with the arithmetic of a single-precision
    implementation emulated around them (see the module docstring)."""
    rng = np.random.default_rng(seed)
    Op = implicit.ImplicitOp
    mv, rmv, common = Op.matvec, Op.rmatvec, implicit._common
    sketch, es = philox.sketch, rsvd.einsumsvd
    qr, svd = torch.linalg.qr, torch.linalg.svd

    def qr32(A, *a, **k):
        return tuple(x.to(A.dtype) for x in qr(A.to(torch.complex64), *a, **k))

    def svd32(A, *a, **k):
        U, S, V = svd(A.to(torch.complex64), *a, **k)
        return U.to(A.dtype), S.to(torch.float64), V.to(A.dtype)

    def common32(*arrays):
        return [torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)) for a in arrays]

    def in32(f):
        def g(self, X):
            implicit._common = common32
            try:
                return f(self, X).astype(np.complex128)
            finally:
                implicit._common = common
        return g

    def sketch32(N, ell, sd, inst, is_c, kind="gauss"):
        flat = philox.draw_elements(N * ell, sd, inst, philox.TAG_SKETCH, is_c, kind, single=True)
        return _c64(flat.reshape(ell, N).T)

    def noisy(x):
        e = 2.0 ** -24 * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)) / np.sqrt(2.0)
        return _c64(x * (1.0 + e))

    def es32(*a, **k):
        U, W, s, l = es(*a, **k)
        return noisy(U), noisy(W), s, l

    Op.matvec, Op.rmatvec = in32(mv), in32(rmv)
    philox.sketch, bmps.einsumsvd = sketch32, es32
    torch.linalg.qr, torch.linalg.svd = qr32, svd32
    try:
        yield
    finally:
        Op.matvec, Op.rmatvec = mv, rmv
        philox.sketch, bmps.einsumsvd = sketch, es
        torch.linalg.qr, torch.linalg.svd = qr, svd


def replay(cfg, ket, seed, alternate=False):
    with single_precision(seed):
        rec = []
        la, _ = bmps.contract(ket, ket, cfg.m, cfg.p, cfg.q, cfg.omega_seed, record=rec, alternate=alternate)
    return la, rec


def main():
    alternate = "--alternate" in sys.argv[1:]
    cfg = synth.config("c2")
    ket = synth.peps_for(cfg)
    if alternate:
        rec = []
        la, _ = bmps.contract(ket, ket, cfg.m, cfg.p, cfg.q, cfg.omega_seed, record=rec, alternate=True)
        gold = {"log_norm": la, "steps": [{"row": r["row"], "col": r["col"], "sigma": r["sigma"]} for r in rec]}
    else:
        gold = json.load(open(os.path.join(ROOT, "tests", "golden", "c2_sweep.json")))
    env = np.zeros(len(gold["steps"]))
    dlog = []
    for seed in SEEDS:
        la, rec = replay(cfg, ket, seed, alternate)
        dlog.append(la - gold["log_norm"])
        for i, (r, g) in enumerate(zip(rec, gold["steps"])):
            ref = np.asarray(g["sigma"])
            env[i] = max(env[i], float(np.max(np.abs(np.asarray(r["sigma"]) - ref)) / ref[0]))
    out = {"workload": cfg.name, "seeds": list(SEEDS), "alternate": alternate,
           "generator": "tests/golden/make_c2_envelope.py (oracle.bmps.contract with single-precision "
                        "emulation wrappers)",
           "steps": [{"row": g["row"], "col": g["col"], "envelope": float(e)} for g, e in zip(gold["steps"], env)],
           "dlog": dlog}
    name = "c2_envelope_alternate.json" if alternate else "c2_envelope.json"
    with open(os.path.join(ROOT, "tests", "golden", name), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()

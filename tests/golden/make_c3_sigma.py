"""Write tests/golden/c3_sigma.json: the singular values and log(sigma_1) of
every instance of the 512-instance batched einsumsvd workload (one zip-up
step per instance, Algorithm 3's einsumsvd line with Algorithm 4 inside;
m ~ U{16..128}, D ~ U{2..6}, rank k = m, real FP32-rounded N(0,1) operands),
computed by the FP64 oracle only.  Instance i draws its sketch from Philox
stream i.  Run from the repository root:

    python tests/golden/make_c3_sigma.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import rsvd  # noqa: E402


def main():
    cfg = synth.config("c3")
    out = []
    t0 = time.time()
    for i, (m, D) in enumerate(synth.batched_dims(cfg)):
        inst = synth.batched_instance(cfg, i, m, D)
        _, _, s, logs1 = rsvd.einsumsvd(inst["V"], inst["S"], inst["ket"], inst["bra"], m, cfg.p, cfg.q,
                                        cfg.omega_seed, i)
        out.append({"i": i, "m": m, "D": D, "logs1": logs1, "sigma": [float("%.13e" % v) for v in s]})
    doc = {"workload": cfg.name, "p": cfg.p, "q": cfg.q, "seed": cfg.omega_seed,
           "generator": "tests/golden/make_c3_sigma.py (oracle.rsvd.einsumsvd per instance)",
           "seconds": time.time() - t0, "instances": out}
    with open(os.path.join(ROOT, "tests", "golden", "c3_sigma.json"), "w") as f:
        json.dump(doc, f)


if __name__ == "__main__":
    main()

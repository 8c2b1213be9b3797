"""Full-size parity of the 16 x 16, D = 8, m = 256 norm contraction (complex64,
mixed precision: tcgen05 3xTF32 products): the singular values of every
einsumsvd step of the first zip-up row (Algorithm 3 on rows one and two,
identical network inputs on both sides) against the FP64 oracle's values
stored in tests/golden/c5_row1.json (written by tests/golden/make_c5_row1.py,
which calls only the oracle).  Error per step: max_i |sigma_i - sigma_i^ref| /
sigma_1^ref.

The first step of the row sees exactly the oracle's inputs: bound 1e-5, the
single-precision tolerance of the workload (measured 2.4e-6 mixed, 4.3e-6
plain FP32).  Every later step takes the previous step's carry W, which the
GPU holds in single precision and the oracle in FP64; that rounding alone
moves the next singular values by up to ~1.2e-5 relative to sigma_1 on this
workload (the plain FP32 path measures the same 1.2e-5), so those steps are
held to 2e-5."""
import json
import os

import numpy as np
import pytest

import synth
from paper_2006_15234_gb300 import libpeps
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c5_row1.json")


@pytest.mark.parametrize("prec", [libpeps.PREC_MIXED])
def test_c5_first_row_sigma_matches_oracle(prec):
    gold = json.load(open(GOLDEN))
    cfg = synth.config("c5")
    assert (gold["m"], gold["p"], gold["q"], gold["seed"]) == (cfg.m, cfg.p, cfg.q, cfg.omega_seed)
    k = to_dev(synth.peps_for(cfg), "c64")
    plan = libpeps.ContractPlan(k, k, libpeps.make_opts(cfg.m, cfg.p, cfg.q, cfg.omega_seed, prec=prec))
    plan.execute()
    la, ph, sig = plan.result(with_sigma=True)
    assert np.isfinite(la)
    pos, errs = 0, []
    for st in gold["steps"]:
        ref = np.asarray(st["sigma"])
        got = sig[pos:pos + len(ref)]
        pos += len(ref)
        errs.append(np.max(np.abs(got - ref)) / ref[0])
    msg = ["%.2e" % e for e in errs]
    assert errs[0] <= 1e-5, msg
    assert max(errs) <= 2e-5, msg

"""The whole 512-instance batched einsumsvd workload (m ~ U{16..128},
D ~ U{2..6}, rank k = m, real FP32 operands) in ONE plan, replayed as one
CUDA graph, against the FP64 oracle's stored singular values
(tests/golden/c3_sigma.json, written by tests/golden/make_c3_sigma.py from
the oracle alone): every singular value of every instance within 1e-5 of
its sigma_1, and log(sigma_1) within 1e-5, on both the plain path and the
mixed path (where every instance runs on the tensor cores, 437 of them
through a zero-padded copy)."""
import json
import os

import numpy as np
import pytest
import torch

import synth
from paper_2006_15234_gb300 import libpeps

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c3_sigma.json")


@pytest.mark.parametrize("prec", [libpeps.PREC_PLAIN, libpeps.PREC_MIXED])
def test_c3_all_instances_match_oracle(prec):
    gold = json.load(open(GOLDEN))
    cfg = synth.config("c3")
    dims = synth.batched_dims(cfg)
    assert (gold["p"], gold["q"], gold["seed"]) == (cfg.p, cfg.q, cfg.omega_seed)
    assert len(gold["instances"]) == len(dims) == 512
    shapes, ios, outs = [], [], []
    for m, D in dims:
        R = D * D
        shapes.append((m, R, m, m, cfg.d, D, D, D, D, D, D, D, D, m))
    plan = libpeps.EinsumsvdPlan(torch.float32, shapes, libpeps.make_opts(128, cfg.p, cfg.q, cfg.omega_seed, prec=prec),
                                 instance_ids=list(range(len(dims))))
    for i, (m, D) in enumerate(dims):
        inst = synth.batched_instance(cfg, i, m, D)
        ops = [torch.tensor(np.asarray(inst[k]), dtype=torch.float32, device="cuda") for k in ("V", "S", "ket", "bra")]
        k = plan.ranks[i]
        R = D * D
        U = torch.empty((m * R, k), dtype=torch.float32, device="cuda")
        W = torch.empty((k, R * m * R), dtype=torch.float32, device="cuda")
        sg = torch.empty(k, dtype=torch.float64, device="cuda")
        lg = torch.empty(1, dtype=torch.float64, device="cuda")
        ios.append(tuple(ops) + (U, W, sg, lg))
        outs.append((sg, lg))
    plan.execute(ios)
    torch.cuda.synchronize()
    errs, lerr = [], []
    for (sg, lg), ref in zip(outs, gold["instances"]):
        r = np.asarray(ref["sigma"])
        g = sg.cpu().numpy()
        errs.append(np.max(np.abs(g[: len(r)] - r)) / r[0])
        lerr.append(abs(float(lg.cpu()[0]) - ref["logs1"]))
    errs, lerr = np.array(errs), np.array(lerr)
    print(f"prec {prec}: max sigma error {errs.max():.2e} (instance {errs.argmax()}), "
          f"max log sigma_1 error {lerr.max():.2e}")
    assert errs.max() <= 1e-5, np.argsort(errs)[-5:]
    assert lerr.max() <= 1e-5

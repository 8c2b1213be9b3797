"""The tensor-core tile autotuner: every candidate MMA width of every GEMM
shape timed on the device, the fastest kept.  Tiling changes neither which
products are summed nor their order along K, so the tuned contraction must
reproduce the untuned one bit for bit; the table round-trips through its
text form into a fresh plan."""
import numpy as np
import pytest

import synth
from paper_2006_15234_gb300 import libpeps
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def test_autotuned_plan_reproduces_results_and_table_round_trips():
    cfg = synth.config("c2")
    k = to_dev(synth.peps_for(cfg), "c64")
    opts = libpeps.make_opts(cfg.m, cfg.p, cfg.q, cfg.omega_seed, prec=libpeps.PREC_MIXED)
    plan = libpeps.ContractPlan(k, k, opts)
    plan.execute()
    ref = plan.result(with_sigma=True)
    plan.autotune(reps=2)
    table = plan.tune_table()
    lines = [x for x in table.splitlines() if x]
    assert lines and all(x.rsplit(" = ", 1)[1] in ("64", "128", "192", "256") for x in lines)
    plan.execute()
    tuned = plan.result(with_sigma=True)
    assert tuned[0] == ref[0] and tuned[1] == ref[1] and np.array_equal(tuned[2], ref[2])
    fresh = libpeps.ContractPlan(k, k, opts)
    fresh.set_tune_table(table)
    fresh.execute()
    again = fresh.result(with_sigma=True)
    assert again[0] == ref[0] and np.array_equal(again[2], ref[2])
    assert fresh.tune_table() == table
    with pytest.raises(libpeps.PepsError):
        fresh.set_tune_table("c1 s1 = 100\n")

"""The plan's device status word (failure detection without a GPU fault).

* A clean contraction leaves no error bit.
* A tensor-core wait limit of 1 ns makes the GEMM's pipeline waits give up
  (their barriers are not complete that soon): each such kernel raises the
  TIMEOUT bit, drains its own copies and MMAs, frees its tensor memory and
  returns; the result call reports PEPS_ERR_TIMEOUT and peps_poll the bit.
  The same plan with the default limit then reproduces the clean result
  exactly, so the context stayed usable.
* A NaN in one host-side site tensor reaches the small SVD, which raises the
  NONFINITE bit: the result call reports PEPS_ERR_NUMERIC.
"""
import numpy as np
import pytest
import torch

import synth
from paper_2006_15234_gb300 import libpeps
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _c2_plan(prec, sites=None):
    cfg = synth.config("c2")
    ket = synth.peps_for(cfg) if sites is None else sites
    k = to_dev(ket, "c64")
    return libpeps.ContractPlan(k, k, libpeps.make_opts(cfg.m, cfg.p, cfg.q, cfg.omega_seed, prec=prec))


@pytest.mark.parametrize("prec", [libpeps.PREC_PLAIN, libpeps.PREC_MIXED])
def test_clean_run_leaves_no_error_bit(prec):
    plan = _c2_plan(prec)
    plan.execute()
    la, ph = plan.result()
    code, word = plan.poll()
    assert code == 0 and word & (libpeps.STATUS_TIMEOUT | libpeps.STATUS_NONFINITE) == 0, word
    assert np.isfinite(la)


def test_wait_limit_expiry_reports_timeout_and_recovers():
    plan = _c2_plan(libpeps.PREC_MIXED)
    plan.execute()
    ref = plan.result(with_sigma=True)
    plan.set_wait_limit(1)
    plan.execute()
    with pytest.raises(libpeps.PepsError) as e:
        plan.result()
    assert e.value.status == libpeps.ERR_TIMEOUT
    code, word = plan.poll()
    assert code == libpeps.ERR_TIMEOUT and word & libpeps.STATUS_TIMEOUT
    plan.set_wait_limit(0)
    plan.execute()
    again = plan.result(with_sigma=True)
    torch.cuda.synchronize()
    assert again[0] == ref[0] and again[1] == ref[1] and np.array_equal(again[2], ref[2])
    code, word = plan.poll()
    assert code == 0 and word & libpeps.STATUS_TIMEOUT == 0


@pytest.mark.parametrize("prec", [libpeps.PREC_PLAIN, libpeps.PREC_MIXED])
def test_nan_input_reports_numeric(prec):
    cfg = synth.config("c2")
    ket = synth.peps_for(cfg)
    bad = [[np.array(T, copy=True) for T in row] for row in ket]
    bad[3][4].reshape(-1)[7] = np.nan
    plan = _c2_plan(prec, bad)
    plan.execute()
    with pytest.raises(libpeps.PepsError) as e:
        plan.result()
    assert e.value.status == libpeps.ERR_NUMERIC
    code, word = plan.poll()
    assert code == libpeps.ERR_NUMERIC and word & libpeps.STATUS_NONFINITE

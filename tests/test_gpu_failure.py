"""The device failure path, exercised without a fault.

paw_set_wait_limit(probe = 1) makes every persistent tensor-core launch first wait on a
device word that nothing writes, before it issues any copy or MMA.  The bounded wait runs
out (1 ms here), the launch gives up and records it; the asynchronous filter call returns
PAW_OK, and the failure is reported by paw_sync_status and by the next synchronising calls
(PAW_ERR_TIMEOUT).  With the probe off the same handle computes correct results again.
"""
import numpy as np
import pytest

import inputs
from oracle import cheb
from tests.gpu_util import gpu_fe, oracle_ops, rel_err, to_dev

pytestmark = pytest.mark.gpu


def _timeout(fn):
    from paper_2604_26037_gb300 import PawError
    with pytest.raises(PawError) as e:
        fn()
    return e.value.status


def test_wait_probe_reports_timeout_then_recovers():
    import torch
    fe = gpu_fe("tiny", block=16)
    op = oracle_ops("tiny")
    X = inputs.start_columns("tiny", range(16))
    Xd = to_dev(X)
    lam = np.linspace(-0.4, 0.3, 16)
    bounds = (-0.6, 0.35, 95.0)
    ref = cheb.rchfsi_filter(op.apply_H, op.apply_S, op.apply_Sinv_approx, X, lam, 4, *bounds)

    fe.set_wait_limit(1e-3, probe=True)
    fe.cheb_filter(Xd, lam, 4, bounds, prec="tf32")         # enqueued; the launches give up
    assert _timeout(fe.sync_status) == "PAW_ERR_TIMEOUT"
    fe.sync_status()                                        # read once, then cleared
    # a synchronising tensor-core call reports its own launch
    assert _timeout(lambda: fe.apply_H(Xd.float(), prec="tf32")) == "PAW_ERR_TIMEOUT"
    # the next synchronising call reports a failure left by an asynchronous one
    fe.cheb_filter(Xd, lam, 4, bounds, prec="tf32")
    assert _timeout(lambda: fe.rayleigh_ritz(Xd.clone())) == "PAW_ERR_TIMEOUT"

    fe.set_wait_limit(2.0, probe=False)
    out = fe.cheb_filter(Xd, lam, 4, bounds, prec="tf32")
    fe.sync_status()
    assert rel_err(out.cpu().numpy(), ref) < 2e-2
    torch.cuda.synchronize()
    fe.close()


def test_wait_limit_arguments():
    from paper_2604_26037_gb300 import PawError
    fe = gpu_fe("tiny", block=16)
    for bad in (0.0, 1e-4, 61.0, float("nan")):
        with pytest.raises(PawError):
            fe.set_wait_limit(bad)
    fe.set_wait_limit(5.0)
    fe.close()

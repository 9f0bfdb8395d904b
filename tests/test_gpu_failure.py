"""Failure handling on the GPU without a fault: every device-side wait is bounded, and a wait
that runs out reaches the host as KAFMM_ERR_TIMEOUT while the device stays usable.

* Report-only threshold (KAFMM_OPT_WAIT_REPORT_US = 0): every wait records a timeout but
  completes normally, so the status reaches the host and the results are unchanged.
* A real expiry (KAFMM_OPT_TEST_STALL): each near-field block first waits on a barrier that
  nothing completes; the wait runs out after a short limit, the block winds down (no copy in
  flight, no output), and the next evaluation without the stall is correct.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from paper_2010_15155_gb300 import kafmm as K  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_15155_gb300 import build
    build.build()


def _problem(n=20000):
    pts, f = W.stokes_uniform(n, seed=31, dtype=np.float32)
    return torch.from_numpy(pts).cuda(), torch.from_numpy(f).cuda()


@pytest.mark.parametrize("sync", [True, False])
def test_report_only_wait_threshold_reaches_the_host(sync):
    y, s = _problem()
    plan = K.Plan(K.STOKESLET, p=8, q=64, precision=K.PREC_MIXED, variant=K.ML_L4, sync=sync)
    plan.set_points(y)
    ref = plan.eval(s)
    torch.cuda.synchronize()
    K.kafmm_status(plan.h)
    K.kafmm_set_option(plan.h, K.OPT_WAIT_REPORT_US, 0)
    g = torch.empty_like(ref)
    if sync:
        with pytest.raises(K.KafmmError) as e:
            K.kafmm_eval(plan.h, s, g, K.F32)
        assert e.value.code == -4
    else:
        K.kafmm_eval(plan.h, s, g, K.F32)   # enqueued only; the status is sticky
        with pytest.raises(K.KafmmError) as e:
            K.kafmm_status(plan.h)
        assert e.value.code == -4
    torch.cuda.synchronize()
    assert torch.equal(g, ref)   # the waits completed normally: same bits
    K.kafmm_set_option(plan.h, K.OPT_WAIT_REPORT_US, -1)
    K.kafmm_eval(plan.h, s, g, K.F32)
    K.kafmm_status(plan.h)   # clean again
    assert torch.equal(g, ref)
    plan.close()


def test_expired_wait_winds_down_and_the_device_stays_usable():
    y, s = _problem()
    plan = K.Plan(K.STOKESLET, p=6, q=64, precision=K.PREC_MIXED, variant=K.ML_L4)
    plan.set_points(y)
    ref = plan.eval(s)
    K.kafmm_set_option(plan.h, K.OPT_WAIT_LIMIT_US, 2000)   # 2 ms per block
    K.kafmm_set_option(plan.h, K.OPT_TEST_STALL, 1)
    with pytest.raises(K.KafmmError) as e:
        plan.eval(s)
    assert e.value.code == -4
    K.kafmm_set_option(plan.h, K.OPT_TEST_STALL, 0)
    K.kafmm_set_option(plan.h, K.OPT_WAIT_LIMIT_US, 2_000_000)
    g = plan.eval(s)   # the context and the plan are intact
    assert torch.equal(g, ref)
    plan.close()
    # and a fresh plan on the same device works too
    p2 = K.Plan(K.STOKESLET, p=6, q=64, precision=K.PREC_MIXED, variant=K.ML_L4)
    p2.set_points(y)
    assert torch.equal(p2.eval(s), ref)
    p2.close()

"""kafmm_rpy_velocity_noalloc: the RPY sphere-velocity pass for callers that cannot allocate
device memory during the call (their own pool owns the memory, or they must not trigger the
device-wide synchronisation of cudaMalloc/cudaFree).  Its work arrays live in a fixed device
array instead of fresh allocations; its output must equal that of kafmm_rpy_velocity, on two
calls in a row (the shared array keeps the last call's contents, so each call must clear what
has to start at zero).  This file sorts last so a stop-at-first-failure run has already run
every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import direct as D  # noqa: E402
from paper_2010_15155_gb300 import kafmm as K  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_15155_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", [K.PREC_FP64, K.PREC_FP32])
def test_noalloc_velocity_equals_allocating_entry_point(prec):
    dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
    code = K.F64 if prec == K.PREC_FP64 else K.F32
    plan = K.Plan(K.RPY, p=6, q=48, precision=prec, variant=K.ML_L4)
    outs = []
    for seed in (6, 7):  # two calls in a row on different inputs
        pts, f, a = W.rpy_clusters(3000, seed=seed, n_clusters=4, sigma=0.05, a_lo=0.004,
                                   a_hi=0.012, dtype=np.float32)
        y = torch.from_numpy(pts).to(dt).cuda()
        s = torch.from_numpy(np.concatenate([f, a[:, None]], axis=1)).to(dt).cuda()
        ac = torch.from_numpy(a).to(dt).cuda()
        plan.set_points(y)
        g = plan.eval(s)
        ref = torch.empty((len(pts), 3), dtype=dt, device="cuda")
        K.kafmm_rpy_velocity(plan.h, s, ac, g, ref, code)
        ua = torch.full((len(pts), 3), float("nan"), dtype=dt, device="cuda")
        allocs = K.kafmm_get_counters(plan.h)["device_allocations"]
        K.kafmm_rpy_velocity_noalloc(plan.h, s, ac, g, ua, code)
        torch.cuda.synchronize()
        # the library made no device allocation during the call
        assert K.kafmm_get_counters(plan.h)["device_allocations"] == allocs
        r, u = ref.double().cpu().numpy(), ua.double().cpu().numpy()
        assert np.all(np.isfinite(u))
        assert D.rel_l2(u, r) < (1e-12 if prec == K.PREC_FP64 else 1e-6)
        outs.append(u)
    assert D.rel_l2(outs[0], outs[1]) > 1e-3  # the second call really computed new values
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    plan = K.Plan(K.RPY, p=4, q=64, precision=K.PREC_FP64, variant=K.ML_L4, near_only=True)
    n = 900_000
    pts, f, a = W.rpy_clusters(n, seed=3, n_clusters=8, sigma=0.1, dtype=np.float64)
    y = torch.from_numpy(pts).cuda()
    s = torch.from_numpy(np.concatenate([f, a[:, None]], axis=1)).cuda()
    plan.set_points(y)
    g = torch.zeros((n, 6), dtype=torch.float64, device="cuda")
    ua = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(K.KafmmError) as e:
        K.kafmm_rpy_velocity_noalloc(plan.h, s, torch.from_numpy(a).cuda(), g, ua, K.F64)
    assert e.value.code == -1 and "scratch" in str(e.value)
    plan.close()

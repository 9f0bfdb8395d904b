"""Stokeslet above a no-slip wall on the GPU (KAFMM_BC_WALL, Sec. III.C): three KAFMM sums
over the sources and their images assembled at the targets.

* FP64 GPU form against the oracle's plain CPU KAFMM of the same three sums, assembled the same
  way (oracle/wall.py): relative L2 <= 1e-7.
* FP64 and mixed forms against the direct sum of Blake's image system (the plain definition):
  within the FMM error of the order (FP64) and within 1e-5 (mixed).
* No slip: targets on the wall see a velocity at the level of the FMM error.
* Points below the wall are rejected with KAFMM_ERR_DOMAIN.
* RPY above the wall (four sums, Table tab:rpywall): FP64 form against the oracle's CPU KAFMM of
  the four sums (1e-7), FP64 and mixed forms against the direct sums of the table (pinned to the
  definition (1 + b^2/6 lap_y) G_wall f), including lap u; no slip.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import direct as D  # noqa: E402
from oracle import wall as Wl  # noqa: E402
from oracle.kafmm import KAFMM  # noqa: E402
from paper_2010_15155_gb300 import kafmm as K  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_15155_gb300 import build
    build.build()


def _upper(n, seed):
    """Points in the upper half of the unit cube (the wall is the plane z = 1/2)."""
    rng = np.random.default_rng(seed)
    p = rng.random((n, 3))
    p[:, 2] = 0.5 + 0.5 * p[:, 2]
    return np.minimum(p, 1.0 - 2.0 ** -24), rng.standard_normal((n, 3))


def _wall_eval(pts, f, prec, p, q, trg=None):
    dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
    plan = K.Plan(K.STOKESLET, p=p, q=q, bc=K.BC_WALL, precision=prec)
    y = torch.from_numpy(pts).to(dt).cuda()
    x = None if trg is None else torch.from_numpy(trg).to(dt).cuda()
    plan.set_points(y, x)
    g = plan.eval(torch.from_numpy(f).to(dt).cuda()).double().cpu().numpy()
    info = plan.info()
    plan.close()
    return g, info


def test_fp64_wall_matches_cpu_kafmm_of_the_three_sums():
    pts, f = _upper(2000, 1)
    p, q = 6, 40
    yy = np.concatenate([pts, Wl.images(pts, 0.5)])
    fs, sd, sdz = Wl.table_sources(pts, f, 0.5)
    uS = KAFMM("stokeslet_l4", p, q).evaluate(yy, fs, trg=pts)
    lap = KAFMM("laplace_qd", p, q)
    ref = Wl.assemble(pts, uS, lap.evaluate(yy, sd, trg=pts), lap.evaluate(yy, sdz, trg=pts), 0.5)
    g, _ = _wall_eval(pts, f, K.PREC_FP64, p, q)
    assert D.rel_l2(g, ref) < 1e-7


@pytest.mark.parametrize("prec,p,tol", [(K.PREC_FP64, 10, 1e-6), (K.PREC_MIXED, 10, 1e-5)])
def test_wall_forms_against_blake_direct_sum(prec, p, tol):
    """The three sums' FMM errors (about 1e-7 each at p = 10) reach the assembled velocity
    enlarged by the cancellation between its terms: measured 4.6e-7 (FP64) and 9.0e-6
    (mixed) against Blake's direct sum."""
    pts, f = _upper(60000, 2)
    idx = np.arange(0, 60000, 30)
    ref = Wl.blake(pts[idx], pts, f, 0.5)
    g, _ = _wall_eval(pts, f, prec, p, 64)
    err = D.rel_l2(g[idx], ref)
    print("wall vs Blake", prec, p, err)
    assert err < tol


def test_wall_velocity_vanishes_on_the_wall():
    pts, f = _upper(20000, 3)
    rng = np.random.default_rng(4)
    trg = rng.random((500, 3))
    trg[:, 2] = 0.5
    g, _ = _wall_eval(pts, f, K.PREC_FP64, 10, 64, trg=trg)
    above = trg.copy()
    above[:, 2] = 0.6
    ga, _ = _wall_eval(pts, f, K.PREC_FP64, 10, 64, trg=above)
    assert np.linalg.norm(g) < 1e-6 * np.linalg.norm(ga)


def _upper_rpy(n, seed):
    """Spheres of radius U(0.002, 0.006) whose centres lie at least 0.02 above the wall (a
    sphere reaching the wall is outside the image system's use; there the b^2 image terms grow
    like b^2 / h^3 and the sums cancel to FP32 rounding)."""
    pts, f = _upper(n, seed)
    pts[:, 2] = 0.52 + (pts[:, 2] - 0.5) * (0.48 / 0.5)
    b = np.random.default_rng(seed + 100).uniform(0.002, 0.006, (n, 1))
    return np.minimum(pts, 1.0 - 2.0 ** -24), np.concatenate([f, b], axis=1)


def _rpy_wall_eval(pts, fb, prec, p, q, trg=None):
    dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
    plan = K.Plan(K.RPY, p=p, q=q, bc=K.BC_WALL, precision=prec)
    plan.set_points(torch.from_numpy(pts).to(dt).cuda(),
                    None if trg is None else torch.from_numpy(trg).to(dt).cuda())
    g = plan.eval(torch.from_numpy(fb).to(dt).cuda()).double().cpu().numpy()
    plan.close()
    return g


def test_rpy_wall_fp64_matches_cpu_kafmm_of_the_four_sums():
    pts, fb = _upper_rpy(2000, 11)
    p, q = 6, 40
    yy = np.concatenate([pts, Wl.images(pts, 0.5)])
    rpy, sd, sdz, quad = Wl.rpy_table_sources(pts, fb, 0.5)
    lap = KAFMM("laplace_qd", p, q)
    ref = Wl.rpy_assemble(pts, KAFMM("rpy_l4", p, q).evaluate(yy, rpy, trg=pts), lap.evaluate(yy, sd, trg=pts),
                          lap.evaluate(yy, sdz, trg=pts), KAFMM("laplace_quad", p, q).evaluate(yy, quad, trg=pts),
                          0.5)
    g = _rpy_wall_eval(pts, fb, K.PREC_FP64, p, q)
    assert D.rel_l2(g, ref) < 1e-7


@pytest.mark.parametrize("prec,tol_u,tol_lap", [(K.PREC_FP64, 1e-6, 1e-5), (K.PREC_MIXED, 2e-5, 1e-4)])
def test_rpy_wall_against_direct_four_sums(prec, tol_u, tol_lap):
    """[u, lap u] against the table's direct sums on sampled targets, p = 10 (lap u, a second
    derivative field, carries a larger FMM error)."""
    pts, fb = _upper_rpy(40000, 12)
    idx = np.arange(0, 40000, 40)
    ref = Wl.rpy_table(pts[idx], pts, fb, 0.5)
    g = _rpy_wall_eval(pts, fb, prec, 10, 64)[idx]
    eu, el = D.rel_l2(g[:, :3], ref[:, :3]), D.rel_l2(g[:, 3:], ref[:, 3:])
    print("rpy wall", prec, eu, el)
    assert eu < tol_u and el < tol_lap


def test_rpy_wall_velocity_vanishes_on_the_wall():
    pts, fb = _upper_rpy(20000, 13)
    rng = np.random.default_rng(14)
    trg = rng.random((500, 3))
    trg[:, 2] = 0.5
    g = _rpy_wall_eval(pts, fb, K.PREC_FP64, 10, 64, trg=trg)
    above = trg.copy()
    above[:, 2] = 0.6
    ga = _rpy_wall_eval(pts, fb, K.PREC_FP64, 10, 64, trg=above)
    assert np.linalg.norm(g[:, :3]) < 1e-6 * np.linalg.norm(ga[:, :3])


def test_points_below_the_wall_are_rejected():
    plan = K.Plan(K.STOKESLET, p=4, q=32, bc=K.BC_WALL, precision=K.PREC_FP64)
    bad = torch.tensor([[0.5, 0.5, 0.7], [0.2, 0.3, 0.4]], dtype=torch.float64, device="cuda")
    with pytest.raises(K.KafmmError) as e:
        plan.set_points(bad)
    assert e.value.code == -2
    plan.close()
    with pytest.raises(K.KafmmError) as e:
        K.Plan(K.LAPLACE, p=4, q=32, bc=K.BC_WALL)
    assert e.value.code == -1

"""GPU parity of the singly and doubly periodic boundaries (PX, PXY; Sec. III.B), alone and
with the no-slip wall (Sec. III.C), through the C ABI, against the oracle: the tree and its
lists with wrap along the periodic axes (integer-exact), the FP64 KAFMM against the oracle's
plain KAFMM with the same far-image operator definition (rel L2 <= 1e-7), the FP32 and mixed
forms against the extrapolated lattice sum (O1) and under a shift along the periodic axes (the
paper's translation test), the RPY sphere velocities with contacts across the periodic
boundary, and the wall's image system summed over the lattice.  The lattice sums of the
larger cases are stored by tests/golden/lattice_refs.py (oracle only), which also defines
their seeded inputs."""
import functools
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import workloads as W  # noqa: E402
from oracle import direct as D  # noqa: E402
from oracle import lattice as La  # noqa: E402
from oracle.kafmm import KAFMM  # noqa: E402
from oracle.tree import Tree  # noqa: E402
from paper_2010_15155_gb300 import kafmm as K  # noqa: E402
sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import lattice_refs as G  # noqa: E402

pytestmark = pytest.mark.gpu

BC = {"px": K.BC_PX, "pxy": K.BC_PXY}
AXES = {"px": "x", "pxy": "xy"}
KERN = {"laplace": K.LAPLACE, "stokeslet": K.STOKESLET, "rpy": K.RPY, "stokeslet_reg": K.STOKES_REG,
        "laplace_qd": K.LAPLACE_QD, "laplace_quad": K.LAPLACE_QUAD}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_15155_gb300 import build
    build.build()


def _code(sh):
    return (sh[0] + 1) + 3 * (sh[1] + 1) + 9 * (sh[2] + 1)


@pytest.mark.parametrize("bc", ["px", "pxy"])
@pytest.mark.parametrize("case", ["uniform", "clustered"])
def test_tree_and_lists_with_partial_wrap_match_oracle(case, bc):
    if case == "uniform":
        pts, _ = W.laplace_uniform(5000, seed=31)
        q = 40
    else:
        pts, _, _ = W.rpy_clusters(4000, seed=32, n_clusters=5, sigma=0.03, dtype=np.float64)
        q = 24
    T = Tree(pts, q=q, periodic=AXES[bc])
    plan = K.Plan(K.LAPLACE, p=4, q=q, precision=K.PREC_FP64, near_only=True, bc=BC[bc])
    plan.set_points(torch.from_numpy(np.ascontiguousarray(pts)).cuda())
    nb = plan.info()["nbox"]
    level, anchor, parent, leaf = K.kafmm_get_tree(plan.h, nb)
    assert nb == T.nbox
    assert np.array_equal(level, T.level) and np.array_equal(anchor, T.anchor)
    assert np.array_equal(parent, T.parent) and np.array_equal(leaf.astype(bool), T.is_leaf)
    for kind, name in enumerate("UVWX"):
        off, ent, sh = K.kafmm_get_list(plan.h, kind, nb)
        ref = getattr(T, name)
        for b in range(nb):
            got = set(zip(ent[off[b]:off[b + 1]].tolist(), sh[off[b]:off[b + 1]].tolist()))
            assert got == {(a, _code(s)) for (a, s) in ref[b]}, (name, b)
    plan.close()


def _neutral(kernel, n, seed):
    """Sources neutral in the kernel's monopole (charges, forces minus their mean); radii b or
    blob widths eps in the fourth column of RPY and the regularized Stokeslet."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    ks = K.KDIM[KERN[kernel]][0]
    s = rng.standard_normal((n, ks))
    for c in La.MONOPOLE[kernel]:
        s[:, c] -= s[:, c].mean()
    if kernel in ("rpy", "stokeslet_reg"):
        s[:, 3] = rng.uniform(0.0, 2e-3, n)
    return pts, s


@functools.lru_cache(maxsize=None)
def _t_m2l(ml, p, bc):
    return La.t_m2l(ml, p, bc)


@pytest.mark.parametrize("problem,kernel,bc", [
    ("laplace", "laplace", "px"), ("stokeslet_g", "stokeslet", "px"), ("rpy_g", "rpy", "px"),
    ("laplace", "laplace", "pxy"), ("stokeslet_g", "stokeslet", "pxy"), ("rpy_g", "rpy", "pxy"),
    ("stokeslet_reg_g", "stokeslet_reg", "pxy"), ("laplace_qd", "laplace_qd", "pxy"),
    ("laplace_quad", "laplace_quad", "px")])
def test_fp64_gpu_kafmm_matches_cpu_kafmm(problem, kernel, bc):
    """FP64 GPU KAFMM with the far-image operator of the line or plane lattice against the
    oracle's plain KAFMM with its own operator (same definition: the extrapolated image sum
    over max|n| >= 2, projected onto neutral densities): rel L2 <= 1e-7."""
    pts, s = _neutral(kernel, 1500, seed=33)
    p, q = 6, 32
    ml = "laplace" if kernel.startswith("laplace") else "stokeslet"
    ref = KAFMM(problem, p, q, bc=bc, t_m2l=_t_m2l(ml, p, bc)).evaluate(pts, s)
    plan = K.Plan(KERN[kernel], p=p, q=q, bc=BC[bc], precision=K.PREC_FP64, variant=K.ML_G)
    plan.set_points(torch.from_numpy(pts).cuda())
    g = plan.eval(torch.from_numpy(s).cuda()).cpu().numpy()
    plan.close()
    err = D.rel_l2(g, ref)
    print(problem, bc, err)
    assert err < 1e-7


@pytest.mark.parametrize("bc", ["px", "pxy"])
@pytest.mark.parametrize("prec,p,tol", [(K.PREC_FP32, 8, 5e-5), (K.PREC_MIXED, 10, 2e-5)])
def test_stokeslet_against_lattice_sum_and_translation(bc, prec, p, tol):
    """Stokeslet (G table), FP32 and mixed (tensor-core M->L) forms against the extrapolated
    lattice sum of the direct kernel on sampled targets, and a rigid shift along the periodic
    axes (modulo the period) changes the result by no more than the two evaluations' errors."""
    pts, f = G.stokeslet_case()
    ref = G.load(f"stokeslet_{bc}")   # the lattice sum on the sampled targets (tests/golden)
    plan = K.Plan(K.STOKESLET, p=p, q=64, bc=BC[bc], precision=prec, variant=K.ML_G)
    plan.set_points(torch.from_numpy(pts.astype(np.float32)).cuda())
    g0 = plan.eval(torch.from_numpy(f.astype(np.float32)).cuda()).double().cpu().numpy()
    if prec == K.PREC_MIXED:
        assert K.kafmm_get_counters(plan.h)["tensor_core_m2l"] == 1
    sh = np.array([0.4173, 0.2281 if bc == "pxy" else 0.0, 0.0])
    moved = np.minimum(((pts + sh) % 1.0).astype(np.float32), np.float32(1) - np.float32(2 ** -24))
    plan.set_points(torch.from_numpy(moved).cuda())
    g1 = plan.eval(torch.from_numpy(f.astype(np.float32)).cuda()).double().cpu().numpy()
    plan.close()
    e0 = D.rel_l2(g0[G.IDX_LAT], ref)
    print(bc, prec, e0, D.rel_l2(g1, g0))
    assert e0 < tol
    assert D.rel_l2(g1, g0) < 2 * tol


def test_rpy_sphere_velocities_across_the_periodic_boundary():
    """Singly periodic RPY: kafmm_eval + kafmm_rpy_velocity (the assembly and the overlap pass,
    whose contact search wraps along x) against the lattice sum of the far-form pair mobility
    plus the overlap corrections of the images with shift -1, 0, 1 along x, FP64."""
    pts, fb = G.rpy_cluster_case()
    n, a = len(pts), fb[:, 3]
    ref = G.load("rpy_velocity_px")   # lattice sum + overlap corrections (tests/golden)
    # p = 10: the assembled velocities lose about one digit to the overlap corrections (the
    # oracle's own KAFMM: 3.0e-6 at p = 8, 1.6e-7 at p = 10)
    plan = K.Plan(K.RPY, p=10, q=32, bc=K.BC_PX, precision=K.PREC_FP64, variant=K.ML_G)
    plan.set_points(torch.from_numpy(pts).cuda())
    st = torch.from_numpy(fb).cuda()
    gg = plan.eval(st)
    ua = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    K.kafmm_rpy_velocity(plan.h, st, torch.from_numpy(a).cuda(), gg, ua, K.F64)
    plan.close()
    d = pts[:, None] - pts[None]
    wrap = np.abs(d[..., 0]) > 0.5
    d[..., 0] = (d[..., 0] + 0.5) % 1.0 - 0.5      # nearest image along x
    close = np.linalg.norm(d, axis=2) < a[:, None] + a[None]
    assert np.sum(wrap & close) > 100   # contacts across the periodic boundary
    err = D.rel_l2(ua.cpu().numpy(), ref)
    print("rpy px", err)
    assert err < 1e-6


WALL = {"px": K.BC_WALL_PX, "pxy": K.BC_WALL_PXY}


@pytest.mark.parametrize("bc", ["px", "pxy"])
@pytest.mark.parametrize("prec,tol", [(K.PREC_FP64, 2e-6), (K.PREC_MIXED, 2e-5)])
def test_periodic_wall_stokeslet_against_lattice_sum(bc, prec, tol):
    """Stokeslets above the wall, periodic along x (and y), p = 10, forces with a net part:
    the three image-system sums as singly / doubly periodic child plans, against the lattice
    sums of the same sums assembled (pinned to the lattice sum of Blake's solution)."""
    pts, f = G.upper_case(G.N_WALL, 36)
    ref = G.load(f"wall_{bc}")   # the lattice sums of the three sums, assembled (tests/golden)
    dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
    plan = K.Plan(K.STOKESLET, p=10, q=64, bc=WALL[bc], precision=prec)
    plan.set_points(torch.from_numpy(pts).to(dt).cuda())
    g = plan.eval(torch.from_numpy(f).to(dt).cuda()).double().cpu().numpy()
    plan.close()
    err = D.rel_l2(g[G.IDX_WALL], ref)
    print("wall", bc, prec, err)
    assert err < tol


def test_doubly_periodic_rpy_wall_against_lattice_sums():
    """RPY above the wall, doubly periodic, FP64, p = 10: [u, lap u] against the lattice sums of
    the table's four sums, assembled (pinned to the lattice sum of the RPY definition)."""
    pts, fb = G.upper_case(G.N_RPY_WALL, 37, rpy=True)
    idx = G.IDX_RPY_WALL
    ref = G.load("rpy_wall_pxy")   # the lattice sums of the four sums, assembled (tests/golden)
    plan = K.Plan(K.RPY, p=10, q=64, bc=K.BC_WALL_PXY, precision=K.PREC_FP64)
    plan.set_points(torch.from_numpy(pts).cuda())
    g = plan.eval(torch.from_numpy(fb).cuda()).cpu().numpy()[idx]
    plan.close()
    eu, el = D.rel_l2(g[:, :3], ref[:, :3]), D.rel_l2(g[:, 3:], ref[:, 3:])
    print("rpy wall pxy", eu, el)
    assert eu < 2e-6 and el < 2e-5

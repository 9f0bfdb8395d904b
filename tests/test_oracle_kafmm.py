"""Pins for the oracle's octree, interaction lists and plain KAFMM (oracle/tree.py,
oracle/kafmm.py).

* Tree: every point in exactly one leaf; the refinement rule (Sec. III) holds box by box.
* Lists: every (target leaf, source leaf[, image]) pair is reached by exactly one route
  (U, W, V of an ancestor pair, X of an ancestor) -- the partition property the U/V/W/X
  lists exist to provide, checked by brute force.
* KAFMM: equals the direct sum to round-off when the tree has no far field; converges to
  the direct sum exponentially in the order m (Sec. III); the four-channel Laplace
  aggregation of the Stokeslet reproduces the Stokeslet exactly for point sources.
"""
import numpy as np
import pytest

import workloads as W
from oracle import direct as D
from oracle.kafmm import KAFMM, PROBLEMS
from oracle.tree import Tree, cells


def _tree_points():
    pts, _ = W.laplace_uniform(700, seed=21)
    clu, _, _ = W.rpy_clusters(700, seed=22, n_clusters=4, sigma=0.04, dtype=np.float64)
    return [pts, clu]


@pytest.mark.parametrize("which", [0, 1])
def test_tree_partition_and_refinement_rule(which):
    pts = _tree_points()[which]
    q = 16
    T = Tree(pts, q=q)
    owner = np.full(len(pts), -1)
    for b in T.leaves():
        assert np.all(owner[T.src_idx[b]] == -1)
        owner[T.src_idx[b]] = b
        assert len(T.src_idx[b]) <= q or T.level[b] == 20
    assert np.all(owner >= 0)
    I = cells(pts)
    for b in range(T.nbox):
        lv = int(T.level[b])
        inside = np.all((I >> (20 - lv)) == T.anchor[b], axis=1)
        assert np.array_equal(np.sort(np.nonzero(inside)[0]), np.sort(T.src_idx[b]))
        if not T.is_leaf[b]:
            assert len(T.src_idx[b]) > q
    # breadth-first numbering: levels non-decreasing, Morton order inside a level
    assert np.all(np.diff(T.level) >= 0)


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("which", [0, 1])
def test_lists_reach_every_pair_exactly_once(periodic, which):
    pts = _tree_points()[which][:300]
    T = Tree(pts, q=12, periodic=periodic)
    lv = T.leaves()
    assert len(lv) > 20 and T.nlevels >= 3
    for b in range(T.nbox):  # faster membership tests
        T.U[b], T.V[b], T.W[b], T.X[b] = set(T.U[b]), set(T.V[b]), set(T.W[b]), set(T.X[b])
    bad = [(tb, sb, sh) for tb in lv for sb in lv for sh in T._shifts()
           if T.route_count(tb, sb, sh) != 1]
    assert not bad


@pytest.mark.parametrize("problem", list(PROBLEMS))
def test_kafmm_without_far_field_is_the_direct_sum(problem):
    """Depth-0 tree (N <= q): only the U list is used, so KAFMM == O1 to round-off."""
    rng = np.random.default_rng(1)
    ks, kt, _, _ = PROBLEMS[problem]
    pts = rng.random((50, 3))
    s = rng.standard_normal((50, ks))
    if problem in WIDTH_PROBLEMS:   # radius b / blob width eps in the fourth column
        s[:, 3] = rng.uniform(0.001, 0.01, 50)
    kern = KERNEL_OF[problem]
    g = KAFMM(problem, 4, q=64).evaluate(pts, s)
    assert D.rel_l2(g, D.direct(kern, pts, pts, s)) < 1e-14


def test_l4_aggregation_reproduces_stokeslet_exactly():
    """With the true point sources as 'equivalent' charges, the four-channel Laplace form of
    the Stokeslet equals the Stokeslet (for any reference centre)."""
    rng = np.random.default_rng(2)
    y = rng.random((30, 3))
    f = rng.standard_normal((30, 3))
    x = rng.random((20, 3)) + 2.0
    F = KAFMM("stokeslet_l4", 4, 8)
    for c in (np.zeros(3), np.array([0.3, -0.7, 1.1])):
        q = np.concatenate([f, np.sum((y - c) * f, axis=1)[:, None]], axis=1)
        u = F._equiv_to_targets(x, y, q, c)
        assert D.rel_l2(u, D.direct("stokeslet", x, y, f)) < 1e-13
    # shifting the reference moves channel 4 by (c - c') . q_{1:3}
    c0, c1 = np.array([0.1, 0.2, 0.3]), np.array([-0.4, 0.9, 0.0])
    q0 = np.concatenate([f, np.sum((y - c0) * f, axis=1)[:, None]], axis=1)
    q1 = np.concatenate([f, np.sum((y - c1) * f, axis=1)[:, None]], axis=1)
    assert np.allclose(F._shift(q0, c0, c1), q1, rtol=1e-13, atol=1e-14)


WIDTH_PROBLEMS = ("rpy_g", "rpy_l4", "stokeslet_reg_g")
KERNEL_OF = {"laplace": "laplace", "stokeslet_g": "stokeslet", "stokeslet_l4": "stokeslet",
             "rpy_g": "rpy", "rpy_l4": "rpy", "stokeslet_reg_g": "stokeslet_reg",
             "laplace_qd": "laplace_qd", "stokes_dl_pv": "stokes_dl", "stokes_pvel": "stokes_pvel",
             "stokes_pvel_grad": "stokes_pvel_grad", "stokes_pvel_lapl": "stokes_pvel_lapl",
             "stokes_pvel_traction": "stokes_pvel_traction", "stokes_dl_grad": "stokes_dl_grad",
             "stokes_dl_lapl": "stokes_dl_lapl", "stokes_dl_traction": "stokes_dl_traction",
             "laplace_quad": "laplace_quad"}


def _inputs(problem, n, seed=0):
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    ks = PROBLEMS[problem][0]
    s = rng.standard_normal((n, ks))
    if problem in WIDTH_PROBLEMS:
        s[:, 3] = rng.uniform(0.0, 2e-3, n)
    return pts, s


@pytest.mark.parametrize("problem,n,q,orders,bound", [
    ("laplace", 3000, 48, (4, 6, 8), 1e-6),
    ("stokeslet_l4", 2000, 40, (4, 6, 8), 1e-5),
    ("stokeslet_g", 1200, 40, (4, 6), 1e-3),
    ("rpy_l4", 2000, 40, (4, 6, 8), 1e-5),
    ("rpy_g", 1200, 40, (4, 6), 1e-3),
    ("stokeslet_reg_g", 1200, 40, (4, 6), 1e-3),
    ("laplace_qd", 2000, 48, (4, 6, 8), 1e-5),
    ("laplace_quad", 2000, 48, (4, 6, 8), 1e-4),
    ("stokes_dl_pv", 1200, 40, (4, 6), 1e-3),
    ("stokes_pvel", 1200, 40, (4, 6), 1e-3),
    ("stokes_pvel_grad", 1200, 40, (4, 6), 3e-3),
    ("stokes_dl_traction", 1200, 40, (4, 6), 3e-3),
])
def test_kafmm_converges_to_direct_sum(problem, n, q, orders, bound):
    """eps_L2 against the direct sum falls exponentially with the order m (Sec. III)."""
    pts, s = _inputs(problem, n)
    kern = KERNEL_OF[problem]
    ref = D.direct(kern, pts, pts, s)
    errs = []
    for m in orders:
        F = KAFMM(problem, m, q)
        g = F.evaluate(pts, s)
        assert F.tree.nlevels >= 3 and sum(len(v) for v in F.tree.V) > 0
        errs.append(D.rel_l2(g, ref))
    assert all(b < a / 8 for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < bound, errs


def test_kafmm_adaptive_tree_with_w_and_x_lists():
    """A clustered cloud exercises W and X lists; the result still converges."""
    pts, f, _ = W.rpy_clusters(2500, seed=8, n_clusters=3, sigma=0.05, dtype=np.float64)
    ref = D.direct("stokeslet", pts, pts, f)
    F = KAFMM("stokeslet_l4", 8, 24)
    g = F.evaluate(pts, f)
    T = F.tree
    assert sum(len(v) for v in T.W) > 0 and sum(len(v) for v in T.X) > 0
    assert D.rel_l2(g, ref) < 2e-5


def test_kafmm_is_linear_in_source_values():
    pts, s = _inputs("stokeslet_l4", 800, seed=4)
    _, s2 = _inputs("stokeslet_l4", 800, seed=5)
    F = KAFMM("stokeslet_l4", 5, 32)
    g = F.evaluate(pts, 2.0 * s - 0.5 * s2)
    ref = 2.0 * F.evaluate(pts, s) - 0.5 * F.evaluate(pts, s2)
    assert D.rel_l2(g, ref) < 1e-9   # pinv amplifies FP64 rounding by ~1/rcond

"""GPU parity of batched evaluation (kafmm_set_points_batched): many independent kernel sums
of uneven size in one forest.

* The forest is the union of the single-problem octrees: box for box and list for list equal
  (integer-exact) to the oracle's tree of each problem.
* Plain FP64 form: each problem's slice equals the oracle CPU KAFMM of that problem alone
  (rel L2 <= 1e-7) and the GPU's own single-problem evaluation (<= 1e-12).
* Mixed form (tcgen05 M->L): each slice within 1e-5 of the plain FP64 form of that problem.
* Full size (512 problems, about 8 million points, p = 8, q = 64, as timed by the batched
  bench): 8 whole problems against the FP64 direct sum and against their FP64 GPU form.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads as W  # noqa: E402
from oracle import direct as D  # noqa: E402
from oracle.kafmm import KAFMM  # noqa: E402
from oracle.tree import Tree  # noqa: E402
from paper_2010_15155_gb300 import kafmm as K  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_15155_gb300 import build
    build.build()


def _problems(sizes, seed, clustered=(), dtype=np.float64):
    """Uniform problems (Gaussian clusters for the indices in `clustered`), forces N(0,1)^3."""
    pts, fs = [], []
    for k, n in enumerate(sizes):
        rng = np.random.default_rng([seed, k])
        if k in clustered:
            c = rng.random((3, 3)) * 0.6 + 0.2
            p = c[rng.integers(0, 3, n)] + 0.04 * rng.standard_normal((n, 3))
            p = np.clip(p, 0.0, 1.0 - 2.0 ** -40)
        else:
            p = rng.random((n, 3))
        pts.append(p)
        fs.append(rng.standard_normal((n, 3)))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(pts).astype(dtype), np.concatenate(fs).astype(dtype), off


def _code(sh):
    return (sh[0] + 1) + 3 * (sh[1] + 1) + 9 * (sh[2] + 1)


def test_forest_is_the_union_of_single_problem_trees():
    sizes = [0, 1, 37, 700, 3000, 64, 2000]
    pts, _, off = _problems(sizes, seed=31, clustered=(4,))
    q = 40
    plan = K.Plan(K.LAPLACE, p=4, q=q, precision=K.PREC_FP64, near_only=True)
    plan.set_points_batched(torch.from_numpy(pts).cuda(), off)
    info = plan.info()
    nb = info["nbox"]
    assert info["n_prob"] == len(sizes)
    level, anchor, parent, leaf = K.kafmm_get_tree(plan.h, nb)
    lists = {name: K.kafmm_get_list(plan.h, kind, nb) for kind, name in enumerate("UVWX")}
    plan.close()
    # problem of every box: follow the parents up to the root (root of problem k is box k)
    prob = np.empty(nb, np.int64)
    for b in range(nb):
        r = b
        while parent[r] >= 0:
            r = parent[r]
        prob[b] = r
    assert np.array_equal(level[:len(sizes)], np.zeros(len(sizes)))
    for k, n in enumerate(sizes):
        mine = np.flatnonzero(prob == k)
        if n == 0:
            assert list(mine) == [k] and leaf[k] == 1
            continue
        T = Tree(pts[off[k]:off[k + 1]], q=q)
        assert len(mine) == T.nbox, k
        local = {int(g): i for i, g in enumerate(mine)}
        assert np.array_equal(level[mine], T.level)
        assert np.array_equal(anchor[mine], T.anchor)
        assert np.array_equal(leaf[mine].astype(bool), T.is_leaf)
        par = np.array([local[int(parent[g])] if parent[g] >= 0 else -1 for g in mine])
        assert np.array_equal(par, T.parent)
        for name in "UVWX":
            o, ent, sh = lists[name]
            ref = getattr(T, name)
            for i, g in enumerate(mine):
                got = {(local[int(e)], int(c)) for e, c in zip(ent[o[g]:o[g + 1]], sh[o[g]:o[g + 1]])}
                want = {(a, _code(s)) for (a, s) in ref[i]}
                assert got == want, (k, name, i)


def test_batched_fp64_matches_oracle_and_single_problems():
    sizes = [0, 1, 200, 2500, 900, 64, 1700]
    pts, f, off = _problems(sizes, seed=32, clustered=(3,))
    p, q = 6, 40
    plan = K.Plan(K.STOKESLET, p=p, q=q, precision=K.PREC_FP64, variant=K.ML_L4)
    plan.set_points_batched(torch.from_numpy(pts).cuda(), off)
    g = plan.eval(torch.from_numpy(f).cuda()).cpu().numpy()
    for k, n in enumerate(sizes):
        a, b = off[k], off[k + 1]
        if n <= 1:
            assert np.all(g[a:b] == 0.0)
            continue
        ref = KAFMM("stokeslet_l4", p, q).evaluate(pts[a:b], f[a:b])
        assert D.rel_l2(g[a:b], ref) < 1e-7, k
        plan.set_points(torch.from_numpy(pts[a:b]).cuda())
        single = plan.eval(torch.from_numpy(f[a:b]).cuda()).cpu().numpy()
        assert D.rel_l2(g[a:b], single) < 1e-12, k
    plan.close()


def test_batched_laplace_with_separate_targets():
    """Sources and targets as separate sets per problem (offsets differ)."""
    rng = np.random.default_rng(33)
    ns, nt = [300, 0, 1500, 40], [100, 50, 800, 0]
    y = rng.random((sum(ns), 3))
    x = rng.random((sum(nt), 3))
    q_ = rng.uniform(-1, 1, (sum(ns), 1))
    so = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    to = np.concatenate([[0], np.cumsum(nt)]).astype(np.int64)
    plan = K.Plan(K.LAPLACE, p=8, q=32, precision=K.PREC_FP64)
    plan.set_points_batched(torch.from_numpy(y).cuda(), so, torch.from_numpy(x).cuda(), to)
    g = plan.eval(torch.from_numpy(q_).cuda()).cpu().numpy()
    plan.close()
    for k in range(len(ns)):
        gk = g[to[k]:to[k + 1]]
        if nt[k] == 0:
            continue
        if ns[k] == 0:
            assert np.all(gk == 0.0)
            continue
        ref = KAFMM("laplace", 8, 32).evaluate(y[so[k]:so[k + 1]], q_[so[k]:so[k + 1]],
                                               trg=x[to[k]:to[k + 1]])
        assert D.rel_l2(gk, ref) < 1e-7, k


def test_batched_mixed_tensor_core_form_matches_fp64_form():
    sizes = W.batched_sizes(24, lo=1024, hi=16384, seed=34)
    pts, f, off = W.batched_stokes(sizes, seed=34)
    out = {}
    for prec in (K.PREC_FP64, K.PREC_MIXED):
        dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
        plan = K.Plan(K.STOKESLET, p=8, q=64, precision=prec, variant=K.ML_L4)
        plan.set_points_batched(torch.from_numpy(pts).to(dt).cuda(), off)
        out[prec] = plan.eval(torch.from_numpy(f).to(dt).cuda()).double().cpu().numpy()
        if prec == K.PREC_MIXED:
            assert K.kafmm_get_counters(plan.h)["tensor_core_m2l"] == 1
        plan.close()
    for k in range(len(sizes)):
        a, b = off[k], off[k + 1]
        assert D.rel_l2(out[K.PREC_MIXED][a:b], out[K.PREC_FP64][a:b]) < 1e-5, k


def test_batched_argument_errors():
    pts = torch.rand((100, 3), dtype=torch.float64, device="cuda") * 0.99
    plan = K.Plan(K.STOKESLET, p=4, q=32, precision=K.PREC_FP64)
    # rejected on the host before any device access: decreasing offsets, a first offset
    # other than 0, no problems
    for bad in ([0, 60, 50, 100], [1, 50, 100], [0]):
        with pytest.raises(K.KafmmError) as e:
            K.kafmm_set_points_batched(plan.h, len(bad) - 1, bad, bad, pts, pts, K.F64)
        assert e.value.code == -1
    plan.close()
    per = K.Plan(K.STOKESLET, p=4, q=32, bc=K.BC_PXYZ, precision=K.PREC_FP64, variant=K.ML_G)
    with pytest.raises(K.KafmmError) as e:
        per.set_points_batched(pts, [0, 50, 100])
    assert e.value.code == -1
    per.close()
    rpy = K.Plan(K.RPY, p=4, q=32, precision=K.PREC_FP64)
    rpy.set_points_batched(pts, [0, 50, 100])
    s = torch.zeros((100, 4), dtype=torch.float64, device="cuda")
    g = rpy.eval(s)
    ua = torch.empty((100, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(K.KafmmError) as e:
        K.kafmm_rpy_velocity(rpy.h, s, torch.ones(100, dtype=torch.float64, device="cuda") * 1e-3,
                             g, ua, K.F64)
    assert e.value.code == -1
    rpy.close()


def test_batched_full_size_sampled_problems():
    """512 problems, N_k log-uniform in [1024, 65536] (about 8 million points), p = 8, q = 64,
    mixed form, in the configuration the batched bench times; 8 whole problems checked."""
    sizes = W.batched_sizes(512)
    pts, f, off = W.batched_stokes(sizes)
    plan = K.Plan(K.STOKESLET, p=8, q=64, precision=K.PREC_MIXED, variant=K.ML_L4)
    plan.set_points_batched(torch.from_numpy(pts).cuda(), off)
    g = plan.eval(torch.from_numpy(f).cuda()).double().cpu().numpy()
    assert plan.info()["n_prob"] == 512
    plan.close()
    pick = np.random.default_rng(35).choice(512, 8, replace=False)
    ref64 = K.Plan(K.STOKESLET, p=8, q=64, precision=K.PREC_FP64, variant=K.ML_L4)
    for k in pick:
        a, b = off[k], off[k + 1]
        p64 = pts[a:b].astype(np.float64)
        f64 = f[a:b].astype(np.float64)
        direct = D.direct("stokeslet", p64, p64, f64)
        ref64.set_points(torch.from_numpy(p64).cuda())
        fp64 = ref64.eval(torch.from_numpy(f64).cuda()).cpu().numpy()
        assert D.rel_l2(g[a:b], fp64) < 1e-5, k
        assert D.rel_l2(g[a:b], direct) < 1e-4, k
    ref64.close()

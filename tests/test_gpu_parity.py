"""GPU parity: the CUDA evaluator (through the C ABI) against the CPU oracle.

* Octree and U/V/W/X lists: identical (integer-exact) to the oracle's, box by box.
* Near field (U-list S->T) per kernel: FP64 to 1e-12, FP32 to 2e-5 (relative L2).
* Full KAFMM, plain FP64 GPU form vs the FP64 CPU KAFMM (same order, same tables):
  relative L2 <= 1e-7.
* FP32 form vs the FP64 GPU form: relative L2 <= 1e-5.
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

KERN = {"laplace": K.LAPLACE, "stokeslet": K.STOKESLET, "rpy": K.RPY, "stokes_dl": K.STOKES_DL,
        "stokeslet_reg": K.STOKES_REG, "laplace_qd": K.LAPLACE_QD, "stokes_pvel": K.STOKES_PVEL,
        "stokes_pvel_grad": K.STOKES_PVEL_GRAD, "stokes_pvel_lapl": K.STOKES_PVEL_LAPL,
        "stokes_pvel_traction": K.STOKES_PVEL_TRACTION, "stokes_dl_grad": K.STOKES_DL_GRAD,
        "stokes_dl_lapl": K.STOKES_DL_LAPL, "stokes_dl_traction": K.STOKES_DL_TRACTION,
        "laplace_quad": K.LAPLACE_QUAD}
DERIV = ["stokes_pvel_grad", "stokes_pvel_lapl", "stokes_pvel_traction", "stokes_dl_grad", "stokes_dl_lapl",
         "stokes_dl_traction"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_15155_gb300 import build
    build.build()


def _gpu_tree(pts, q, dtype=torch.float64, periodic=False):
    plan = K.Plan(K.LAPLACE, p=4, q=q, precision=K.PREC_FP64, near_only=True,
                  bc=K.BC_PXYZ if periodic else K.BC_OPEN)
    y = torch.from_numpy(np.ascontiguousarray(pts)).to(dtype).cuda()
    plan.set_points(y)
    info = plan.info()
    nb = info["nbox"]
    level, anchor, parent, leaf = K.kafmm_get_tree(plan.h, nb)
    lists = {}
    for kind, name in enumerate("UVWX"):
        off, ent, sh = K.kafmm_get_list(plan.h, kind, nb)
        lists[name] = [set(zip(ent[off[b]:off[b + 1]].tolist(), sh[off[b]:off[b + 1]].tolist()))
                       for b in range(nb)]
    plan.close()
    return info, level, anchor, parent, leaf, lists


def _code(sh):
    return (sh[0] + 1) + 3 * (sh[1] + 1) + 9 * (sh[2] + 1)


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("case", ["uniform", "clustered", "tiny"])
def test_tree_and_lists_match_oracle(case, periodic):
    if case == "uniform":
        pts, _ = W.laplace_uniform(6000, seed=3)
        q = 40
    elif case == "clustered":
        pts, _, _ = W.rpy_clusters(5000, seed=4, n_clusters=5, sigma=0.03, dtype=np.float64)
        q = 24
    else:
        pts, _ = W.laplace_uniform(30, seed=5)
        q = 64
    T = Tree(pts, q=q, periodic=periodic)
    info, level, anchor, parent, leaf, lists = _gpu_tree(pts, q, periodic=periodic)
    assert info["nbox"] == T.nbox and info["nlevels"] == T.nlevels
    assert np.array_equal(level, T.level)
    assert np.array_equal(anchor, T.anchor)
    assert np.array_equal(parent, T.parent)
    assert np.array_equal(leaf.astype(bool), T.is_leaf)
    for name in "UVWX":
        ref = getattr(T, name)
        for b in range(T.nbox):
            want = {(a, _code(sh)) for (a, sh) in ref[b]}
            assert lists[name][b] == want, (name, b)


def _inputs(kernel, n, seed, dtype=np.float64):
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    ks = K.KDIM[KERN[kernel]][0]
    s = rng.standard_normal((n, ks))
    if kernel in ("rpy", "stokeslet_reg"):   # radius b / blob width eps per source
        s[:, 3] = rng.uniform(0.0, 2e-3, n)
    return pts.astype(dtype), s.astype(dtype)


def _near_oracle(kernel, pts, s, q):
    """U-list sums only, from the oracle tree (plain loops)."""
    T = Tree(pts, q=q)
    g = np.zeros((len(pts), K.KDIM[KERN[kernel]][1]))
    for b in T.leaves():
        ti = T.trg_idx[b]
        for (a, sh) in T.U[b]:
            si = T.src_idx[a]
            g[ti] += D.direct(kernel, pts[ti], pts[si], s[si])
    return g


@pytest.mark.parametrize("kernel", ["laplace", "stokeslet", "rpy", "stokes_dl", "stokeslet_reg",
                                    "laplace_qd", "stokes_pvel", "laplace_quad"] + DERIV)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_near_field_matches_oracle(kernel, prec):
    n, q = 3000, 50
    pts, s = _inputs(kernel, n, seed=7)
    if prec == "fp32":   # the oracle sees the points and values the FP32 form computes with
        pts = pts.astype(np.float32).astype(np.float64)
        s = s.astype(np.float32).astype(np.float64)
    ref = _near_oracle(kernel, pts, s, q)
    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = K.Plan(KERN[kernel], p=4, q=q, precision=K.PREC_FP64 if prec == "fp64" else K.PREC_FP32,
                  near_only=True)
    plan.set_points(torch.from_numpy(pts).to(dt).cuda())
    g = plan.eval(torch.from_numpy(s).to(dt).cuda()).double().cpu().numpy()
    plan.close()
    tol = 1e-12 if prec == "fp64" else 2e-5
    assert D.rel_l2(g, ref) < tol


@pytest.mark.parametrize("problem,kernel,variant,n,p,q", [
    ("laplace", "laplace", K.ML_L4, 4096, 8, 64),
    ("stokeslet_l4", "stokeslet", K.ML_L4, 3000, 6, 40),
    ("stokeslet_g", "stokeslet", K.ML_G, 1500, 4, 32),
    ("rpy_l4", "rpy", K.ML_L4, 2500, 6, 40),
    ("rpy_g", "rpy", K.ML_G, 1500, 4, 32),
    ("stokeslet_reg_g", "stokeslet_reg", K.ML_G, 1500, 4, 32),
    ("laplace_qd", "laplace_qd", K.ML_L4, 3000, 6, 40),
    ("stokes_dl_pv", "stokes_dl", K.ML_L4, 1500, 6, 40),
    ("stokes_pvel", "stokes_pvel", K.ML_L4, 1500, 6, 40),
    ("laplace_quad", "laplace_quad", K.ML_L4, 3000, 6, 40),
] + [(k, k, K.ML_L4, 1500, 6, 40) for k in DERIV])
def test_fp64_gpu_kafmm_matches_cpu_kafmm(problem, kernel, variant, n, p, q):
    if problem == "laplace":
        pts, s = W.laplace_uniform(n, seed=0)
    else:
        pts, s = _inputs(kernel, n, seed=11)
    ref = KAFMM(problem, p, q).evaluate(pts, s)
    plan = K.Plan(KERN[kernel], p=p, q=q, precision=K.PREC_FP64, variant=variant)
    plan.set_points(torch.from_numpy(pts).cuda())
    g = plan.eval(torch.from_numpy(s).cuda()).cpu().numpy()
    plan.close()
    assert D.rel_l2(g, ref) < 1e-7


@pytest.mark.parametrize("kernel", DERIV)
def test_derivative_targets_mixed_form_against_direct_sum(kernel):
    """Gradient, Laplacian and traction target values of the mixed form (FP32 near field,
    tensor-core M->L) and of the FP64 form at p = 10 against the oracle's direct sum on 500
    sampled targets (measured on a GB300: FP64 form 2e-10 .. 3.5e-8, mixed 1.9e-7 .. 3.4e-7)."""
    pts, s = _inputs(kernel, 40000, seed=17, dtype=np.float32)
    idx = np.arange(0, 40000, 80)
    ref = D.direct(kernel, pts.astype(np.float64)[idx], pts.astype(np.float64), s.astype(np.float64))
    err = {}
    for prec in (K.PREC_FP64, K.PREC_MIXED):
        dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
        plan = K.Plan(KERN[kernel], p=10, q=64, precision=prec)
        plan.set_points(torch.from_numpy(pts).to(dt).cuda())
        g = plan.eval(torch.from_numpy(s).to(dt).cuda()).double().cpu().numpy()
        if prec == K.PREC_MIXED:
            assert K.kafmm_get_counters(plan.h)["tensor_core_m2l"] == 1
        plan.close()
        err[prec] = D.rel_l2(g[idx], ref)
    print(kernel, err)
    assert err[K.PREC_FP64] < 2e-7 and err[K.PREC_MIXED] < 2e-6, err


def test_fp64_gpu_kafmm_adaptive_tree_matches_cpu_kafmm():
    pts, f, _ = W.rpy_clusters(4000, seed=8, n_clusters=3, sigma=0.05, dtype=np.float64)
    F = KAFMM("stokeslet_l4", 6, 24)
    ref = F.evaluate(pts, f)
    T = F.tree
    assert sum(map(len, T.W)) > 0 and sum(map(len, T.X)) > 0
    plan = K.Plan(K.STOKESLET, p=6, q=24, precision=K.PREC_FP64, variant=K.ML_L4)
    plan.set_points(torch.from_numpy(pts).cuda())
    g = plan.eval(torch.from_numpy(f).cuda()).cpu().numpy()
    plan.close()
    assert D.rel_l2(g, ref) < 1e-7


@pytest.mark.parametrize("kernel,variant", [("laplace", K.ML_L4), ("stokeslet", K.ML_L4),
                                            ("stokeslet", K.ML_G), ("rpy", K.ML_L4)])
def test_fp32_form_matches_fp64_form(kernel, variant):
    """The FP32 form (pseudo-inverse cutoff 1e-7) is as accurate as the FP64 form (cutoff
    1e-9) against the direct sum, up to 1e-5."""
    pts, s = _inputs(kernel, 20000, seed=13, dtype=np.float32)
    ref = D.direct(kernel, pts, pts, s)
    err = {}
    for prec in (K.PREC_FP64, K.PREC_FP32):
        dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
        plan = K.Plan(KERN[kernel], p=6, q=64, precision=prec, variant=variant)
        plan.set_points(torch.from_numpy(pts).to(dt).cuda())
        g = plan.eval(torch.from_numpy(s).to(dt).cuda()).double().cpu().numpy()
        plan.close()
        err[prec] = D.rel_l2(g, ref)
    assert err[K.PREC_FP32] < err[K.PREC_FP64] + 1e-5, err


def test_errors_are_reported_not_trapped():
    for kern in (K.LAPLACE_QD, K.LAPLACE_QUAD):   # open boundary only
        with pytest.raises(K.KafmmError) as e:
            K.Plan(kern, p=4, q=32, bc=K.BC_PXYZ)
        assert e.value.code == -1
    plan = K.Plan(K.STOKESLET, p=4, q=32, precision=K.PREC_FP32)
    bad = torch.tensor([[0.5, 0.5, 1.5], [0.1, 0.2, 0.3]], dtype=torch.float32, device="cuda")
    with pytest.raises(K.KafmmError) as e:
        plan.set_points(bad)
    assert e.value.code == -2
    with pytest.raises(K.KafmmError) as e:
        plan.eval(torch.zeros((2, 3), device="cuda"))
    assert e.value.code == -6
    plan.close()


@pytest.mark.parametrize("n,p,q", [(20000, 6, 64), (262144, 10, 128)])
def test_mixed_tensor_core_form_matches_fp64_form(n, p, q):
    """Split-BF16x3 tcgen05 M->L (mixed form) vs the plain FP64 GPU form: rel L2 <= 1e-5."""
    pts, f = W.stokes_uniform(n, seed=1, dtype=np.float32)
    out = {}
    for prec in (K.PREC_FP64, K.PREC_MIXED):
        dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
        plan = K.Plan(K.STOKESLET, p=p, q=q, precision=prec, variant=K.ML_L4)
        plan.set_points(torch.from_numpy(pts).to(dt).cuda())
        out[prec] = plan.eval(torch.from_numpy(f).to(dt).cuda()).double().cpu().numpy()
        if prec == K.PREC_MIXED:
            assert K.kafmm_get_counters(plan.h)["tensor_core_m2l"] == 1
        plan.close()
    assert D.rel_l2(out[K.PREC_MIXED], out[K.PREC_FP64]) < 1e-5


@pytest.mark.parametrize("kernel,bc,p,split", [
    ("laplace", "open", 8, K.TC_TF32X3),      # R = 296: one 128-row block per CTA
    ("stokeslet", "open", 6, K.TC_TF32X3),    # G table, R = 456: two row blocks per CTA
    ("stokeslet", "open", 8, K.TC_BF16X3),    # G table, R = 888
    ("stokeslet", "pxyz", 8, K.TC_AUTO),      # periodic G table (root operator on CUDA cores)
    ("rpy", "open", 6, K.TC_AUTO),            # RPY on the G table
    ("laplace_qd", "open", 8, K.TC_AUTO),     # charges + dipoles -> phi, grad, Hessian
    ("stokes_dl", "open", 8, K.TC_AUTO),      # double layer on the StokesPVel table, R = 4n
    ("stokes_pvel", "open", 10, K.TC_AUTO),   # [f, q] -> [p, u], BF16x3
])
def test_mixed_tensor_core_single_column_tables_match_fp64_form(kernel, bc, p, split):
    """Single-column ML tables (Laplace; the Stokeslet G table, open and periodic) with the
    M->L, M->M, L->L and pseudo-inverse gather-GEMMs on the tensor cores: within 1e-5 of the
    FP32 form (same rounded operators on the CUDA cores), and no further from the plain FP64
    form than the FP32 form is, plus 1e-5.  (At p = 6 the FP32 form itself differs from the
    FP64 form by about 1e-4: its pseudo-inverse cutoff, 1e-7, drops more singular values.)"""
    n = 30000
    pts, s = _neutral(kernel, n, seed=41) if bc == "pxyz" else _inputs(kernel, n, seed=41)
    pts = np.minimum(pts, 1.0 - 2.0 ** -24)   # below 1 after rounding to FP32
    out = {}
    for prec in (K.PREC_FP64, K.PREC_FP32, K.PREC_MIXED):
        dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
        plan = K.Plan(KERN[kernel], p=p, q=64, bc=K.BC_PXYZ if bc == "pxyz" else K.BC_OPEN,
                      precision=prec, variant=K.ML_G, tc_split=split)
        plan.set_points(torch.from_numpy(pts).to(dt).cuda())
        out[prec] = plan.eval(torch.from_numpy(s).to(dt).cuda()).double().cpu().numpy()
        if prec == K.PREC_MIXED:
            assert K.kafmm_get_counters(plan.h)["tensor_core_m2l"] == 1
        plan.close()
    tc_err = D.rel_l2(out[K.PREC_MIXED], out[K.PREC_FP32])
    err = D.rel_l2(out[K.PREC_MIXED], out[K.PREC_FP64])
    assert tc_err < 1e-5
    assert err < D.rel_l2(out[K.PREC_FP32], out[K.PREC_FP64]) + 1e-5


@pytest.mark.parametrize("workload", ["uniform_l4", "clusters_l4", "uniform_g"])
def test_m2l_tilings_agree(workload):
    """Tensor-core M->L tiled per parent neighbour (per-box partials, combined in neighbour
    order) and with whole V lists per tile compute the same translations: equal up to the
    summation order of the split products (2.6e-6 measured, uniform, p = 8), each within 1e-5
    of the FP64 form; both are deterministic."""
    if workload == "clusters_l4":
        pts, f, _ = W.rpy_clusters(100000, seed=7, n_clusters=16)
        kern, variant, p = K.STOKESLET, K.ML_L4, 8
    else:
        pts, f = W.stokes_uniform(60000, seed=8, dtype=np.float32)
        kern, variant, p = K.STOKESLET, (K.ML_L4 if workload == "uniform_l4" else K.ML_G), 8
    y = torch.from_numpy(pts).cuda()
    s = torch.from_numpy(f).cuda()
    out = {}
    for tiling in (1, 2):
        plan = K.Plan(kern, p=p, q=64, precision=K.PREC_MIXED, variant=variant)
        K.kafmm_set_option(plan.h, K.OPT_TC_TILING, tiling)
        plan.set_points(y)
        g = plan.eval(s)
        assert torch.equal(plan.eval(s), g)
        c = K.kafmm_get_counters(plan.h)
        assert c["tensor_core_m2l"] == 1
        assert c["m2l_tiling"] == ("whole V lists" if tiling == 1 else "per parent neighbour")
        out[tiling] = g.double().cpu().numpy()
        plan.close()
    p64 = K.Plan(kern, p=p, q=64, precision=K.PREC_FP64, variant=variant)
    p64.set_points(y.double())
    ref = p64.eval(s.double()).cpu().numpy()
    p64.close()
    print("tilings", workload, D.rel_l2(out[2], out[1]), D.rel_l2(out[1], ref), D.rel_l2(out[2], ref))
    assert D.rel_l2(out[2], out[1]) < 1e-5
    assert D.rel_l2(out[1], ref) < 1e-5 and D.rel_l2(out[2], ref) < 1e-5


@pytest.mark.parametrize("p", [8, 10])
def test_regularized_stokeslet_mixed_form(p):
    """Regularized Stokeslet, blob widths eps ~ U(0, 1e-4) per source as in the paper's
    benchmark (Sec. III.A), 60000 uniform points: the mixed form (G table on the tensor cores)
    within 1e-5 of the plain FP64 GPU form, and both forms within their FMM error of the FP64
    direct sum on sampled targets."""
    rng = np.random.default_rng(44)
    n = 60000
    pts = np.minimum(rng.random((n, 3)), 1.0 - 2.0 ** -24)
    s = np.concatenate([rng.standard_normal((n, 3)), rng.uniform(0.0, 1e-4, (n, 1))], axis=1)
    idx = W.sample_targets(n, 1024)
    ref = D.direct("stokeslet_reg", pts[idx], pts, s)
    out = {}
    for prec in (K.PREC_FP64, K.PREC_MIXED):
        dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
        plan = K.Plan(K.STOKES_REG, p=p, q=64, precision=prec)
        plan.set_points(torch.from_numpy(pts).to(dt).cuda())
        out[prec] = plan.eval(torch.from_numpy(s).to(dt).cuda()).double().cpu().numpy()
        if prec == K.PREC_MIXED:
            assert K.kafmm_get_counters(plan.h)["tensor_core_m2l"] == 1
        plan.close()
    assert D.rel_l2(out[K.PREC_MIXED], out[K.PREC_FP64]) < 1e-5
    assert D.rel_l2(out[K.PREC_FP64][idx], ref) < (1e-5 if p == 8 else 1e-6)
    assert D.rel_l2(out[K.PREC_MIXED][idx], ref) < 2e-5


@pytest.mark.parametrize("prec,tol", [(K.PREC_FP64, 1e-6), (K.PREC_FP32, 2e-5)])
def test_rpy_sphere_velocities_with_overlap_match_brute_force(prec, tol):
    """kafmm_eval ([u, lap u]) + kafmm_rpy_velocity (assembly u + a^2/6 lap u and the overlap
    pass) against the oracle's brute-force pair mobility over all pairs (Sec. II.B)."""
    pts, f, a = W.rpy_clusters(3000, seed=6, n_clusters=4, sigma=0.05, a_lo=0.004, a_hi=0.012,
                               dtype=np.float64)
    fb = np.concatenate([f, a[:, None]], axis=1)
    ref = D.rpy_velocity(pts, a, pts, fb, same_set=True)
    dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
    if dt == torch.float32:  # keep every point below 1 after rounding to FP32
        pts = np.minimum(pts.astype(np.float32), np.float32(1) - np.float32(2 ** -24)).astype(np.float64)
        fb = np.concatenate([f, a[:, None]], axis=1)
        ref = D.rpy_velocity(pts, a, pts, fb, same_set=True)
    plan = K.Plan(K.RPY, p=8, q=48, precision=prec, variant=K.ML_L4)
    plan.set_points(torch.from_numpy(pts).to(dt).cuda())
    s = torch.from_numpy(fb).to(dt).cuda()
    g = plan.eval(s)
    ua = torch.empty((len(pts), 3), dtype=dt, device="cuda")
    K.kafmm_rpy_velocity(plan.h, s, torch.from_numpy(a).to(dt).cuda(), g, ua,
                         K.F64 if dt == torch.float64 else K.F32)
    plan.close()
    nover = np.sum(np.linalg.norm(pts[:, None] - pts[None], axis=2) < a[:, None] + a[None]) - len(pts)
    assert nover > 1000  # the case really exercises the overlap pass
    assert D.rel_l2(ua.double().cpu().numpy(), ref) < tol


def _neutral(kernel, n, seed, dtype=np.float64):
    """Zero net source (periodic sums): charges or forces minus their mean; the regularized
    Stokeslet's blob widths eps ~ U(0, 2e-3) in the fourth column."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    if kernel.startswith("stokes_dl"):          # double layer: sum of tr D = 0
        s = rng.standard_normal((n, 9))
        s[:, [0, 4, 8]] -= (s[:, 0] + s[:, 4] + s[:, 8]).mean() / 3.0
        return pts.astype(dtype), s.astype(dtype)
    if kernel.startswith("stokes_pvel"):        # [f, q]: sum of f = 0 and sum of q = 0
        s = rng.standard_normal((n, 4))
        return pts.astype(dtype), (s - s.mean(axis=0)).astype(dtype)
    kt = 1 if kernel == "laplace" else 3
    s = rng.standard_normal((n, kt))
    s = s - s.mean(axis=0)
    if kernel == "stokeslet_reg":
        s = np.concatenate([s, rng.uniform(0.0, 2e-3, (n, 1))], axis=1)
    return pts.astype(dtype), s.astype(dtype)


@pytest.mark.parametrize("problem,kernel", [("laplace", "laplace"), ("stokeslet_g", "stokeslet"),
                                            ("stokeslet_reg_g", "stokeslet_reg"), ("stokes_pvel", "stokes_pvel"),
                                            ("stokes_dl_pv", "stokes_dl"),
                                            ("stokes_pvel_traction", "stokes_pvel_traction"),
                                            ("stokes_dl_grad", "stokes_dl_grad")])
def test_periodic_fp64_gpu_kafmm_matches_cpu_kafmm(problem, kernel):
    """Triply periodic KAFMM (far images through the root operator) vs the oracle's periodic
    plain KAFMM, FP64 both: rel L2 <= 1e-7."""
    from oracle import periodic as Pd
    pts, s = _neutral(kernel, 1500, seed=21)
    p, q = 6, 32
    # the ML-tree kernel of the table
    ml = "laplace" if kernel == "laplace" else ("stokes_pvel" if kernel.startswith(("stokes_pvel", "stokes_dl"))
                                                else "stokeslet")
    ref = KAFMM(problem, p, q, bc="pxyz", t_m2l=Pd.t_m2l(ml, p)).evaluate(pts, s)
    plan = K.Plan(KERN[kernel], p=p, q=q, bc=K.BC_PXYZ, precision=K.PREC_FP64, variant=K.ML_G)
    plan.set_points(torch.from_numpy(pts).cuda())
    g = plan.eval(torch.from_numpy(s).cuda()).cpu().numpy()
    plan.close()
    assert D.rel_l2(g, ref) < 1e-7


@pytest.mark.parametrize("kernel", ["stokes_pvel", "stokes_dl"])
def test_periodic_pvel_table_mixed_form(kernel):
    """Triply periodic StokesPVel and double layer in the mixed form (tensor-core M->L on the
    4-row table, FP32 near field) against the FP64 form (pinned above to the oracle's periodic
    KAFMM, and through it to the Ewald sum): rel L2 <= 1e-5 at p = 10."""
    pts, s = _neutral(kernel, 30000, seed=23, dtype=np.float32)
    out = {}
    for prec in (K.PREC_FP64, K.PREC_MIXED):
        dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
        plan = K.Plan(KERN[kernel], p=10, q=64, bc=K.BC_PXYZ, precision=prec)
        plan.set_points(torch.from_numpy(pts).to(dt).cuda())
        out[prec] = plan.eval(torch.from_numpy(s).to(dt).cuda()).double().cpu().numpy()
        if prec == K.PREC_MIXED:
            assert K.kafmm_get_counters(plan.h)["tensor_core_m2l"] == 1
        plan.close()
    err = D.rel_l2(out[K.PREC_MIXED], out[K.PREC_FP64])
    print(kernel, err)
    assert err < 1e-5


def test_periodic_fp32_gpu_kafmm_against_ewald_and_translation():
    """Periodic Stokeslet, FP32 form: error against the Ewald sum at the FMM level, and the
    translation error (Sec. III.B): a rigid shift modulo the cell changes nothing beyond it."""
    from oracle import periodic as Pd
    pts, f = _neutral("stokeslet", 6000, seed=22)
    idx = np.arange(0, 6000, 24)
    ref = Pd.ewald_sum("stokeslet", pts[idx], pts, f)
    plan = K.Plan(K.STOKESLET, p=8, q=48, bc=K.BC_PXYZ, precision=K.PREC_FP32, variant=K.ML_G)
    plan.set_points(torch.from_numpy(pts.astype(np.float32)).cuda())
    g0 = plan.eval(torch.from_numpy(f.astype(np.float32)).cuda()).double().cpu().numpy()
    shifted = ((pts + np.array([0.4173, 0.2281, 0.9011])) % 1.0).astype(np.float32)
    shifted = np.minimum(shifted, np.float32(1) - np.float32(2 ** -24))
    plan.set_points(torch.from_numpy(shifted).cuda())
    g1 = plan.eval(torch.from_numpy(f.astype(np.float32)).cuda()).double().cpu().numpy()
    plan.close()
    assert D.rel_l2(g0[idx], ref) < 5e-5
    assert D.rel_l2(g1, g0) < 5e-5



def test_periodic_full_size_mixed_form():
    """Triply periodic Stokeslet at full size (2^22 uniform points, forces minus their mean,
    p = 12, q = 128) in the mixed form (G table on the tensor cores): within 1e-5 of the FP32
    CUDA-core form (pinned to the Ewald sum and the oracle's periodic KAFMM at small sizes by
    the tests above; at full size the mixed form is checked against the Ewald sum directly in
    test_gpu_parity_full.py), and a rigid shift modulo the cell (Sec. III.B) changes the result
    by less than the sum of the two evaluations' errors, 2 x 1e-5 (measured 1.1e-5 in
    compressed coordinates, each evaluation 4.9e-6 from the Ewald sum)."""
    n = 1 << 22
    pts, f = W.stokes_uniform(n, seed=4, zero_mean=True)
    y = torch.from_numpy(pts).cuda()
    s = torch.from_numpy(f).cuda()
    plan = K.Plan(K.STOKESLET, p=12, q=128, bc=K.BC_PXYZ, precision=K.PREC_MIXED, variant=K.ML_G)
    plan.set_points(y)
    g0 = plan.eval(s)
    assert K.kafmm_get_counters(plan.h)["tensor_core_m2l"] == 1
    sh = ((pts.astype(np.float64) + np.array([0.4173, 0.2281, 0.9011])) % 1.0).astype(np.float32)
    sh = np.minimum(sh, np.float32(1) - np.float32(2 ** -24))
    plan.set_points(torch.from_numpy(sh).cuda())
    g1 = plan.eval(s)
    plan.close()
    p32 = K.Plan(K.STOKESLET, p=12, q=128, bc=K.BC_PXYZ, precision=K.PREC_FP32, variant=K.ML_G)
    p32.set_points(y)
    g32 = p32.eval(s)
    p32.close()

    def rel(a, b):
        return float(torch.linalg.norm(a.double() - b.double()) / torch.linalg.norm(b.double()))
    assert rel(g0, g32) < 1e-5
    assert rel(g1, g0) < 2e-5


def test_eval_is_graph_capturable():
    """With KAFMM_OPT_SYNC = 0 a kafmm_eval after the first one enqueues work only: captured in
    a CUDA graph and replayed it reproduces the eager result bit for bit, for new source values
    written into the captured input buffer too."""
    pts, f = W.stokes_uniform(40000, seed=2, dtype=np.float32)
    y = torch.from_numpy(pts).cuda()
    s = torch.from_numpy(f).cuda()
    g = torch.empty((len(pts), 3), dtype=torch.float32, device="cuda")
    plan = K.Plan(K.STOKESLET, p=8, q=64, precision=K.PREC_MIXED, variant=K.ML_L4, sync=False)
    plan.set_points(y)
    plan.eval(s, g)
    torch.cuda.synchronize()
    ref = g.clone()
    f2 = torch.from_numpy(np.random.default_rng(3).standard_normal(f.shape).astype(np.float32)).cuda()
    plan.eval(f2, g)
    torch.cuda.synchronize()
    ref2 = g.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        K.kafmm_set_option(plan.h, K.OPT_STREAM, torch.cuda.current_stream().cuda_stream)
        K.kafmm_eval(plan.h, s, g, K.F32)
    K.kafmm_set_option(plan.h, K.OPT_STREAM, torch.cuda.current_stream().cuda_stream)
    g.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(g, ref)
    s.copy_(f2)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(g, ref2)
    K.kafmm_status(plan.h)
    plan.close()


@pytest.mark.parametrize("p", [6, 8, 10])
def test_tensor_core_pipeline_depths_agree_bit_for_bit(p):
    """Two stages of 128-byte operand rows and four stages of 64-byte rows issue the same MMAs
    in the same order: the mixed form (M->L, M->M, L->L, pseudo-inverse factors on the tensor
    cores) gives identical bits with either."""
    pts, f = W.stokes_uniform(30000, seed=9, dtype=np.float32)
    y = torch.from_numpy(pts).cuda()
    s = torch.from_numpy(f).cuda()
    out = {}
    for stages in (2, 4):
        plan = K.Plan(K.STOKESLET, p=p, q=64, precision=K.PREC_MIXED, variant=K.ML_L4, tc_stages=stages)
        plan.set_points(y)
        out[stages] = plan.eval(s)
        assert K.kafmm_get_counters(plan.h)["tensor_core_m2l"] == 1
        plan.close()
    assert torch.equal(out[2], out[4])


@pytest.mark.parametrize("compress,tiling", [(0, 2), (0, 1), (2, 2), (2, 1)])
def test_tensor_core_tiles_per_cta_agree_bit_for_bit(compress, tiling):
    """One, two or four consecutive tiles per CTA of the gather-GEMM issue the same MMAs per tile
    in the same order: identical bits, dense and compressed, grouped and per-class tiles, on an
    adaptive cloud whose tile count is not a multiple of four."""
    pts = W.lognormal_points(70001, seed=12).astype(np.float32)
    f = np.random.default_rng(12).standard_normal((len(pts), 3)).astype(np.float32)
    y = torch.from_numpy(pts).cuda()
    s = torch.from_numpy(f).cuda()
    out = {}
    for tiles in (1, 2, 4):
        plan = K.Plan(K.STOKESLET, p=10, q=64, precision=K.PREC_MIXED, variant=K.ML_L4, compress=compress)
        K.kafmm_set_option(plan.h, K.OPT_TC_TILING, tiling)
        K.kafmm_set_option(plan.h, K.OPT_TC_TILES, tiles)
        plan.set_points(y)
        out[tiles] = plan.eval(s)
        assert K.kafmm_get_counters(plan.h)["tensor_core_m2l"] == 1
        plan.close()
    assert torch.equal(out[1], out[2]) and torch.equal(out[1], out[4])


def test_tensor_core_tiles_option_is_validated():
    plan = K.Plan(K.STOKESLET, p=6, q=64, precision=K.PREC_MIXED)
    for bad in (0, 3, 8):
        with pytest.raises(K.KafmmError) as e:
            K.kafmm_set_option(plan.h, K.OPT_TC_TILES, bad)
        assert e.value.code == -1
    plan.close()


def test_autotune_picks_a_valid_configuration():
    """kafmm_autotune times the tensor-core pipeline depth and slot-range counts on the current
    points and keeps the fastest; evaluation afterwards equals an evaluation with those options
    set by hand and stays within the mixed-form tolerance of the FP64 form."""
    pts, f = W.stokes_uniform(60000, seed=10, dtype=np.float32)
    y = torch.from_numpy(pts).cuda()
    s = torch.from_numpy(f).cuda()
    g = torch.empty((len(pts), 3), dtype=torch.float32, device="cuda")
    plan = K.Plan(K.STOKESLET, p=8, q=64, precision=K.PREC_MIXED, variant=K.ML_L4)
    plan.set_points(y)
    chosen = K.kafmm_autotune(plan.h, s, g, K.F32)
    assert chosen["tc_stages"] in (2, 4) and chosen["tc_ranges"] in (1, 2, 4, 8)
    assert chosen["tc_tiling"] in (1, 2) and chosen["leaf_stage"] in (256, 640, 1280)
    assert chosen["tc_tiles"] in (1, 2, 4)
    tuned = plan.eval(s)
    plan.close()
    ref = K.Plan(K.STOKESLET, p=8, q=64, precision=K.PREC_MIXED, variant=K.ML_L4,
                 tc_stages=chosen["tc_stages"])
    K.kafmm_set_option(ref.h, K.OPT_TC_RANGES, chosen["tc_ranges"])
    K.kafmm_set_option(ref.h, K.OPT_TC_TILING, chosen["tc_tiling"])
    K.kafmm_set_option(ref.h, K.OPT_LEAF_STAGE, chosen["leaf_stage"])
    K.kafmm_set_option(ref.h, K.OPT_TC_TILES, chosen["tc_tiles"])
    ref.set_points(y)
    assert torch.equal(ref.eval(s), tuned)
    ref.close()
    p64 = K.Plan(K.STOKESLET, p=8, q=64, precision=K.PREC_FP64, variant=K.ML_L4)
    p64.set_points(y.double())
    g64 = p64.eval(s.double())
    p64.close()
    assert float(torch.linalg.norm(tuned.double() - g64) / torch.linalg.norm(g64)) < 1e-5


def _rpy_velocity_run(pts, fb, a, prec, contact):
    dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
    plan = K.Plan(K.RPY, p=8, q=64 if len(pts) < 200000 else 128, precision=prec, variant=K.ML_L4)
    K.kafmm_set_option(plan.h, K.OPT_RPY_CONTACT, contact)
    plan.set_points(torch.from_numpy(pts).to(dt).cuda())
    s = torch.from_numpy(fb).to(dt).cuda()
    g = plan.eval(s)
    ua = torch.empty((len(pts), 3), dtype=dt, device="cuda")
    K.kafmm_rpy_velocity(plan.h, s, torch.from_numpy(a).to(dt).cuda(), g, ua,
                         K.F64 if dt == torch.float64 else K.F32)
    plan.close()
    return ua.double().cpu().numpy()


def _rpy_brute(pts, fb, a, idx):
    p64, fb64, a64 = pts.astype(np.float64), fb.astype(np.float64), a.astype(np.float64)
    ref = D.rpy_velocity(p64[idx], a64[idx], p64, fb64, same_set=False)
    return ref - fb64[idx, :3] / (6 * np.pi * a64[idx, None])   # without the self mobility


def test_rpy_contact_split_is_exact_bookkeeping_in_fp64():
    """In FP64, leaving contact pairs out of the near field (and adding their whole mobility in
    the velocity pass) equals the paper's order (full kernel sum, then overlap correction)."""
    pts, f, a = W.rpy_clusters(60000, seed=12, n_clusters=8, sigma=0.03, dtype=np.float64)
    fb = np.concatenate([f, a[:, None]], axis=1)
    u0 = _rpy_velocity_run(pts, fb, a, K.PREC_FP64, 0)
    u1 = _rpy_velocity_run(pts, fb, a, K.PREC_FP64, 1)
    assert D.rel_l2(u1, u0) < 1e-10   # equal up to the summation order of the far forms


@pytest.mark.parametrize("n", [131072, 1 << 20])
def test_rpy_cluster_sphere_velocities_fp32(n):
    """Clustered spheres (64 Gaussian clusters, sigma 0.02, radii U(0.002, 0.006)); the mixed
    form with the contact split against brute-force pair mobilities on sampled targets.  At
    2^20 points this is the RPY cluster workload at full size (p = 8, q = 128)."""
    pts, f, a = W.rpy_clusters(n)
    fb = np.concatenate([f, a[:, None]], axis=1).astype(np.float32)
    idx = W.sample_targets(n, 1024)
    ref = _rpy_brute(pts, fb, a, idx)
    ua = _rpy_velocity_run(pts, fb, a, K.PREC_MIXED, 1)
    err = D.rel_l2(ua[idx], ref)
    print("rpy cluster", n, err)
    assert err < 2e-5   # measured 9.7e-6 (2^17) and 1.3e-5 (2^20); FP64 form 1.7e-6 at 2^20

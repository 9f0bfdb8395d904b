"""Pins for the oracle's triply periodic sums (oracle/periodic.py, Ewald in oracle/direct.c)
and its periodic KAFMM.

* The regular part of the periodic Green's function at the source point reproduces two
  classical lattice constants: the simple-cubic Madelung constant of the Laplace kernel
  (-2.837297479480619 / (4 pi L)) and Hasimoto's periodic-array Stokeslet correction
  (-2.837297479480619 / (6 pi L) I), the same number for both kernels by cubic symmetry.
* The Ewald split parameter drops out; the sums are periodic in each direction.
* The periodic KAFMM (tree with wrapped lists + far-image operator on the root) converges
  to the Ewald sum in the order m and is invariant under a rigid translation modulo the cell
  (the translation error of Sec. III.B).
"""
import numpy as np
import pytest

from oracle import direct as D
from oracle import periodic as Pd
from oracle.kafmm import KAFMM

MADELUNG_SC = -2.837297479480619


def test_lattice_constants():
    y = np.array([[0.3, 0.4, 0.5]])
    for L in (1.0, 2.5):
        g = Pd.ewald_sum("laplace", y * L, y * L, [1.0], L=L)
        assert abs(g[0, 0] * 4 * np.pi * L - MADELUNG_SC) < 1e-12
        u = Pd.ewald_sum("stokeslet", y * L, y * L, [[0.2, -1.0, 0.7]], L=L)
        assert np.allclose(u[0] * 6 * np.pi * L, MADELUNG_SC * np.array([0.2, -1.0, 0.7]),
                           rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("kernel", ["laplace", "stokeslet"])
def test_ewald_split_independent_and_periodic(kernel):
    rng = np.random.default_rng(3)
    y = rng.random((6, 3))
    kt = 1 if kernel == "laplace" else 3
    s = rng.standard_normal((6, kt))
    s -= s.mean(axis=0)
    x = rng.random((4, 3))
    a = Pd.ewald_sum(kernel, x, y, s, xi_l=3.0, nreal=3, nfour=12)
    b = Pd.ewald_sum(kernel, x, y, s, xi_l=5.5, nreal=3, nfour=14)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-13)
    c = Pd.ewald_sum(kernel, x, y, s)
    assert np.allclose(a, c, rtol=1e-12, atol=1e-13)
    # periodicity: move one source by a lattice vector (difference stays inside (-L, L)^3)
    y2 = y.copy()
    y2[0, 0] = y2[0, 0] - 1.0 if y2[0, 0] > 0.5 else y2[0, 0] + 1.0
    xs = np.clip(x, 0.0, 1.0)
    if np.all(np.abs(xs[:, None, :] - y2[None, :, :]) < 1.0):
        assert np.allclose(Pd.ewald_sum(kernel, xs, y2, s), Pd.ewald_sum(kernel, xs, y, s),
                           rtol=1e-11, atol=1e-12)


def _neutral(kernel, n, seed):
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    kt = 1 if kernel == "laplace" else 3
    s = rng.standard_normal((n, kt))
    return pts, s - s.mean(axis=0)


@pytest.mark.parametrize("problem,kernel", [("laplace", "laplace"), ("stokeslet_g", "stokeslet")])
def test_periodic_kafmm_converges_to_ewald_sum(problem, kernel):
    pts, s = _neutral(kernel, 400, seed=5)
    ref = Pd.ewald_sum(kernel, pts, pts, s)
    # the self images are part of the periodic sum; the KAFMM skips only the r = 0 self pair
    errs = []
    for p in (4, 6):
        T = Pd.t_m2l(kernel, p)
        F = KAFMM(problem, p, 16, bc="pxyz", t_m2l=T)
        g = F.evaluate(pts, s)
        assert F.tree.nlevels >= 3
        errs.append(D.rel_l2(g, ref))
    assert errs[1] < errs[0] / 8 and errs[1] < 5e-4, errs


def test_periodic_kafmm_translation_invariance():
    pts, s = _neutral("stokeslet", 300, seed=9)
    p = 6
    F = KAFMM("stokeslet_g", p, 16, bc="pxyz", t_m2l=Pd.t_m2l("stokeslet", p))
    g0 = F.evaluate(pts, s)
    shift = np.array([0.3719, 0.1183, 0.7242])
    g1 = F.evaluate((pts + shift) % 1.0, s)
    ref = Pd.ewald_sum("stokeslet", pts, pts, s)
    e_fmm = D.rel_l2(g0, ref)
    assert D.rel_l2(g1, g0) < 3 * e_fmm + 1e-12


@pytest.mark.parametrize("kernel", ["laplace", "stokeslet"])
def test_sampled_ewald_equals_converged_ewald_sum(kernel):
    """The structure-factor Ewald evaluation (used at full size, many sources, few targets)
    equals the pairwise Ewald sum converged to FP64 round-off, on targets that are sources
    (self images by the regular limit) and on targets that are not."""
    rng = np.random.default_rng(17)
    n = 300
    y = rng.random((n, 3))
    kq = 1 if kernel == "laplace" else 3
    s = rng.standard_normal((n, kq))
    s -= s.mean(axis=0)
    x = np.concatenate([y[:40], rng.random((40, 3))])
    ref = Pd.ewald_sum(kernel, x, y, s)
    got = Pd.ewald_sum_sampled(kernel, x, y, s, chunk=64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-11
    # a different cell size and split parameter give the same sum (scale and split invariance)
    got2 = Pd.ewald_sum_sampled(kernel, 2.0 * x, 2.0 * y, s, L=2.0, xi_l=11.0, kmax=18)
    scale = 0.5   # both kernels are homogeneous of degree -1
    assert np.linalg.norm(got2 - scale * ref) / np.linalg.norm(ref) < 1e-11
    # the cheaper split of the full-size checks: truncation erfc(4) ~ 1.5e-8
    got3 = Pd.ewald_sum_sampled(kernel, x, y, s, xi_l=8.0, kmax=12)
    assert np.linalg.norm(got3 - ref) / np.linalg.norm(ref) < 1e-7

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
import functools

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


def test_periodic_pvel_kernel_from_the_pinned_kernels():
    """Periodic StokesPVel block: u <- f is the (pinned) periodic Stokeslet; p <- f and u <- q
    are -f . grad G_per and (q/2) grad G_per, checked against central differences of the
    pinned periodic Laplace sum; p <- q is zero; the split parameter drops out."""
    rng = np.random.default_rng(31)
    y = rng.random((5, 3))
    x = rng.random((3, 3))
    sv = rng.standard_normal((5, 4))
    sv -= sv.mean(axis=0)
    g = Pd.ewald_sum("stokes_pvel", x, y, sv)
    assert np.allclose(g, Pd.ewald_sum("stokes_pvel", x, y, sv, xi_l=6.0, nreal=3, nfour=12),
                       rtol=1e-11, atol=1e-12)
    assert np.allclose(g[:, 1:] - Pd.ewald_sum("stokes_pvel", x, y, np.c_[np.zeros((5, 3)), sv[:, 3]])[:, 1:],
                       Pd.ewald_sum("stokeslet", x, y, sv[:, :3]), rtol=1e-12, atol=1e-13)
    h = 1e-5
    grad = np.zeros((len(x), 3, len(y)))   # d G_per(x_a - y_b) / d x_k
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        for b in range(len(y)):
            one = np.zeros(len(y))
            one[b] = 1.0
            gp = Pd.ewald_sum("laplace", x + e, y, one)[:, 0]
            gm = Pd.ewald_sum("laplace", x - e, y, one)[:, 0]
            grad[:, k, b] = (gp - gm) / (2 * h)
    p_ref = -np.einsum("akb,bk->a", grad, sv[:, :3])
    u_q = 0.5 * np.einsum("akb,b->ak", grad, sv[:, 3])
    only_q = Pd.ewald_sum("stokes_pvel", x, y, np.c_[np.zeros((5, 3)), sv[:, 3]])
    assert np.allclose(g[:, 0], p_ref, rtol=1e-7, atol=1e-8 * np.abs(p_ref).max())
    assert np.allclose(only_q[:, 1:], u_q, rtol=1e-7, atol=1e-8 * np.abs(u_q).max())
    assert np.abs(only_q[:, 0]).max() < 1e-13


def _force_pairs(y, Dm, eps=1e-6):
    """A double layer D at y as its definition's limit: force pairs -+sym(D)_{.k} / eps at
    y +- eps e_k / 2 and a source q = tr D at y ([f, q] records for the StokesPVel kernel)."""
    P, S = [], []
    for yi, Di in zip(y, Dm.reshape(-1, 3, 3)):
        Sy = 0.5 * (Di + Di.T)
        for k in range(3):
            e = np.zeros(3)
            e[k] = eps / 2
            f = -Sy[:, k] / eps
            P += [yi + e, yi - e]
            S += [np.r_[f, 0.0], np.r_[-f, 0.0]]
        P.append(yi)
        S.append(np.r_[0.0, 0.0, 0.0, np.trace(Sy)])
    return np.array(P), np.array(S)


@pytest.mark.parametrize("problem", ["stokes_pvel", "stokes_dl_pv", "stokes_pvel_grad"])
def test_periodic_pvel_table_kafmm_converges_to_ewald_sum(problem):
    """Periodic KAFMM on the StokesPVel table (far images through the root operator of the
    periodic StokesPVel kernel, plus the constant shifts of the moments equivalent densities do
    not carry) against the Ewald sum: [f, q] sources directly; double-layer sources through
    their force-pair limit (on targets away from the sources); the gradient outputs against
    central differences of the Ewald sum."""
    rng = np.random.default_rng(41)
    n = 300
    pts = rng.random((n, 3))
    x = rng.random((40, 3))
    if problem == "stokes_dl_pv":
        s = rng.standard_normal((n, 9))
        tr = s[:, 0] + s[:, 4] + s[:, 8]
        s[:, [0, 4, 8]] -= tr.mean() / 3.0
        P, S = _force_pairs(pts, s)
        ref = Pd.ewald_sum("stokes_pvel", x, P, S)
    else:
        s = rng.standard_normal((n, 4))
        s -= s.mean(axis=0)
        ref = Pd.ewald_sum("stokes_pvel", x, pts, s)
        if problem == "stokes_pvel_grad":
            h = 1e-5
            cols = [ref]
            cols.append(np.stack([(Pd.ewald_sum("stokes_pvel", x + h * e, pts, s)[:, 0]
                                   - Pd.ewald_sum("stokes_pvel", x - h * e, pts, s)[:, 0]) / (2 * h)
                                  for e in np.eye(3)], axis=1))
            du = np.stack([(Pd.ewald_sum("stokes_pvel", x + h * e, pts, s)[:, 1:]
                            - Pd.ewald_sum("stokes_pvel", x - h * e, pts, s)[:, 1:]) / (2 * h)
                           for e in np.eye(3)], axis=2)   # [target, i, j] = d u_i / d x_j
            cols.append(du.reshape(len(x), 9))
            ref = np.concatenate(cols, axis=1)
    errs = []
    for p in (6, 8):
        F = KAFMM(problem, p, 40, bc="pxyz", t_m2l=_pvel_t_m2l(p))
        errs.append(D.rel_l2(F.evaluate(pts, s, trg=x), ref))
    assert errs[1] < errs[0] / 4 and errs[1] < 1e-5, errs


@functools.lru_cache(maxsize=None)
def _pvel_t_m2l(p):
    return Pd.t_m2l("stokes_pvel", p)

"""Pins of the singly and doubly periodic oracle (``oracle.lattice``; boundaries PX and PXY of
Sec. III.B) against results fixed by the mathematics, not by the oracle's own formula:

* the doubly periodic Laplace sum equals the 2D Ewald sum (Parry's split: erfc real part, the
  Fourier modes of the plane with erfc-weighted exponentials in z, and the k = 0 plane term),
  which is independent of its splitting parameter;
* the singly periodic Laplace sum equals its Fourier series along the axis, whose modes are
  modified Bessel functions K_0 of the distance to the axis;
* the mean over the periodic directions satisfies the reduced equations: for a plane lattice
  the 1D Poisson / Stokes equations in z (a neutral layer gives a potential or velocity jump
  sum q z / A), for a line lattice the 2D Poisson / Stokes equations in the cross-section
  (line charges and line forces of strength s / L);
* periodicity along the lattice, invariance under a common shift, rejection of non-neutral
  sources;
* the interaction lists with wrap along some axes reach every pair of leaves exactly once;
* above a no-slip wall: the lattice sums of the image-system table equal the lattice sum of
  Blake's solution (and, for RPY, of its definition with the source Laplacian), and the plane
  mean is the layered shear flow fixed by the reduced 1D Stokes equation with no slip;
* the CPU KAFMM with the far-image operator converges to the lattice sum with the order and
  is invariant under a shift of all points along the periodic axes (the paper's translation
  test, Sec. III.B).
"""
import functools

import numpy as np
import pytest
from scipy.special import erf, erfc, k0

from oracle import direct as D
from oracle import lattice as La
from oracle import wall as Wl
from oracle.kafmm import KAFMM
from oracle.tree import Tree


def _neutral(n, ks, seed, lo=0.0, hi=1.0):
    rng = np.random.default_rng(seed)
    y = lo + (hi - lo) * rng.random((n, 3))
    s = rng.standard_normal((n, ks))
    return y, s - s.mean(axis=0)


def _ewald2d_laplace(x, y, q, alpha, kmax, nreal=4, L=1.0):
    """Doubly periodic sum of q / (4 pi r) by the 2D Ewald split (neutral charges)."""
    A = L * L
    out = np.zeros(len(x))
    sp = np.sqrt(np.pi)
    for i, xi in enumerate(x):
        d = xi - y
        z = d[:, 2]
        acc = 0.0
        for a in range(-nreal, nreal + 1):
            for b in range(-nreal, nreal + 1):
                r = np.linalg.norm(d + np.array([a * L, b * L, 0.0]), axis=1)
                acc += np.sum(q * erfc(alpha * r) / r)
        for a in range(-kmax, kmax + 1):
            for b in range(-kmax, kmax + 1):
                if a == 0 and b == 0:
                    continue
                kx, ky = 2 * np.pi * a / L, 2 * np.pi * b / L
                k = np.hypot(kx, ky)
                ph = np.cos(kx * d[:, 0] + ky * d[:, 1])
                acc += np.pi / A * np.sum(q * ph / k * (np.exp(k * z) * erfc(k / (2 * alpha) + alpha * z)
                                                        + np.exp(-k * z) * erfc(k / (2 * alpha) - alpha * z)))
        acc -= 2 * sp / A * np.sum(q * (np.exp(-(alpha * z) ** 2) / alpha + sp * z * erf(alpha * z)))
        out[i] = acc / (4 * np.pi)
    return out


def test_doubly_periodic_laplace_equals_2d_ewald():
    y, q = _neutral(12, 1, seed=1)
    x = np.random.default_rng(2).random((6, 3))
    e1 = _ewald2d_laplace(x, y, q[:, 0], alpha=3.0, kmax=30)
    e2 = _ewald2d_laplace(x, y, q[:, 0], alpha=5.0, kmax=40)
    assert np.abs(e1 - e2).max() < 1e-13 * np.abs(e1).max()   # split independence
    g = La.lattice_sum("laplace", x, y, q, "pxy")[:, 0]
    assert np.abs(g - e1).max() < 2e-9 * np.abs(e1).max(), np.abs(g - e1).max()


def test_singly_periodic_laplace_equals_bessel_series():
    y, q = _neutral(10, 1, seed=3)
    rng = np.random.default_rng(4)
    x = rng.random((200, 3))
    rho = np.hypot(x[:, None, 1] - y[None, :, 1], x[:, None, 2] - y[None, :, 2])
    x = x[rho.min(axis=1) > 0.08][:8]
    assert len(x) >= 4
    ref = np.zeros(len(x))
    m = np.arange(1, 160)
    for i, xi in enumerate(x):
        dx = xi[0] - y[:, 0]
        r = np.hypot(xi[1] - y[:, 1], xi[2] - y[:, 2])
        modes = k0(2 * np.pi * np.outer(r, m)) * np.cos(2 * np.pi * np.outer(dx, m))
        ref[i] = np.sum(q[:, 0] * (-2 * np.log(r) + 4 * modes.sum(axis=1))) / (4 * np.pi)
    g = La.lattice_sum("laplace", x, y, q, "px")[:, 0]
    assert np.abs(g - ref).max() < 1e-10 * np.abs(ref).max(), np.abs(g - ref).max()


def _plane_grid(z, M=16, L=1.0):
    a = (np.arange(M) + 0.37) * L / M
    X, Y = np.meshgrid(a, a, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(M * M, z)], axis=1)


@pytest.mark.parametrize("kernel", ["laplace", "stokeslet"])
def test_doubly_periodic_plane_mean_solves_1d_equation(kernel):
    """Mean over x, y: -d2/dz2 mean = sum s delta(z - z_j) / A (Laplace; the Stokeslet's
    tangential components alike with mu = 1, its normal component constant = 0)."""
    ks = 1 if kernel == "laplace" else 3
    y, s = _neutral(20, ks, seed=6, lo=0.3, hi=0.7)
    for z in (-0.1, 1.15, 0.52):
        xs = _plane_grid(z)
        g = La.lattice_sum(kernel, xs, y, s, "pxy").mean(axis=0)
        w = -0.5 * np.abs(z - y[:, 2])
        if kernel == "laplace":
            ref = np.array([np.sum(w * s[:, 0])])
        else:
            ref = np.array([np.sum(w * s[:, 0]), np.sum(w * s[:, 1]), 0.0])
        if z == 0.52:
            # inside the source layer the other Fourier modes do not vanish on the grid: only
            # the jump across the layer is checked there (next loop)
            continue
        assert np.abs(g - ref).max() < 1e-9 * np.abs(s).max(), (z, g, ref)
    # the jump across the layer: sum s_j z_j / A
    lo = La.lattice_sum(kernel, _plane_grid(-0.2), y, s, "pxy").mean(axis=0)
    hi = La.lattice_sum(kernel, _plane_grid(1.2), y, s, "pxy").mean(axis=0)
    jump = s.T @ y[:, 2]
    if kernel == "laplace":
        assert abs((hi - lo)[0] - jump[0]) < 1e-9
    else:
        assert np.abs((hi - lo)[:2] - jump[:2]).max() < 1e-9 and abs(hi[2] - lo[2]) < 1e-9


@pytest.mark.parametrize("kernel", ["laplace", "stokeslet"])
def test_singly_periodic_line_mean_solves_2d_equation(kernel):
    """Mean over x: the 2D free-space solution of line charges / line forces s / L
    (Laplace: -ln(rho) / (2 pi L); Stokeslet: axial -ln(rho) / (2 pi L), cross-section
    (-ln(rho) I + rho rho^T / rho^2) / (4 pi L)), exact for neutral sources."""
    ks = 1 if kernel == "laplace" else 3
    y, s = _neutral(16, ks, seed=7, lo=0.35, hi=0.65)
    M = 16
    for (py, pz) in ((1.3, 0.5), (0.5, -0.4), (-0.2, 1.1)):
        xs = np.stack([(np.arange(M) + 0.21) / M, np.full(M, py), np.full(M, pz)], axis=1)
        g = La.lattice_sum(kernel, xs, y, s, "px").mean(axis=0)
        d = np.array([py, pz]) - y[:, 1:]
        r2 = np.sum(d * d, axis=1)
        lg = -0.5 * np.log(r2)
        if kernel == "laplace":
            ref = np.array([np.sum(s[:, 0] * lg) / (2 * np.pi)])
        else:
            ux = np.sum(s[:, 0] * lg) / (2 * np.pi)
            dF = np.sum(d * s[:, 1:], axis=1)
            uc = (lg[:, None] * s[:, 1:] + d * (dF / r2)[:, None]).sum(axis=0) / (4 * np.pi)
            ref = np.array([ux, uc[0], uc[1]])
        assert np.abs(g - ref).max() < 1e-9 * np.abs(s).max(), (g, ref)


@pytest.mark.parametrize("bc", ["px", "pxy"])
def test_lattice_sum_periodic_and_shift_invariant(bc):
    y, s = _neutral(24, 3, seed=8)
    x = np.random.default_rng(9).random((10, 3))
    g = La.lattice_sum("stokeslet", x, y, s, bc)
    e = np.array([1.0, 0.0, 0.0]) if bc == "px" else np.array([0.0, 1.0, 0.0])
    # targets one period away sit off centre in the truncation window, where the plane's
    # extrapolation (N <= 128) is good to about 1e-8
    tol = 1e-12 if bc == "px" else 1e-7
    assert D.rel_l2(La.lattice_sum("stokeslet", x + e, y, s, bc), g) < tol
    sh = np.array([0.317, 0.0 if bc == "px" else 0.622, 0.0])
    g2 = La.lattice_sum("stokeslet", (x + sh) % 1.0, (y + sh) % 1.0, s, bc)
    assert D.rel_l2(g2, g) < tol


def test_lattice_sum_rejects_non_neutral_sources():
    y, s = _neutral(8, 1, seed=10)
    with pytest.raises(ValueError):
        La.lattice_sum("laplace", y, y, s + 0.1, "pxy")


@pytest.mark.parametrize("axes", ["x", "xy"])
def test_lists_with_partial_wrap_reach_every_pair_once(axes):
    rng = np.random.default_rng(11)
    pts = np.concatenate([rng.random((150, 3)), 0.5 + 0.1 * rng.standard_normal((150, 3))])
    T = Tree(np.clip(pts, 0, 0.999), q=12, periodic=axes)
    lv = T.leaves()
    assert len(lv) > 20 and T.nlevels >= 3
    for b in range(T.nbox):
        T.U[b], T.V[b], T.W[b], T.X[b] = set(T.U[b]), set(T.V[b]), set(T.W[b]), set(T.X[b])
    shifts = T._shifts()
    assert len(shifts) == (3 if axes == "x" else 9)
    assert all(sh[2] == 0 and (axes == "xy" or sh[1] == 0) for sh in shifts)
    bad = [(tb, sb, sh) for tb in lv for sb in lv for sh in shifts if T.route_count(tb, sb, sh) != 1]
    assert not bad


@functools.lru_cache(maxsize=None)
def _t(ml, p, bc):
    return La.t_m2l(ml, p, bc)


@pytest.mark.parametrize("bc", ["px", "pxy"])
@pytest.mark.parametrize("problem,kernel,ml", [("laplace", "laplace", "laplace"),
                                               ("stokeslet_g", "stokeslet", "stokeslet")])
def test_kafmm_converges_to_lattice_sum(bc, problem, kernel, ml):
    ks = 1 if kernel == "laplace" else 3
    pts, s = _neutral(200, ks, seed=12)
    ref = La.lattice_sum(kernel, pts, pts, s, bc)
    errs = []
    for p in (4, 6):
        F = KAFMM(problem, p, 16, bc=bc, t_m2l=_t(ml, p, bc))
        errs.append(D.rel_l2(F.evaluate(pts, s), ref))
        assert F.tree.nlevels >= 3
    assert errs[1] < errs[0] / 10 and errs[1] < 3e-4, errs


def test_kafmm_doubly_periodic_translation_invariance():
    pts, s = _neutral(200, 3, seed=13)
    p = 6
    F = KAFMM("stokeslet_g", p, 16, bc="pxy", t_m2l=_t("stokeslet", p, "pxy"))
    g0 = F.evaluate(pts, s)
    sh = np.array([0.4137, 0.2291, 0.0])
    g1 = F.evaluate((pts + sh) % 1.0, s)
    ref = La.lattice_sum("stokeslet", pts, pts, s, "pxy")
    e = D.rel_l2(g0, ref)
    assert D.rel_l2(g1, g0) < 3 * e + 1e-12, (D.rel_l2(g1, g0), e)


def _above(n, seed, lo=0.6, hi=0.9):
    rng = np.random.default_rng(seed)
    y = rng.random((n, 3))
    y[:, 2] = lo + (hi - lo) * y[:, 2]
    return y, rng.standard_normal((n, 3))


@pytest.mark.parametrize("bc", ["px", "pxy"])
def test_periodic_wall_table_equals_blake_lattice_sum(bc):
    """The wall's three neutral sums over the lattice, assembled (Table tab:rpywall, b = 0),
    equal the lattice sum of Blake's closed-form image system for forces with a net part."""
    y, f = _above(10, seed=14)
    x, _ = _above(6, seed=15, lo=0.5, hi=1.0)
    a = La.wall_blake(x, y, f, bc, 0.5)
    b = La.wall_table(x, y, f, bc, 0.5)
    assert D.rel_l2(b, a) < 1e-10


def test_doubly_periodic_wall_mean_flow_is_the_layered_shear():
    """Mean over x, y above a wall at z_w with no slip: d2/dz2 mean u = -sum f delta(z - z_j) / A
    and mean u = 0 on the wall, so the tangential mean is sum f_j min(z - z_w, h_j) / A (a shear
    below each layer, uniform above it) and the normal mean vanishes."""
    y, f = _above(8, seed=16, lo=0.75, hi=0.8)
    M = 24
    a = (np.arange(M) + 0.37) / M
    X, Y = np.meshgrid(a, a, indexing="ij")
    for z in (0.53, 0.99):
        xs = np.stack([X.ravel(), Y.ravel(), np.full(M * M, z)], axis=1)
        u = La.wall_blake(xs, y, f, "pxy", 0.5).mean(axis=0)
        w = np.minimum(z - 0.5, y[:, 2] - 0.5)
        ref = np.array([np.sum(f[:, 0] * w), np.sum(f[:, 1] * w), 0.0])
        assert np.abs(u - ref).max() < 1e-8 * np.abs(ref).max(), (z, u, ref)


def test_periodic_rpy_wall_table_equals_the_definition():
    """RPY above the wall, singly periodic: the lattice sums of the four table sums, assembled,
    equal the lattice sum of the definition (1 + b^2/6 lap_y) G_wall f."""
    rng = np.random.default_rng(17)
    y, f = _above(3, seed=17, lo=0.65, hi=0.85)
    fb = np.concatenate([f, rng.uniform(0.02, 0.05, (3, 1))], axis=1)
    x, _ = _above(4, seed=18, lo=0.55, hi=0.95)
    ref = La._extrapolated(lambda xs: Wl.blake_rpy(xs, y, fb, 0.5), x, 3, "px", 1.0, 16, 6)
    got = La.wall_rpy_table(x, y, fb, "px", 0.5)[:, :3]
    assert D.rel_l2(got, ref) < 1e-9


def test_doubly_periodic_pvel_and_double_layer_plane_means():
    """Mean over x, y outside a layer of StokesPVel and double-layer sources (1D Stokes
    equations with mu = 1): forces give the tangential flow -sum f |z - z_j| / (2A) and no
    normal flow; a source q sends -q / (4A) each way (its flux -q/2 split between the two
    sides); a double layer D is the force dipole -sym(D) plus the source tr D, so the mean flow
    jumps by -(D_az + D_za) / (2A) tangentially and by -tr D / (2A) normally across it."""
    rng = np.random.default_rng(19)
    y = 0.3 + 0.4 * rng.random((20, 3))
    s = rng.standard_normal((20, 4))
    s[:, :3] -= s[:, :3].mean(axis=0)
    for z in (-0.2, 1.2):
        g = La.lattice_sum("stokes_pvel", _plane_grid(z), y, s, "pxy").mean(axis=0)
        sg, dz = np.sign(z - y[:, 2]), np.abs(z - y[:, 2])
        ref = np.array([np.sum(s[:, 2] * sg) / 2, -0.5 * np.sum(s[:, 0] * dz), -0.5 * np.sum(s[:, 1] * dz),
                        -np.sum(s[:, 3] * sg) / 4])
        assert np.abs(g - ref).max() < 1e-8, (z, g, ref)
    Dd = rng.standard_normal((20, 9))
    lo = La.lattice_sum("stokes_dl", _plane_grid(-0.2), y, Dd, "pxy").mean(axis=0)
    hi = La.lattice_sum("stokes_dl", _plane_grid(1.2), y, Dd, "pxy").mean(axis=0)
    Dm = Dd.reshape(-1, 3, 3)
    jump = np.array([0.0, -np.sum(Dm[:, 0, 2] + Dm[:, 2, 0]) / 2, -np.sum(Dm[:, 1, 2] + Dm[:, 2, 1]) / 2,
                     -np.sum(np.trace(Dm, axis1=1, axis2=2)) / 2])
    assert np.abs((hi - lo) - jump).max() < 1e-8, (hi - lo, jump)


@pytest.mark.parametrize("bc,problem,kernel", [("px", "stokes_pvel", "stokes_pvel"),
                                               ("pxy", "stokes_dl_pv", "stokes_dl")])
def test_kafmm_pvel_table_converges_to_lattice_sum(bc, problem, kernel):
    """The StokesPVel table ([f, q] and double-layer sources) with the far-image operator of
    the line or plane lattice converges to the lattice sum: unlike the triply periodic Ewald
    convention, the real-space image sums depend only on the field outside the cell, so no
    moment shifts enter."""
    rng = np.random.default_rng(20)
    pts = rng.random((200, 3))
    ks = 4 if kernel == "stokes_pvel" else 9
    s = rng.standard_normal((200, ks))
    if ks == 4:
        s[:, :3] -= s[:, :3].mean(axis=0)
    ref = La.lattice_sum(kernel, pts, pts, s, bc)
    errs = [D.rel_l2(KAFMM(problem, p, 16, bc=bc, t_m2l=_t("stokes_pvel", p, bc)).evaluate(pts, s), ref)
            for p in (4, 6)]
    assert errs[1] < errs[0] / 10 and errs[1] < 1e-3, errs

"""Pins for the oracle's direct kernel sums (oracle/direct.c).

Each test checks the oracle against something other than its own formula: conservation laws
(Gauss's law, momentum balance, the double-layer net flux stated in Sec. II.C), PDEs the
kernels solve (checked by finite differences), textbook special cases (equal-radius RPY and
its overlap form), symmetry, and the SPD property of the RPY mobility (Sec. II.B).
"""
import numpy as np
import pytest

from oracle import direct as D

PI = np.pi


def sphere_quadrature(R, centre=(0.0, 0.0, 0.0), nt=40, nphi=80):
    """Gauss-Legendre in cos(theta) x trapezoid in phi: nodes, outward normals, weights."""
    ct, wt = np.polynomial.legendre.leggauss(nt)
    phi = np.arange(nphi) * 2 * PI / nphi
    st = np.sqrt(1 - ct ** 2)
    n = np.stack([np.outer(st, np.cos(phi)), np.outer(st, np.sin(phi)),
                  np.outer(ct, np.ones(nphi))], axis=-1).reshape(-1, 3)
    w = np.outer(wt, np.full(nphi, 2 * PI / nphi)).reshape(-1) * R * R
    return np.asarray(centre) + R * n, n, w


def fd_grad(fun, x, h=1e-4):
    """Central-difference gradient of a vector field: returns [..., comp, dir]."""
    out = []
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        out.append((fun(x + e) - fun(x - e)) / (2 * h))
    return np.stack(out, axis=-1)


def fd_laplacian(fun, x, h=1e-3):
    acc = -6.0 * fun(x)
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        acc = acc + fun(x + e) + fun(x - e)
    return acc / (h * h)


def test_surface_point_count_formula():
    """M = 6(m-1)^2 + 2 boundary nodes of an m^3 grid (Sec. III) = m^3 - (m-2)^3."""
    from oracle.kafmm import surface
    for m in range(2, 17):
        assert len(surface(m)) == 6 * (m - 1) ** 2 + 2 == m ** 3 - (m - 2) ** 3


def test_laplace_gauss_law_and_harmonic():
    """Flux of grad phi through any sphere around a charge q is -q; phi is harmonic."""
    y = np.array([[0.1, -0.2, 0.05]])
    q = np.array([[0.7]])
    for R in (0.3, 1.7):
        pts, n, w = sphere_quadrature(R, centre=(0.2, -0.1, 0.0))
        g = D.direct("laplace_pgradgrad", pts, y, q)
        flux = np.sum(w * np.sum(g[:, 1:4] * n, axis=1))
        assert abs(flux + 0.7) < 1e-10
    x = np.array([0.9, 0.4, -0.3])
    lap = fd_laplacian(lambda z: D.direct("laplace", z[None], y, q)[0, 0], x)
    assert abs(lap) < 1e-5


def test_laplace_derivatives_match_finite_differences():
    rng = np.random.default_rng(7)
    y = rng.random((5, 3))
    q = rng.standard_normal((5, 1))
    x = np.array([1.3, -0.4, 0.8])
    g = D.direct("laplace_pgradgrad", x[None], y, q)[0]
    assert abs(g[0] - D.direct("laplace", x[None], y, q)[0, 0]) < 1e-14
    grad = fd_grad(lambda z: D.direct("laplace", z[None], y, q)[0], x)[0]
    assert np.allclose(g[1:4], grad, rtol=1e-7, atol=1e-9)
    hess = fd_grad(lambda z: D.direct("laplace_pgradgrad", z[None], y, q)[0, 1:4], x)
    h6 = [hess[0, 0], hess[0, 1], hess[0, 2], hess[1, 1], hess[1, 2], hess[2, 2]]
    assert np.allclose(g[4:10], h6, rtol=1e-6, atol=1e-8)
    assert abs(g[4] + g[7] + g[9]) < 1e-10 * np.abs(g[4:10]).max()  # trace-free (harmonic)


def test_laplace_dipole_is_limit_of_charge_pair():
    """A dipole d = q e (e -> 0) equals charges +q at y + e/2 and -q at y - e/2."""
    y = np.array([0.2, 0.3, -0.1])
    d = np.array([0.4, -1.1, 0.6])
    x = np.array([[1.0, 0.5, 0.7], [-0.6, 0.2, 0.4]])
    eps = 1e-5
    ys = np.stack([y + eps * d / 2, y - eps * d / 2])
    pair = D.direct("laplace", x, ys, np.array([1.0 / eps, -1.0 / eps]))
    dip = D.direct("laplace_dipole", x, y[None], d[None])
    assert np.allclose(dip, pair, rtol=1e-8)


def test_stokeslet_divergence_free_symmetric_and_stokes_equation():
    rng = np.random.default_rng(3)
    y = rng.random((3, 3))
    f = rng.standard_normal((3, 3))
    x = np.array([1.4, 0.9, -0.5])
    ufun = lambda z: D.direct("stokeslet", z[None], y, f)[0]
    J = fd_grad(ufun, x)
    assert abs(np.trace(J)) < 1e-6 * np.abs(J).max()           # div u = 0 (Sec. II.C)
    # lap u = grad p with p the pressure of Eq. stkslp, taken here as -div of the Laplace
    # potentials of the force components (a route independent of the Stokeslet routine)
    pfun = lambda z: -sum(D.direct("laplace_pgradgrad", z[None], y, f[:, j])[0, 1 + j]
                          for j in range(3))
    lap_u = fd_laplacian(ufun, x)
    gp = fd_grad(lambda z: np.array([pfun(z)]), x)[0]
    assert np.allclose(lap_u, gp, rtol=1e-5, atol=1e-7)
    # symmetry G(x, y) = G(y, x)^T
    a, b = np.array([[0.1, 0.2, 0.3]]), np.array([[0.7, -0.2, 0.5]])
    Gab = np.stack([D.direct("stokeslet", a, b, e[None])[0] for e in np.eye(3)], axis=1)
    Gba = np.stack([D.direct("stokeslet", b, a, e[None])[0] for e in np.eye(3)], axis=1)
    assert np.allclose(Gab, Gba.T, rtol=1e-14)


def test_stokeslet_momentum_balance_fixes_normalisation():
    """For u = G f and p = f.r/(4 pi r^3): the traction sigma.n = (-p I + grad u + grad u^T) n
    integrates to -f over any sphere around the point force (div sigma = -f delta)."""
    f = np.array([[0.3, -1.2, 0.8]])
    y = np.zeros((1, 3))
    pts, n, w = sphere_quadrature(0.5, nt=24, nphi=48)
    tot = np.zeros(3)
    for xk, nk, wk in zip(pts, n, w):
        J = fd_grad(lambda z: D.direct("stokeslet", z[None], y, f)[0], xk, h=1e-5)
        p = -sum(D.direct("laplace_pgradgrad", xk[None], y, f[:, j])[0, 1 + j] for j in range(3))
        sig = -p * np.eye(3) + J + J.T
        tot += wk * sig @ nk
    assert np.allclose(tot, -f[0], rtol=1e-6, atol=1e-7)


def test_rpy_equal_radius_is_classical_rpy_and_biharmonic():
    """[u, lap u] assembled as u + a^2/6 lap u (Eq. RPYtrgvel) with b = a equals the classical
    Rotne-Prager tensor (1/8 pi r)[(1 + 2a^2/3r^2) I + (1 - 2a^2/r^2) rr/r^2] for r > 2a."""
    a = 0.05
    y = np.array([[0.0, 0.0, 0.0]])
    x = np.array([[0.31, -0.12, 0.2]])
    r = x[0] - y[0]
    rn = np.linalg.norm(r)
    for e in np.eye(3):
        g = D.direct("rpy", x, y, np.concatenate([e, [a]])[None])[0]
        ua = g[:3] + a * a / 6.0 * g[3:]
        ref = ((1 + 2 * a * a / (3 * rn * rn)) * e
               + (1 - 2 * a * a / (rn * rn)) * r * (r @ e) / (rn * rn)) / (8 * PI * rn)
        assert np.allclose(ua, ref, rtol=1e-14, atol=1e-16)
    # lap lap G = 0 (Sec. II.B): the Laplacian output is harmonic
    fb = np.array([[0.2, 0.5, -0.4, 0.01]])
    lap2 = fd_laplacian(lambda z: D.direct("rpy", z[None], y, fb)[0, 3:], np.array([0.6, 0.3, 0.2]))
    assert np.abs(lap2).max() < 1e-4 * np.abs(D.direct("rpy", x, y, fb)[0, 3:]).max()
    # lap u output equals the finite-difference Laplacian of the Stokeslet field
    ufun = lambda z: D.direct("stokeslet", z[None], y, fb[:, :3])[0]
    lapu = fd_laplacian(ufun, np.array([0.6, 0.3, 0.2]))
    assert np.allclose(D.direct("rpy", np.array([[0.6, 0.3, 0.2]]), y, fb)[0, 3:], lapu,
                       rtol=1e-5)


def test_rpy_far_tends_to_stokeslet():
    """RPY -> Stokeslet as a/r -> 0 with relative difference O(a^2/r^2)."""
    y = np.zeros((1, 3))
    x = np.array([[0.4, 0.3, -0.2]])
    f = np.array([0.3, 0.1, -0.7])
    u0 = D.direct("stokeslet", x, y, f[None])[0]
    prev = None
    for b in (1e-1, 1e-2, 1e-3):
        u = D.direct("rpy", x, y, np.concatenate([f, [b]])[None])[0, :3]
        rel = np.linalg.norm(u - u0) / np.linalg.norm(u0)
        if prev is not None:
            assert 80 < prev / rel < 120      # quadratic in b
        prev = rel


def test_rpy_overlap_continuity_and_equal_radius_form():
    rng = np.random.default_rng(11)
    rhat = rng.standard_normal(3)
    rhat /= np.linalg.norm(rhat)
    for ai, aj in ((0.03, 0.05), (0.05, 0.05), (0.02, 0.09)):
        s, d = ai + aj, abs(ai - aj)
        out = D.rpy_pair(rhat * s * (1 + 1e-12), ai, aj)
        inn = D.rpy_pair(rhat * s * (1 - 1e-12), ai, aj)
        assert np.allclose(out, inn, rtol=1e-9)                     # continuous at contact
        if d > 0:
            o2 = D.rpy_pair(rhat * d * (1 + 1e-12), ai, aj)
            i2 = D.rpy_pair(rhat * d * (1 - 1e-12), ai, aj)
            assert np.allclose(o2, i2, rtol=1e-9, atol=1e-12)       # continuous inside
            assert np.allclose(i2, np.eye(3) / (6 * PI * max(ai, aj)), rtol=1e-14)
    a = 0.04
    for r in (0.01, 0.05, 0.079):
        m = D.rpy_pair(rhat * r, a, a)
        ref = ((1 - 9 * r / (32 * a)) * np.eye(3)
               + (3 * r / (32 * a)) * np.outer(rhat, rhat)) / (6 * PI * a)
        assert np.allclose(m, ref, rtol=1e-13)
    assert np.allclose(D.rpy_pair(np.zeros(3), a, a), np.eye(3) / (6 * PI * a))


def test_rpy_mobility_is_symmetric_positive_definite():
    """The RPY mobility of a set of (overlapping, polydisperse) spheres is SPD (Sec. II.B)."""
    rng = np.random.default_rng(5)
    n = 40
    x = 0.3 * rng.random((n, 3))
    a = rng.uniform(0.02, 0.06, n)
    Mob = np.zeros((3 * n, 3 * n))
    for i in range(n):
        Mob[3 * i:3 * i + 3, 3 * i:3 * i + 3] = np.eye(3) / (6 * PI * a[i])
        for j in range(n):
            if i != j:
                Mob[3 * i:3 * i + 3, 3 * j:3 * j + 3] = D.rpy_pair(x[i] - x[j], a[i], a[j])
    assert np.abs(Mob - Mob.T).max() < 1e-12 * np.abs(Mob).max()
    assert np.linalg.eigvalsh(Mob).min() > 0
    # and rpy_velocity is that matrix without the self blocks
    f = rng.standard_normal((n, 3))
    u = D.rpy_velocity(x, a, x, np.concatenate([f, a[:, None]], axis=1), same_set=True)
    off = Mob.copy()
    for i in range(n):
        off[3 * i:3 * i + 3, 3 * i:3 * i + 3] = 0
    assert np.allclose(u.reshape(-1), off @ f.reshape(-1), rtol=1e-12)


def test_rpy_overlap_correction_matches_brute_force_velocity():
    """kernel sum [u, lap u] + assembly + overlap correction == brute-force pair mobility."""
    rng = np.random.default_rng(9)
    n = 60
    x = 0.25 * rng.random((n, 3))
    a = rng.uniform(0.01, 0.05, n)
    f = rng.standard_normal((n, 3))
    fb = np.concatenate([f, a[:, None]], axis=1)
    g = D.direct("rpy", x, x, fb)
    ua = g[:, :3] + (a[:, None] ** 2 / 6.0) * g[:, 3:]
    ua = D.rpy_overlap_correction(x, a, x, fb, same_set=True, g=ua)
    ref = D.rpy_velocity(x, a, x, fb, same_set=True)
    assert np.allclose(ua, ref, rtol=1e-11, atol=1e-12)


def test_double_layer_net_flux_and_stokes_equation():
    """Net flow out of a sphere around a tensor source D is -1/2 tr D, for any radius
    (Sec. II.C); the double-layer flow is divergence-free away from the source and solves
    lap u = grad p with its own pressure (Eq. stkdlp)."""
    rng = np.random.default_rng(2)
    Dm = rng.standard_normal((3, 3))
    y = np.zeros((1, 3))
    for R in (0.2, 3.0):
        pts, n, w = sphere_quadrature(R)
        u = D.direct("stokes_dl", pts, y, Dm.reshape(1, 9))[:, 1:]
        assert abs(np.sum(w * np.sum(u * n, axis=1)) + 0.5 * np.trace(Dm)) < 1e-10
    x = np.array([0.5, -0.3, 0.4])
    fun = lambda z: D.direct("stokes_dl", z[None], y, Dm.reshape(1, 9))[0]
    lap = fd_laplacian(lambda z: fun(z)[1:], x)
    gp = fd_grad(lambda z: fun(z)[:1], x)[0]
    assert np.allclose(lap, gp, rtol=1e-5, atol=1e-6)
    # p is harmonic: its FD Laplacian is truncation-sized against the scale |p| / |x|^2
    assert abs(fd_laplacian(lambda z: fun(z)[0], x)) < 1e-3 * abs(fun(x)[0]) / (x @ x)
    J = fd_grad(lambda z: fun(z)[1:], x)
    assert abs(np.trace(J)) < 1e-6 * np.abs(J).max()


def test_two_point_roundoff_under_translation():
    """The paper's two-point test (Sec. III.B): translating a pair at distance ~1e-4 changes
    the FP64 kernel value by ~1e-12 relative, from the rounding of r alone."""
    rng = np.random.default_rng(4)
    y = np.array([[0.3, 0.6, 0.1]])
    x = y + 1e-4 * rng.standard_normal((1, 3)) / np.sqrt(3)
    f = np.array([[1.0, -0.5, 0.25]])
    errs = []
    for _ in range(20):
        t = rng.random(3) * 7.0
        u0 = D.direct("stokeslet", x, y, f)
        u1 = D.direct("stokeslet", x + t, y + t, f)
        errs.append(D.rel_l2(u1, u0))
    assert 1e-15 < np.median(errs) < 1e-10


def _blob(rr, eps):
    """Spreading function of the regularized Stokeslet (Sec. II.B), integral 1."""
    return 15 * eps ** 4 / (8 * PI * (rr + eps * eps) ** 3.5)


def test_regularized_stokeslet_limits_and_divergence():
    """eps = 0 gives the Stokeslet; the regularized flow is divergence-free (it is the Stokes
    flow of a spread force); far from the blob G^eps = G + (eps^2/4) lap G + O(eps^4 / r^5):
    with b^2 / 6 = eps^2 / 4 the oracle's RPY field is G + (eps^2/4) lap G, and the
    remainder drops 16-fold when eps halves."""
    rng = np.random.default_rng(31)
    y = rng.random((4, 3))
    f = rng.standard_normal((4, 3))
    x = rng.random((5, 3)) + 1.0
    s0 = np.concatenate([f, np.zeros((4, 1))], axis=1)
    assert np.allclose(D.direct("stokeslet_reg", x, y, s0), D.direct("stokeslet", x, y, f),
                       rtol=1e-13, atol=0)
    eps = np.array([0.3, 0.5, 0.2, 0.7])
    s = np.concatenate([f, eps[:, None]], axis=1)
    xt = np.array([0.6, 0.4, 0.7])   # within a blob width of the sources
    J = fd_grad(lambda z: D.direct("stokeslet_reg", z[None], y, s)[0], xt, h=1e-5)
    assert abs(np.trace(J)) < 1e-8 * np.abs(J).max()
    one = np.array([[0.0, 0.0, 0.0]])
    xr = np.array([[0.6, -0.5, 0.62]])   # |r| = 1
    res = []
    for e in (0.02, 0.01):
        ureg = D.direct("stokeslet_reg", xr, one, np.array([[0.3, -1.1, 0.7, e]]))
        urpy = D.direct("rpy", xr, one, np.array([[0.3, -1.1, 0.7, np.sqrt(1.5) * e]]))[:, :3]
        res.append(np.abs(ureg - urpy).max())
    assert 15.5 < res[0] / res[1] < 16.5, res


@pytest.mark.parametrize("eps,xt", [(0.5, (0.5, 0.4, -0.3)), (0.2, (0.1, -0.25, 0.12))])
def test_regularized_stokeslet_is_the_flow_of_the_blob_force(eps, xt):
    """u(x) = int G(x - y) psi_eps(y) dy f (Sec. II.B: the force f spread by the blob psi_eps
    around the source), by quadrature in spherical coordinates about the target: with z =
    x - y = rho n, G(z) dz = (I + n n^T) rho / (8 pi) drho dOmega, a smooth integrand.
    Panels of Gauss-Legendre in rho (tail rho > 6 mapped to (0, 1]), Gauss-Legendre in the
    cosine of the angle to x and trapezoid in the azimuth."""
    x = np.array(xt)
    f = np.array([0.4, -0.9, 1.3])
    ez = x / np.linalg.norm(x)
    ex = np.cross(ez, [0.3, 0.5, 0.8])
    ex /= np.linalg.norm(ex)
    ey = np.cross(ez, ex)
    ct, wt = np.polynomial.legendre.leggauss(96)
    phi = np.arange(64) * 2 * PI / 64
    st = np.sqrt(1 - ct ** 2)
    n = (ct[:, None, None] * ez + (st[:, None] * np.cos(phi))[:, :, None] * ex
         + (st[:, None] * np.sin(phi))[:, :, None] * ey).reshape(-1, 3)
    wang = np.outer(wt, np.full(64, 2 * PI / 64)).reshape(-1)
    gl, gw = np.polynomial.legendre.leggauss(24)
    edges = np.concatenate([np.linspace(0, 2, 21), [3, 4, 6]])
    rho, wr = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        rho.append(0.5 * (b - a) * gl + 0.5 * (a + b))
        wr.append(0.5 * (b - a) * gw)
    t = 0.5 * gl + 0.5                                # rho = 6 / t on (0, 1]
    rho.append(6 / t)
    wr.append(0.5 * gw * 6 / t ** 2)
    rho, wr = np.concatenate(rho), np.concatenate(wr)
    u = np.zeros(3)
    for rk, wk in zip(rho, wr):
        y = x - rk * n                                  # source points of this shell
        psi = _blob(np.sum(y * y, axis=1), eps)
        nf = n @ f
        u += wk * rk / (8 * PI) * ((wang * psi) @ (f[None, :] + n * nf[:, None]))
    ref = D.direct("stokeslet_reg", x[None], np.zeros((1, 3)), np.concatenate([f, [eps]])[None])[0]
    assert np.allclose(u, ref, rtol=1e-8, atol=1e-10), (u, ref)


def test_laplace_charge_dipole_gradients_and_hessian():
    """[q, d] -> [phi, grad phi, grad grad phi] (Table tab:ktab_lapqdpgradgrad): charges alone
    equal the charge routine, the potential of dipoles alone equals the (separately pinned)
    dipole potential, the gradient and Hessian equal central differences of the potential
    and of the gradient, and the Hessian is trace-free (phi is harmonic off the sources)."""
    rng = np.random.default_rng(41)
    y = rng.random((5, 3))
    sv = rng.standard_normal((5, 4))
    x = np.array([[1.3, 0.7, -0.4], [0.2, 1.9, 1.1]])
    q_only = sv.copy()
    q_only[:, 1:] = 0
    assert np.allclose(D.direct("laplace_qd", x, y, q_only), D.direct("laplace_pgradgrad", x, y, sv[:, :1]),
                       rtol=1e-13, atol=0)
    d_only = sv.copy()
    d_only[:, 0] = 0
    assert np.allclose(D.direct("laplace_qd", x, y, d_only)[:, 0],
                       D.direct("laplace_dipole", x, y, sv[:, 1:])[:, 0], rtol=1e-13, atol=0)
    hidx = {(0, 0): 4, (0, 1): 5, (0, 2): 6, (1, 1): 7, (1, 2): 8, (2, 2): 9}
    for xt in x:
        g = D.direct("laplace_qd", xt[None], y, sv)[0]
        phi = lambda z: D.direct("laplace_qd", z[None], y, sv)[0, :1]
        grad = lambda z: D.direct("laplace_qd", z[None], y, sv)[0, 1:4]
        assert np.allclose(fd_grad(phi, xt, h=1e-5)[0], g[1:4], rtol=1e-7, atol=1e-9)
        H = fd_grad(grad, xt, h=1e-5)
        for (i, j), k in hidx.items():
            assert np.isclose(H[i, j], g[k], rtol=1e-6, atol=1e-8)
        assert abs(g[4] + g[7] + g[9]) < 1e-12 * np.abs(g[4:]).max()


def test_stokes_pvel_pressure_source_and_stokes_equation():
    """StokesPVel [f, q] -> [p, u] (Eqs. stkslp, stkslvel): with q = 0 the velocity is the
    Stokeslet's and the pressure is -sum_j d_j (f_j / (4 pi r)) (from the Laplace oracle);
    the flow out of any sphere around the source is -q / 2 (the net flow a double layer
    leaves, -1/2 tr D, is matched by q = tr D); lap u = grad p and div u = 0 off the source."""
    rng = np.random.default_rng(51)
    y = rng.random((3, 3))
    sv = rng.standard_normal((3, 4))
    x = np.array([[1.4, 0.9, -0.5], [-0.3, 1.7, 0.8]])
    f_only = sv.copy()
    f_only[:, 3] = 0
    g = D.direct("stokes_pvel", x, y, f_only)
    assert np.allclose(g[:, 1:], D.direct("stokeslet", x, y, sv[:, :3]), rtol=1e-13, atol=0)
    for k, xt in enumerate(x):
        p_ref = -sum(D.direct("laplace_pgradgrad", xt[None], y, sv[:, j])[0, 1 + j] for j in range(3))
        assert np.isclose(g[k, 0], p_ref, rtol=1e-13)
    one = np.zeros((1, 3))
    src = np.array([[0.7, -0.4, 1.1, 2.3]])
    for R in (0.3, 2.5):
        pts, n, w = sphere_quadrature(R)
        u = D.direct("stokes_pvel", pts, one, src)[:, 1:]
        assert abs(np.sum(w * np.sum(u * n, axis=1)) + 0.5 * src[0, 3]) < 1e-10
    xt = np.array([0.5, -0.3, 0.4])
    fun = lambda z: D.direct("stokes_pvel", z[None], y, sv)[0]
    lap = fd_laplacian(lambda z: fun(z)[1:], xt)
    gp = fd_grad(lambda z: fun(z)[:1], xt)[0]
    assert np.allclose(lap, gp, rtol=1e-5, atol=1e-6)
    J = fd_grad(lambda z: fun(z)[1:], xt)
    assert abs(np.trace(J)) < 1e-6 * np.abs(J).max()


def test_direct_sums_do_not_depend_on_the_thread_count():
    """The OpenMP loops split targets only: one thread and all threads give the same bits."""
    rng = np.random.default_rng(61)
    y = rng.random((500, 3))
    f = rng.standard_normal((500, 3))
    x = rng.random((64, 3))
    g_all = D.direct("stokeslet", x, y, f)
    prev = D.set_threads(1)
    try:
        g_one = D.direct("stokeslet", x, y, f)
    finally:
        D.set_threads(prev)
    assert np.array_equal(g_all, g_one)


@pytest.mark.parametrize("base,ks", [("stokes_pvel", 4), ("stokes_dl", 9)])
def test_derivative_kernels_against_finite_differences(base, ks):
    """PVelGrad / PVelLaplacian / Traction target values (Tables tab:ktab_stkslpvelgrad,
    tab:ktab_stkdlpvelgrad, Eq. stressdef) against central differences of the [p, u] kernel
    (pinned above): grad p, grad u and lap u by finite differences, [p, u] unchanged; the
    traction assembled from those differences."""
    rng = np.random.default_rng(61 if ks == 4 else 62)
    y = rng.random((4, 3))
    sv = rng.standard_normal((4, ks))
    fun = lambda z: D.direct(base, z[None], y, sv)[0]
    for xt in (np.array([1.3, 0.2, -0.6]), np.array([0.45, 0.5, 0.55]), np.array([-0.7, 1.9, 0.9])):
        pu = fun(xt)
        gr = D.direct(base + "_grad", xt[None], y, sv)[0]
        lp = D.direct(base + "_lapl", xt[None], y, sv)[0]
        tr = D.direct(base + "_traction", xt[None], y, sv)[0]
        assert np.allclose(gr[:4], pu, rtol=1e-13, atol=1e-15)
        assert np.allclose(lp[:4], pu, rtol=1e-13, atol=1e-15)
        J = fd_grad(fun, xt, h=1e-5)                       # [component, direction]
        scale = np.abs(J).max()
        assert np.allclose(gr[4:7], J[0], rtol=1e-6, atol=1e-7 * scale)
        assert np.allclose(gr[7:].reshape(3, 3), J[1:], rtol=1e-6, atol=1e-7 * scale)
        # Richardson-extrapolated 7-point Laplacian (error O(h^4))
        l1 = fd_laplacian(lambda z: fun(z)[1:], xt, h=2e-3)
        l2 = fd_laplacian(lambda z: fun(z)[1:], xt, h=1e-3)
        lap = (4.0 * l2 - l1) / 3.0
        assert np.allclose(lp[4:], lap, rtol=1e-6, atol=1e-6 * np.abs(lap).max())
        sig = -pu[0] * np.eye(3) + J[1:] + J[1:].T
        assert np.allclose(tr.reshape(3, 3), sig, rtol=1e-6, atol=1e-7 * scale)


@pytest.mark.parametrize("base,ks", [("stokes_pvel", 4), ("stokes_dl", 9)])
def test_derivative_kernels_solve_stokes(base, ks):
    """Off the sources the fields are Stokes flows: lap u (worked out from the velocity) equals
    grad p (worked out from the pressure), div u = tr grad u = 0 (the PVel source term q is a
    potential flow), and the traction is symmetric with trace -3 p."""
    rng = np.random.default_rng(63 if ks == 4 else 64)
    y = rng.random((6, 3))
    sv = rng.standard_normal((6, ks))
    x = rng.random((20, 3)) * 3 - 1
    gr = D.direct(base + "_grad", x, y, sv)
    lp = D.direct(base + "_lapl", x, y, sv)
    tr = D.direct(base + "_traction", x, y, sv).reshape(-1, 3, 3)
    scale = np.abs(gr[:, 4:7]).max()
    assert np.allclose(lp[:, 4:], gr[:, 4:7], rtol=1e-11, atol=1e-12 * scale)
    G = gr[:, 7:].reshape(-1, 3, 3)
    assert np.abs(np.trace(G, axis1=1, axis2=2)).max() < 1e-12 * np.abs(G).max()
    assert np.allclose(tr, np.transpose(tr, (0, 2, 1)), rtol=0, atol=1e-13 * np.abs(tr).max())
    assert np.allclose(np.trace(tr, axis1=1, axis2=2), -3 * gr[:, 0], rtol=1e-11,
                       atol=1e-12 * np.abs(gr[:, 0]).max())


def test_laplace_quadrupole_against_the_pinned_dipole_kernel():
    """Quadrupoles Q -> [phi, grad phi, grad grad phi] (LapQPGradGrad): phi = Q_jk d_j d_k L is
    minus the divergence of dipole potentials, phi_Q = -sum_k d_k phi_D(d = Q_{., k}), checked by
    central differences of the pinned dipole kernel; grad phi_Q = -sum_k H_D(Q_{., k})_{ik} from
    the pinned charge + dipole Hessian; the Hessian by central differences of the gradient, and
    trace-free (phi_Q is harmonic off the sources)."""
    rng = np.random.default_rng(71)
    y = rng.random((3, 3))
    Q = rng.standard_normal((3, 9))
    hidx = {(0, 0): 4, (0, 1): 5, (0, 2): 6, (1, 1): 7, (1, 2): 8, (2, 2): 9}
    for xt in (np.array([1.4, -0.3, 0.8]), np.array([0.2, 0.9, -0.6])):
        g = D.direct("laplace_quad", xt[None], y, Q)[0]
        phi_ref = 0.0
        grad_ref = np.zeros(3)
        for k in range(3):
            dk = Q.reshape(3, 3, 3)[:, :, k]           # dipoles Q_{., k} of every source
            fun = lambda z, dk=dk: D.direct("laplace_dipole", z[None], y, dk)[0, :1]
            phi_ref -= fd_grad(fun, xt, h=1e-5)[0, k]
            qd = np.concatenate([np.zeros((3, 1)), dk], axis=1)
            Hd = D.direct("laplace_qd", xt[None], y, qd)[0]
            for i in range(3):
                grad_ref[i] -= Hd[hidx[(min(i, k), max(i, k))]]
        assert np.isclose(g[0], phi_ref, rtol=1e-7, atol=1e-9)
        assert np.allclose(g[1:4], grad_ref, rtol=1e-12, atol=1e-13 * np.abs(grad_ref).max())
        H = fd_grad(lambda z: D.direct("laplace_quad", z[None], y, Q)[0, 1:4], xt, h=1e-5)
        for (i, j), k in hidx.items():
            assert np.isclose(H[i, j], g[k], rtol=1e-6, atol=1e-8 * np.abs(g[4:]).max())
        assert abs(g[4] + g[7] + g[9]) < 1e-12 * np.abs(g[4:]).max()

"""ORACLE -- triply periodic sums (test infrastructure).

The paper imposes periodicity with a precomputed operator that adds the far field of the
periodic images and depends only on the M->L kernel (Sec. III, App. B).  Its construction is
in the authors' earlier work and not in the paper; the reading used here:

* The tree, with its lists taken modulo the cube, covers every source image whose shift n lies
  in {-1, 0, 1}^3.  All images with max|n| >= 2 enter through
      T_M2L[i, j] = G_per(dc_i - ue_j) - sum_{max|n| <= 1} K(dc_i - ue_j - n L),
  applied to the root's upward equivalent density and added to the root's downward check
  potential (dc, ue: the root's surfaces).
* G_per is the Ewald sum with the k = 0 mode removed (zero-mean field; the sources must be
  neutral / force-free), evaluated in C (``direct.c``: Laplace, the Stokeslet by Hasimoto's
  splitting, and StokesPVel from the two: its pressure of a force and flow of a source are
  gradients of the Laplace Green's function).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import direct as D
from .kafmm import ALPHA, ml_matrix, surface

# Ewald parameters: xi L = 4; real images |n| <= 2 (erfc(8) ~ 1e-29), Fourier |m| <= 8
# (exp(-pi^2 m^2 / 16) ~ 7e-18 at m = 8) -- converged to FP64 round-off.
XI_L, NREAL, NFOUR = 4.0, 2, 8


def _lib():
    L = D.lib()
    if not hasattr(L, "_ewald_ready"):
        p, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        L.orc_ewald_sum.argtypes = [i32, p, i64, p, i64, p, dbl, dbl, i32, i32, p]
        L.orc_ewald_matrix.argtypes = [i32, p, i64, p, i64, dbl, dbl, i32, i32, p]
        L.orc_ewald_real_mi.argtypes = [i32, p, i64, p, i64, p, dbl, dbl, dbl, p]
        L._ewald_ready = True
    return L


_KID = {"laplace": (0, 1), "stokeslet": (1, 3), "stokes_pvel": (2, 4)}


def ewald_sum(kernel: str, x, y, s, L=1.0, xi_l=XI_L, nreal=NREAL, nfour=NFOUR):
    """sum_b K_per(x_a - y_b) s_b (FP64); kernel 'laplace', 'stokeslet' or 'stokes_pvel'
    ([f, q] -> [p, u])."""
    kid, kt = _KID[kernel]
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, 3))
    y = np.ascontiguousarray(np.asarray(y, np.float64).reshape(-1, 3))
    s = np.ascontiguousarray(np.asarray(s, np.float64).reshape(len(y), kt))
    g = np.zeros((len(x), kt))
    _lib().orc_ewald_sum(kid, x.ctypes.data, len(x), y.ctypes.data, len(y), s.ctypes.data,
                         float(L), xi_l / L, nreal, nfour, g.ctypes.data)
    return g


def ewald_matrix(kernel: str, x, y, L=1.0, xi_l=XI_L, nreal=NREAL, nfour=NFOUR):
    kid, kt = _KID[kernel]
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, 3))
    y = np.ascontiguousarray(np.asarray(y, np.float64).reshape(-1, 3))
    out = np.zeros((kt * len(x), kt * len(y)))
    _lib().orc_ewald_matrix(kid, x.ctypes.data, len(x), y.ctypes.data, len(y), float(L),
                            xi_l / L, nreal, nfour, out.ctypes.data)
    return out


def t_m2l(ml: str, p: int, L=1.0, origin=0.0):
    """The far-image operator of the root (real coordinates), maps the root's upward
    equivalent density to its downward check potential."""
    unit = surface(p)
    r0 = L / 2.0
    c = origin + r0
    dc = c + ALPHA["dc"] * r0 * unit
    ue = c + ALPHA["ue"] * r0 * unit
    T = ewald_matrix(ml, dc, ue, L)
    for n in [(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)]:
        with np.errstate(divide="ignore", invalid="ignore"):
            K = ml_matrix(ml, dc, ue + np.array(n) * L)
        # dc and ue coincide point by point (both at 1.05 half-widths): there the Ewald
        # routine already returned the regular limit (own images only), so the n = 0 term
        # is absent for those entries
        T -= np.where(np.isfinite(K), K, 0.0)
    return T


def ewald_sum_sampled(kernel: str, x, y, s, L=1.0, xi_l=10.0, kmax=16, chunk=16384):
    """The same periodic sum as :func:`ewald_sum` for many sources and few targets (FP64).

    Ewald's split with the Fourier part through structure factors,
        S_q(k) = sum_b s_bq exp(-i k.y_b),   k = 2 pi m / L,  |m|_inf <= kmax,
    one per pair {k, -k} (half space, weight 2), evaluated at the targets as
    (1/V) sum_k 2 w(k) Re[exp(i k.x) M(k) S(k)] with w, M of the blocks in ``direct.c``
    (Laplace: w = exp(-k^2/4xi^2)/k^2, M = 1; Stokeslet: w = (1 + k^2/4xi^2) exp(-k^2/4xi^2)/k^2,
    M = I - k k^T/k^2), and the real part in C with the minimum image and cutoff L/2.  With
    xi L = 10 and kmax = 16 both truncations are below 1e-12 (erfc(5), exp(-pi^2 17^2/100)).
    The structure factors are contracted axis by axis: exp(-i k.y) = e_x^a e_y^b e_z^c, the
    (a, b) factors per source times the (c, q) factors, summed over sources by a matrix
    product."""
    kid = 0 if kernel == "laplace" else 1
    kq = 1 if kid == 0 else 3
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, 3))
    y = np.ascontiguousarray(np.asarray(y, np.float64).reshape(-1, 3))
    s = np.ascontiguousarray(np.asarray(s, np.float64).reshape(len(y), kq))
    xi = xi_l / L
    V = L ** 3
    g = np.zeros((len(x), kq))
    _lib().orc_ewald_real_mi(kid, x.ctypes.data, len(x), y.ctypes.data, len(y), s.ctypes.data,
                             float(L), xi, L / 2.0, g.ctypes.data)
    if kid == 0:
        g[:, 0] += -s[:, 0].sum() / (4.0 * xi * xi * V)
    tw = 2.0 * np.pi / L
    ma = np.arange(0, kmax + 1)
    mb = np.arange(-kmax, kmax + 1)
    na, nb = len(ma), len(mb)
    S = np.zeros((na * nb, nb * kq), dtype=np.complex128)
    for j0 in range(0, len(y), chunk):
        yc, sc = y[j0:j0 + chunk], s[j0:j0 + chunk]
        ex = np.exp(-1j * tw * np.outer(ma, yc[:, 0]))
        ey = np.exp(-1j * tw * np.outer(mb, yc[:, 1]))
        ez = np.exp(-1j * tw * np.outer(mb, yc[:, 2]))
        xy = (ex[:, None, :] * ey[None, :, :]).reshape(na * nb, -1)
        zs = (ez[:, None, :] * sc.T[None, :, :]).reshape(nb * kq, -1)
        S += xy @ zs.T
    S = S.reshape(na, nb, nb, kq)
    A, B, C = np.meshgrid(ma, mb, mb, indexing="ij")
    half = (A > 0) | ((A == 0) & ((B > 0) | ((B == 0) & (C > 0))))
    kv = tw * np.stack([A[half], B[half], C[half]], axis=1).astype(np.float64)
    Sh = S[half]                                   # [nk, kq]
    k2 = np.sum(kv * kv, axis=1)
    e = np.exp(-k2 / (4.0 * xi * xi))
    if kid == 0:
        P = (2.0 * e / k2 / V)[:, None] * Sh
    else:
        w = 2.0 * (1.0 + k2 / (4.0 * xi * xi)) * e / k2 / V
        kS = np.sum(kv * Sh, axis=1)               # k . S(k)
        P = w[:, None] * (Sh - kv * (kS / k2)[:, None])
    for i0 in range(0, len(x), 256):
        E = np.exp(1j * (x[i0:i0 + 256] @ kv.T))  # [nt, nk]
        g[i0:i0 + 256] += (E @ P).real
    return g

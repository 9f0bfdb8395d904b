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
  neutral / force-free), evaluated in C (``direct.c``: Laplace, and the Stokeslet by
  Hasimoto's splitting).
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
        L._ewald_ready = True
    return L


def ewald_sum(kernel: str, x, y, s, L=1.0, xi_l=XI_L, nreal=NREAL, nfour=NFOUR):
    """sum_b K_per(x_a - y_b) s_b (FP64); kernel 'laplace' or 'stokeslet'."""
    kid = 0 if kernel == "laplace" else 1
    kt = 1 if kid == 0 else 3
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, 3))
    y = np.ascontiguousarray(np.asarray(y, np.float64).reshape(-1, 3))
    s = np.ascontiguousarray(np.asarray(s, np.float64).reshape(len(y), kt))
    g = np.zeros((len(x), kt))
    _lib().orc_ewald_sum(kid, x.ctypes.data, len(x), y.ctypes.data, len(y), s.ctypes.data,
                         float(L), xi_l / L, nreal, nfour, g.ctypes.data)
    return g


def ewald_matrix(kernel: str, x, y, L=1.0, xi_l=XI_L, nreal=NREAL, nfour=NFOUR):
    kid = 0 if kernel == "laplace" else 1
    kt = 1 if kid == 0 else 3
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

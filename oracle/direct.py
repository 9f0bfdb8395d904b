"""ORACLE O1 -- direct FP64 kernel sums (test infrastructure).

The definition of the result (Eq. kernelsumlinear, Sec. I): g_i(x_a) = sum_b K_ij(x_a, y_b) s_j(y_b),
evaluated pair by pair in C (``direct.c``).  Pairs at zero distance are skipped, which removes
the self term when sources and targets are one set.

Kernels (dimensions k_s x k_t, Table tab:implement):
  laplace            q -> phi                     1 x 1   (Sec. II.A)
  laplace_pgradgrad  q -> phi, grad, grad grad    1 x 10  (Table tab:ktab_lapqdpgradgrad)
  laplace_dipole     d -> phi                     3 x 1   (Sec. II.A)
  laplace_qd         [q, d] -> phi, grad, grad grad  4 x 10  (Table tab:ktab_lapqdpgradgrad)
  laplace_quad       Q -> phi, grad, grad grad    9 x 10  (LapQPGradGrad, Table tab:implement)
  stokeslet          f -> u                       3 x 3   (Sec. II.B)
  stokeslet_reg      [f, eps] -> u                4 x 3   (regularized Stokeslet, Table tab:ktab_reg)
  stokes_pvel        [f, q] -> [p, u]             4 x 4   (StokesPVel, Eqs. stkslp, stkslvel)
  rpy                [f, b] -> [u, lap u]         4 x 6   (Eqs. RPYflow, RPYkernel)
  stokes_dl          D -> [p, u]                  9 x 4   (Eqs. stkdlp, stkdlvel)
  stokes_pvel_grad   [f, q] -> [p, u, grad p, grad u]  4 x 16  (Table tab:ktab_stkslpvelgrad)
  stokes_pvel_lapl   [f, q] -> [p, u, lap u]      4 x 7   (Table tab:ktab_stkslpvelgrad)
  stokes_pvel_traction [f, q] -> sigma            4 x 9   (Eq. stressdef, mu = 1)
  stokes_dl_grad     D -> [p, u, grad p, grad u]  9 x 16  (Table tab:ktab_stkdlpvelgrad)
  stokes_dl_lapl     D -> [p, u, lap u]           9 x 7   (Table tab:ktab_stkdlpvelgrad)
  stokes_dl_traction D -> sigma                   9 x 9   (Eq. stressdef, mu = 1)
grad u is d u_i / d x_j at 3 i + j; sigma_ij = -p delta_ij + d_j u_i + d_i u_j at 3 i + j.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_lib = None

KDIM = {  # kernel -> (k_s, k_t)
    "laplace": (1, 1),
    "laplace_pgradgrad": (1, 10),
    "laplace_dipole": (3, 1),
    "laplace_qd": (4, 10),
    "laplace_quad": (9, 10),
    "stokeslet": (3, 3),
    "stokeslet_reg": (4, 3),
    "stokes_pvel": (4, 4),
    "rpy": (4, 6),
    "stokes_dl": (9, 4),
    "stokes_pvel_grad": (4, 16),
    "stokes_pvel_lapl": (4, 7),
    "stokes_pvel_traction": (4, 9),
    "stokes_dl_grad": (9, 16),
    "stokes_dl_lapl": (9, 7),
    "stokes_dl_traction": (9, 9),
}


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        p = ctypes.c_void_p
        i64 = ctypes.c_int64
        for name in KDIM:
            fn = getattr(_lib, "orc_" + name)
            fn.argtypes = [p, i64, p, i64, p, p]
            fn.restype = None
        for name in ("orc_rpy_velocity", "orc_rpy_overlap_correction"):
            fn = getattr(_lib, name)
            fn.argtypes = [p, p, i64, p, i64, p, ctypes.c_int, p]
            fn.restype = None
        _lib.orc_rpy_pair.argtypes = [p, ctypes.c_double, ctypes.c_double, p]
        _lib.orc_rpy_pair.restype = None
        _lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib.orc_set_threads.restype = ctypes.c_int
    return _lib


def set_threads(n: int) -> int:
    """Threads of the direct sums (n > 0); returns the previous maximum."""
    return int(lib().orc_set_threads(int(n)))


def _f64(a, shape1=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape1 is not None:
        a = a.reshape(-1, shape1)
    return a


def direct(kernel: str, x, y, s, g=None) -> np.ndarray:
    """g += sum over sources of K(x, y) s, FP64.  Returns g ([nt, k_t])."""
    ks, kt = KDIM[kernel]
    x = _f64(x, 3)
    y = _f64(y, 3)
    s = _f64(s, ks)
    assert s.shape[0] == y.shape[0]
    if g is None:
        g = np.zeros((x.shape[0], kt))
    assert g.dtype == np.float64 and g.flags.c_contiguous and g.shape == (x.shape[0], kt)
    if x.shape[0] and y.shape[0]:
        getattr(lib(), "orc_" + kernel)(x.ctypes.data, x.shape[0], y.ctypes.data, y.shape[0],
                                        s.ctypes.data, g.ctypes.data)
    return g


def rpy_pair(r, ai: float, aj: float) -> np.ndarray:
    """3x3 RPY pair mobility (far form outside contact, overlap form inside)."""
    r = _f64(r).reshape(3)
    m = np.zeros(9)
    lib().orc_rpy_pair(r.ctypes.data, float(ai), float(aj), m.ctypes.data)
    return m.reshape(3, 3)


def rpy_velocity(x, a, y, fb, same_set: bool) -> np.ndarray:
    """Sphere velocities sum_b M(x_a - y_b; a_a, b_b) f_b with the overlap form, brute force."""
    x = _f64(x, 3)
    y = _f64(y, 3)
    a = _f64(a).reshape(-1)
    fb = _f64(fb, 4)
    g = np.zeros((x.shape[0], 3))
    lib().orc_rpy_velocity(x.ctypes.data, a.ctypes.data, x.shape[0], y.ctypes.data,
                           y.shape[0], fb.ctypes.data, int(same_set), g.ctypes.data)
    return g


def rpy_overlap_correction(x, a, y, fb, same_set: bool, g=None) -> np.ndarray:
    """g += sum over overlapping pairs of (M_overlap - M_far) f (brute force over all pairs)."""
    x = _f64(x, 3)
    y = _f64(y, 3)
    a = _f64(a).reshape(-1)
    fb = _f64(fb, 4)
    if g is None:
        g = np.zeros((x.shape[0], 3))
    lib().orc_rpy_overlap_correction(x.ctypes.data, a.ctypes.data, x.shape[0], y.ctypes.data,
                                     y.shape[0], fb.ctypes.data, int(same_set), g.ctypes.data)
    return g


def rel_l2(a, b) -> float:
    """Relative L2 error ||a - b|| / ||b|| over all entries (Sec. III, eps_L2)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))

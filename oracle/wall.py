"""ORACLE -- Stokeslet above a no-slip wall (test infrastructure).

The paper (Sec. III.C, Table tab:rpywall with b = 0) evaluates the flow of point forces above a
no-slip wall as one Stokeslet sum and two Laplace charge + dipole sums over the sources and
their mirror images, assembled at the targets as
    u = u^S + grad phi^SDZ + x_3 grad phi^SD - [0, 0, phi^SD]       (wall at x_3 = 0),
with the Laplace kernels L = 1/(4 pi r), L^D = -dL/dx (Sec. II.A).  Two definitions here:

* ``blake`` -- the direct sum of Blake's closed-form image system (``direct.c``), the plain
  definition of the result;
* ``table`` -- the paper's three sums, each a direct FP64 sum, assembled as above.

Reading: the printed table gives the Laplace charges of phi^SD as f_3 at y and -f_3 at y^I;
with those the assembled field vanishes on the wall but is not the flow of the force f (its
normal part has another strength).  The charges -f_3 / 2 at y and +f_3 / 2 at y^I make the
assembly equal Blake's solution to round-off, and are used everywhere (source heights
h = y_3 above the wall):
    u^S:    f_12 = (f_1, f_2, 0) at y,  -f_12 at y^I                       (Stokeslet)
    SD:     charge -f_3 / 2 at y;  charge f_3 / 2 and dipole h (-f_1, -f_2, f_3) at y^I
    SDZ:    charge h f_3 / 2 at y;  charge -h f_3 / 2 at y^I
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import direct as D


def _lib():
    L = D.lib()
    if not hasattr(L, "_wall_ready"):
        p, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        L.orc_stokeslet_wall.argtypes = [p, i64, p, i64, p, dbl, p]
        L._wall_ready = True
    return L


def blake(x, y, f, zw=0.0):
    """sum_b of Blake's wall Stokeslet at x from forces f at y (all above x_3 = zw), FP64."""
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, 3))
    y = np.ascontiguousarray(np.asarray(y, np.float64).reshape(-1, 3))
    f = np.ascontiguousarray(np.asarray(f, np.float64).reshape(-1, 3))
    g = np.zeros((len(x), 3))
    _lib().orc_stokeslet_wall(x.ctypes.data, len(x), y.ctypes.data, len(y), f.ctypes.data, float(zw),
                              g.ctypes.data)
    return g


def images(y, zw=0.0):
    yI = np.array(y, dtype=np.float64, copy=True).reshape(-1, 3)
    yI[:, 2] = 2.0 * zw - yI[:, 2]
    return yI


def table_sources(y, f, zw=0.0):
    """Sources of the three sums over [y; y^I]: Stokeslet forces [2n, 3], the SD charges and
    dipoles [2n, 4] and the SDZ charges and dipoles [2n, 4] (see the module docstring)."""
    y = np.asarray(y, np.float64).reshape(-1, 3)
    f = np.asarray(f, np.float64).reshape(-1, 3)
    n = len(y)
    h = y[:, 2] - zw
    fs = np.zeros((2 * n, 3))
    fs[:n, :2] = f[:, :2]
    fs[n:, :2] = -f[:, :2]
    sd = np.zeros((2 * n, 4))
    sd[:n, 0] = -0.5 * f[:, 2]
    sd[n:, 0] = 0.5 * f[:, 2]
    sd[n:, 1] = -h * f[:, 0]
    sd[n:, 2] = -h * f[:, 1]
    sd[n:, 3] = h * f[:, 2]
    sdz = np.zeros((2 * n, 4))
    sdz[:n, 0] = 0.5 * h * f[:, 2]
    sdz[n:, 0] = -0.5 * h * f[:, 2]
    return fs, sd, sdz


def assemble(x, uS, sd_out, sdz_out, zw=0.0):
    """u = u^S + grad phi^SDZ + x_3 grad phi^SD - [0, 0, phi^SD]; sd_out, sdz_out are the
    [phi, grad phi, ...] outputs of the Laplace sums (columns 0..3 used)."""
    x3 = (np.asarray(x, np.float64).reshape(-1, 3)[:, 2] - zw)[:, None]
    u = uS + sdz_out[:, 1:4] + x3 * sd_out[:, 1:4]
    u[:, 2] -= sd_out[:, 0]
    return u


def table(x, y, f, zw=0.0):
    """The paper's three sums as direct FP64 sums over the sources and their images."""
    x = np.asarray(x, np.float64).reshape(-1, 3)
    y = np.asarray(y, np.float64).reshape(-1, 3)
    yy = np.concatenate([y, images(y, zw)])
    fs, sd, sdz = table_sources(y, f, zw)
    uS = D.direct("stokeslet", x, yy, fs)
    sd_out = D.direct("laplace_qd", x, yy, sd)
    sdz_out = D.direct("laplace_qd", x, yy, sdz)
    return assemble(x, uS, sd_out, sdz_out, zw)

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

RPY kernel above the wall (Table tab:rpywall with radius b > 0).  The plain definition is the
RPY kernel sum's source operator applied to Blake's solution, u = (1 + b^2/6 lap_y) G_wall f
(``blake_rpy``: the y-Laplacian by a Richardson-extrapolated central difference, error
O(h^4)).  The table's four sums, assembled as
    u     = u^S + grad phi^SDZ + x_3 grad phi^SD + x_3 grad phi^Q - [0, 0, phi^SD + phi^Q],
    lap u = lap u^S + 2 d_3 grad (phi^SD + phi^Q),
with, besides the Stokeslet reading above:
    u^S:    RPY sum of (f_12, b) at y and (-f_12, b) at y^I     ([u, lap u] per target)
    SDZ:    adds the dipole (b^2/6) (0, 0, f_3) at y and at y^I
    Q:      the quadrupole (b^2/3) [[f_3, 0, 0], [0, f_3, 0], [f_1, f_2, 0]] (phi = Q_jk d_j d_k L)
Reading: the table prints the quadrupole under "source at y" with 0 at y^I; placed at y^I it
makes the assembly equal (1 + b^2/6 lap_y) of Blake's solution (a least-squares fit of the
candidate b^2 terms to that definition gives coefficient 1/3 at y^I and 0 at y), and is used
everywhere.
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


def blake_rpy(x, y, fb, zw=0.0, h=2e-4):
    """u = sum_b (1 + b_b^2 / 6 lap_y) G_wall(x, y_b) f_b (RPY kernel sum above the wall), FP64;
    fb = [f, b] per source.  lap_y by the 7-point stencil at h and h / 2, Richardson-extrapolated.
    A target on a source gets only that source's image field (the free-space self pair is left
    out, as in every kernel sum here).  Sources must lie more than h above the wall."""
    x = np.asarray(x, np.float64).reshape(-1, 3)
    y = np.asarray(y, np.float64).reshape(-1, 3)
    fb = np.asarray(fb, np.float64).reshape(-1, 4)
    u = blake(x, y, fb[:, :3], zw)
    for j in range(len(y)):
        b = fb[j, 3]
        if b == 0.0:
            continue
        f = fb[j:j + 1, :3]
        on = np.all(x == y[j], axis=1)          # targets on this source: image part only

        def g(yj):
            v = blake(x, yj, f, zw)
            if on.any():
                v[on] -= D.direct("stokeslet", x[on], yj, f)
            return v
        c = g(y[j:j + 1])
        lap = []
        for hh in (h, 0.5 * h):
            acc = -6.0 * c
            for k in range(3):
                e = np.zeros(3)
                e[k] = hh
                acc = acc + g(y[j:j + 1] + e) + g(y[j:j + 1] - e)
            lap.append(acc / (hh * hh))
        u += b * b / 6.0 * (4.0 * lap[1] - lap[0]) / 3.0
    return u


def rpy_table_sources(y, fb, zw=0.0):
    """Sources of the four sums over [y; y^I] (module docstring): RPY [2n, 4] (f_12, b), SD and
    SDZ charges + dipoles [2n, 4], quadrupoles [2n, 9] (Q_jk at 3j + k)."""
    y = np.asarray(y, np.float64).reshape(-1, 3)
    fb = np.asarray(fb, np.float64).reshape(-1, 4)
    f, b = fb[:, :3], fb[:, 3]
    n = len(y)
    _, sd, sdz = table_sources(y, f, zw)
    rpy = np.zeros((2 * n, 4))
    rpy[:n, :2] = f[:, :2]
    rpy[n:, :2] = -f[:, :2]
    rpy[:n, 3] = b
    rpy[n:, 3] = b
    bb = b * b
    sdz[:n, 3] += bb / 6.0 * f[:, 2]
    sdz[n:, 3] += bb / 6.0 * f[:, 2]
    quad = np.zeros((2 * n, 9))
    quad[n:, 0] = bb / 3.0 * f[:, 2]
    quad[n:, 4] = bb / 3.0 * f[:, 2]
    quad[n:, 6] = bb / 3.0 * f[:, 0]
    quad[n:, 7] = bb / 3.0 * f[:, 1]
    return rpy, sd, sdz, quad


def rpy_assemble(x, rpy_out, sd_out, sdz_out, q_out, zw=0.0):
    """[u, lap u] from the four sums' target values: rpy_out [u, lap u] (6), the Laplace sums
    [phi, grad phi, Hessian xx xy xz yy yz zz] (10)."""
    x3 = (np.asarray(x, np.float64).reshape(-1, 3)[:, 2] - zw)[:, None]
    u = rpy_out[:, :3] + sdz_out[:, 1:4] + x3 * (sd_out[:, 1:4] + q_out[:, 1:4])
    u[:, 2] -= sd_out[:, 0] + q_out[:, 0]
    h = sd_out + q_out
    lap = rpy_out[:, 3:6] + 2.0 * h[:, [6, 8, 9]]   # 2 d_3 grad(phi^SD + phi^Q): xz, yz, zz
    return np.concatenate([u, lap], axis=1)


def rpy_table(x, y, fb, zw=0.0):
    """The paper's four sums as direct FP64 sums over the sources and their images."""
    x = np.asarray(x, np.float64).reshape(-1, 3)
    y = np.asarray(y, np.float64).reshape(-1, 3)
    yy = np.concatenate([y, images(y, zw)])
    rpy, sd, sdz, quad = rpy_table_sources(y, fb, zw)
    return rpy_assemble(x, D.direct("rpy", x, yy, rpy), D.direct("laplace_qd", x, yy, sd),
                        D.direct("laplace_qd", x, yy, sdz), D.direct("laplace_quad", x, yy, quad), zw)

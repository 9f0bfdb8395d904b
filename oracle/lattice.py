"""ORACLE -- singly and doubly periodic sums (test infrastructure).

The paper offers periodicity along one axis (PX), two axes (PXY) or all three (PXYZ) for every
kernel, through a precomputed operator that adds the far field of the periodic images to the
root (Sec. III.B, Table tab:implement; the construction is in the authors' earlier work, not in
the paper).  The reading used here for PX and PXY:

* Lattice: images y + n L with n = (a, 0, 0) (PX) or n = (a, b, 0) (PXY); the other axes are
  open.  Sources must be neutral in the kernel's monopole (sum of q = 0 for Laplace charges,
  sum of f = 0 for Stokeslet-type forces): a net charge or force makes the image sum diverge
  (logarithmically along a line, linearly over a plane).
* The periodic sum is the limit of the symmetric square-shell truncations
      g_N(x) = sum_{max|n| <= N} sum_b K(x - y_b - n L) s_b,   N -> infinity,
  which exists for neutral sources (the dipole-type terms of n and -n cancel, what remains
  falls off like 1/N).  The limit is taken by Richardson extrapolation of the partial sums at
  N = n0 2^k (the tail is a power series in 1/N: a lattice sum of smooth functions over the
  cells outside a square, expanded by the midpoint rule).  Over a plane, with N up to 128,
  the extrapolated sum is within about 1e-9 of the 2D Ewald sum; along a line, with N up to
  2048, within rounding of the Bessel series (both pinned in the tests).
* KAFMM (``kafmm.KAFMM`` with bc 'px' or 'pxy'): the tree covers the images with shift in
  {-1, 0, 1} along the periodic axes (lists with wrap, ``tree.Tree``); all farther images
  (max|n| >= 2) enter through T_M2L[i, j] = lim sum_{2 <= max|n| <= N} K(dc_i - ue_j - n L),
  applied to the root's upward equivalent density and added to its downward check potential.
  The raw partial sums grow with N along the monopole direction (a constant matrix per
  component pair); the operator is projected onto neutral densities by subtracting, per
  output row and source component, the mean over the equivalent points, which changes
  nothing for a neutral density and removes the divergent part.
* No-slip wall with PX / PXY (``wall_table``, ``wall_rpy_table``, ``wall_blake``): the image
  system of ``oracle.wall`` with every sum taken over the lattice.
* StokesPVel table ([f, q] and double-layer sources): only the forces must be neutral; the
  fields of q and D fall off like 1/r^2 and are odd, so their symmetric sums converge.  The
  far-image operator is projected on the force columns only.  Being real-space image sums of
  the field outside the cell, these need none of the moment shifts of the triply periodic
  Ewald convention (pinned by the KAFMM's convergence to the lattice sum).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import direct as D
from . import wall as Wl
from .kafmm import ALPHA, surface

AXES = {"px": 1, "pxy": 2}
# partial sums at N = n0 2^k, k < nlev: N = 16 ... 2048 along a line (4097 images, the
# extrapolated sum to rounding), N = 4 ... 128 over a plane (66049 images, about 1e-9)
EXTRAP = {"px": (16, 8), "pxy": (4, 6)}

# source columns that carry the kernel's monopole (must sum to zero)
# (StokesPVel: the forces; its sources q and the double layer's D have fields that fall off
# like 1/r^2 and odd, whose symmetric sums converge without a condition)
MONOPOLE = {"laplace": [0], "laplace_pgradgrad": [0], "laplace_qd": [0], "laplace_quad": [],
            "stokeslet": [0, 1, 2], "stokeslet_reg": [0, 1, 2], "rpy": [0, 1, 2],
            "stokes_pvel": [0, 1, 2], "stokes_pvel_grad": [0, 1, 2], "stokes_pvel_lapl": [0, 1, 2],
            "stokes_pvel_traction": [0, 1, 2], "stokes_dl": [], "stokes_dl_grad": [], "stokes_dl_lapl": [],
            "stokes_dl_traction": []}


def _lib():
    L = D.lib()
    if not hasattr(L, "_lattice_ready"):
        p, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        L.orc_lattice_matrix.argtypes = [i32, i32, p, i64, p, i64, dbl, i32, i32, i32, p]
        L.orc_lattice_matrix.restype = None
        L._lattice_ready = True
    return L


def richardson(parts, n0: int):
    """Limit N -> infinity of partial sums parts[k] at N = n0 2^k, removing the terms in
    1/N, 1/N^2, ... (one per extra level) by repeated extrapolation."""
    t = [np.asarray(v, dtype=np.float64) for v in parts]
    for j in range(1, len(t)):
        f = 2.0 ** j
        t = [(f * t[k + 1] - t[k]) / (f - 1.0) for k in range(len(t) - 1)]
    return t[0]


def shifts(bc: str, s: int) -> np.ndarray:
    """Integer image shifts (a, b, 0) of the square shell max|n| = s."""
    if s == 0:
        return np.zeros((1, 3), dtype=np.int64)
    if AXES[bc] == 1:
        return np.array([[-s, 0, 0], [s, 0, 0]], dtype=np.int64)
    a = np.arange(-s, s + 1)
    ring = [(i, j) for i in a for j in a if max(abs(i), abs(j)) == s]
    return np.array([(i, j, 0) for i, j in ring], dtype=np.int64)


def check_neutral(kernel: str, s) -> None:
    s = np.asarray(s, dtype=np.float64)
    cols = MONOPOLE.get(kernel)
    if cols is None:
        raise ValueError(f"no singly/doubly periodic sum for kernel {kernel}")
    for c in cols:
        if abs(s[:, c].sum()) > 1e-12 * max(1.0, np.abs(s[:, c]).sum()):
            raise ValueError("singly/doubly periodic sums need neutral sources "
                             f"(column {c} sums to {s[:, c].sum():.3e})")


def _extrapolated(fn, x, kt: int, bc: str, L: float, n0: int | None, nlev: int | None) -> np.ndarray:
    """sum over the lattice of fn(x - n L) (fn: the sum over the sources at the given targets,
    [m, kt]), in square shells, extrapolated in the truncation N."""
    n0 = n0 or EXTRAP[bc][0]
    nlev = nlev or EXTRAP[bc][1]
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    g = np.zeros((len(x), kt))
    parts = []
    snaps = [n0 << k for k in range(nlev)]
    batch = []

    def flush():
        # K(x - (y + n L)) as K((x - n L) - y): the images of the targets, one call per batch
        if batch:
            n = np.concatenate(batch).astype(np.float64) * L
            xs = (x[None, :, :] - n[:, None, :]).reshape(-1, 3)
            g[:] += fn(xs).reshape(len(n), len(x), kt).sum(axis=0)
            batch.clear()
    for sh in range(0, snaps[-1] + 1):
        batch.append(shifts(bc, sh))
        if sh in snaps or sum(len(v) for v in batch) * len(x) > 200000:
            flush()
        if sh in snaps:
            parts.append(g.copy())
    return richardson(parts, n0)


def lattice_sum(kernel: str, x, y, s, bc: str, L: float = 1.0, n0: int | None = None,
                nlev: int | None = None) -> np.ndarray:
    """O1 for PX / PXY: the symmetric lattice sum of ``direct.direct(kernel)`` over all images,
    extrapolated in the truncation N (FP64).  Pairs at zero distance are skipped."""
    ks, kt = D.KDIM[kernel]
    y = np.asarray(y, dtype=np.float64).reshape(-1, 3)
    s = np.asarray(s, dtype=np.float64).reshape(len(y), ks)
    check_neutral(kernel, s)
    return _extrapolated(lambda xs: D.direct(kernel, xs, y, s), x, kt, bc, L, n0, nlev)


def wall_blake(x, y, f, bc: str, zw: float, L: float = 1.0) -> np.ndarray:
    """Stokeslets above a no-slip wall at x_3 = zw, periodic along x (and y): the lattice sum
    of Blake's image system (``wall.blake``).  Its far field falls off like 1/r^3 along the
    wall, so the sum converges for any net force."""
    y = np.asarray(y, dtype=np.float64).reshape(-1, 3)
    f = np.asarray(f, dtype=np.float64).reshape(-1, 3)
    return _extrapolated(lambda xs: Wl.blake(xs, y, f, zw), x, 3, bc, L, None, None)


def wall_table(x, y, f, bc: str, zw: float, L: float = 1.0) -> np.ndarray:
    """The paper's three sums of the wall (Table tab:rpywall, b = 0), each summed over the
    lattice (each is neutral: a source and its image carry opposite charges or forces), and
    assembled at the targets."""
    x = np.asarray(x, np.float64).reshape(-1, 3)
    y = np.asarray(y, np.float64).reshape(-1, 3)
    yy = np.concatenate([y, Wl.images(y, zw)])
    fs, sd, sdz = Wl.table_sources(y, f, zw)
    return Wl.assemble(x, lattice_sum("stokeslet", x, yy, fs, bc, L), lattice_sum("laplace_qd", x, yy, sd, bc, L),
                       lattice_sum("laplace_qd", x, yy, sdz, bc, L), zw)


def wall_rpy_table(x, y, fb, bc: str, zw: float, L: float = 1.0) -> np.ndarray:
    """RPY above the wall, periodic along x (and y): the four sums of Table tab:rpywall over the
    lattice, assembled into [u, lap u]."""
    x = np.asarray(x, np.float64).reshape(-1, 3)
    y = np.asarray(y, np.float64).reshape(-1, 3)
    yy = np.concatenate([y, Wl.images(y, zw)])
    rpy, sd, sdz, quad = Wl.rpy_table_sources(y, fb, zw)
    return Wl.rpy_assemble(x, lattice_sum("rpy", x, yy, rpy, bc, L), lattice_sum("laplace_qd", x, yy, sd, bc, L),
                           lattice_sum("laplace_qd", x, yy, sdz, bc, L),
                           lattice_sum("laplace_quad", x, yy, quad, bc, L), zw)


def lattice_matrix(ml: str, x, y, bc: str, L: float = 1.0, nmin: int = 2, n0: int | None = None,
                   nlev: int | None = None) -> np.ndarray:
    """Kernel matrix (ml 'laplace', 'stokeslet' or 'stokes_pvel') summed over the images with
    nmin <= max|n| <= N, extrapolated in N.  Rows: targets x (by component), columns:
    sources y (by component)."""
    n0 = n0 or EXTRAP[bc][0]
    nlev = nlev or EXTRAP[bc][1]
    kid = {"laplace": 0, "stokeslet": 1, "stokes_pvel": 2}[ml]
    kt = (1, 3, 4)[kid]
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, 3))
    y = np.ascontiguousarray(np.asarray(y, np.float64).reshape(-1, 3))
    out = np.zeros((nlev, kt * len(x), kt * len(y)))
    _lib().orc_lattice_matrix(kid, AXES[bc], x.ctypes.data, len(x), y.ctypes.data, len(y),
                              float(L), int(nmin), int(n0), int(nlev), out.ctypes.data)
    return richardson(list(out), n0)


def t_m2l(ml: str, p: int, bc: str, L: float = 1.0, origin: float = 0.0) -> np.ndarray:
    """The far-image operator of the root for PX / PXY (real coordinates): maps the root's
    upward equivalent density to its downward check potential; images with max|n| >= 2,
    projected onto neutral densities."""
    unit = surface(p)
    r0 = L / 2.0
    c = origin + r0
    dc = c + ALPHA["dc"] * r0 * unit
    ue = c + ALPHA["ue"] * r0 * unit
    T = lattice_matrix(ml, dc, ue, bc, L)
    kt = {"laplace": 1, "stokeslet": 3, "stokes_pvel": 4}[ml]
    n = len(unit)
    Tv = T.reshape(T.shape[0], n, kt)
    mono = [0] if ml == "laplace" else [0, 1, 2]    # the StokesPVel q column converges as is
    Tv[:, :, mono] -= Tv[:, :, mono].mean(axis=1, keepdims=True)
    return Tv.reshape(T.shape)

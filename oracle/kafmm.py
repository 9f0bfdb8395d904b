"""ORACLE O2 -- plain CPU KAFMM in FP64 (test infrastructure).

The method of Yan & Blackwell (arXiv:2010.15155) step by step, in the paper's order:
the upward pass S->M then M->M (Sec. II, Fig. kifmmgraph), the downward pass M->L (V list),
S->L (X list) and L->L, then at the leaves L->T, M->T (W list) and S->T (U list).  Equivalent
densities come from the check potentials through an SVD pseudo-inverse (Sec. II: PVFMM's
backward-stable SVD in place of Tikhonov).  Each problem uses the kernel table of its
subsection (Tables tab:ktab_rpy etc.); see ``PROBLEMS``.

No blocking, fusion or reordering beyond the algorithm: box by box, list entry by list
entry.  Operators are cached per (level, octant or offset) only to avoid recomputing the
same kernel matrix.

Readings of points the paper leaves open:
* Surfaces: the boundary nodes of an m x m x m grid (M = 6(m-1)^2 + 2 points, Sec. III),
  scaled about the box centre to a half-width of alpha times the box half-width, with
  alpha = 1.05 (upward equivalent), 2.95 (upward check), 2.95 (downward equivalent),
  1.05 (downward check) -- the values of Ying, Biros & Zorin 2004.
* Pseudo-inverse cutoff: singular values below ``rcond`` times the largest are dropped;
  rcond = 1e-9 gives the lowest FP64 error against the direct sum for m = 8..12 (smaller
  cutoffs amplify rounding, larger ones truncate the expansion).
* ``stokeslet_l4`` / ``rpy_l4``: an aggregation of the Stokeslet into four Laplace channels
  (charges f_1, f_2, f_3 and (y - c).f about the box centre c), which is a valid kernel table
  in the paper's sense (linear, low-dimensional ML-tree kernels, Sec. II) but is derived here,
  not printed in the paper:
      u_i = 1/2 [phi_i - (x - c)_j d_i phi_j + d_i phi_4],   phi_k = sum q_k / (4 pi r),
      lap u_i = - d_i d_j phi_j.
  The RPY source term (b^2/6) lap G f adds a Laplace dipole (b^2/3) f to channel 4.  Moving
  a representation from reference c to c' adds (c - c') . q_{1:3} to channel 4.
* Singly and doubly periodic (``bc='px'``, ``'pxy'``): as below with the lattice of images
  along x (and y) and its far-image operator from ``oracle.lattice`` (neutral sources).
* Periodic (``bc='pxyz'``): the tree covers the source images with shift in {-1,0,1}^3 (lists
  with wrap, ``oracle.tree``); all farther images enter through one operator T_M2L applied to
  the root's multipole density and added to the root's downward check potential.  For the
  Laplace kernel the zero-mean (Ewald) periodic Green's function is not harmonic
  (lap G_per = 1/V), so the result depends on the trace of the second charge moment,
  sum q |y - c|^2, which equivalent charges do not carry; the constant
  (sum_j q_j |y_j - c|^2 - sum_k M_k |ue_k - c|^2) / (6 V) is added back at the end
  (c: root centre, M: the root's equivalent charges).  The Stokeslet needs no such step: a
  uniform body force is balanced by pressure alone.
* Periodic StokesPVel table (the [f, q] and double-layer problems): the zero-mean periodic
  pressure of a force and flow of a source are gradients of the periodic Laplace function,
  grad G_per = grad(harmonic) + r / (3 V), and Hasimoto's Stokeslet carries the matching
  backflow.  Two source moments are then not fixed by the far field the equivalent density
  reproduces, and each shifts the result by a constant: the trace of the force dipole
  tr M = sum f.(y - c) (an isotropic force dipole has no free-space field), which shifts the
  pressure by tr M / (3 V); and the split of the potential-dipole field between the source
  dipole d = sum q (y - c) and the force quadrupole, whose potential-dipole content is
  a = (2 v - w) / 5 with v = sum f |y - c|^2, w = sum (f.(y - c)) (y - c) (the remaining
  second moments are traceless or have no field).  d + a is fixed by the far field, but the
  two pieces extend periodically with different constants, shifting the velocity by
  -d / (6 V) + a / (3 V).  The differences of these constants between the true sources and
  the root's equivalent density are added at the end (derived here; pinned by the periodic
  Ewald sums of the StokesPVel kernel).  A double-layer source D is a force dipole -sym(D)
  and a source q = tr D at its point (the kernel sees only sym(D)).
"""
from __future__ import annotations

import numpy as np

from . import direct as D
from .tree import Tree

# periodic axes of each boundary (the ``periodic`` argument of ``Tree``)
PERIODIC_AXES = {"open": False, "px": "x", "pxy": "xy", "pxyz": True}

PI = np.pi
ALPHA = dict(ue=1.05, uc=2.95, de=2.95, dc=1.05)

# problem -> (k_s, k_t, ML-tree kernel, ML columns)
PROBLEMS = {
    "laplace": (1, 1, "laplace", 1),
    "stokeslet_g": (3, 3, "stokeslet", 1),
    "stokeslet_l4": (3, 3, "laplace", 4),
    "rpy_g": (4, 6, "stokeslet", 1),
    "rpy_l4": (4, 6, "laplace", 4),
    # regularized Stokeslet [f, eps] -> u, Table tab:ktab_reg: G^eps from S (to M, L and T),
    # the singular Stokeslet G between equivalent surfaces and from them to T
    "stokeslet_reg_g": (4, 3, "stokeslet", 1),
    # charges and dipoles to potential, gradient and Hessian, Table tab:ktab_lapqdpgradgrad:
    # L and L^D from S, charges on M and L, L + grad L + grad grad L to T
    "laplace_qd": (4, 10, "laplace", 1),
    # quadrupoles to potential, gradient and Hessian (LapQPGradGrad, Table tab:implement; the
    # phi^Q sum of Table tab:rpywall): the quadrupole potential from S, charges on M and L,
    # L + grad L + grad grad L to T
    "laplace_quad": (9, 10, "laplace", 1),
    # Stokes double layer D -> [p, u], Table tab:ktab_stkdlpvelgrad: K from S, the StokesPVel
    # kernel G^P ([f, q] -> [p, u]) between and from the equivalent surfaces
    "stokes_dl_pv": (9, 4, "stokes_pvel", 1),
    # StokesPVel [f, q] -> [p, u] (Sec. II.C): G^P for all interactions
    "stokes_pvel": (4, 4, "stokes_pvel", 1),
    # the same ML tree with derivative target values (the T column of Tables
    # tab:ktab_stkslpvelgrad and tab:ktab_stkdlpvelgrad): G^P + grad G^P (16), G^P + lap G^P
    # (7), and the traction (9, Eq. stressdef) from [f, q] or from D sources
    "stokes_pvel_grad": (4, 16, "stokes_pvel", 1),
    "stokes_pvel_lapl": (4, 7, "stokes_pvel", 1),
    "stokes_pvel_traction": (4, 9, "stokes_pvel", 1),
    "stokes_dl_grad": (9, 16, "stokes_pvel", 1),
    "stokes_dl_lapl": (9, 7, "stokes_pvel", 1),
    "stokes_dl_traction": (9, 9, "stokes_pvel", 1),
}

# target value kind of the derivative problems (suffix of the direct-sum kernel names)
_DERIV = {"stokes_pvel_grad": "grad", "stokes_pvel_lapl": "lapl", "stokes_pvel_traction": "traction",
          "stokes_dl_grad": "grad", "stokes_dl_lapl": "lapl", "stokes_dl_traction": "traction"}


def surface(m: int) -> np.ndarray:
    """Boundary nodes of the m x m x m grid on [-1, 1]^3, [6(m-1)^2 + 2, 3]."""
    t = np.linspace(-1.0, 1.0, m)
    pts = [(a, b, c) for i, a in enumerate(t) for j, b in enumerate(t) for k, c in enumerate(t)
           if min(i, j, k) == 0 or max(i, j, k) == m - 1]
    return np.array(pts, dtype=np.float64)


def ml_matrix(ml: str, trg: np.ndarray, src: np.ndarray) -> np.ndarray:
    """Kernel matrix of the ML-tree kernel: Laplace [nt, ns], Stokeslet [3nt, 3ns] or
    StokesPVel [4nt, 4ns] (rows p, u per target point; columns f, q per source point)."""
    r = trg[:, None, :] - src[None, :, :]
    rn = np.sqrt(np.sum(r * r, axis=2))
    if ml == "laplace":
        return 1.0 / (4.0 * PI * rn)
    nt, ns = rn.shape
    if ml == "stokes_pvel":
        K = np.zeros((nt, 4, ns, 4))
        for b in range(3):
            K[:, 0, :, b] = r[:, :, b] / (4.0 * PI * rn ** 3)
        for a in range(3):
            for b in range(3):
                K[:, 1 + a, :, b] = ((1.0 if a == b else 0.0) / rn
                                     + r[:, :, a] * r[:, :, b] / rn ** 3) / (8.0 * PI)
            K[:, 1 + a, :, 3] = -r[:, :, a] / (8.0 * PI * rn ** 3)
        return K.reshape(4 * nt, 4 * ns)
    K = np.zeros((nt, 3, ns, 3))
    for a in range(3):
        for b in range(3):
            K[:, a, :, b] = ((1.0 if a == b else 0.0) / rn
                             + r[:, :, a] * r[:, :, b] / rn ** 3) / (8.0 * PI)
    return K.reshape(3 * nt, 3 * ns)


class KAFMM:
    """Plain KAFMM for one problem type, order m (= p), leaf size q."""

    def __init__(self, problem: str, p: int, q: int, rcond: float = 1e-9, bc: str = "open",
                 origin: float = 0.0, L: float = 1.0, t_m2l=None):
        self.problem = problem
        self.ks, self.kt, self.ml, self.cols = PROBLEMS[problem]
        self.p, self.q, self.rcond = int(p), int(q), float(rcond)
        self.bc, self.origin, self.L = bc, float(origin), float(L)
        self.unit = surface(self.p)
        self.n = len(self.unit)
        self.dim = {"laplace": 1, "stokeslet": 3, "stokes_pvel": 4}[self.ml]  # rows per point
        self.t_m2l = t_m2l
        self._cache = {}

    # ---- operators (cached) ------------------------------------------------------------
    def _surf(self, kind: str, centre, lv: int) -> np.ndarray:
        r = self.L / float(1 << (lv + 1))
        return np.asarray(centre) + ALPHA[kind] * r * self.unit

    def _pinv(self, kind: str, lv: int) -> np.ndarray:
        key = ("pinv", kind, lv)
        if key not in self._cache and self.ml == "stokes_pvel":
            # StokesPVel mixes degrees (p and the q-term of u fall as 1/r^2, the f-term of u as
            # 1/r): the pseudo-inverse is taken for the unit box in scaled units, check values
            # [h p, u] times h and equivalent densities [f, q / h] (h: half-width at level lv),
            # so its cutoff does not depend on the level
            h = self.L / float(1 << (lv + 1))
            z = np.zeros(3)
            ck, ek = ("uc", "ue") if kind == "up" else ("dc", "de")
            Ku = ml_matrix(self.ml, ALPHA[ck] * self.unit, ALPHA[ek] * self.unit)
            P = np.linalg.pinv(Ku, rcond=self.rcond)
            chk_scale = np.tile([h, 1.0, 1.0, 1.0], self.n)
            eq_scale = np.tile([1.0, 1.0, 1.0, h], self.n)
            self._cache[key] = h * eq_scale[:, None] * P * chk_scale[None, :]
        if key not in self._cache:
            z = np.zeros(3)
            if kind == "up":
                K = ml_matrix(self.ml, self._surf("uc", z, lv), self._surf("ue", z, lv))
            else:
                K = ml_matrix(self.ml, self._surf("dc", z, lv), self._surf("de", z, lv))
            self._cache[key] = np.linalg.pinv(K, rcond=self.rcond)
        return self._cache[key]

    def _op(self, kind: str, lv: int, rel: tuple) -> np.ndarray:
        """Kernel matrix between two surfaces whose centres differ by ``rel`` (in units of
        the level-lv box side for m2l, of the child half-width for m2m/l2l)."""
        key = (kind, lv, rel)
        if key not in self._cache:
            z = np.zeros(3)
            h = self.L / float(1 << lv)             # box side at level lv
            if kind == "m2l":                        # dc(B) <- ue(A), c_A - c_B = rel * h
                K = ml_matrix(self.ml, self._surf("dc", z, lv),
                              self._surf("ue", np.array(rel) * h, lv))
            elif kind == "m2m":                      # uc(parent) <- ue(child at octant rel)
                cc = (np.array(rel) - 0.5) * h       # child centre (child level lv)
                K = ml_matrix(self.ml, self._surf("uc", z, lv - 1), self._surf("ue", cc, lv))
            else:                                    # l2l: dc(child) <- de(parent)
                cc = (np.array(rel) - 0.5) * h
                K = ml_matrix(self.ml, self._surf("dc", cc, lv), self._surf("de", z, lv - 1))
            self._cache[key] = K
        return self._cache[key]

    # ---- kernel-table entries -------------------------------------------------------------
    def _src_to_check(self, chk, y, s, centre) -> np.ndarray:
        """S->M / S->L: check potentials of the ML-tree kernel, [rows, cols]."""
        pr = self.problem
        if pr == "laplace":
            return D.direct("laplace", chk, y, s)
        if pr == "laplace_qd":
            return D.direct("laplace", chk, y, s[:, :1]) + D.direct("laplace_dipole", chk, y, s[:, 1:])
        if pr == "laplace_quad":
            return D.direct("laplace_quad", chk, y, s)[:, :1]
        if pr in ("stokeslet_g", "rpy_g", "stokeslet_reg_g"):
            kern = {"stokeslet_g": "stokeslet", "rpy_g": "rpy", "stokeslet_reg_g": "stokeslet_reg"}[pr]
            g = D.direct(kern, chk, y, s)
            return g[:, :3].reshape(-1, 1)
        if pr in ("stokes_dl_pv", "stokes_pvel") or pr in _DERIV:
            kern = "stokes_dl" if pr == "stokes_dl_pv" or pr.startswith("stokes_dl_") else "stokes_pvel"
            return D.direct(kern, chk, y, s).reshape(-1, 1)
        f = s[:, :3]
        out = np.zeros((len(chk), 4))
        for j in range(3):
            out[:, j] = D.direct("laplace", chk, y, f[:, j])[:, 0]
        out[:, 3] = D.direct("laplace", chk, y, np.sum((y - centre) * f, axis=1))[:, 0]
        if pr == "rpy_l4":
            bb = s[:, 3] ** 2
            out[:, 3] += D.direct("laplace_dipole", chk, y, (bb / 3.0)[:, None] * f)[:, 0]
        return out

    def _equiv_to_targets(self, x, eq, dens, centre) -> np.ndarray:
        """M->T / L->T: field of the equivalent densities at the targets, [nt, k_t]."""
        pr = self.problem
        if pr == "laplace":
            return D.direct("laplace", x, eq, dens[:, 0])
        if pr in ("laplace_qd", "laplace_quad"):
            return D.direct("laplace_pgradgrad", x, eq, dens[:, 0])
        if pr in ("stokes_dl_pv", "stokes_pvel"):
            return D.direct("stokes_pvel", x, eq, dens.reshape(-1, 4))
        if pr in _DERIV:
            return D.direct("stokes_pvel_" + _DERIV[pr], x, eq, dens.reshape(-1, 4))
        if pr in ("stokeslet_g", "stokeslet_reg_g"):
            return D.direct("stokeslet", x, eq, dens.reshape(-1, 3))
        if pr == "rpy_g":
            fb = np.concatenate([dens.reshape(-1, 3), np.zeros((len(eq), 1))], axis=1)
            return D.direct("rpy", x, eq, fb)
        H = [D.direct("laplace_pgradgrad", x, eq, dens[:, k]) for k in range(4)]
        xc = x - centre
        u = np.zeros((len(x), 3))
        for i in range(3):
            u[:, i] = 0.5 * (H[i][:, 0] - sum(xc[:, j] * H[j][:, 1 + i] for j in range(3))
                             + H[3][:, 1 + i])
        if pr == "stokeslet_l4":
            return u
        hidx = {(0, 0): 4, (0, 1): 5, (0, 2): 6, (1, 1): 7, (1, 2): 8, (2, 2): 9}
        lap = np.zeros((len(x), 3))
        for i in range(3):
            lap[:, i] = -sum(H[j][:, hidx[(min(i, j), max(i, j))]] for j in range(3))
        return np.concatenate([u, lap], axis=1)

    def _src_to_targets(self, x, y, s) -> np.ndarray:
        if self.problem in _DERIV or self.problem == "laplace_quad":
            return D.direct(self.problem, x, y, s)
        kern = {"laplace": "laplace", "stokeslet_g": "stokeslet", "stokeslet_l4": "stokeslet",
                "rpy_g": "rpy", "rpy_l4": "rpy", "stokeslet_reg_g": "stokeslet_reg",
                "laplace_qd": "laplace_qd", "stokes_dl_pv": "stokes_dl",
                "stokes_pvel": "stokes_pvel"}[self.problem]
        return D.direct(kern, x, y, s)

    def _shift(self, dens, c_from, c_to) -> np.ndarray:
        """Re-reference a four-channel density: q_4 += (c_from - c_to) . q_{1:3}."""
        if self.cols != 4:
            return dens
        out = dens.copy()
        out[:, 3] += dens[:, :3] @ (np.asarray(c_from) - np.asarray(c_to))
        return out

    def _pvel_periodic_shift(self, src, s, root_eq, c0):
        """Constant pressure and velocity shifts of the periodic StokesPVel table (module
        notes): the moment differences between the true sources and the root's equivalent
        density (real units [f, q] at the root's upward equivalent points)."""
        def moments(dy, f, q, Mi):
            # dy: positions - c0; f: forces; q: sources; Mi: intrinsic force dipoles [n, 3, 3]
            trM = np.sum(f * dy) + np.trace(Mi, axis1=1, axis2=2).sum()
            d = np.sum(q[:, None] * dy, axis=0)
            v = np.sum(f * np.sum(dy * dy, axis=1)[:, None], axis=0) + 2.0 * np.einsum("njk,nk->j", Mi, dy)
            w = (np.sum(np.sum(f * dy, axis=1)[:, None] * dy, axis=0)
                 + np.einsum("njj,nl->l", Mi, dy) + np.einsum("njl,nj->l", Mi, dy))
            return trM, d, (2.0 * v - w) / 5.0
        dy = src - c0
        if self.ks == 9:   # double layer: force dipole -sym(D), source tr D
            Dm = s.reshape(-1, 3, 3)
            S = 0.5 * (Dm + np.transpose(Dm, (0, 2, 1)))
            mt = moments(dy, np.zeros_like(dy), np.trace(S, axis1=1, axis2=2), -S)
        else:
            mt = moments(dy, s[:, :3], s[:, 3], np.zeros((len(src), 3, 3)))
        ue = self._surf("ue", c0, 0) - c0
        E = root_eq.reshape(-1, 4)
        me = moments(ue, E[:, :3], E[:, 3], np.zeros((len(E), 3, 3)))
        V = self.L ** 3
        dp = (mt[0] - me[0]) / (3.0 * V)
        du = -(mt[1] - me[1]) / (6.0 * V) + (mt[2] - me[2]) / (3.0 * V)
        return dp, du

    # ---- evaluation ------------------------------------------------------------------------
    def evaluate(self, src, s, trg=None, tree: Tree | None = None, near_only: bool = False):
        """g at the targets (sources if trg is None), [nt, k_t]."""
        src = np.asarray(src, dtype=np.float64).reshape(-1, 3)
        s = np.asarray(s, dtype=np.float64).reshape(len(src), self.ks)
        T = tree or Tree(src, trg, q=self.q, origin=self.origin, L=self.L,
                         periodic=PERIODIC_AXES[self.bc])
        self.tree = T
        x = T.trg
        nb = T.nbox
        per = self.bc != "open"
        L = self.L
        M = [None] * nb
        Lden = [None] * nb

        if not near_only:
            # upward pass: S->M at leaves, M->M at parents, deepest level first
            for lv in range(T.nlevels - 1, -1, -1):
                for b in np.nonzero(T.level == lv)[0]:
                    c = T.centre(b)
                    if T.is_leaf[b]:
                        si = T.src_idx[b]
                        chk = self._src_to_check(self._surf("uc", c, lv), src[si], s[si], c)
                    else:
                        chk = np.zeros((self.n * self.dim, self.cols))
                        for o, ch in enumerate(T.children[b]):
                            if ch < 0:
                                continue
                            rel = (o & 1, (o >> 1) & 1, (o >> 2) & 1)
                            dm = self._shift(M[ch], T.centre(ch), c)
                            chk += self._op("m2m", lv + 1, rel) @ dm
                    M[b] = self._pinv("up", lv) @ chk
            self.root_equiv = M[0]

            # downward pass: V (M->L), X (S->L), L->L, then L = DC2DE * check
            for lv in range(T.nlevels):
                for b in np.nonzero(T.level == lv)[0]:
                    c = T.centre(b)
                    chk = np.zeros((self.n * self.dim, self.cols))
                    for (a, sh) in T.V[b]:
                        ca = T.centre(a) + np.array(sh) * L
                        rel = tuple(int(v) for v in (T.anchor[a] + np.array(sh) * (1 << lv)
                                                     - T.anchor[b]))
                        chk += self._op("m2l", lv, rel) @ self._shift(M[a], ca, c)
                    for (a, sh) in T.X[b]:
                        si = T.src_idx[a]
                        ys = src[si] + np.array(sh) * L
                        chk += self._src_to_check(self._surf("dc", c, lv), ys, s[si], c)
                    if T.parent[b] >= 0:
                        pb = T.parent[b]
                        o = int(np.sum((T.anchor[b] & 1) * np.array([1, 2, 4])))
                        rel = (o & 1, (o >> 1) & 1, (o >> 2) & 1)
                        chk += self._op("l2l", lv, rel) @ self._shift(Lden[pb], T.centre(pb), c)
                    elif per:
                        if self.t_m2l is None:
                            raise ValueError("periodic evaluation needs the T_M2L operator")
                        chk += (self.t_m2l @ M[b].reshape(-1)).reshape(chk.shape)
                    Lden[b] = self._pinv("down", lv) @ chk

        # leaves: L->T, M->T (W), S->T (U)
        g = np.zeros((len(x), self.kt))
        if self.bc == "pxyz" and self.problem == "laplace" and not near_only:
            c0 = T.centre(0)
            ue0 = self._surf("ue", c0, 0)
            second = np.sum(s[:, 0] * np.sum((src - c0) ** 2, axis=1))
            second_eq = np.sum(M[0][:, 0] * np.sum((ue0 - c0) ** 2, axis=1))
            g += (second - second_eq) / (6.0 * self.L ** 3)
        if self.bc == "pxyz" and self.ml == "stokes_pvel" and not near_only:
            dp, du = self._pvel_periodic_shift(src, s, M[0], T.centre(0))
            if self.problem in ("stokes_pvel_traction", "stokes_dl_traction"):
                g[:, [0, 4, 8]] -= dp           # sigma = -p I + ...
            else:
                g[:, 0] += dp
                g[:, 1:4] += du
        for b in T.leaves():
            ti = T.trg_idx[b]
            if len(ti) == 0:
                continue
            xt = x[ti]
            lv = int(T.level[b])
            c = T.centre(b)
            acc = np.zeros((len(ti), self.kt))
            if not near_only:
                acc += self._equiv_to_targets(xt, self._surf("de", c, lv), Lden[b], c)
                for (a, sh) in T.W[b]:
                    ca = T.centre(a) + np.array(sh) * L
                    acc += self._equiv_to_targets(xt, self._surf("ue", ca, int(T.level[a])),
                                                  M[a], ca)
            for (a, sh) in T.U[b]:
                si = T.src_idx[a]
                acc += self._src_to_targets(xt, src[si] + np.array(sh) * L, s[si])
            g[ti] += acc
        return g

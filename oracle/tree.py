"""ORACLE -- adaptive octree and U/V/W/X interaction lists (test infrastructure).

The paper builds its octree by recursive refinement until every leaf holds at most a fixed
number of points (Sec. III, "no more than 2000 target points"; here the limit q is a
parameter) and classifies boxes into the U, V, W, X lists of kernel-independent FMM (Sec. II,
the lists defined by Ying, Biros & Zorin 2004, which the paper uses unmodified).

Readings used here (the paper defers the details):
* Root = the cube [origin, origin + L)^3.  A box is split while it holds more than q points
  and its level is below MAX_LEVEL (20).  When sources and targets are one set a point
  counts once; otherwise sources and targets are both counted.  Empty children are dropped.
* Point membership uses integer cells at the finest level:
  I = clamp(floor((p - origin) / L * 2^20), 0, 2^20 - 1) per coordinate (in FP64), and a box
  (level l, anchor a) holds the points with I >> (20 - l) == a.
* Boxes are numbered level by level, each level in Morton order (octant bit 0 = x, 1 = y,
  2 = z), i.e. in breadth-first order of the refinement.
* "Adjacent" means the closed boxes intersect.  No 2:1 balance is enforced.
* U(B), leaf B: all leaves adjacent to B (B included).
  V(B): children of the colleagues of parent(B) that are not adjacent to B.
  W(B), leaf B: descendants A of B's colleagues with A not adjacent to B and parent(A)
  adjacent to B.
  X(B): all A with B in W(A).
* Periodic (``periodic=True`` or "xyz": triply; "x": singly, along x; "xy": doubly, along x
  and y): adjacency and colleagues are taken modulo the cube along the periodic axes; every
  list entry carries the integer image shift (in units of L) applied to the source box, zero
  along the other axes.
"""
from __future__ import annotations

import numpy as np

MAX_LEVEL = 20


def periodic_axes(periodic) -> tuple:
    """(x, y, z) flags of the periodic axes: False/None -> none, True -> all three, or a
    string naming the axes ("x", "xy", "xyz")."""
    if periodic is None or periodic is False:
        return (False, False, False)
    if periodic is True:
        return (True, True, True)
    if isinstance(periodic, str):
        return tuple(a in periodic for a in "xyz")
    return tuple(bool(v) for v in periodic)


def cells(points, origin=0.0, L=1.0) -> np.ndarray:
    """Finest-level integer cell coordinates, int64 [n, 3]."""
    p = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    c = np.floor((p - origin) / L * float(1 << MAX_LEVEL))
    return np.clip(c, 0, (1 << MAX_LEVEL) - 1).astype(np.int64)


class Tree:
    """Adaptive octree over sources (and targets, if a separate set)."""

    def __init__(self, src, trg=None, q=64, origin=0.0, L=1.0, periodic=False):
        self.origin = float(origin)
        self.L = float(L)
        self.q = int(q)
        self.axes = periodic_axes(periodic)
        self.periodic = any(self.axes)
        self.same = trg is None
        self.src = np.asarray(src, dtype=np.float64).reshape(-1, 3)
        self.trg = self.src if self.same else np.asarray(trg, dtype=np.float64).reshape(-1, 3)
        cs = cells(self.src, origin, L)
        ct = cs if self.same else cells(self.trg, origin, L)

        # breadth-first refinement
        self.level, self.anchor, self.parent = [0], [(0, 0, 0)], [-1]
        self.src_idx = [np.arange(len(cs))]
        self.trg_idx = [np.arange(len(ct))]
        self.children = []
        b = 0
        while b < len(self.level):
            lv = self.level[b]
            si, ti = self.src_idx[b], self.trg_idx[b]
            count = len(si) if self.same else len(si) + len(ti)
            kids = [-1] * 8
            if count > self.q and lv < MAX_LEVEL:
                sh = MAX_LEVEL - (lv + 1)
                a = self.anchor[b]
                for o in range(8):
                    ca = (2 * a[0] + (o & 1), 2 * a[1] + ((o >> 1) & 1),
                          2 * a[2] + ((o >> 2) & 1))
                    ms = np.all((cs[si] >> sh) == ca, axis=1)
                    mt = ms if self.same else np.all((ct[ti] >> sh) == ca, axis=1)
                    if ms.any() or mt.any():
                        kids[o] = len(self.level)
                        self.level.append(lv + 1)
                        self.anchor.append(ca)
                        self.parent.append(b)
                        self.src_idx.append(si[ms])
                        self.trg_idx.append(ti[mt] if not self.same else si[ms])
            self.children.append(kids)
            b += 1
        self.nbox = len(self.level)
        self.level = np.array(self.level, dtype=np.int64)
        self.anchor = np.array(self.anchor, dtype=np.int64).reshape(-1, 3)
        self.parent = np.array(self.parent, dtype=np.int64)
        self.children = np.array(self.children, dtype=np.int64).reshape(-1, 8)
        self.is_leaf = np.all(self.children < 0, axis=1)
        self.nlevels = int(self.level.max()) + 1
        self.lookup = {(int(self.level[i]), tuple(int(v) for v in self.anchor[i])): i
                       for i in range(self.nbox)}
        self._build_lists()

    # ---- geometry -------------------------------------------------------------------
    def half_width(self, lv: int) -> float:
        return self.L / float(1 << (lv + 1))

    def centre(self, b: int) -> np.ndarray:
        lv = int(self.level[b])
        return self.origin + (self.anchor[b] + 0.5) * (self.L / float(1 << lv))

    def _span(self, b: int, shift=(0, 0, 0)):
        """Closed box [lo, hi] in finest-level integer units, shifted by whole domains."""
        sh = MAX_LEVEL - int(self.level[b])
        lo = (self.anchor[b] << sh) + np.array(shift, dtype=np.int64) * (1 << MAX_LEVEL)
        return lo, lo + (1 << sh)

    def adjacent(self, a: int, b: int, shift=(0, 0, 0)) -> bool:
        """Do closed boxes a (moved by ``shift`` domains) and b intersect?"""
        la, ha = self._span(a, shift)
        lb, hb = self._span(b)
        return bool(np.all(la <= hb) and np.all(lb <= ha))

    def _shifts(self):
        r = [(-1, 0, 1) if a else (0,) for a in self.axes]
        return [(i, j, k) for i in r[0] for j in r[1] for k in r[2]]

    def colleagues(self, b: int):
        """Same-level boxes (with their image shift) adjacent to b, b itself included."""
        lv = int(self.level[b])
        n = 1 << lv
        out = []
        for d in [(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)]:
            a = self.anchor[b] + np.array(d)
            shift = np.floor_divide(a, n) * np.array(self.axes, dtype=np.int64)
            a = a - shift * n
            if np.any(a < 0) or np.any(a >= n):
                continue
            c = self.lookup.get((lv, tuple(int(v) for v in a)))
            if c is not None:
                key = (c, tuple(int(v) for v in shift))
                if key not in out:
                    out.append(key)
        return out

    # ---- lists ------------------------------------------------------------------------
    def _build_lists(self):
        nb = self.nbox
        self.U = [[] for _ in range(nb)]
        self.V = [[] for _ in range(nb)]
        self.W = [[] for _ in range(nb)]
        self.X = [[] for _ in range(nb)]
        for b in range(nb):
            lv = int(self.level[b])
            # V: children of parent's colleagues, not adjacent to b.  With periodic wrap the
            # root's colleagues are its images, so level-1 boxes get a V list too.
            if lv >= 2 or (self.periodic and lv >= 1):
                for (c, sh) in self.colleagues(int(self.parent[b])):
                    for ch in self.children[c]:
                        if ch >= 0 and not self.adjacent(int(ch), b, sh):
                            self.V[b].append((int(ch), sh))
            if not self.is_leaf[b]:
                continue
            # U: all leaves adjacent to b -- descend from the root (and its images)
            for sh in self._shifts():
                stack = [0]
                while stack:
                    c = stack.pop()
                    if not self.adjacent(c, b, sh):
                        continue
                    if self.is_leaf[c]:
                        if (c, sh) not in self.U[b]:
                            self.U[b].append((c, sh))
                    else:
                        stack.extend(int(ch) for ch in self.children[c] if ch >= 0)
            # W: descendants of colleagues, non-adjacent, with an adjacent parent
            for (c, sh) in self.colleagues(b):
                if c == b and sh == (0, 0, 0):
                    continue
                stack = [int(ch) for ch in self.children[c] if ch >= 0]
                while stack:
                    d = stack.pop()
                    if self.adjacent(d, b, sh):
                        stack.extend(int(ch) for ch in self.children[d] if ch >= 0)
                    elif (d, sh) not in self.W[b]:
                        self.W[b].append((d, sh))
        # X is the dual of W: A in X(B) iff B in W(A); the shift flips sign
        for a in range(nb):
            for (b, sh) in self.W[a]:
                self.X[b].append((a, tuple(-v for v in sh)))
        for lst in (self.U, self.V, self.W, self.X):
            for b in range(nb):
                lst[b].sort()

    # ---- helpers ----------------------------------------------------------------------
    def leaves(self):
        return np.nonzero(self.is_leaf)[0]

    def ancestors(self, b: int):
        """b and all its ancestors up to the root."""
        out = [b]
        while self.parent[out[-1]] >= 0:
            out.append(int(self.parent[out[-1]]))
        return out

    def route_count(self, tb: int, sb: int, sh=(0, 0, 0)) -> int:
        """Number of list routes by which the sources of leaf sb (moved by sh domains) reach
        the targets of leaf tb.  A correct set of lists gives exactly 1 for every pair of
        leaves (and every image shift of the near image block when periodic)."""
        n = 0
        sh = tuple(sh)
        if (sb, sh) in self.U[tb]:
            n += 1
        anc_s = self.ancestors(sb)
        anc_t = self.ancestors(tb)
        for a in anc_s:
            if (a, sh) in self.W[tb]:
                n += 1
        for bt in anc_t:
            for a in anc_s:
                if (a, sh) in self.V[bt]:
                    n += 1
            if (sb, sh) in self.X[bt]:
                n += 1
        return n

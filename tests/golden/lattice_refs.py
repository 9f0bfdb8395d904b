"""Expected values of the singly / doubly periodic GPU tests (tests/test_gpu_lattice.py),
written by this script from ``oracle/`` alone: the extrapolated lattice sums (O1) of seeded
synthetic cases, whose FP64 direct sums over up to 66049 images take minutes on the host.

    python tests/golden/lattice_refs.py        # rewrites tests/golden/lattice/*.txt

The cases are defined here (seeded generators, no arithmetic of the method) and imported by the
tests, which rebuild the same inputs and load the stored sums.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "lattice")

N_LAT = 6000                                   # Stokeslet, no wall
IDX_LAT = np.arange(0, N_LAT, N_LAT // 24)
N_WALL = 2000                                  # Stokeslet above the wall
IDX_WALL = np.arange(0, N_WALL, N_WALL // 24)
N_RPY_WALL = 1200                              # RPY above the wall
IDX_RPY_WALL = np.arange(0, N_RPY_WALL, N_RPY_WALL // 24)
N_RPY = 900                                    # RPY spheres across the periodic boundary


def stokeslet_case():
    """Uniform points (rounded to FP32 and kept below 1) and forces minus their mean."""
    rng = np.random.default_rng(34)
    pts = rng.random((N_LAT, 3))
    f = rng.standard_normal((N_LAT, 3))
    f -= f.mean(axis=0)
    pts = np.minimum(pts.astype(np.float32), np.float32(1) - np.float32(2 ** -24)).astype(np.float64)
    return pts, f


def upper_case(n, seed, rpy=False):
    """Points in the upper half of the unit cube (wall at z = 1/2) with forces that keep their
    net part; RPY spheres of radius U(0.002, 0.006) at least 0.02 above the wall."""
    rng = np.random.default_rng(seed)
    p = rng.random((n, 3))
    p[:, 2] = (0.52 + 0.48 * p[:, 2]) if rpy else (0.5 + 0.5 * p[:, 2])
    s = rng.standard_normal((n, 3))
    if rpy:
        s = np.concatenate([s, rng.uniform(0.002, 0.006, (n, 1))], axis=1)
    return np.minimum(p, 1.0 - 2.0 ** -24), s


def rpy_cluster_case():
    """A Gaussian cluster of spheres straddling the periodic boundary x = 0, radii
    U(0.004, 0.012), forces minus their mean."""
    rng = np.random.default_rng(35)
    pts = np.array([0.0, 0.5, 0.5]) + 0.04 * rng.standard_normal((N_RPY, 3))
    pts[:, 0] %= 1.0
    pts = np.clip(pts, 0.0, 1.0 - 1e-12)
    a = rng.uniform(0.004, 0.012, N_RPY)
    f = rng.standard_normal((N_RPY, 3))
    f -= f.mean(axis=0)
    return pts, np.concatenate([f, a[:, None]], axis=1)


def path(name):
    return os.path.join(OUT, name + ".txt")


def load(name):
    return np.loadtxt(path(name), ndmin=2)


def main():
    sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
    from oracle import direct as D
    from oracle import lattice as La
    os.makedirs(OUT, exist_ok=True)

    def save(name, a):
        np.savetxt(path(name), a, fmt="%.17e")
        print(name, a.shape, flush=True)
    pts, f = stokeslet_case()
    for bc in ("px", "pxy"):
        save(f"stokeslet_{bc}", La.lattice_sum("stokeslet", pts[IDX_LAT], pts, f, bc))
    pts, fb = rpy_cluster_case()
    a = fb[:, 3]
    g = La.lattice_sum("rpy", pts, pts, fb, "px")
    ref = g[:, :3] + (a * a / 6.0)[:, None] * g[:, 3:]
    for s in (-1, 0, 1):   # overlap corrections of the nearest images along x
        ref = D.rpy_overlap_correction(pts, a, pts + np.array([s, 0.0, 0.0]), fb, same_set=(s == 0), g=ref)
    save("rpy_velocity_px", ref)
    pts, f = upper_case(N_WALL, 36)
    for bc in ("px", "pxy"):
        save(f"wall_{bc}", La.wall_table(pts[IDX_WALL], pts, f, bc, 0.5))
    pts, fb = upper_case(N_RPY_WALL, 37, rpy=True)
    save("rpy_wall_pxy", La.wall_rpy_table(pts[IDX_RPY_WALL], pts, fb, "pxy", 0.5))


if __name__ == "__main__":
    main()

"""Pins for the oracle's Stokeslet above a no-slip wall (oracle/wall.py, Sec. III.C).

Blake's image system is fixed here by what the physics demands, not by its formula:
* no slip: the velocity vanishes on the wall;
* incompressible: finite-difference divergence zero;
* reciprocal (Lorentz): B_ij(x, y) = B_ji(y, x);
* near the source the field is the free-space Stokeslet plus a regular field.
The paper's three-sum assembly (Table tab:rpywall at b = 0, with the reading of the charges
stated in oracle/wall.py) must equal Blake's solution to round-off.
"""
import numpy as np
import pytest

from oracle import direct as D
from oracle import wall as Wl


def _above(n, rng, zw=0.0):
    p = rng.random((n, 3))
    p[:, 2] = zw + 0.05 + p[:, 2]
    return p


@pytest.mark.parametrize("zw", [0.0, 0.5])
def test_blake_vanishes_on_the_wall(zw):
    rng = np.random.default_rng(1)
    y = _above(40, rng, zw)
    f = rng.standard_normal((40, 3))
    xw = rng.random((30, 3)) * 3 - 1
    xw[:, 2] = zw
    u = Wl.blake(xw, y, f, zw)
    scale = np.abs(D.direct("stokeslet", xw, y, f)).max()
    assert np.abs(u).max() < 1e-13 * scale


def test_blake_is_divergence_free():
    rng = np.random.default_rng(2)
    y = _above(10, rng)
    f = rng.standard_normal((10, 3))
    x = _above(20, rng) + np.array([0.0, 0.0, 0.3])
    e = 1e-5
    div = np.zeros(len(x))
    for k in range(3):
        d = np.zeros(3)
        d[k] = e
        div += (Wl.blake(x + d, y, f)[:, k] - Wl.blake(x - d, y, f)[:, k]) / (2 * e)
    scale = np.abs(Wl.blake(x, y, f)).max() / 0.3
    assert np.abs(div).max() < 1e-7 * scale


def test_blake_is_reciprocal():
    rng = np.random.default_rng(3)
    a, b = _above(1, rng)[0], _above(1, rng)[0]
    B = np.stack([Wl.blake(a[None], b[None], np.eye(3)[j][None])[0] for j in range(3)], axis=1)
    Bt = np.stack([Wl.blake(b[None], a[None], np.eye(3)[j][None])[0] for j in range(3)], axis=1)
    assert np.allclose(B, Bt.T, rtol=1e-12, atol=1e-14)


def test_blake_near_the_source_is_the_free_stokeslet_plus_a_regular_field():
    y = np.array([[0.3, 0.4, 0.6]])
    f = np.array([[0.2, -0.5, 0.9]])
    d = np.array([1.0, 2.0, -1.5]) / np.sqrt(7.25)
    reg = []
    for eps in (1e-3, 1e-4, 1e-5):
        x = y + eps * d
        reg.append(Wl.blake(x, y, f)[0] - D.direct("stokeslet", x, y, f)[0])
    # the image field is smooth at the source: it converges as the target approaches it
    assert np.linalg.norm(reg[1] - reg[2]) < 1e-3 * np.linalg.norm(reg[2])
    assert np.linalg.norm(reg[0] - reg[2]) < 1e-2 * np.linalg.norm(reg[2])


@pytest.mark.parametrize("zw", [0.0, 0.5])
def test_three_sum_assembly_equals_blake(zw):
    rng = np.random.default_rng(4)
    y = _above(200, rng, zw)
    f = rng.standard_normal((200, 3))
    x = np.concatenate([_above(150, rng, zw), y[:20]])   # targets off and on the sources
    ref = Wl.blake(x, y, f, zw)
    got = Wl.table(x, y, f, zw)
    assert D.rel_l2(got, ref) < 1e-12


def _rpy_above(n, rng, zw=0.0):
    y = _above(n, rng, zw)
    fb = np.concatenate([rng.standard_normal((n, 3)), rng.uniform(0.005, 0.03, (n, 1))], axis=1)
    return y, fb


@pytest.mark.parametrize("zw", [0.0, 0.5])
def test_rpy_wall_four_sums_equal_the_definition(zw):
    """The four-sum assembly of Table tab:rpywall (with the quadrupole at the image) equals
    (1 + b^2/6 lap_y) of Blake's solution (the RPY kernel sum above the wall), targets off and
    on the sources; with b = 0 it is the Stokeslet wall's three-sum assembly."""
    rng = np.random.default_rng(5)
    y, fb = _rpy_above(60, rng, zw)
    x = np.concatenate([_above(80, rng, zw), y[:10]])
    got = Wl.rpy_table(x, y, fb, zw)
    assert D.rel_l2(got[:, :3], Wl.blake_rpy(x, y, fb, zw)) < 1e-8
    fb0 = fb.copy()
    fb0[:, 3] = 0.0
    assert D.rel_l2(Wl.rpy_table(x, y, fb0, zw)[:, :3], Wl.table(x, y, fb[:, :3], zw)) < 1e-13


def test_rpy_wall_laplacian_and_no_slip():
    """lap u of the assembly equals a Richardson-extrapolated 7-point Laplacian of its u in x,
    and u vanishes on the wall (the source operator acts on y, Blake's field vanishes on the
    wall for every y)."""
    rng = np.random.default_rng(6)
    y, fb = _rpy_above(20, rng)
    x = _above(10, rng) + np.array([0.0, 0.0, 0.2])
    got = Wl.rpy_table(x, y, fb)
    lap = []
    for h in (2e-3, 1e-3):
        acc = -6.0 * Wl.rpy_table(x, y, fb)[:, :3]
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            acc = acc + Wl.rpy_table(x + e, y, fb)[:, :3] + Wl.rpy_table(x - e, y, fb)[:, :3]
        lap.append(acc / (h * h))
    fd = (4.0 * lap[1] - lap[0]) / 3.0
    assert D.rel_l2(got[:, 3:], fd) < 1e-6
    xw = rng.random((30, 3)) * 3 - 1
    xw[:, 2] = 0.0
    uw = Wl.rpy_table(xw, y, fb)[:, :3]
    assert np.abs(uw).max() < 1e-12 * np.abs(Wl.rpy_table(xw + [0, 0, 0.3], y, fb)[:, :3]).max()

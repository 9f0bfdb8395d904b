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

"""Pins for the oracle's quadrature rules (closed forms and published tables)."""
import json
import math
import os

import numpy as np
import pytest

from oracle.quadrature import gauss_legendre, gauss_lobatto, level_symmetric_2d, level_symmetric_octant

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_gauss_legendre_exactness(n):
    x, w = gauss_legendre(n)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14
    if n <= 3:
        assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-8


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_gauss_lobatto_exactness(n):
    x, w = gauss_lobatto(n)
    assert x[0] == 0.0 and x[-1] == 1.0
    for k in range(2 * n - 2):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14


def test_gauss_lobatto_closed_forms():
    x, w = gauss_lobatto(3)
    assert np.allclose(x, [0, 0.5, 1], atol=1e-15) and np.allclose(w, [1 / 6, 2 / 3, 1 / 6], atol=1e-15)
    x, w = gauss_lobatto(4)
    r = 0.5 / math.sqrt(5.0)
    assert np.allclose(x, [0, 0.5 - r, 0.5 + r, 1], atol=1e-15)
    assert np.allclose(w, [1 / 12, 5 / 12, 5 / 12, 1 / 12], atol=1e-15)


@pytest.mark.parametrize("N,count", [(2, 4), (4, 12), (6, 24), (8, 40), (10, 60), (12, 84)])
def test_level_symmetric_moments(N, count):
    om, w = level_symmetric_2d(N)
    assert len(w) == count and np.all(w > 0)
    fp = 4 * math.pi
    assert abs(w.sum() - fp) < 1e-13
    ox, oy = om[:, 0], om[:, 1]
    # first and second moments: int Omega = 0, int Omega_i Omega_j = 4pi/3 delta_ij
    assert abs(np.sum(w * ox)) < 1e-13 and abs(np.sum(w * oy)) < 1e-13
    assert abs(np.sum(w * ox * ox) - fp / 3) < 1e-13
    assert abs(np.sum(w * oy * oy) - fp / 3) < 1e-13
    assert abs(np.sum(w * ox * oy)) < 1e-13
    # odd third moments vanish
    for a, b, c in [(ox, ox, ox), (ox, ox, oy), (ox, oy, oy), (oy, oy, oy)]:
        assert abs(np.sum(w * a * b * c)) < 1e-13
    if N >= 4:
        assert abs(np.sum(w * ox ** 4) - fp / 5) < 1e-12
        assert abs(np.sum(w * ox ** 2 * oy ** 2) - fp / 15) < 1e-12
    if N >= 8:
        assert abs(np.sum(w * ox ** 6) - fp / 7) < 1e-12
    # octant (quadrant) symmetry: reflections map the set onto itself
    s = {(round(a, 12), round(b, 12), round(c, 12)) for (a, b), c in zip(om, w)}
    for sx, sy in [(-1, 1), (1, -1), (-1, -1)]:
        assert {(round(sx * a, 12), round(sy * b, 12), c) for (a, b, c) in s} == s
    # transposition symmetry Omega_x <-> Omega_y
    assert {(b, a, c) for (a, b, c) in s} == s


def test_level_symmetric_unit_vectors():
    for N in (4, 6, 8, 10, 12):
        cos, w = level_symmetric_octant(N)
        assert np.allclose(np.sum(cos ** 2, axis=1), 1.0, atol=1e-14)
        assert abs(w.sum() - 1.0) < 1e-14


def test_level_symmetric_matches_published_tables():
    gold = json.load(open(os.path.join(GOLD, "lq_weights.json")))
    for N in (6, 8, 12):
        _, w = level_symmetric_octant(N)
        assert np.allclose(np.unique(np.round(w, 12))[::-1][: len(gold[str(N)])].sum(), sum(gold[str(N)]), atol=5e-7)
        for ref in gold[str(N)]:
            assert np.min(np.abs(w - ref)) < 5e-7

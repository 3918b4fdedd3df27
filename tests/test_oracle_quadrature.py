"""Pins of the oracle's triangle rules against exact monomial integrals.

Exact: the integral of l1^a l2^b l3^c over a triangle of area A is
2 A a! b! c! / (a + b + c + 2)!  (barycentric coordinates).
"""
from math import factorial

import numpy as np
import pytest

from oracle.quadrature import radon7, collapsed_gauss, subdivided


def exact(a, b, c):
    # normalised to area 1
    return 2.0 * factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 2)


def max_err(rule, deg):
    pts, w = rule
    err = 0.0
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            c = deg - a - b
            v = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
            err = max(err, abs(v - exact(a, b, c)) / exact(a, b, c))
    return err


def test_radon7_degree5_exact_and_not_6():
    r = radon7()
    assert abs(r[1].sum() - 1.0) < 1e-15
    for d in range(6):
        assert max_err(r, d) < 1e-13, d
    assert max_err(r, 6) > 1e-6


@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_collapsed_gauss_degree(n):
    r = collapsed_gauss(n)
    for d in range(2 * n - 1):
        assert max_err(r, d) < 1e-12, (n, d)
    assert max_err(r, 2 * n) > 1e-12


def test_subdivided_keeps_degree():
    r = subdivided(radon7(), 2)
    assert r[0].shape[0] == 7 * 16
    for d in range(6):
        assert max_err(r, d) < 1e-13

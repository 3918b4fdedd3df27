"""Triangle quadrature rules (barycentric points, weights summing to one).

The paper states no quadrature rule (its Sec. IV-B leaves the projection and
integration rules open).  Two rule families are used:

* radon7: Radon's classical 7-point rule, exact for polynomials of degree 5.
  Closed form: the centroid (weight 9/40) and two 3-point orbits
  (a, a, 1-2a) with a = (6 -+ sqrt 15)/21 and weights (155 -+ sqrt 15)/1200.
* collapsed_gauss(n): the conical product of n-point Gauss-Legendre rules on the
  square mapped onto the triangle by (u, v) -> (u, v (1 - u)); exact for degree
  2n - 2 (the Jacobian 1 - u costs one degree).
* subdivided(rule, levels): the rule applied on each of 4**levels congruent
  sub-triangles (midpoint refinement).
"""
from __future__ import annotations

import numpy as np


def radon7():
    s15 = np.sqrt(15.0)
    a1 = (6.0 - s15) / 21.0
    a2 = (6.0 + s15) / 21.0
    w1 = (155.0 - s15) / 1200.0
    w2 = (155.0 + s15) / 1200.0
    pts = [(1.0 / 3, 1.0 / 3, 1.0 / 3)]
    wts = [9.0 / 40.0]
    for a, w in ((a1, w1), (a2, w2)):
        b = 1.0 - 2.0 * a
        pts += [(a, a, b), (a, b, a), (b, a, a)]
        wts += [w, w, w]
    return np.array(pts), np.array(wts)


def centroid1():
    return np.array([[1.0 / 3, 1.0 / 3, 1.0 / 3]]), np.array([1.0])


def collapsed_gauss(n):
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    u, v = np.meshgrid(x, x, indexing="ij")
    wu, wv = np.meshgrid(w, w, indexing="ij")
    l1 = u.ravel()
    l2 = (v * (1.0 - u)).ravel()
    wt = (wu * wv * (1.0 - u)).ravel() * 2.0     # reference triangle area 1/2
    pts = np.stack([1.0 - l1 - l2, l1, l2], axis=1)
    return pts, wt


def subdivided(rule, levels):
    """Apply `rule` (pts, wts) on 4**levels midpoint sub-triangles."""
    pts, wts = rule
    tris = [np.eye(3)]                     # sub-triangle vertices in barycentrics
    for _ in range(levels):
        nxt = []
        for t in tris:
            a, b, c = t
            ab, bc, ca = 0.5 * (a + b), 0.5 * (b + c), 0.5 * (c + a)
            nxt += [np.array([a, ab, ca]), np.array([ab, b, bc]), np.array([ca, bc, c]),
                    np.array([bc, ca, ab])]
        tris = nxt
    P = np.concatenate([pts @ t for t in tris])
    W = np.concatenate([wts / len(tris) for _ in tris])
    return P, W


def rule_points(rule, p0, p1, p2):
    """Map barycentric rule points onto triangles.

    p0, p1, p2: [..., 3] vertex arrays.  Returns points [..., Q, 3]."""
    bary, _ = rule
    return (bary[:, 0, None] * p0[..., None, :] + bary[:, 1, None] * p1[..., None, :]
            + bary[:, 2, None] * p2[..., None, :])

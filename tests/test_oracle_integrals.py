"""Pins of the oracle's panel integrals (Eq. RWG, Eq. Zb).

* closed-form potential integrals K0, K1 against brute force: a 200x200-point
  product rule for points off the triangle, and polar coordinates around the
  projected point (where the 1/R singularity cancels with the area element)
  for points inside the triangle;
* the Gram closed form against Radon's rule, exact for the quadratic integrand;
* Gram invariants: one triangle's block is symmetric positive semidefinite and
  the branch self term G_ii > 0;
* the inductive blocks: symmetric under exchange of the two triangles, equal
  to (int f_k).(int f_l)/R plus O(a/R) for far pairs (the first moment of
  f_k about the centroid does not vanish), where
  int_T (r - v_k)/(2A) dS = (c - v_k)/2;
* brute force for coplanar and edge-sharing pairs: a fully numerical 4-D
  integral with the inner integral done in polar coordinates.
"""
import numpy as np
import pytest

from oracle.integrals import potential_integrals, gram_local, pair_blocks, tri_geometry
from oracle.quadrature import collapsed_gauss, radon7, rule_points
from oracle import native

A0 = np.array([0.0, 0.0, 0.0])
A1 = np.array([1.0, 0.2, 0.0])
A2 = np.array([0.3, 0.9, 0.0])


def brute_offplane(r, a0, a1, a2, n=200):
    pts, w = collapsed_gauss(n)
    P = pts[:, 0, None] * a0 + pts[:, 1, None] * a1 + pts[:, 2, None] * a2
    A = 0.5 * np.linalg.norm(np.cross(a1 - a0, a2 - a0))
    nrm = np.cross(a1 - a0, a2 - a0)
    nrm /= np.linalg.norm(nrm)
    rho = r - ((r - a0) @ nrm) * nrm
    d = np.linalg.norm(P - r, axis=1)
    return A * np.sum(w / d), A * np.sum(w[:, None] * (P - rho) / d[:, None], axis=0)


def polar_inside(r, a0, a1, a2, n=400):
    """r inside the (planar) triangle: sum over the 3 sub-triangles (r, p, q),
    int dtheta int_0^rmax (1/rho) rho drho = int rmax dtheta (and rmax^2/2 u for K1)."""
    x, w = np.polynomial.legendre.leggauss(n)
    s, ws = 0.5 * (x + 1), 0.5 * w
    k0, k1 = 0.0, np.zeros(3)
    for p, q in ((a0, a1), (a1, a2), (a2, a0)):
        X = p[None] + s[:, None] * (q - p)[None]
        d = np.linalg.norm(X - r, axis=1)
        dth = np.linalg.norm(np.cross(X - r, (q - p)[None]), axis=1) / d ** 2
        k0 += np.sum(ws * dth * d)
        k1 += np.sum((ws * dth * d ** 2 / 2)[:, None] * (X - r) / d[:, None], axis=0)
    return k0, k1


@pytest.mark.parametrize("r", [[2.0, 1.0, 0.5], [0.4, 0.3, 0.3], [0.4, 0.3, 0.05],
                               [1.5, -0.2, 0.0], [-0.3, 0.5, -0.7], [0.2, 0.1, -0.02]])
def test_potential_integrals_offplane(r):
    r = np.array(r)
    k0, k1 = potential_integrals(r, A0, A1, A2)
    b0, b1 = brute_offplane(r, A0, A1, A2)
    tol = 1e-12 if abs(r[2]) > 0.2 or r[0] > 1.2 else 1e-6   # brute force loses near the plane
    assert abs(k0 - b0) / abs(b0) < tol
    assert np.abs(k1 - b1).max() / abs(b0) < tol


@pytest.mark.parametrize("r", [[0.4, 0.3, 0.0], [0.05, 0.02, 0.0], [0.5, 0.5, 0.0], [0.3, 0.8, 0.0]])
def test_potential_integrals_inside(r):
    r = np.array(r)
    k0, k1 = potential_integrals(r, A0, A1, A2)
    b0, b1 = polar_inside(r, A0, A1, A2)
    assert abs(k0 - b0) / b0 < 1e-12
    assert np.abs(k1 - b1).max() / b0 < 1e-12


def test_native_potentials_match():
    rng = np.random.default_rng(0)
    pT = rng.standard_normal((50, 3, 3))
    pS = rng.standard_normal((50, 3, 3))
    g = lambda p: 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1)
    a = pair_blocks(pT, g(pT), pS, g(pS), radon7())
    b = native.pair_blocks(pT, g(pT), pS, g(pS), radon7())
    assert np.abs(a - b).max() / np.abs(a).max() < 1e-12


def test_gram_closed_form_vs_exact_rule():
    rng = np.random.default_rng(1)
    p = rng.standard_normal((20, 3, 3))
    area = 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1)
    g = gram_local(p, area)
    rq = rule_points(radon7(), p[:, 0], p[:, 1], p[:, 2])
    w = radon7()[1]
    for t in range(20):
        f = (rq[t][:, None, :] - p[t][None, :, :]) / (2 * area[t])
        ref = area[t] * np.einsum("q,qki,qli->kl", w, f, f)
        assert np.abs(g[t] - ref).max() / np.abs(ref).max() < 1e-13
        ev = np.linalg.eigvalsh(g[t])
        assert ev.min() > -1e-12 * ev.max()


def test_gram_equilateral_closed_form():
    # unit equilateral triangle: int_T |r - v_k|^2 dS / (4A^2) = (a^2 A/ ... ) check
    # against the polar-moment identity  int_T |r - v|^2 dS = A (|c - v|^2 + J_c/A),
    # J_c = A a^2 / 12 for an equilateral triangle of side a.
    a = 1.0
    p = np.array([[[0, 0, 0], [a, 0, 0], [a / 2, a * np.sqrt(3) / 2, 0]]], float)
    A = np.sqrt(3) / 4 * a * a
    g = gram_local(p, np.array([A]))[0]
    c = p[0].mean(axis=0)
    ref = A * (np.sum((c - p[0, 0]) ** 2) + a * a / 12.0) / (4 * A * A)
    assert abs(g[0, 0] - ref) < 1e-14


def test_block_symmetry_and_far_limit():
    rng = np.random.default_rng(2)
    base = np.array([[0, 0, 0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.1]])
    other = np.array([[0, 0, 0], [0.8, -0.2, 0.3], [0.1, 0.7, -0.2]])
    errs = []
    for dist in [3.0, 10.0, 100.0, 1000.0]:
        off = np.array([dist, 0.3 * dist, -0.2 * dist])
        pT = base[None]
        pS = (other + off)[None]
        aT = np.array([0.5 * np.linalg.norm(np.cross(base[1] - base[0], base[2] - base[0]))])
        aS = np.array([0.5 * np.linalg.norm(np.cross(other[1] - other[0], other[2] - other[0]))])
        b1 = pair_blocks(pT, aT, pS, aS, collapsed_gauss(12))[0]
        b2 = pair_blocks(pS, aS, pT, aT, collapsed_gauss(12))[0]
        if dist <= 100.0:   # beyond, the closed form's logarithms cancel (about 1e-7 at 1000)
            assert np.abs(b1 - b2.T).max() / np.abs(b1).max() < 1e-8
        cT, cS = base.mean(0), (other + off).mean(0)
        fT = (cT - base) / 2.0          # int_T (r - v_k)/(2A) dS
        fS = (cS - (other + off)) / 2.0
        far = fT @ fS.T / np.linalg.norm(cT - cS)
        errs.append(np.abs(b1 - far).max() / np.abs(far).max())
        assert errs[-1] < 1.0 / dist
    # first order: ten times farther, ten times smaller
    assert 8.0 < errs[2] / errs[3] < 12.0


def brute_block(pT, pS, n_outer=24, n_polar=120):
    """4-D brute force: outer collapsed Gauss, inner integral in polar coordinates
    around each outer point's projection (coplanar pairs only)."""
    AT = 0.5 * np.linalg.norm(np.cross(pT[1] - pT[0], pT[2] - pT[0]))
    AS = 0.5 * np.linalg.norm(np.cross(pS[1] - pS[0], pS[2] - pS[0]))
    bary, w = collapsed_gauss(n_outer)
    R = bary @ pT
    x, wx = np.polynomial.legendre.leggauss(n_polar)
    s, ws = 0.5 * (x + 1), 0.5 * wx
    out = np.zeros((3, 3))
    for q in range(R.shape[0]):
        r = R[q]
        inner = np.zeros((3, 3))      # inner[l] = int (r' - v_l)/R dS'
        for p0, p1 in ((pS[0], pS[1]), (pS[1], pS[2]), (pS[2], pS[0])):
            X = p0[None] + s[:, None] * (p1 - p0)[None]
            d = np.linalg.norm(X - r, axis=1)
            cr = np.cross(X - r, (p1 - p0)[None])
            sgn = np.sign(cr[:, 2])      # signed angle (triangles in the z = 0 plane)
            dth = sgn * np.linalg.norm(cr, axis=1) / d ** 2
            u = (X - r) / d[:, None]
            # int_0^rmax (r + rho u - v_l)/rho rho drho = (r - v_l) rmax + u rmax^2/2
            for l in range(3):
                inner[l] += np.sum((ws * dth)[:, None] * ((r - pS[l])[None] * d[:, None]
                                                           + u * (d ** 2 / 2)[:, None]), axis=0)
        for k in range(3):
            for l in range(3):
                out[k, l] += w[q] * AT * np.dot(r - pT[k], inner[l])
    return out / (4 * AT * AS)


@pytest.mark.parametrize("case", ["self", "edge", "vertex"])
def test_singular_blocks_vs_brute_force(case):
    pT = np.array([[0, 0, 0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.0]])
    if case == "self":
        pS = pT.copy()
    elif case == "edge":
        pS = np.array([[1.0, 0.1, 0.0], [1.1, 1.0, 0.0], [0.2, 0.9, 0.0]])
    else:
        pS = np.array([[1.0, 0.1, 0.0], [1.9, 0.3, 0.0], [1.5, 0.9, 0.0]])
    aT = 0.5 * np.linalg.norm(np.cross(pT[1] - pT[0], pT[2] - pT[0]))
    aS = 0.5 * np.linalg.norm(np.cross(pS[1] - pS[0], pS[2] - pS[0]))
    ref = brute_block(pT, pS)
    got = pair_blocks(pT[None], np.array([aT]), pS[None], np.array([aS]), collapsed_gauss(24))[0]
    assert np.abs(got - ref).max() / np.abs(ref).max() < 2e-5
    # 16x16 outer (the pFFT near-field rule) stays within 1e-4 of the brute force
    got16 = pair_blocks(pT[None], np.array([aT]), pS[None], np.array([aS]), collapsed_gauss(16))[0]
    assert np.abs(got16 - ref).max() / np.abs(ref).max() < 1e-4

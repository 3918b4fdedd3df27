"""Pins of the dense MoM oracle against closed forms and invariants.

Closed forms (well-developed skin effect, Sec. II-A, Eq. ImpedanceOp):
* a long isolated round (polygonal) wire carries a uniform surface current by
  symmetry, so R = l / (sigma delta P_n), P_n the polygon's perimeter, and
  R grows as sqrt(f);
* its external inductance is the partial self-inductance of a thin tube, the
  Neumann mutual inductance of two filaments at the tube radius:
  L = mu0 l / (2 pi) [asinh(l/a) - sqrt(1 + (a/l)^2) + a/l];
  the surface impedance adds an internal reactance equal to R, so
  L_ext = (Im Z - Re Z) / w.
Invariants: Z = Z^T (reciprocity), Re Z and Im Z positive definite
(passivity), Z independent of the spanning tree (Sec. III-A: any tree gives an
independent and complete loop set).
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.mom import DenseMoM, resistance_inductance, surface_impedance
from oracle.integrals import MU0

UM = 1e-6


@pytest.fixture(scope="module")
def wire():
    m = synth.wire_array_mesh(1, 10 * UM, 400 * UM, 0.0, n_sides=8, n_seg=40, jitter=0.0,
                              sigma=4.1e7, name="wire")
    return m, DenseMoM(m)


def test_wire_resistance_uniform_perimeter(wire):
    m, D = wire
    f = np.array([1e9, 1e10])
    Z = D.port_impedance(f)
    R, _ = resistance_inductance(Z, f)
    a, l, n, sigma = 10 * UM, 400 * UM, 8, 4.1e7
    perim = n * 2 * a * np.sin(np.pi / n)
    for i, fi in enumerate(f):
        delta = np.sqrt(2.0 / (2 * np.pi * fi * MU0 * sigma))
        R0 = l / (sigma * delta * perim)
        # end caps add a little resistance
        assert 1.0 < R[i, 0, 0] / R0 < 1.03, (fi, R[i, 0, 0], R0)
    assert abs(R[1, 0, 0] / R[0, 0, 0] / np.sqrt(10.0) - 1.0) < 0.01


def test_wire_external_inductance_tube(wire):
    m, D = wire
    f = np.array([1e10])
    Z = D.port_impedance(f)[0, 0, 0]
    w = 2 * np.pi * f[0]
    Lext = (Z.imag - Z.real) / w
    a, l = 10 * UM, 400 * UM
    Lt = MU0 * l / (2 * np.pi) * (np.arcsinh(l / a) - np.sqrt(1 + (a / l) ** 2) + a / l)
    assert abs(Lext / Lt - 1.0) < 0.03, (Lext, Lt)


def test_surface_impedance_convention():
    # e^{jwt}, principal root: Z_s = (1+j)/(sigma delta)
    w, s = 2 * np.pi * 1e9, 5.8e7
    delta = np.sqrt(2.0 / (w * MU0 * s))
    zs = surface_impedance(w, s)
    assert abs(zs - (1 + 1j) / (s * delta)) < 1e-15
    assert abs(zs * zs - 1j * w * MU0 / s) < 1e-12 * abs(zs * zs)


@pytest.fixture(scope="module")
def two_port():
    m = synth.tiny_wires()
    return m, DenseMoM(m)


def test_reciprocity_and_passivity(two_port):
    m, D = two_port
    f = np.array([1e9, 5e9])
    Z = D.port_impedance(f)
    R, L = resistance_inductance(Z, f)
    for i in range(len(f)):
        assert np.abs(Z[i] - Z[i].T).max() < 1e-10 * np.abs(Z[i]).max()
        assert np.linalg.eigvalsh(0.5 * (R[i] + R[i].T)).min() > 0
        assert np.linalg.eigvalsh(0.5 * (L[i] + L[i].T)).min() > 0
        # mutual inductance of parallel wires is positive and below the self terms
        assert 0 < L[i, 0, 1] < min(L[i, 0, 0], L[i, 1, 1])


def test_tree_independence(two_port):
    m, D = two_port
    f = np.array([2e9])
    Z1 = D.port_impedance(f)
    L2 = build_loops(m, root="highest")
    D2 = DenseMoM(m, L2, Lt=D.Lt)           # same branches, other tree
    assert np.array_equal(L2.br_tri, D.loops.br_tri)
    Z2 = D2.port_impedance(f)
    assert np.abs(Z1 - Z2).max() < 1e-9 * np.abs(Z1).max()


def test_dense_loop_matrix_symmetric_and_inductive_pd(two_port):
    m, D = two_port
    A = D.loops.A.toarray()[:, :D.loops.nb]
    K = A @ D.Lt @ A.T
    assert np.abs(K - K.T).max() < 1e-12 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).min() > 0          # magnetic energy > 0

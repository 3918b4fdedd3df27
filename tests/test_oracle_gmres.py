"""Pins of the plain GMRES oracle with the paper's preconditioner (Sec. IV-A).

* P = A diag(Z_b) A^T is symmetric (Sec. IV-A states it) and sparse;
* GMRES converges to the direct solution of the same loop system;
* its residual estimate equals the true preconditioned residual;
* the preconditioner cuts the iteration count (the trend of Sec. V);
* port impedance through pFFT + GMRES agrees with the dense MoM.
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.mom import DenseMoM
from oracle.pfft import PfftSystem, PfftParams
from oracle.gmres import gmres, Precond, precond_matrix


@pytest.fixture(scope="module")
def system():
    m = synth.tiny_wires()
    L = build_loops(m)
    D = DenseMoM(m, L)
    S = PfftSystem(m, L, PfftParams(grid=(16, 8, 4), near_factor=5.0))
    return m, L, D, S


def test_precond_symmetric(system):
    m, L, D, S = system
    w = 2 * np.pi * 3e9
    P = precond_matrix(L, S.diag_Zb(w))
    assert abs(P - P.T).max() == 0.0


def test_gmres_matches_direct(system):
    m, L, D, S = system
    w = 2 * np.pi * 3e9
    Zl = D.Zl(w)
    pc = Precond(L, np.diag(D.Zb(w)))
    b = np.zeros(L.nl, complex)
    b[L.port_loop(1)] = 1.0
    x, it, hist = gmres(lambda v: Zl @ v, b, pc, tol=1e-11)
    xd = np.linalg.solve(Zl, b)
    assert np.linalg.norm(x - xd) < 1e-8 * np.linalg.norm(xd)
    r = pc.solve(b - Zl @ x)
    assert abs(np.linalg.norm(r) / np.linalg.norm(pc.solve(b)) - hist[-1]) < 1e-3 * hist[-1] + 1e-14


def test_gmres_restart_converges(system):
    m, L, D, S = system
    w = 2 * np.pi * 3e9
    Zl = D.Zl(w)
    b = synth.complex_gaussian(L.nl, 1, seed=9)[0]
    x, it, hist = gmres(lambda v: Zl @ v, b, None, tol=1e-8, restart=10, maxit=3000)
    assert np.linalg.norm(Zl @ x - b) < 1e-6 * np.linalg.norm(b)


def test_preconditioner_reduces_iterations(system):
    m, L, D, S = system
    w = 2 * np.pi * 3e9
    b = np.zeros(L.nl, complex)
    b[L.port_loop(0)] = 1.0
    mv = lambda v: S.matvec(v, w)
    _, it_p, _ = gmres(mv, b, Precond(L, S.diag_Zb(w)), tol=1e-6)
    _, it_n, _ = gmres(mv, b, None, tol=1e-6, maxit=1000)
    assert it_p < it_n


def test_pfft_gmres_port_impedance_vs_dense(system):
    m, L, D, S = system
    f = 3e9
    w = 2 * np.pi * f
    Zd = D.port_impedance([f])[0]
    pc = Precond(L, S.diag_Zb(w))
    Y = np.zeros((2, 2), complex)
    for p in range(2):
        b = np.zeros(L.nl, complex)
        b[L.port_loop(p)] = 1.0
        x, it, _ = gmres(lambda v: S.matvec(v, w), b, pc, tol=1e-8)
        for q in range(2):
            Y[q, p] = x[L.port_loop(q)]
    Z = np.linalg.inv(Y)
    assert np.abs(Z.real - Zd.real).max() < 1e-3 * np.abs(Zd.real).max()
    assert np.abs(Z.imag - Zd.imag).max() < 1e-3 * np.abs(Zd.imag).max()

"""Plain restarted GMRES with the paper's left preconditioner (Sec. IV-A).

Eq. (Precond): P = A Z_b^N A^T with Z_b^N = diag(Z_b) (the Gram and inductive
self terms of each branch; a port link carries no impedance).  Eq. (LoopWithP):
GMRES is run on P^-1 Z_l I_l = P^-1 V_l.  P is factorised directly (the paper
uses a sparse direct solver; here scipy's sparse LU).

Readings: x0 = 0; restart m; the stop test is the left-preconditioned residual
||P^-1 (V - Z_l I)|| / ||P^-1 V|| < tol.  Arnoldi by modified Gram-Schmidt,
least squares by Givens rotations.
Parity: pinned against the dense direct solution and against its own
monotone residual (tests/test_oracle_gmres.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def precond_matrix(loops, diag_zb):
    nb = loops.nb
    A = loops.A.tocsr()
    d = np.concatenate([diag_zb, np.zeros(loops.n_ports)])
    return (A @ sp.diags(d) @ A.T).tocsc()


class Precond:
    def __init__(self, loops, diag_zb):
        self.P = precond_matrix(loops, diag_zb)
        self.lu = spla.splu(self.P.astype(complex))

    def solve(self, y):
        return self.lu.solve(np.asarray(y, dtype=complex))


def gmres(matvec, b, precond=None, tol=1e-6, restart=200, maxit=2000):
    """Returns (x, iterations, history of preconditioned relative residuals)."""
    Mi = (lambda v: v) if precond is None else precond.solve
    b = np.asarray(b, dtype=complex)
    n = b.shape[0]
    x = np.zeros(n, dtype=complex)
    pb = Mi(b)
    nb = np.linalg.norm(pb)
    if nb == 0.0:
        return x, 0, [0.0]
    hist = [1.0]
    it = 0
    while it < maxit:
        r = Mi(b - matvec(x))
        beta = np.linalg.norm(r)
        if beta / nb < tol:
            break
        m = min(restart, maxit - it)
        V = np.zeros((m + 1, n), dtype=complex)
        Hh = np.zeros((m + 1, m), dtype=complex)
        cs = np.zeros(m, dtype=complex)
        sn = np.zeros(m, dtype=complex)
        g = np.zeros(m + 1, dtype=complex)
        g[0] = beta
        V[0] = r / beta
        k_done = 0
        for k in range(m):
            w = Mi(matvec(V[k]))
            for i in range(k + 1):
                Hh[i, k] = np.vdot(V[i], w)
                w = w - Hh[i, k] * V[i]
            Hh[k + 1, k] = np.linalg.norm(w)
            if Hh[k + 1, k] != 0:
                V[k + 1] = w / Hh[k + 1, k]
            # rotation i: [[conj c, conj s], [-s, c]] (unitary, zeroes H[i+1, i])
            for i in range(k):
                t = np.conj(cs[i]) * Hh[i, k] + np.conj(sn[i]) * Hh[i + 1, k]
                Hh[i + 1, k] = -sn[i] * Hh[i, k] + cs[i] * Hh[i + 1, k]
                Hh[i, k] = t
            a, bb = Hh[k, k], Hh[k + 1, k]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[k] = a / den if den else 1.0
            sn[k] = bb / den if den else 0.0
            Hh[k, k] = den
            Hh[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = np.conj(cs[k]) * g[k]
            it += 1
            k_done = k + 1
            hist.append(abs(g[k + 1]) / nb)
            if abs(g[k + 1]) / nb < tol:
                break
        y = np.linalg.solve(np.triu(Hh[:k_done, :k_done]), g[:k_done])
        x = x + V[:k_done].T @ y
        if hist[-1] < tol:
            break
    return x, it, hist

"""Dense method of moments of the MQS SIE and port impedance extraction (O1).

This is the plain definition the pFFT product approximates: every triangle
pair integrated (Eq. Zb), the branch system turned into the loop system
Z_l = A Z_b A^T (Eq. LoopVandI / FinalME), solved directly for one unit voltage
source per port (Sec. III-C), and the port impedance Z = Y^-1 with
Y[q, p] = current of port q's loop when port p is driven (R = Re Z,
L = Im Z / w; the loop values R_o, L_o of Sec. V-D follow from Z).

Per frequency (Eq. ImpedanceOp, with the e^{jwt} convention and the principal
root): Z_s = sqrt(j w mu0 / sigma) = (1 + j) sqrt(w mu0 / (2 sigma)).
Thickness-aware variant (the low-frequency remedy Sec. II-A names; reading in
the design notes): a conductor given an effective thickness t (twice its
cross-section area over its perimeter) uses the impedance of one face of a slab
of thickness t, Z_s = (gamma / sigma) coth(gamma t / 2) with
gamma = (1 + j) sqrt(w mu0 sigma / 2) = (1 + j) / delta.  It tends to the value
above when delta << t and to the DC sheet value 2 / (sigma t) as w -> 0, where
a uniform perimeter current gives the bar's DC resistance rho L / (w t).
Parity: pinned by closed forms (uniform-perimeter skin resistance of a long
polygonal wire, R proportional to sqrt(f), Neumann inductance of a long tube)
and invariants (Z = Z^T, R > 0, L > 0, tree independence) in
tests/test_oracle_mom.py.
"""
from __future__ import annotations

import numpy as np

from .graph import build_loops
from .integrals import (MU0, gram_matrix, symmetric_blocks, tri_branches, dense_rules)


def surface_impedance(omega, sigma, t_eff=0.0):
    """Z_s of a conductor; t_eff > 0 selects the slab form (module docstring)."""
    sigma = np.asarray(sigma, dtype=float)
    t_eff = np.broadcast_to(np.asarray(t_eff, dtype=float), sigma.shape)
    classic = (1.0 + 1.0j) * np.sqrt(omega * MU0 / (2.0 * sigma))
    gamma = (1.0 + 1.0j) * np.sqrt(omega * MU0 * sigma / 2.0)
    z = gamma * t_eff / 2.0
    # z coth z: its Taylor series where |z| is small, 1 / tanh otherwise
    small = np.abs(z) < 1e-2
    zs_ = np.where(small, 1.0, z)
    zcoth = np.where(small, 1.0 + z ** 2 / 3.0 - z ** 4 / 45.0, zs_ / np.tanh(zs_))
    slab = 2.0 / (sigma * np.where(t_eff > 0, t_eff, 1.0)) * zcoth
    out = np.where(t_eff > 0, slab, classic)
    return out[()] if out.ndim == 0 else out


def branch_zs(mesh, loops, omega, t_eff=None):
    """Z_s of each branch's conductor (both triangles of a branch share it);
    t_eff: effective thickness per conductor (None or 0: the classic form)."""
    cond = mesh.cond[loops.br_tri[:, 0]]
    t = np.zeros(mesh.ncond) if t_eff is None else np.asarray(t_eff, dtype=float)
    return surface_impedance(omega, mesh.sigma[cond], t[cond])


def assemble_from_blocks(mesh, loops, pi, pj, blocks):
    """Branch matrix sum over triangle pairs (i, j) of s_i s_j blocks[k, l],
    dense [nb, nb]."""
    tb, ts = tri_branches(mesh.nt, loops)
    nb = loops.nb
    out = np.zeros((nb, nb))
    for k in range(3):
        for l in range(3):
            bi = tb[pi, k]
            bj = tb[pj, l]
            ok = (bi >= 0) & (bj >= 0)
            np.add.at(out, (bi[ok], bj[ok]), ts[pi[ok], k] * ts[pj[ok], l] * blocks[ok, k, l])
    return out


def dense_Lt(mesh, loops, rules=None, far_ratio=4.0):
    """Dense Lt [nb, nb] = int int f_i . f_j / |r - r'| (no mu0/4pi), every pair
    with the closed-form inner integral; outer rule by proximity."""
    rt, rm, rf = dense_rules() if rules is None else rules
    nt = mesh.nt
    iu, ju = np.triu_indices(nt)
    blk = symmetric_blocks(mesh, iu, ju, rt, rf, far_ratio=far_ratio, rule_mid=rm)
    pi = np.concatenate([iu, ju[iu != ju]])
    pj = np.concatenate([ju, iu[iu != ju]])
    blocks = np.concatenate([blk, np.transpose(blk[iu != ju], (0, 2, 1))])
    return assemble_from_blocks(mesh, loops, pi, pj, blocks)


class DenseMoM:
    """Dense loop system of one mesh; Z(f) by direct solves."""

    def __init__(self, mesh, loops=None, Lt=None, t_eff=None):
        self.mesh = mesh
        self.loops = build_loops(mesh) if loops is None else loops
        self.G = gram_matrix(mesh, self.loops).toarray()
        self.Lt = dense_Lt(mesh, self.loops) if Lt is None else Lt
        self.t_eff = t_eff

    def Zb(self, omega):
        zs = branch_zs(self.mesh, self.loops, omega, self.t_eff)
        return zs[:, None] * self.G + (1j * omega * MU0 / (4.0 * np.pi)) * self.Lt

    def Zl(self, omega):
        nb = self.loops.nb
        A = self.loops.A.toarray()[:, :nb]
        return A @ self.Zb(omega) @ A.T

    def matvec(self, x, omega):
        """Loop-space product y = A Z_b A^T x (x: [nl] complex)."""
        nb = self.loops.nb
        A = self.loops.A[:, :nb]
        return A @ (self.Zb(omega) @ (A.T @ x))

    def port_impedance(self, freqs):
        """Z [nf, np, np] complex, by dense LU."""
        P = self.loops.n_ports
        out = np.zeros((len(freqs), P, P), dtype=complex)
        for fi, f in enumerate(freqs):
            w = 2.0 * np.pi * f
            Zl = self.Zl(w)
            V = np.zeros((self.loops.nl, P), dtype=complex)
            for p in range(P):
                V[self.loops.port_loop(p), p] = 1.0
            I = np.linalg.solve(Zl, V)
            Y = np.array([[I[self.loops.port_loop(q), p] for p in range(P)] for q in range(P)])
            out[fi] = np.linalg.inv(Y)
        return out


def bar_effective_thickness(width, thickness):
    """2 A / P of a width x thickness rectangle: the slab thickness whose DC
    sheet impedance makes a uniform perimeter current carry the bar's DC resistance."""
    return width * thickness / (width + thickness)


def resistance_inductance(Z, freqs):
    w = 2.0 * np.pi * np.asarray(freqs)
    return Z.real, Z.imag / w[:, None, None]

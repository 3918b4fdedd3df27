"""Lossy-conductor grid kernel and its grid convolution (oracle, test infrastructure only).

Plain FP64 CPU code used by the tests; the GPU library never imports it.

Sec. IV-B, step 2 evaluates the Toeplitz product phi_g = H Q_g of the grid
potentials with a kernel sampled at the node offsets; the paper's kernel is
the static Green's function G_0 = 1/(4 pi R) of Eq. (StaticGF), the MQS choice
of Sec. II-A for the exterior region.  The paper gives no interior kernel.  The
reading used for the lossy variant of step 2: inside a conductor of
conductivity sigma the MQS field obeys the lossy Helmholtz equation whose
free-space kernel is exp(-j k R)/(4 pi R) with

    k = (1 - j) / delta,   delta = sqrt(2 / (w mu0 sigma))   (the skin depth),

in the same e^{j w t} convention as Z_s of Eq. (ImpedanceOp), so
|exp(-j k R)| = exp(-R / delta) decays over a few skin depths and the kernel
tends to the static one as w -> 0.  As for the static kernel, the grid kernel
drops the 1/(4 pi) (applied with mu0 by the caller), takes the value h0 at zero
offset and, on the zero-padded 2N grid, is sampled at the signed offsets; the
offset +-N_d is never used by the aperiodic product and is set to zero.

The lossy variant of the whole product (Sec. IV-B steps 1-4 with that kernel in
place of the static one; reading in the design notes): per angular frequency
w the inductive term uses

    Lt_k[i, j] = int int f_i(r) . f_j(r') exp(-j k R) / R dS' dS,

split as the static integral 1/R (closed-form inner integral, oracle.integrals)
plus the bounded remainder (exp(-j k R) - 1)/R, which tends to -j k = -(1 + j)/delta
as R -> 0 and is integrated by the product of the 7-point Radon rule on both
triangles.  That product rule is symmetric in the two triangles, so the
blocks keep Lt_k = Lt_k^T.  The pre-corrected near blocks are
L_d = L_direct,k - (I H_k B)_near with H_k the lossy grid kernel.  The rule
resolves the remainder while |k| times the panel diameter is of order one or
below; the pins state the accuracy there.
"""
from __future__ import annotations

import numpy as np

from .quadrature import radon7, rule_points

MU0 = 4e-7 * np.pi


def skin_wavenumber(omega, sigma):
    """k = (1 - j)/delta with delta = sqrt(2/(omega mu0 sigma))."""
    delta = np.sqrt(2.0 / (omega * MU0 * sigma))
    return (1.0 - 1.0j) / delta


def lossy_kernel(d, h, k, h0=0.0):
    """exp(-j k r)/r at integer node offsets d [..., 3], r = |d o h|; h0 at d = 0."""
    r = np.linalg.norm(np.asarray(d, dtype=float) * np.asarray(h, dtype=float), axis=-1)
    zero = np.all(np.asarray(d) == 0, axis=-1)
    rs = np.where(zero, 1.0, r)
    return np.where(zero, complex(h0), np.exp(-1j * k * rs) / rs)


def padded_kernel(N, h, k, h0=0.0):
    """The kernel on the zero-padded [2N_x][2N_y][2N_z] grid at signed offsets,
    zero on the unused offset planes +-N_d."""
    M = 2 * np.asarray(N)
    ax = [np.where(np.arange(m) < m // 2, np.arange(m), np.arange(m) - m) for m in M]
    dx, dy, dz = np.meshgrid(*ax, indexing="ij")
    H = lossy_kernel(np.stack([dx, dy, dz], axis=-1), h, k, h0)
    for a, m in enumerate(M):
        sl = [slice(None)] * 3
        sl[a] = m // 2
        H[tuple(sl)] = 0.0
    return H


def convolve_lossy(Qg, h, k, h0=0.0):
    """phi_g = H_k Q_g for one grid Q_g [N_x, N_y, N_z] (zero-padded FFT)."""
    N = np.array(Qg.shape)
    M = 2 * N
    pad = np.zeros(tuple(M), dtype=complex)
    pad[:N[0], :N[1], :N[2]] = Qg
    out = np.fft.ifftn(np.fft.fftn(pad) * np.fft.fftn(padded_kernel(N, h, k, h0)))
    return out[:N[0], :N[1], :N[2]]


def convolve_lossy_direct(Qg, h, k, h0=0.0):
    """The same product by the direct O(N_g^2) sum over node pairs (tiny grids)."""
    Nx, Ny, Nz = Qg.shape
    idx = np.stack(np.meshgrid(np.arange(Nx), np.arange(Ny), np.arange(Nz), indexing="ij"),
                   axis=-1).reshape(-1, 3)
    Hm = lossy_kernel(idx[:, None, :] - idx[None, :, :], h, k, h0)
    return (Hm @ Qg.reshape(-1)).reshape(Qg.shape)


# ---------------------------------------------------------------- the lossy product (Sec. IV-B, lossy kernel)

def inv_skin_depth(omega, sigma):
    """1/delta = sqrt(omega mu0 sigma / 2)."""
    return np.sqrt(omega * MU0 * sigma / 2.0)


def smooth_remainder(R, inv_delta):
    """(exp(-j k R) - 1) / R with k = (1 - j)/delta, for R >= 0.

    With a = R/delta, exp(-j k R) = exp(-a) (cos a - j sin a); the real part of
    the numerator is written expm1(-a) cos a - 2 sin^2(a/2), which keeps its
    relative accuracy for small a.  At R = 0 the value is the limit -(1 + j)/delta."""
    R = np.asarray(R, dtype=float)
    a = R * inv_delta
    num = (np.expm1(-a) * np.cos(a) - 2.0 * np.sin(0.5 * a) ** 2) - 1j * np.exp(-a) * np.sin(a)
    with np.errstate(divide="ignore", invalid="ignore"):
        out = num / R
    return np.where(R > 0, out, -(1.0 + 1.0j) * inv_delta)


def remainder_blocks(pT, aT, pS, aS, inv_delta, rule=None):
    """3x3 blocks of the remainder for triangle pairs (T, S):
    Blk[k, l] = int_T int_S (r - v_k)/(2 A_T) . (r' - v'_l)/(2 A_S) g(|r - r'|)
    with g = smooth_remainder, by the product of `rule` (Radon 7) on T and S:
    A_T A_S sum_p sum_q w_p w_q ... = (1/4) sum_p sum_q w_p w_q (r_p - v_k).(r'_q - v'_l) g."""
    rule = radon7() if rule is None else rule
    w = rule[1]
    ro = rule_points(rule, pT[:, 0], pT[:, 1], pT[:, 2])           # [m, Q, 3]
    ri = rule_points(rule, pS[:, 0], pS[:, 1], pS[:, 2])
    d = np.linalg.norm(ro[:, :, None, :] - ri[:, None, :, :], axis=-1)
    g = smooth_remainder(d, inv_delta)
    fo = ro[:, :, None, :] - pT[:, None, :, :]                       # [m, Q, 3, 3]
    fi = ri[:, :, None, :] - pS[:, None, :, :]
    return 0.25 * np.einsum("p,q,mpki,mqli,mpq->mkl", w, w, fo, fi, g)


def grid_blocks_complex(op, ti, tj, Hpad):
    """(I H B) blocks of the pairs (ti, tj) for a complex padded kernel: the grid
    blocks are linear in the kernel table, so they are the blocks of its real
    part plus j times those of its imaginary part (each the plain C double sum
    of oracle.native, pinned against the numpy double sum)."""
    from .native import grid_blocks
    re = grid_blocks(ti, tj, op.start, op.lw, op.mom, np.ascontiguousarray(Hpad.real))
    im = grid_blocks(ti, tj, op.start, op.lw, op.mom, np.ascontiguousarray(Hpad.imag))
    return re + 1j * im


class LossyPfft:
    """pFFT operator of the lossy kernel at one (omega, sigma), built on a static
    oracle.pfft.Pfft (same grid, stencils, projection B and near list)."""

    def __init__(self, static, omega, sigma, native=True):
        self.s = static
        self.omega, self.sigma = omega, sigma
        self.inv_delta = inv_skin_depth(omega, sigma)
        k = (1.0 - 1.0j) * self.inv_delta
        self.Hpad = padded_kernel(static.N, static.h, k, static.p.h0)
        self.Hhat = np.fft.fftn(self.Hpad)
        g = static.geo
        i, j = static.near_i, static.near_j
        rem = remainder_blocks(g["p"][i], g["area"][i], g["p"][j], g["area"][j], self.inv_delta)
        self.L_direct = static.L_direct + rem
        if native:
            self.L_grid = grid_blocks_complex(static, i, j, self.Hpad)
        else:
            Hs = static.Hpad
            static.Hpad = self.Hpad
            try:
                self.L_grid = static.grid_blocks(i, j, native=False)
            finally:
                static.Hpad = Hs
        self.L_d = self.L_direct - self.L_grid
        self._near = static.near_matrix(self.L_d)

    def convolve(self, Qg):
        N = self.s.N
        pad = np.zeros(tuple(2 * N), dtype=complex)
        pad[:N[0], :N[1], :N[2]] = Qg
        return np.fft.ifftn(np.fft.fftn(pad) * self.Hhat)[:N[0], :N[1], :N[2]]

    def far(self, alpha):
        Qg = (self.s.B @ alpha).reshape(3, *self.s.N)
        phi = np.stack([self.convolve(Qg[c]) for c in range(3)]).reshape(-1)
        return self.s.B.T @ phi

    def Lt_apply(self, alpha):
        return self.far(alpha) + self._near @ alpha

    def diag_Lt(self):
        """Self terms Lt_k[e, e] of every branch (from the direct near blocks)."""
        return self.s.near_matrix(self.L_direct).diagonal()


class LossyPfftSystem:
    """Loop-space product y = A (Z_s G + j w mu0/4pi (L_d,k + I H_k B)) A^T x with the
    lossy kernel of conductivity sigma at each w (operators cached per w)."""

    def __init__(self, mesh, loops, params, sigma=None, targets=None):
        from .pfft import PfftSystem
        self.base = PfftSystem(mesh, loops, params, targets=targets)
        self.mesh, self.loops = mesh, loops
        self.sigma = float(mesh.sigma[0]) if sigma is None else float(sigma)
        self.A = self.base.A
        self.G = self.base.G
        self._ops = {}

    def op(self, omega):
        if omega not in self._ops:
            self._ops[omega] = LossyPfft(self.base.op, omega, self.sigma)
        return self._ops[omega]

    def branch_product(self, alpha, omega):
        from .mom import branch_zs
        zs = branch_zs(self.mesh, self.loops, omega)
        return zs * (self.G @ alpha) + (1j * omega * MU0 / (4.0 * np.pi)) * self.op(omega).Lt_apply(alpha)

    def matvec(self, x, omega):
        return self.A @ self.branch_product(self.A.T @ x, omega)

    def diag_Zb(self, omega):
        from .mom import branch_zs
        zs = branch_zs(self.mesh, self.loops, omega)
        return zs * self.G.diagonal() + (1j * omega * MU0 / (4.0 * np.pi)) * self.op(omega).diag_Lt()


def dense_Lt_lossy(mesh, loops, omega, sigma, static_Lt=None):
    """Dense Lt_k [nb, nb] (no mu0/4pi): the dense static Lt of oracle.mom (every pair,
    closed-form inner integral) plus the remainder of every pair by the Radon 7 x 7
    product rule."""
    from .mom import dense_Lt, assemble_from_blocks
    from .integrals import tri_geometry
    Lt0 = dense_Lt(mesh, loops) if static_Lt is None else static_Lt
    g = tri_geometry(mesh.xyz, mesh.tri)
    nt = mesh.nt
    pi, pj = np.meshgrid(np.arange(nt), np.arange(nt), indexing="ij")
    pi, pj = pi.ravel(), pj.ravel()
    rem = remainder_blocks(g["p"][pi], g["area"][pi], g["p"][pj], g["area"][pj], inv_skin_depth(omega, sigma))
    Rr = assemble_from_blocks(mesh, loops, pi, pj, rem.real)
    Ri = assemble_from_blocks(mesh, loops, pi, pj, rem.imag)
    return Lt0 + Rr + 1j * Ri

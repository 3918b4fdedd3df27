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
"""
from __future__ import annotations

import numpy as np

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

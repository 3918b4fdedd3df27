"""Pins of the lossy grid kernel and its convolution (oracle/lossy.py).

* the FFT product equals the direct sum over node pairs (Toeplitz embedding);
* as w -> 0 the lossy kernel tends to the static 1/R one (closed-form limit);
* kernel values: |K| = exp(-r/delta)/r and arg K = -r/delta (mod 2 pi);
* the operator is complex symmetric (K(d) = K(-d)): <u, K v> = <v, K u>
  without conjugation, and it is not Hermitian;
* a planted mistake (a conjugated k, i.e. a growing exponential) fails the
  value pin.
"""
import numpy as np
import pytest

from oracle.lossy import (MU0, skin_wavenumber, lossy_kernel, padded_kernel, convolve_lossy,
                          convolve_lossy_direct)

H = np.array([1.5e-6, 2.0e-6, 0.7e-6])
SIG = 5.8e7


def rand_grid(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("f", [1e6, 1e9, 2e10])
def test_fft_product_equals_direct_sum(f):
    k = skin_wavenumber(2 * np.pi * f, SIG)
    q = rand_grid((6, 4, 4), 1)
    a = convolve_lossy(q, H, k, h0=0.3)
    b = convolve_lossy_direct(q, H, k, h0=0.3)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_static_limit():
    """w -> 0: exp(-jkR) = 1 - jkR + ..., so the relative change is O(|k| R_max)."""
    k = skin_wavenumber(2 * np.pi * 1e-3, SIG)     # delta ~ 2 m against a ~10 um grid
    q = rand_grid((6, 4, 4), 2)
    a = convolve_lossy_direct(q, H, k)
    idx = np.stack(np.meshgrid(np.arange(6), np.arange(4), np.arange(4), indexing="ij"), -1).reshape(-1, 3)
    d = idx[:, None, :] - idx[None, :, :]
    r = np.linalg.norm(d * H, axis=-1)
    Hs = np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), 0.0)
    b = (Hs @ q.reshape(-1)).reshape(q.shape)
    rmax = np.linalg.norm(np.array([5, 3, 3]) * H)
    assert np.abs(a - b).max() < 2 * abs(k) * rmax * np.abs(b).max()
    assert np.abs(a - b).max() > 0.0


def test_kernel_values_closed_form():
    w = 2 * np.pi * 3e9
    delta = np.sqrt(2.0 / (w * MU0 * SIG))
    assert abs(delta - 1.0 / np.sqrt(np.pi * 3e9 * MU0 * SIG)) < 1e-15   # the 1/sqrt(pi f mu sigma) form
    assert 1.20e-6 < delta < 1.21e-6                                      # Cu at 3 GHz
    d = np.array([[1, 0, 0], [2, 3, 1], [0, 0, 5]])
    r = np.linalg.norm(d * H, axis=-1)
    K = lossy_kernel(d, H, skin_wavenumber(w, SIG))
    assert np.allclose(np.abs(K), np.exp(-r / delta) / r, rtol=1e-13)
    assert np.allclose(np.angle(K), np.angle(np.exp(-1j * r / delta)), atol=1e-12)
    assert lossy_kernel(np.zeros(3, int), H, 1.0, h0=0.25) == 0.25
    # a conjugated wavenumber grows instead of decaying: the value pin catches it
    Kbad = lossy_kernel(d, H, np.conj(skin_wavenumber(w, SIG)))
    assert not np.allclose(np.abs(Kbad), np.exp(-r / delta) / r, rtol=1e-3)


def test_complex_symmetric_not_hermitian():
    k = skin_wavenumber(2 * np.pi * 1e9, SIG)
    u, v = rand_grid((5, 4, 3), 3), rand_grid((5, 4, 3), 4)
    Kv, Ku = convolve_lossy(v, H, k), convolve_lossy(u, H, k)
    assert abs(np.sum(u * Kv) - np.sum(v * Ku)) < 1e-12 * abs(np.sum(u * Kv))
    assert abs(np.vdot(u, Kv) - np.conj(np.vdot(v, Ku))) > 1e-3 * abs(np.vdot(u, Kv))


def test_padded_kernel_layout_matches_static_convention():
    """Same offsets, wrap and zeroed +-N planes as the static kernel table."""
    k = skin_wavenumber(2 * np.pi * 1e-3, SIG)
    N = np.array([4, 4, 2])

    Kp = padded_kernel(N, H, k)
    ax = [np.where(np.arange(m) < m // 2, np.arange(m), np.arange(m) - m) for m in 2 * N]
    for a, m in enumerate(2 * N):
        sl = [slice(None)] * 3
        sl[a] = m // 2
        assert np.all(Kp[tuple(sl)] == 0)
    dx, dy, dz = np.meshgrid(*ax, indexing="ij")
    r = np.linalg.norm(np.stack([dx, dy, dz], -1) * H, axis=-1)
    live = (r > 0) & (Kp != 0)
    # exp(-jkr)/r = 1/r - jk + O(k^2 r): within 2|k| of 1/r at the signed offsets
    assert np.abs(Kp[live] - 1 / r[live]).max() < 2 * abs(k)

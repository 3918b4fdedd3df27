"""Pins of the thickness-aware (slab) surface impedance in the oracle.

Closed forms fix it: a straight bar driven end face to end face carries a
uniform perimeter current at DC on its side faces, so with the slab impedance at
effective thickness t = 2A/P each unit of length adds exactly rho / (w t) of
resistance (the volume value); the end faces are the contacts, and the halves of
the basis functions lying on them add a length correction that vanishes in
proportion to the end-face mesh size.  The slab impedance tends to the classic
(1+j)/(sigma delta) when delta << t and to 2 / (sigma t) as w -> 0; its
small-argument series and direct evaluation agree.
"""
import numpy as np
import pytest

import synth
from oracle.integrals import MU0
from oracle.mom import DenseMoM, surface_impedance, bar_effective_thickness

UM = 1e-6
SIG = 5.8e7


def dc_resistance(L, W, T, nx, ny, nz, jitter=0.0):
    m = synth.box_mesh(L * UM, W * UM, T * UM, nx, ny, nz, jitter=jitter, seed=5, sigma=SIG)
    Z = DenseMoM(m, t_eff=[bar_effective_thickness(W * UM, T * UM)]).port_impedance([0.0])[0, 0, 0]
    assert abs(Z.imag) < 1e-12 * abs(Z.real)
    return Z.real


@pytest.mark.parametrize("ny,nz", [(2, 1), (4, 2)])
def test_dc_resistance_per_length_is_rho_over_wt(ny, nz):
    """Same end faces, lengths 100 and 200 um: R(200) - R(100) = rho 100 um / (w t)."""
    W, T = 20, 10
    r1 = dc_resistance(100, W, T, 10, ny, nz)
    r2 = dc_resistance(200, W, T, 20, ny, nz)
    slope = 100 * UM / (SIG * W * UM * T * UM)
    assert abs((r2 - r1) / slope - 1.0) < 1e-6, (r1, r2, slope)   # dense LU of the DC system


def test_dc_resistance_converges_to_rho_l_over_wt():
    """The end-face correction halves when the end-face mesh spacing halves."""
    L, W, T = 100, 20, 10
    R0 = L * UM / (SIG * W * UM * T * UM)
    e1 = dc_resistance(L, W, T, 10, 4, 2) / R0 - 1.0
    e2 = dc_resistance(L, W, T, 10, 8, 4) / R0 - 1.0
    assert 0 < e2 < e1 < 0.05
    assert abs(e1 / e2 - 2.0) < 1e-6, (e1, e2)


def test_classic_form_has_no_dc_result_but_slab_does():
    m = synth.tiny_bar()
    D = DenseMoM(m)
    assert np.allclose(D.Zb(0.0), 0.0)            # Z_s(0) = 0 and c_L = 0: singular loop system
    t = bar_effective_thickness(20 * UM, 10 * UM)
    Dg = DenseMoM(m, Lt=D.Lt, t_eff=[t])
    s = np.linalg.svd(Dg.Zl(0.0), compute_uv=False)
    assert s.min() > 1e-8 * s.max()


def test_slab_limits():
    sigma, t = 4.1e7, 8 * UM
    # DC sheet value
    assert abs(surface_impedance(0.0, sigma, t) - 2.0 / (sigma * t)) < 1e-15 * 2.0 / (sigma * t)
    # delta << t: within the exponentially small coth correction of the classic value
    for f in (1e10, 1e11):
        w = 2 * np.pi * f
        delta = np.sqrt(2.0 / (w * MU0 * sigma))
        zc = surface_impedance(w, sigma)
        zg = surface_impedance(w, sigma, t)
        assert abs(zg / zc - 1.0) < 3.0 * np.exp(-t / delta), (f, zg, zc)
    # the classic value is unchanged by t_eff = 0
    w = 2 * np.pi * 1e9
    assert surface_impedance(w, sigma, 0.0) == surface_impedance(w, sigma)


def test_slab_series_and_direct_agree_at_the_switch():
    sigma, t = 5.8e7, 10 * UM
    # |z| = |gamma| t / 2 = 1e-2  <=>  w = 2 (2e-2 / t)^2 / (2 mu0 sigma)
    w0 = (2e-2 / t) ** 2 / (MU0 * sigma)
    lo = surface_impedance(w0 * (1 - 1e-9), sigma, t)
    hi = surface_impedance(w0 * (1 + 1e-9), sigma, t)
    assert abs(lo - hi) < 1e-12 * abs(hi)
    # and the slab value at moderate argument against coth from exponentials
    w = 2 * np.pi * 1e8
    g = (1 + 1j) * np.sqrt(w * MU0 * sigma / 2)
    z = g * t / 2
    ref = g / sigma * (np.exp(z) + np.exp(-z)) / (np.exp(z) - np.exp(-z))
    assert abs(surface_impedance(w, sigma, t) - ref) < 1e-13 * abs(ref)

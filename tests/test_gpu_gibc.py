"""GPU parity of the thickness-aware (slab) surface impedance.

The slab form Z_s = (gamma/sigma) coth(gamma t/2) (oracle/mom.py) changes only
the per-frequency scalars of Eq. ImpedanceOp, so the matvec and the
preconditioner must match the oracle built with the same thicknesses to the
usual bounds (FP64 1e-10, mixed 1e-5, preconditioner 1e-9), DC included.  The
solve must give the bar's DC resistance per length rho / (w t) of the closed
form (oracle pin) and R, L within 1e-3 of the dense oracle at 1 GHz.
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.mom import DenseMoM, bar_effective_thickness
from oracle.pfft import PfftSystem, PfftParams
from oracle.gmres import Precond

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, SieError, SPACE_LOOP, PREC_FP64, PREC_MIXED  # noqa: E402

UM = 1e-6
P_WIRES = dict(grid=(16, 8, 4), order=3, near_factor=5.0, near_min_diam=2.0, n_touch=16, h0=0.0)
T_WIRE = 10 * UM   # 2 A / P of a round wire of radius r is r


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


@pytest.fixture(scope="module")
def wires():
    m = synth.tiny_wires()
    O = build_loops(m)
    t = np.full(m.ncond, T_WIRE)
    S = PfftSystem(m, O, PfftParams(grid=P_WIRES["grid"], order=3, near_factor=5.0, near_min_diam=2.0,
                                    n_touch=16), t_eff=t)
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, P_WIRES)
    P.set_surface_model(t)
    return m, O, S, P


def test_matvec_with_slab_surface_model(wires):
    m, O, S, P = wires
    om = 2 * np.pi * np.array([0.0, 1e5, 1e7, 1e9])
    x = synth.complex_gaussian(O.nl, om.size, seed=81)
    ref = np.stack([S.matvec(x[r], om[r]) for r in range(om.size)])
    y64 = api.pfft_matvec(P, torch.from_numpy(x).cuda(), om, SPACE_LOOP, PREC_FP64).cpu().numpy()
    y32 = api.pfft_matvec(P, torch.from_numpy(x).cuda(), om, SPACE_LOOP, PREC_MIXED).cpu().numpy()
    assert rel(y64, ref).max() < 1e-10
    assert rel(y32, ref).max() < 1e-5


def test_precond_with_slab_surface_model(wires):
    m, O, S, P = wires
    om = 2 * np.pi * np.array([0.0, 1e6, 1e9])
    y = synth.complex_gaussian(O.nl, om.size, seed=82)
    ref = np.stack([Precond(O, S.diag_Zb(om[r])).solve(y[r]) for r in range(om.size)])
    z = api.pfft_precond_apply(P, torch.from_numpy(y).cuda(), om, prec=PREC_FP64).cpu().numpy()
    assert rel(z, ref).max() < 1e-9


def test_surface_model_switches_and_rejects():
    m = synth.tiny_bar()
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, dict(grid=(16, 8, 8), order=3, near_factor=5.0, near_min_diam=2.0, n_touch=16, h0=0.0))
    with pytest.raises(SieError):
        api.sie_solve(P, [0.0])                      # classic model: no DC
    P.set_surface_model([bar_effective_thickness(20 * UM, 10 * UM)])
    Z, st = api.sie_solve(P, [0.0, 1e9], tol=1e-10)
    assert st["converged"] and abs(Z[0, 0, 0].imag) < 1e-9 * abs(Z[0, 0, 0].real)
    P.set_surface_model(None)                        # back to classic: cached factors rebuilt
    Zc, _ = api.sie_solve(P, [1e9], tol=1e-10)
    assert abs(Zc[0, 0, 0] - Z[1, 0, 0]) > 1e-6 * abs(Zc[0, 0, 0])
    with pytest.raises(SieError):
        P.set_surface_model([-1.0])


@pytest.mark.parametrize("ny,nz", [(2, 1), (4, 2)])
def test_dc_resistance_per_length(ny, nz):
    """Bars of 100 and 200 um with the same end faces: R(200) - R(100) = rho 100 um / (w t)."""
    W, T, sig = 20, 10, 5.8e7
    R = []
    for Lum, nx in ((100, 10), (200, 20)):
        m = synth.box_mesh(Lum * UM, W * UM, T * UM, nx, ny, nz, jitter=0.0, seed=5, sigma=sig)
        M = api.Mesh.from_synth(m)
        L = api.Loops(M, m.ports)
        P = api.Plan(M, L, dict(grid=(32 if Lum == 100 else 64, 8, 8), order=3, near_factor=5.0,
                                near_min_diam=2.0, n_touch=16, h0=0.0))
        P.set_surface_model([bar_effective_thickness(W * UM, T * UM)])
        Z, st = api.sie_solve(P, [0.0], tol=1e-11, restart=300, max_iter=3000)
        assert st["converged"]
        R.append(Z[0, 0, 0].real)
    slope = 100 * UM / (sig * W * UM * T * UM)
    assert abs((R[1] - R[0]) / slope - 1.0) < 1e-6, (R, slope)


def test_bar_r_l_vs_dense_oracle_with_slab_model():
    m = synth.tiny_bar()
    t = bar_effective_thickness(20 * UM, 10 * UM)
    D = DenseMoM(m, t_eff=[t])
    f = np.array([0.0, 1e8, 1e9])
    Zd = D.port_impedance(f)
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, dict(grid=(16, 8, 8), order=3, near_factor=5.0, near_min_diam=2.0, n_touch=16, h0=0.0))
    P.set_surface_model([t])
    Z, st = api.sie_solve(P, f, tol=1e-10)
    assert st["converged"]
    assert np.all(np.abs(Z.real / Zd.real - 1.0) < 1e-3)
    assert np.all(np.abs(Z[1:].imag / Zd[1:].imag - 1.0) < 1e-3)   # L = Im Z / w (w > 0)

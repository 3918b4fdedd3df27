"""GPU parity of the preconditioner and of the port-impedance solve (Sec. IV-A).

* pfft_precond_apply (P^-1 through the nodal Laplacian, band LDL^T on the
  device) against the oracle's literal P = A diag(Z_b) A^T factorised by a
  sparse LU: relative error per right-hand side <= 1e-9;
* sie_solve (device GMRES) against the oracle's pFFT + GMRES at the same
  tolerance, and R = Re Z, L = Im Z / w against the dense MoM within 1e-3.
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.mom import DenseMoM, resistance_inductance
from oracle.pfft import PfftSystem, PfftParams
from oracle.gmres import gmres, Precond

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, PREC_FP64, PREC_MIXED  # noqa: E402


def make(m, params):
    O = build_loops(m)
    S = PfftSystem(m, O, PfftParams(grid=params["grid"], order=params["order"],
                                    near_factor=params["near_factor"], near_min_diam=params["near_min_diam"],
                                    n_touch=params["n_touch"]))
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    return O, S, api.Plan(M, L, params)


P_WIRES = dict(grid=(16, 8, 4), order=3, near_factor=5.0, near_min_diam=2.0, n_touch=16, h0=0.0)
P_BAR = dict(grid=(16, 8, 8), order=3, near_factor=5.0, near_min_diam=2.0, n_touch=16, h0=0.0)


@pytest.mark.parametrize("make_mesh,params", [(synth.tiny_wires, P_WIRES), (synth.tiny_bar, P_BAR),
                                              (synth.tiny_two_bars, P_BAR)])
def test_precond_matches_oracle(make_mesh, params):
    m = make_mesh()
    O, S, P = make(m, params)
    om = 2 * np.pi * np.array([1e8, 1e9, 1e9, 2e10])
    y = synth.complex_gaussian(O.nl, 4, seed=81)
    z = api.pfft_precond_apply(P, torch.from_numpy(y).cuda(), om).cpu().numpy()
    for r in range(4):
        ref = Precond(O, S.diag_Zb(om[r])).solve(y[r])
        assert np.linalg.norm(z[r] - ref) < 1e-9 * np.linalg.norm(ref), r


def test_precond_mixed_sweeps():
    """FP32 sweeps on the rounded FP64 factor: within FP32 accuracy of the oracle."""
    m = synth.tiny_wires()
    O, S, P = make(m, P_WIRES)
    om = 2 * np.pi * np.array([1e9, 1e10, 1e8])
    y = synth.complex_gaussian(O.nl, 3, seed=83)
    z = api.pfft_precond_apply(P, torch.from_numpy(y).cuda(), om, prec=PREC_MIXED).cpu().numpy()
    for r in range(3):
        ref = Precond(O, S.diag_Zb(om[r])).solve(y[r])
        assert np.linalg.norm(z[r] - ref) < 1e-4 * np.linalg.norm(ref), r


def test_precond_batched_many_rhs():
    """40 right-hand sides over 5 frequencies (several factor slots) on the bar."""
    m = synth.tiny_bar()
    O, S, P = make(m, P_BAR)
    om = 2 * np.pi * np.repeat(np.logspace(8, 10, 5), 8)
    y = synth.complex_gaussian(O.nl, 40, seed=91)
    z = api.pfft_precond_apply(P, torch.from_numpy(y).cuda(), om).cpu().numpy()
    for r in range(0, 40, 7):
        ref = Precond(O, S.diag_Zb(om[r])).solve(y[r])
        assert np.linalg.norm(z[r] - ref) < 1e-9 * np.linalg.norm(ref), r


def test_solve_matches_oracle_gmres_and_dense():
    m = synth.tiny_wires()
    O, S, P = make(m, P_WIRES)
    D = DenseMoM(m, O)
    freqs = np.array([1e9, 1e10])
    Z, st = api.sie_solve(P, freqs, tol=1e-8, restart=60, prec=PREC_FP64)
    assert st["converged"] and st["n_not_converged"] == 0
    Zd = D.port_impedance(freqs)
    for f, fr in enumerate(freqs):
        w = 2 * np.pi * fr
        Y = np.zeros((2, 2), complex)
        for p in range(2):
            b = np.zeros(O.nl, complex)
            b[O.port_loop(p)] = 1.0
            x, _, _ = gmres(lambda v: S.matvec(v, w), b, Precond(O, S.diag_Zb(w)), tol=1e-10)
            Y[:, p] = [x[O.port_loop(q)] for q in range(2)]
        Zo = np.linalg.inv(Y)
        assert np.abs(Z[f] - Zo).max() < 1e-6 * np.abs(Zo).max()
    R, L = resistance_inductance(Z, freqs)
    Rd, Ld = resistance_inductance(Zd, freqs)
    assert np.abs(R - Rd).max() < 1e-3 * np.abs(Rd).max()
    assert np.abs(L - Ld).max() < 1e-3 * np.abs(Ld).max()
    # reciprocity of the solved impedance
    assert np.abs(Z - np.transpose(Z, (0, 2, 1))).max() < 1e-6 * np.abs(Z).max()


def test_solve_mixed_precision():
    m = synth.tiny_wires()
    O, S, P = make(m, P_WIRES)
    freqs = np.array([3e9])
    Z64, _ = api.sie_solve(P, freqs, tol=1e-8, restart=60, prec=PREC_FP64)
    Z32, st = api.sie_solve(P, freqs, tol=1e-6, restart=60, prec=PREC_MIXED)
    assert st["converged"]
    assert np.abs(Z32 - Z64).max() < 1e-4 * np.abs(Z64).max()


def test_solve_mixed_with_fp64_refinement_matches_fp64():
    """Iterative refinement (FP64 restart residuals, mixed Arnoldi cycles):
    the mixed solve converges on the true FP64 residual, so its Z agrees with
    the FP64 solve far more closely than the mixed solve alone."""
    m = synth.tiny_wires()
    O, S, P = make(m, P_WIRES)
    freqs = np.array([1e8, 3e9])
    Z64, st64 = api.sie_solve(P, freqs, tol=1e-10, restart=60, prec=PREC_FP64)
    Zir, st = api.sie_solve(P, freqs, tol=1e-10, restart=60, prec=PREC_MIXED, refine=True)
    assert st["converged"] and st["residual_max"] < 1e-10
    assert np.abs(Zir - Z64).max() < 1e-8 * np.abs(Z64).max()
    # the refined solve alternates precisions on one plan: FP64 matvecs still match the oracle
    om = 2 * np.pi * np.array([2e9])
    x = synth.complex_gaussian(O.nl, 1, seed=5)
    y = api.pfft_matvec(P, torch.from_numpy(x).cuda(), om).cpu().numpy()
    ref = S.matvec(x[0], om[0])
    assert np.linalg.norm(y[0] - ref) < 1e-10 * np.linalg.norm(ref)


def test_solve_without_preconditioner_needs_more_iterations():
    m = synth.tiny_wires()
    O, S, P = make(m, P_WIRES)
    _, with_p = api.sie_solve(P, [5e9], tol=1e-6, restart=100, precond=1)
    _, no_p = api.sie_solve(P, [5e9], tol=1e-6, restart=100, max_iter=600, precond=0)
    assert with_p["iterations_max"] < no_p["iterations_max"]


def test_bar_1500_resistance_inductance_vs_dense():
    """Cu bar 1000 x 20 x 10 um at 1 GHz: R and L within 1e-3 of the dense MoM."""
    w = synth.bar_1500()
    m = w["mesh"]
    params = dict(grid=w["grid"], order=3, near_factor=4.0, near_min_diam=2.0, n_touch=16, h0=0.0)
    O, S, P = make(m, params)
    Z, st = api.sie_solve(P, w["freqs"], tol=1e-8, restart=100)
    assert st["converged"]
    Zd = DenseMoM(m, O).port_impedance(w["freqs"])
    R, L = resistance_inductance(Z, w["freqs"])
    Rd, Ld = resistance_inductance(Zd, w["freqs"])
    assert abs(R[0, 0, 0] / Rd[0, 0, 0] - 1) < 1e-3
    assert abs(L[0, 0, 0] / Ld[0, 0, 0] - 1) < 1e-3


UM = 1e-6
# small near radius: diag(Z_b) needs only the self blocks, and the oracle stays fast
P_WIDE = dict(grid=(32, 8, 8), order=3, near_factor=1.0, near_min_diam=1.0, n_touch=8, h0=0.0)


def wide_bar(seed=7, origin=(0.0, 0.0, 0.0)):
    """Long bar with a 12 x 8-cell cross-section (~80 triangles per ring, 20
    rings): its preconditioner band is wider than a warp."""
    return synth.box_mesh(200 * UM, 24 * UM, 16 * UM, 20, 12, 8, jitter=0.1, seed=seed, origin=origin)


def wide_two_bars():
    return synth.merge([wide_bar(7), wide_bar(8, origin=(0.0, 60 * UM, 0.0))], name="wide_two_bars")


@pytest.mark.parametrize("make_mesh", [wide_bar, wide_two_bars], ids=["one", "two_conductors"])
def test_precond_wide_band_matches_oracle(make_mesh):
    """CTA-wide band sweeps (31 < W < 1024): FP64 within 1e-9 of the oracle's
    sparse LU of P, FP32 sweeps on the rounded factor within 1e-4."""
    m = make_mesh()
    O, S, P = make(m, P_WIDE)
    info = api.precond_info(P)
    assert 31 < info["band_width"] < 1024, info
    om = 2 * np.pi * np.array([1e8, 1e9, 1e9, 2e10, 5e10])
    y = synth.complex_gaussian(O.nl, om.size, seed=85)
    z64 = api.pfft_precond_apply(P, torch.from_numpy(y).cuda(), om).cpu().numpy()
    z32 = api.pfft_precond_apply(P, torch.from_numpy(y).cuda(), om, prec=PREC_MIXED).cpu().numpy()
    for r in range(om.size):
        ref = Precond(O, S.diag_Zb(om[r])).solve(y[r])
        assert np.linalg.norm(z64[r] - ref) < 1e-9 * np.linalg.norm(ref), r
        assert np.linalg.norm(z32[r] - ref) < 1e-4 * np.linalg.norm(ref), r


def test_solve_on_wide_band():
    m = wide_bar()
    O, S, P = make(m, P_WIDE)
    assert api.precond_info(P)["band_width"] > 31
    freqs = np.array([1e8, 1e10])
    Z64, st64 = api.sie_solve(P, freqs, tol=1e-10, restart=100, prec=PREC_FP64)
    Zm, stm = api.sie_solve(P, freqs, tol=1e-10, restart=100, prec=PREC_MIXED, refine=True)
    assert st64["converged"] and stm["converged"]
    assert np.abs(Zm - Z64).max() < 1e-7 * np.abs(Z64).max()

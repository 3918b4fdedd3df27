"""GPU parity of the nested-dissection factorisation of the preconditioner
(Eq. Precond: a direct factorisation of P; SIE_PC_ND).

P^-1 is applied through the nodal Laplacian of the same circuit; with
nested dissection the Laplacian is factorised as a multifrontal LDL^T.  Bars:
* forced on small meshes (a bar, two wires, two bars, a plane pair with vias):
  against the oracle's sparse LU of the literal P = A diag(Z_b) A^T, FP64
  within 1e-9 and the FP32 solves within 1e-4, several frequencies (factor
  slots) in one call;
* against the band factorisation where both apply, within 1e-10;
* a solve through it against the oracle's GMRES (Z within 1e-6);
* the plane pair at full size (517k triangles) takes it by itself (its band
  is thousands wide): the mixed solve with FP64 refinement converges to 1e-6
  with a reciprocal Z, and the FP64 and FP32 solves of P agree.
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.gmres import Precond, gmres
from oracle.pfft import PfftSystem, PfftParams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, native as N, PREC_FP64, PREC_MIXED  # noqa: E402

PARAMS = dict(grid=(16, 8, 8), order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=0.0)


def build(m, params):
    O = build_loops(m)
    S = PfftSystem(m, O, PfftParams(grid=params["grid"], order=params["order"],
                                    near_factor=params["near_factor"], near_min_diam=params["near_min_diam"],
                                    n_touch=params["n_touch"]))
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    return O, S, api.Plan(M, L, params)


MESHES = [("bar", synth.tiny_bar, PARAMS), ("wires", synth.tiny_wires, dict(PARAMS, grid=(16, 8, 4))),
          ("two_bars", synth.tiny_two_bars, PARAMS), ("pdn", synth.tiny_pdn, dict(PARAMS, grid=(32, 32, 16)))]


@pytest.mark.parametrize("name,make,params", MESHES, ids=[m[0] for m in MESHES])
def test_nd_precond_matches_oracle(name, make, params):
    m = make()
    O, S, P = build(m, params)
    api.precond_set_method(P, N.PC_ND)
    info = api.precond_nd_info(P)
    assert info["method"] == N.PC_ND and info["fronts"] >= 1 and info["nnz"] > 0
    om = 2 * np.pi * np.array([1e8, 1e9, 1e9, 2e10])
    y = synth.complex_gaussian(O.nl, om.size, seed=61)
    z64 = api.pfft_precond_apply(P, torch.from_numpy(y).cuda(), om).cpu().numpy()
    z32 = api.pfft_precond_apply(P, torch.from_numpy(y).cuda(), om, prec=PREC_MIXED).cpu().numpy()
    for r in range(om.size):
        ref = Precond(O, S.diag_Zb(om[r])).solve(y[r])
        assert np.linalg.norm(z64[r] - ref) < 1e-9 * np.linalg.norm(ref), (name, r)
        assert np.linalg.norm(z32[r] - ref) < 1e-4 * np.linalg.norm(ref), (name, r)


def test_nd_equals_band():
    m = synth.tiny_wires()
    O, S, P = build(m, dict(PARAMS, grid=(16, 8, 4)))
    om = 2 * np.pi * np.array([5e8, 5e9])
    y = torch.from_numpy(synth.complex_gaussian(O.nl, 2, seed=62)).cuda()
    api.precond_set_method(P, N.PC_BAND)
    zb = api.pfft_precond_apply(P, y, om).cpu().numpy()
    assert api.precond_nd_info(P)["method"] == N.PC_BAND
    api.precond_set_method(P, N.PC_ND)
    zn = api.pfft_precond_apply(P, y, om).cpu().numpy()
    assert np.linalg.norm(zn - zb) < 1e-10 * np.linalg.norm(zb)


def test_nd_solve_matches_oracle():
    m = synth.tiny_pdn()
    O, S, P = build(m, dict(PARAMS, grid=(32, 32, 16)))
    api.precond_set_method(P, N.PC_ND)
    freqs = np.array([1e8, 1e9])
    Z, st = api.sie_solve(P, freqs, tol=1e-10, restart=100, prec=PREC_FP64)
    assert st["converged"]
    npo = O.n_ports
    for fi, f in enumerate(freqs):
        w = 2 * np.pi * f
        pc = Precond(O, S.diag_Zb(w))
        Y = np.zeros((npo, npo), complex)
        for p in range(npo):
            b = np.zeros(O.nl, complex)
            b[O.port_loop(p)] = 1.0
            xs, _, _ = gmres(lambda v: S.matvec(v, w), b, pc, tol=1e-12, restart=200)
            Y[:, p] = [xs[O.port_loop(q)] for q in range(npo)]
        Zo = np.linalg.inv(Y)
        assert np.abs(Z[fi] - Zo).max() < 1e-6 * np.abs(Zo).max()
    Zm, stm = api.sie_solve(P, freqs, tol=1e-10, restart=100, prec=PREC_MIXED, refine=True)
    assert stm["converged"] and np.abs(Zm - Z).max() < 1e-7 * np.abs(Z).max()


@pytest.fixture(scope="module")
def pdn_plan():
    w = synth.pdn_500k()
    m = w["mesh"]
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, dict(grid=w["grid"], order=3, near_factor=4.0, near_min_diam=2.0, n_touch=16, h0=0.0))
    return w, L, P


def test_pdn_takes_nested_dissection(pdn_plan):
    w, L, P = pdn_plan
    assert api.precond_info(P)["band_width"] >= 1024
    info = api.precond_nd_info(P)
    assert info["method"] == N.PC_ND and info["fronts"] > 1000


def test_pdn_precond_fp32_matches_fp64(pdn_plan):
    w, L, P = pdn_plan
    om = 2 * np.pi * np.array([1e6, 1e9])
    y = torch.from_numpy(synth.complex_gaussian(L.nl, 2, seed=63)).cuda()
    z64 = api.pfft_precond_apply(P, y, om).cpu().numpy()
    z32 = api.pfft_precond_apply(P, y, om, prec=PREC_MIXED).cpu().numpy()
    err = np.linalg.norm(z32 - z64, axis=1) / np.linalg.norm(z64, axis=1)
    assert err.max() < 1e-4, err


def test_pdn_solve_converges(pdn_plan):
    w, L, P = pdn_plan
    freqs = np.array([1e7, 1e9])
    Z, st = api.sie_solve(P, freqs, tol=1e-6, restart=100, max_iter=300, prec=PREC_MIXED, refine=True)
    assert st["converged"] and st["residual_max"] < 1e-6
    assert np.abs(Z - np.transpose(Z, (0, 2, 1))).max() < 1e-5 * np.abs(Z).max()
    R = Z.real
    assert np.all(np.diagonal(R, axis1=1, axis2=2) > 0)

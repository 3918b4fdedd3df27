"""GPU parity of the double-float product (SIE_PREC_DF).

Every step of pfft_matvec (Eq. FinalME: loop maps, Eq. Projection, the
zero-padded FFT convolution of Eq. FFTCal, interpolation, the pre-corrected
near field of Eq. Lb and Eq. Zb) runs on pairs of FP32 numbers (about 48
significant bits) with error-free sums and products on the FP32 pipes.  Bars:
* against the oracle pFFT (oracle/pfft.py) within 1e-10 relative 2-norm per
  right-hand side, the FP64 path's bar, and element by element within 1e-9 of
  the largest entry;
* against the FP64 path within 1e-11 (both are rounding away from the exact
  product; the FP64 path's own error is about 1e-15);
on a bar, two wires and a plane pair with vias, with 1, 5, 33 and 70
right-hand sides (both slab shapes and ragged slabs), in loop and branch space;
on a grid whose (y, z) plane takes the large-plane route; at the bond-wire
size (40,192 triangles, 128 right-hand sides) against FP64; and GMRES with
double-float refinement residuals against the FP64-residual refinement and the
plain FP64 solve.

The preconditioner's sweeps (Eq. Precond, the LDL^T solve of the nodal
Laplacian) in double-float agree with FP64 within 1e-11 where the band is
narrow (one warp per sweep), and are the FP64 sweeps elsewhere; the FP32
sweeps of the same factor are far less accurate, which is why double-float
refinement uses them inside its cycles.
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.pfft import PfftSystem, PfftParams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import (api, native as N, SPACE_LOOP, SPACE_BRANCH, PREC_FP64,  # noqa: E402
                                    PREC_MIXED, PREC_DF, REFINE_FP64, REFINE_DF, SieError)

PARAMS = dict(order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=0.0)
MESHES = [("bar", synth.tiny_bar, (16, 8, 8)), ("wires", synth.tiny_wires, (16, 8, 4)),
          ("pdn", synth.tiny_pdn, (32, 32, 16))]


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def build(m, grid):
    O = build_loops(m)
    S = PfftSystem(m, O, PfftParams(grid=grid, **{k: PARAMS[k] for k in ("order", "near_factor",
                                                                          "near_min_diam", "n_touch")}))
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    return O, S, api.Plan(M, L, dict(PARAMS, grid=grid))


@pytest.fixture(scope="module", params=MESHES, ids=[m[0] for m in MESHES])
def system(request):
    name, make, grid = request.param
    m = make()
    return (name,) + build(m, grid)


@pytest.mark.parametrize("R", [1, 5, 33, 70])
def test_df_loop_product_matches_oracle_and_fp64(system, R):
    name, O, S, P = system
    om = 2 * np.pi * np.logspace(6, 10, R)
    x = synth.complex_gaussian(O.nl, R, seed=90 + R)
    xt = torch.from_numpy(x).cuda()
    ydf = api.pfft_matvec(P, xt, om, SPACE_LOOP, PREC_DF).cpu().numpy()
    y64 = api.pfft_matvec(P, xt, om, SPACE_LOOP, PREC_FP64).cpu().numpy()
    assert rel(ydf, y64).max() < 1e-11, (name, R, rel(ydf, y64).max())
    for r in sorted({0, R // 2, R - 1}):
        ref = S.matvec(x[r], om[r])
        assert rel(ydf[r], ref) < 1e-10, (name, R, r)
        assert np.abs(ydf[r] - ref).max() < 1e-9 * np.abs(ref).max(), (name, R, r)


def test_df_branch_product_matches_oracle_and_fp64(system):
    name, O, S, P = system
    R = 6
    om = 2 * np.pi * np.logspace(7, 10, R)
    a = synth.complex_gaussian(O.nb, R, seed=95)
    at = torch.from_numpy(a).cuda()
    ydf = api.pfft_matvec(P, at, om, SPACE_BRANCH, PREC_DF).cpu().numpy()
    y64 = api.pfft_matvec(P, at, om, SPACE_BRANCH, PREC_FP64).cpu().numpy()
    assert rel(ydf, y64).max() < 1e-11
    for r in (0, R - 1):
        ref = S.branch_product(a[r], om[r])
        assert rel(ydf[r], ref) < 1e-10
        assert np.abs(ydf[r] - ref).max() < 1e-9 * np.abs(ref).max()


def test_df_is_much_closer_to_fp64_than_mixed(system):
    name, O, S, P = system
    om = 2 * np.pi * np.array([1e8, 1e9, 1e10, 2e10])
    xt = torch.from_numpy(synth.complex_gaussian(O.nl, om.size, seed=97)).cuda()
    y64 = api.pfft_matvec(P, xt, om, SPACE_LOOP, PREC_FP64).cpu().numpy()
    ydf = api.pfft_matvec(P, xt, om, SPACE_LOOP, PREC_DF).cpu().numpy()
    y32 = api.pfft_matvec(P, xt, om, SPACE_LOOP, PREC_MIXED).cpu().numpy()
    assert rel(ydf, y64).max() < 1e-4 * rel(y32, y64).max()


def test_df_on_large_plane_grid():
    m = synth.tiny_wires()
    O, S, P = build(m, (8, 256, 32))
    om = 2 * np.pi * np.array([1e6, 1e9, 1e10])
    x = synth.complex_gaussian(O.nl, om.size, seed=61)
    xt = torch.from_numpy(x).cuda()
    ydf = api.pfft_matvec(P, xt, om, SPACE_LOOP, PREC_DF).cpu().numpy()
    y64 = api.pfft_matvec(P, xt, om, SPACE_LOOP, PREC_FP64).cpu().numpy()
    assert rel(ydf, y64).max() < 1e-11
    ref = np.stack([S.matvec(x[r], om[r]) for r in range(om.size)])
    assert rel(ydf, ref).max() < 1e-10


def test_df_rejects_the_lossy_kernel():
    m = synth.tiny_wires()
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, dict(PARAMS, grid=(16, 8, 4), kernel=N.KERNEL_LOSSY))
    xt = torch.from_numpy(synth.complex_gaussian(L.nl, 2, seed=3)).cuda()
    with pytest.raises(SieError):
        api.pfft_matvec(P, xt, 2 * np.pi * np.array([1e9, 1e9]), SPACE_LOOP, PREC_DF)
    with pytest.raises(SieError):
        api.sie_solve(P, np.array([1e9]), tol=1e-8, prec=PREC_MIXED, refine=REFINE_DF)


def test_refinement_with_df_residuals_matches_fp64_residuals():
    m = synth.tiny_pdn()
    O, S, P = build(m, (32, 32, 16))
    freqs = np.array([1e8, 1e9, 5e9])
    Z64, st64 = api.sie_solve(P, freqs, tol=1e-10, restart=100, prec=PREC_FP64)
    Zr1, st1 = api.sie_solve(P, freqs, tol=1e-10, restart=100, prec=PREC_MIXED, refine=REFINE_FP64)
    Zr2, st2 = api.sie_solve(P, freqs, tol=1e-10, restart=100, prec=PREC_MIXED, refine=REFINE_DF)
    assert st64["converged"] and st1["converged"] and st2["converged"]
    assert st2["residual_max"] < 1e-10
    assert np.abs(Zr2 - Z64).max() < 1e-8 * np.abs(Z64).max()
    assert np.abs(Zr2 - Zr1).max() < 1e-8 * np.abs(Z64).max()


def test_df_at_bondwire_size_matches_fp64():
    w = synth.bondwires_40k()
    m = w["mesh"]
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, dict(PARAMS, grid=w["grid"], n_touch=16))
    om = np.repeat(2 * np.pi * w["freqs"], len(m.ports))
    xt = torch.from_numpy(synth.complex_gaussian(L.nl, len(om), seed=7)).cuda()
    y64 = api.pfft_matvec(P, xt, om, SPACE_LOOP, PREC_FP64).cpu().numpy()
    ydf = api.pfft_matvec(P, xt, om, SPACE_LOOP, PREC_DF).cpu().numpy()
    assert rel(ydf, y64).max() < 1e-11
    assert np.abs(ydf - y64).max() < 1e-10 * np.abs(y64).max()
    Z, st = api.sie_solve(P, np.array([1e8, 1e10]), tol=1e-6, restart=100, max_iter=400, prec=PREC_MIXED,
                          refine=REFINE_DF)
    assert st["converged"] and st["residual_max"] < 1e-6
    assert np.abs(Z - np.transpose(Z, (0, 2, 1))).max() < 1e-6 * np.abs(Z).max()


@pytest.mark.parametrize("name,make,grid", MESHES, ids=[m[0] for m in MESHES])
def test_df_preconditioner_matches_fp64(name, make, grid):
    m = make()
    O, S, P = build(m, grid)
    om = 2 * np.pi * np.array([1e8, 1e9, 1e9, 2e10])
    y = torch.from_numpy(synth.complex_gaussian(O.nl, om.size, seed=64)).cuda()
    z64 = api.pfft_precond_apply(P, y, om).cpu().numpy()
    zdf = api.pfft_precond_apply(P, y, om, prec=PREC_DF).cpu().numpy()
    z32 = api.pfft_precond_apply(P, y, om, prec=PREC_MIXED).cpu().numpy()
    narrow = api.precond_nd_info(P)["method"] != N.PC_ND and api.precond_info(P)["band_width"] <= 31
    if narrow:
        assert rel(zdf, z64).max() < 1e-11, (name, rel(zdf, z64).max())
        assert rel(zdf, z64).max() < 1e-3 * max(rel(z32, z64).max(), 1e-12)
    else:
        assert np.array_equal(zdf, z64)   # FP64 sweeps where the band is not narrow


def test_df_refinement_at_bondwire_size_takes_fewer_cycles():
    w = synth.bondwires_40k()
    m = w["mesh"]
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, dict(PARAMS, grid=w["grid"], n_touch=16))
    freqs = w["freqs"][::4]
    Z64, st64 = api.sie_solve(P, freqs, tol=1e-6, restart=100, max_iter=400, prec=PREC_FP64)
    Z1, st1 = api.sie_solve(P, freqs, tol=1e-6, restart=100, max_iter=400, prec=PREC_MIXED, refine=REFINE_FP64)
    Z2, st2 = api.sie_solve(P, freqs, tol=1e-6, restart=100, max_iter=400, prec=PREC_MIXED, refine=REFINE_DF)
    assert st1["converged"] and st2["converged"] and st2["residual_max"] < 1e-6
    assert st2["iterations_max"] < st1["iterations_max"]
    assert np.abs(Z2 - Z64).max() < 1e-6 * np.abs(Z64).max()

"""GPU parity on grids whose padded (y, z) plane does not fit one CTA, and on
axes of 256 nodes (padded 512: pencils of the in-register DFT32 four-step split).

For such planes the convolution (Sec. IV-B step 2, Eq. FFTCal) runs as y
pencils through device memory, then z rows that fuse the zero-padded forward
transform, the kernel product and the cropped inverse, then the inverse y
pencils; the kernel spectrum at plan creation takes the same route.  The
oracle's zero-padded FFT product (oracle/lossy.py; the static kernel is its
k = 0 case) is the reference: FP64 within 1e-12, mixed within 1e-6, for the
static kernel (lossy: 1e-12 and 1e-5, the bounds of the lossy tests); and the full matvec on such a grid against the
oracle pFFT (oracle/pfft.py), FP64 within 1e-10, mixed within 1e-5.
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.lossy import convolve_lossy, skin_wavenumber
from oracle.pfft import PfftSystem, PfftParams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, native as N, SPACE_LOOP  # noqa: E402

H0 = 1.3e6
# (N_x, N_y, N_z): a 512 x 64 plane (the PDN-like grid's plane); z rows of 512;
# 128 x 128 and 256 x 64 planes with radix-16 y pencils; x pencils of 512 with a
# plane that fits; and a 512 x 512 plane
GRIDS = [(8, 256, 32), (4, 8, 256), (4, 64, 64), (4, 128, 32), (256, 8, 8), (4, 256, 256)]


@pytest.fixture(scope="module")
def mesh():
    m = synth.tiny_wires()
    M = api.Mesh.from_synth(m)
    return m, M, api.Loops(M, m.ports)


def plan_for(mesh, grid, order=3):
    m, M, L = mesh
    return api.Plan(M, L, dict(grid=grid, order=order, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=H0))


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: "x".join(map(str, g)))
def test_large_grid_convolution_matches_oracle(mesh, grid):
    P = plan_for(mesh, grid)
    h = np.array(P.info()["grid_h"])
    rng = np.random.default_rng(sum(grid) + 1)
    nb = 3
    g = rng.standard_normal((nb,) + grid) + 1j * rng.standard_normal((nb,) + grid)
    ref = np.stack([convolve_lossy(g[b], h, 0.0, H0) for b in range(nb)])
    scale = np.abs(ref).max()
    g64 = api.pfft_convolve(P, torch.from_numpy(g).cuda(), N.PREC_FP64).cpu().numpy()
    assert np.abs(g64 - ref).max() < 1e-12 * scale
    g32 = api.pfft_convolve(P, torch.from_numpy(g.astype(np.complex64)).cuda(), N.PREC_MIXED).cpu().numpy()
    assert np.abs(g32 - ref).max() < 1e-6 * scale
    one = api.pfft_convolve(P, torch.from_numpy(g[2:3].astype(np.complex64)).cuda(), N.PREC_MIXED).cpu().numpy()
    assert np.array_equal(one[0], g32[2])


@pytest.mark.parametrize("grid", [(8, 256, 32), (4, 8, 256)], ids=lambda g: "x".join(map(str, g)))
def test_large_grid_lossy_convolution_matches_oracle(mesh, grid):
    P = plan_for(mesh, grid)
    h = np.array(P.info()["grid_h"])
    om, sig = 2 * np.pi * 1e8, 4.1e7
    k = skin_wavenumber(om, sig)
    rng = np.random.default_rng(7)
    g = rng.standard_normal((2,) + grid) + 1j * rng.standard_normal((2,) + grid)
    ref = np.stack([convolve_lossy(g[b], h, k, H0) for b in range(2)])
    got = api.pfft_convolve_lossy(P, torch.from_numpy(g).cuda(), om, sig).cpu().numpy()
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    got32 = api.pfft_convolve_lossy(P, torch.from_numpy(g.astype(np.complex64)).cuda(), om, sig,
                                    N.PREC_MIXED).cpu().numpy()
    assert np.abs(got32 - ref).max() < 1e-5 * np.abs(ref).max()


def test_matvec_on_large_plane_grid_matches_oracle(mesh):
    m, M, L = mesh
    grid = (8, 256, 32)
    O = build_loops(m)
    S = PfftSystem(m, O, PfftParams(grid=grid, order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8))
    P = api.Plan(M, L, dict(grid=grid, order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=0.0))
    om = 2 * np.pi * np.array([1e6, 1e9, 1e10])
    x = synth.complex_gaussian(O.nl, om.size, seed=61)
    ref = np.stack([S.matvec(x[r], om[r]) for r in range(om.size)])
    for prec, tol in ((N.PREC_FP64, 1e-10), (N.PREC_MIXED, 1e-5)):
        y = api.pfft_matvec(P, torch.from_numpy(x).cuda(), om, SPACE_LOOP, prec).cpu().numpy()
        err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() < tol, (prec, err)


def test_large_plane_rules():
    """A plane larger than one CTA needs N_z >= 16 (8 when N_y = 256); axes above
    256 are rejected."""
    m = synth.tiny_wires()
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    from paper_2210_04891_gb300 import SieError
    for grid in [(512, 8, 8), (4, 256, 4)]:
        with pytest.raises(SieError):
            api.Plan(M, L, dict(grid=grid, order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=0.0))

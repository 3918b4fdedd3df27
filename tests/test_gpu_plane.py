"""GPU parity of the FP32 grid convolution (Sec. IV-B step 2, Eq. FFTCal) over
plane sizes: the paired (y, z) plane kernel is built per padded plane
My x Mz, each with its own four-step splits, so every split shape is checked
against the oracle's zero-padded FFT product.

The static grid kernel 1/R with h0 at zero offset is the lossy oracle kernel
exp(-jkR)/R at k = 0 (oracle/lossy.py states the same sampling and padding
rules), so convolve_lossy(g, h, 0) is the reference here.  FP64 path within
1e-12 of it, the mixed (FP32) path within 1e-6, the bound the other
convolution tests use.
"""
import numpy as np
import pytest

import synth
from oracle.lossy import convolve_lossy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, native as N  # noqa: E402

# (N_x, N_y, N_z) -> padded plane (My, Mz) = (2 N_y, 2 N_z):
# (8, 8) smallest; (16, 64) and (64, 16) with row-pair spacing in the z passes;
# (128, 64) the bond-wire plane; (32, 128) and (16, 256) radix-16 z passes;
# (256, 16) radix-16 y passes.
GRIDS = [(8, 4, 4), (8, 8, 32), (4, 32, 8), (4, 64, 32), (4, 16, 64), (4, 8, 128), (4, 128, 8)]
H0 = 1.7e6


@pytest.fixture(scope="module")
def mesh():
    m = synth.tiny_wires()
    M = api.Mesh.from_synth(m)
    return M, api.Loops(M, m.ports)


@pytest.mark.parametrize("grid", GRIDS, ids=lambda g: "x".join(map(str, g)))
def test_plane_sizes_match_oracle(mesh, grid):
    M, L = mesh
    P = api.Plan(M, L, dict(grid=grid, order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=H0))
    h = np.array(P.info()["grid_h"])
    rng = np.random.default_rng(sum(grid))
    nb = 3
    g = rng.standard_normal((nb,) + grid) + 1j * rng.standard_normal((nb,) + grid)
    ref = np.stack([convolve_lossy(g[b], h, 0.0, H0) for b in range(nb)])
    scale = np.abs(ref).max()
    g64 = api.pfft_convolve(P, torch.from_numpy(g).cuda(), N.PREC_FP64).cpu().numpy()
    assert np.abs(g64 - ref).max() < 1e-12 * scale
    g32 = api.pfft_convolve(P, torch.from_numpy(g.astype(np.complex64)).cuda(), N.PREC_MIXED).cpu().numpy()
    assert np.abs(g32 - ref).max() < 1e-6 * scale
    # a single grid, and the same batch again (results do not depend on the batch)
    one = api.pfft_convolve(P, torch.from_numpy(g[1:2].astype(np.complex64)).cuda(), N.PREC_MIXED).cpu().numpy()
    assert np.array_equal(one[0], g32[1])


@pytest.mark.parametrize("nbatch", [80, 307])
def test_plane_runs_of_grids_match_oracle(mesh, nbatch):
    """Many grids: CTAs then take runs of 2 (80 grids) or 8 (307 grids, last run
    ragged) grids of one x-frequency, with the staged spectrum and twiddles reused
    and the next grid's input prefetched; every grid against the oracle."""
    M, L = mesh
    grid = (16, 8, 4)
    P = api.Plan(M, L, dict(grid=grid, order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=H0))
    h = np.array(P.info()["grid_h"])
    rng = np.random.default_rng(nbatch)
    g = (rng.standard_normal((nbatch,) + grid) + 1j * rng.standard_normal((nbatch,) + grid))
    ref = np.stack([convolve_lossy(g[b], h, 0.0, H0) for b in range(nbatch)])
    g32 = api.pfft_convolve(P, torch.from_numpy(g.astype(np.complex64)).cuda(), N.PREC_MIXED).cpu().numpy()
    err = np.abs(g32 - ref).max(axis=(1, 2, 3)) / np.abs(ref).max(axis=(1, 2, 3))
    assert err.max() < 1e-6

"""GPU parity of pfft_convolve_lossy (Sec. IV-B step 2 with the lossy kernel)
against the oracle's FFT product and direct pair sum (oracle/lossy.py).

Frequencies span a skin depth far above the grid (near-static), comparable to
it and far below it (a kernel that dies within one spacing); grids span
several FFT tiles; batches of 1, 3 and 4 grids.  FP64 within 1e-12 of the
oracle, the mixed (FP32) form within 1e-5.
"""
import numpy as np
import pytest

import synth
from oracle.lossy import skin_wavenumber, convolve_lossy, convolve_lossy_direct

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, native as N  # noqa: E402

SIG = 4.1e7


@pytest.fixture(scope="module")
def plan():
    m = synth.tiny_wires()
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    return api.Plan(M, L, dict(grid=(16, 8, 4), order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=0.0))


@pytest.mark.parametrize("f", [1e6, 1e9, 3e10])
@pytest.mark.parametrize("nbatch", [1, 3, 4])
def test_lossy_convolve_matches_oracle(plan, f, nbatch):
    h = np.array(plan.info()["grid_h"])
    k = skin_wavenumber(2 * np.pi * f, SIG)
    rng = np.random.default_rng(nbatch)
    g = rng.standard_normal((nbatch, 16, 8, 4)) + 1j * rng.standard_normal((nbatch, 16, 8, 4))
    ref = np.stack([convolve_lossy(g[b], h, k) for b in range(nbatch)])
    got = api.pfft_convolve_lossy(plan, torch.from_numpy(g).cuda(), 2 * np.pi * f, SIG).cpu().numpy()
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    got32 = api.pfft_convolve_lossy(plan, torch.from_numpy(g).to(torch.complex64).cuda(), 2 * np.pi * f, SIG,
                                    prec=N.PREC_MIXED).cpu().numpy()
    assert np.abs(got32 - ref).max() < 1e-5 * np.abs(ref).max()


def test_lossy_direct_sum_and_spectrum_cache(plan):
    """Against the O(N^2) pair sum; alternating frequencies rebuilds the spectrum."""
    h = np.array(plan.info()["grid_h"])
    g = synth.complex_gaussian(16 * 8 * 4, 1, seed=3).reshape(1, 16, 8, 4)
    for f in (1e8, 5e9, 1e8):
        k = skin_wavenumber(2 * np.pi * f, SIG)
        ref = convolve_lossy_direct(g[0], h, k)
        got = api.pfft_convolve_lossy(plan, torch.from_numpy(g).cuda(), 2 * np.pi * f, SIG).cpu().numpy()[0]
        assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    # the static product is untouched by the lossy spectrum
    stat = api.pfft_convolve(plan, torch.from_numpy(g).cuda()).cpu().numpy()[0]
    assert np.abs(stat - ref).max() > 1e-3 * np.abs(ref).max()


def test_lossy_rejects_bad_arguments(plan):
    g = torch.zeros((1, 16, 8, 4), dtype=torch.complex128, device="cuda")
    for om, sg in ((0.0, SIG), (1e9, 0.0), (float("nan"), SIG)):
        with pytest.raises(N.SieError):
            api.pfft_convolve_lossy(plan, g, om, sg)

"""pfft_convolve_noalloc against pfft_convolve, through the C ABI.

The no-allocation variant is for callers that may not allocate device memory
when they convolve (a start-up memory budget, a real-time loop, a framework
that owns the allocator).  It must give the same grid potentials as the
allocating entry point, on two calls in a row (its scratch array is shared and
keeps the previous call's contents), and must not grow the plan's memory.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, native as N  # noqa: E402


def call_noalloc(plan, grid, prec):
    rc = N.lib().pfft_convolve_noalloc(plan.h, ctypes.c_void_p(grid.data_ptr()), grid.shape[0], prec,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    N.check(rc)
    return grid


@pytest.mark.parametrize("prec,tol", [(N.PREC_FP64, 1e-13), (N.PREC_MIXED, 1e-6)])
def test_noalloc_matches_convolve_twice(prec, tol):
    m = synth.tiny_wires()
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, dict(grid=(16, 8, 4), order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=0.0))
    bytes0 = P.info()["device_bytes"]
    dt = torch.complex128 if prec == N.PREC_FP64 else torch.complex64
    rng = np.random.default_rng(5)
    for call in range(2):
        g = rng.standard_normal((4, 16, 8, 4)) + 1j * rng.standard_normal((4, 16, 8, 4))
        ref = api.pfft_convolve(P, torch.from_numpy(g).to(dt).cuda(), prec).cpu().numpy()
        got = call_noalloc(P, torch.from_numpy(g).to(dt).cuda(), prec).cpu().numpy()
        assert np.abs(got - ref).max() < tol * np.abs(ref).max(), call
    # the allocating path grew plan scratch; the no-allocation path must not add to it
    bytes1 = P.info()["device_bytes"]
    got2 = call_noalloc(P, torch.from_numpy(g).to(dt).cuda(), prec)
    assert P.info()["device_bytes"] == bytes1
    assert bytes1 >= bytes0


@pytest.mark.parametrize("prec,tol", [(N.PREC_FP64, 1e-13), (N.PREC_MIXED, 1e-6)])
def test_noalloc_fresh_plan_allocates_nothing(prec, tol):
    # a plan that has never convolved: the no-allocation call must neither grow its
    # memory nor differ from the allocating call made afterwards
    m = synth.tiny_bar()
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, dict(grid=(8, 4, 4), order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=0.0))
    before = P.info()["device_bytes"]
    dt = torch.complex128 if prec == N.PREC_FP64 else torch.complex64
    g = torch.from_numpy(synth.complex_gaussian(8 * 4 * 4, 3, seed=2).reshape(3, 8, 4, 4)).to(dt).cuda()
    x = g.clone()
    ref = g.clone()
    call_noalloc(P, g, prec)
    call_noalloc(P, ref, prec)
    assert torch.equal(g, ref)
    assert P.info()["device_bytes"] == before
    conv = api.pfft_convolve(P, x, prec).cpu().numpy()
    got = g.cpu().numpy()
    assert np.abs(got - conv).max() < tol * np.abs(conv).max()


def _plan(mesh, grid):
    M = api.Mesh.from_synth(mesh)
    L = api.Loops(M, mesh.ports)
    return api.Plan(M, L, dict(grid=grid, order=3, near_factor=1.0, near_min_diam=1.0, n_touch=4, h0=0.0))


def test_noalloc_batch_in_pieces():
    # FP64 64 x 16 x 16: one grid's x-padded copy is 512 KiB, so 8 grids fit the
    # 4 MiB scratch and a batch of 10 runs as two pieces
    P = _plan(synth.tiny_bar(), (64, 16, 16))
    rng = np.random.default_rng(11)
    for call in range(2):
        g = rng.standard_normal((10, 64, 16, 16)) + 1j * rng.standard_normal((10, 64, 16, 16))
        ref = api.pfft_convolve(P, torch.from_numpy(g).cuda(), N.PREC_FP64).cpu().numpy()
        got = call_noalloc(P, torch.from_numpy(g).cuda(), N.PREC_FP64).cpu().numpy()
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max(), call


def test_noalloc_large_plane():
    # 8 x 256 x 32: the padded (y, z) plane (512 x 64) does not fit one CTA, so the
    # scratch also holds the y transform: 16 * (256 + 512) * 32 values * 8 B = 3 MiB
    P = _plan(synth.tiny_bar(), (8, 256, 32))
    rng = np.random.default_rng(12)
    for call in range(2):
        g = rng.standard_normal((2, 8, 256, 32)) + 1j * rng.standard_normal((2, 8, 256, 32))
        x = torch.from_numpy(g).to(torch.complex64)
        ref = api.pfft_convolve(P, x.cuda(), N.PREC_MIXED).cpu().numpy()
        got = call_noalloc(P, x.cuda(), N.PREC_MIXED).cpu().numpy()
        assert np.abs(got - ref).max() < 1e-6 * np.abs(ref).max(), call


def test_noalloc_rejects_oversized_grid():
    m = synth.tiny_bar()
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    # 128 x 64 x 32 grid padded along x: 256 * 64 * 32 values = 8 MiB in FP64 (> 4 MiB), 4 MiB in FP32
    P = api.Plan(M, L, dict(grid=(128, 64, 32), order=3, near_factor=1.0, near_min_diam=1.0, n_touch=4, h0=0.0))
    g = torch.zeros((1, 128, 64, 32), dtype=torch.complex128, device="cuda")
    with pytest.raises(N.SieError) as e:
        call_noalloc(P, g, N.PREC_FP64)
    assert e.value.code == -1
    g32 = torch.zeros((1, 128, 64, 32), dtype=torch.complex64, device="cuda")
    call_noalloc(P, g32, N.PREC_MIXED)

"""Pins of the plain pFFT oracle (Sec. IV-B).

* step 2: the FFT convolution on the zero-padded grid equals the direct
  Toeplitz sum phi_i = sum_j H(i - j) Q_j;
* steps 1 and 3: Lagrange stencils of order O_s reproduce polynomials of
  degree < O_s exactly (the projection matches the point source's moments);
  I = B^T (Galerkin);
* step 4: with every pair near, L_d + I H B is the direct product, so the
  pFFT product equals the dense product built with the same near-field rule;
* H(0) does not change the result (every stencil-sharing pair is pre-corrected);
* the pFFT product converges to the dense MoM product as the near radius grows.
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.mom import DenseMoM, assemble_from_blocks
from oracle.pfft import Pfft, PfftParams, PfftSystem, stencil_1d
from oracle.integrals import symmetric_blocks
from oracle.quadrature import collapsed_gauss, radon7


@pytest.fixture(scope="module")
def bar():
    m = synth.tiny_bar()
    L = build_loops(m)
    return m, L


def test_fft_convolution_equals_direct_sum(bar):
    m, L = bar
    P = Pfft(m, L, PfftParams(grid=(6, 5, 4)))
    rng = np.random.default_rng(0)
    Qg = rng.standard_normal((6, 5, 4)) + 1j * rng.standard_normal((6, 5, 4))
    a = P.convolve(Qg)
    b = P.convolve_direct(Qg)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("order", [2, 3, 4])
def test_stencil_reproduces_polynomials(order):
    rng = np.random.default_rng(1)
    n = 12
    t = rng.uniform(0, n - 1, 200)
    start, w = stencil_1d(t, order, n)
    assert np.all(start >= 0) and np.all(start + order <= n)
    for deg in range(order):
        nodes = start[:, None] + np.arange(order)[None]
        assert np.abs((w * nodes ** deg).sum(1) - t ** deg).max() < 1e-9 * (n ** deg)
    # the nearest node is always inside the stencil
    near = np.floor(t + 0.5)
    assert np.all((near >= start) & (near < start + order))


def test_projection_is_interpolation_transpose(bar):
    m, L = bar
    P = Pfft(m, L, PfftParams(grid=(8, 4, 4)))
    rng = np.random.default_rng(2)
    a = rng.standard_normal(L.nb)
    phi = rng.standard_normal(3 * P.ng)
    # <phi, B a> = <B^T phi, a>
    assert abs(phi @ (P.B @ a) - (P.B.T @ phi) @ a) < 1e-12 * np.abs(phi).sum()


def test_all_near_equals_direct(bar):
    m, L = bar
    P = Pfft(m, L, PfftParams(grid=(8, 4, 4), near_factor=1e3))
    assert P.near_i.shape[0] == m.nt * m.nt
    rng = np.random.default_rng(3)
    a = rng.standard_normal(L.nb)
    ii, jj = np.meshgrid(np.arange(m.nt), np.arange(m.nt), indexing="ij")
    blk = symmetric_blocks(m, ii.ravel(), jj.ravel(), collapsed_gauss(16), radon7())
    dense = assemble_from_blocks(m, L, ii.ravel(), jj.ravel(), blk)
    y = P.Lt_apply(a)
    assert np.abs(y - dense @ a).max() < 1e-11 * np.abs(dense @ a).max()


def test_h0_independence(bar):
    m, L = bar
    a = np.random.default_rng(4).standard_normal(L.nb)
    y0 = Pfft(m, L, PfftParams(grid=(12, 4, 4), h0=0.0)).Lt_apply(a)
    y1 = Pfft(m, L, PfftParams(grid=(12, 4, 4), h0=3.7e6)).Lt_apply(a)
    assert np.abs(y0 - y1).max() < 1e-9 * np.abs(y0).max()


def test_converges_to_dense(bar):
    m, L = bar
    D = DenseMoM(m, L)
    x = synth.complex_gaussian(L.nl, 1, seed=5)[0]
    w = 2 * np.pi * 1e9
    yd = D.matvec(x, w)
    errs = []
    for nf in [1.0, 3.0, 6.0]:
        S = PfftSystem(m, L, PfftParams(grid=(16, 6, 6), near_factor=nf, near_min_diam=0.0))
        errs.append(np.linalg.norm(S.matvec(x, w) - yd) / np.linalg.norm(yd))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4


def test_target_rows_equal_full_rows():
    """The near list restricted to target triangles (sampled rows of large
    meshes) gives, on every branch whose two triangles are targets, the same
    rows as the full product; the other rows lose near terms."""
    m = synth.tiny_wires()
    O = build_loops(m)
    prm = PfftParams(grid=(16, 8, 4), order=3, near_factor=5.0, near_min_diam=2.0, n_touch=8)
    full = PfftSystem(m, O, prm)
    rng = np.random.default_rng(4)
    br = np.sort(rng.choice(O.nb, 12, replace=False))
    part = PfftSystem(m, O, prm, targets=O.br_tri[br].ravel())
    a = rng.standard_normal(O.nb) + 1j * rng.standard_normal(O.nb)
    w = 2 * np.pi * 1e9
    yf, yp = full.branch_product(a, w), part.branch_product(a, w)
    assert np.abs(yp[br] - yf[br]).max() < 1e-13 * np.abs(yf[br]).max()
    other = np.setdiff1d(np.arange(O.nb), np.unique(np.nonzero(np.isin(O.br_tri, O.br_tri[br]))[0]))
    assert np.abs(yp[other] - yf[other]).min() > 1e-9 * np.abs(yf).max()


def test_native_grid_blocks_match(bar):
    # the plain C loop of the grid blocks (used for speed) against the numpy
    # version written out node by node, on every 9th near pair of the bar
    # (self, edge- and vertex-adjacent and separated pairs)
    m, L = bar
    P = Pfft(m, L, PfftParams(grid=(8, 4, 4)))
    ti, tj = P.near_i[::9], P.near_j[::9]
    a = P.grid_blocks(ti, tj, native=False)
    b = P.grid_blocks(ti, tj, native=True)
    assert a.shape == b.shape and a.shape[0] > 100 and np.any(ti == tj) and np.any(ti != tj)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("make", [synth.tiny_bar, synth.tiny_wires])
def test_lean_projection_equals_sparse_B(make):
    # steps 1 and 3 applied triangle by triangle (no stored B) against the sparse
    # projection matrix: Q_g = B alpha and B^T phi to rounding, in chunks that
    # split the mesh
    m = make()
    L = build_loops(m)
    prm = PfftParams(grid=(8, 8, 4))
    P = Pfft(m, L, prm)
    Pl = Pfft(m, L, prm, lean=True)
    a = synth.complex_gaussian(L.nb, 1, seed=3)[0]
    q = P.B @ a
    ql = Pl.project(a, chunk=37).reshape(-1)
    assert np.abs(q - ql).max() < 1e-14 * np.abs(q).max()
    phi = synth.complex_gaussian(3 * P.ng, 1, seed=4)[0]
    b = P.B.T @ phi
    bl = Pl.interpolate(phi.reshape(3, *P.N), chunk=41)
    assert np.abs(b - bl).max() < 1e-14 * np.abs(b).max()
    assert np.abs(P.far(a) - Pl.far(a)).max() < 1e-13 * np.abs(P.far(a)).max()

"""GPU parity of pfft_matvec against the oracle (Sec. IV-B, Eq. FinalME).

The CUDA path and the plain pFFT oracle run the same algorithm with the same
parameters on the same seeded inputs, compared element by element:
  FP64 path:  relative 2-norm error per right-hand side <= 1e-10;
  mixed path: <= 1e-5 (FP32 grid/FFT/near field, double-float loop maps);
and against the dense MoM (the definition the pFFT approximates) <= 1e-4.
Beside each norm, an element-wise check: every entry above 1% of the largest
within 100 times the norm bound, so that an error confined to a few entries
(one stage's ragged tail, one tile) cannot hide in the norm.
Grids span several FFT tiles; right-hand-side counts include ragged ones.
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.mom import DenseMoM
from oracle.pfft import PfftSystem, PfftParams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, SPACE_LOOP, SPACE_BRANCH, PREC_FP64, PREC_MIXED  # noqa: E402


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def elementwise_rel(a, b, floor=1e-2):
    # largest relative error over the entries above floor times the largest entry
    big = np.abs(b) > floor * np.abs(b).max()
    return float((np.abs(a - b)[big] / np.abs(b)[big]).max())


def setup(m, params):
    O = build_loops(m)
    S = PfftSystem(m, O, PfftParams(grid=params["grid"], order=params["order"],
                                    near_factor=params["near_factor"], near_min_diam=params["near_min_diam"],
                                    n_touch=params["n_touch"]))
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, params)
    return O, S, P


PARAMS = dict(grid=(16, 8, 4), order=3, near_factor=4.0, near_min_diam=2.0, n_touch=16, h0=0.0)


@pytest.fixture(scope="module")
def wires():
    m = synth.tiny_wires()
    return (m,) + setup(m, PARAMS)


def test_plan_matches_oracle_sizes(wires):
    m, O, S, P = wires
    info = P.info()
    assert info["n_near_pairs"] == S.op.near_i.shape[0]
    assert np.allclose(info["grid_h"], S.op.h, rtol=1e-15)
    assert abs(info["r_near"] - S.op.r_near) <= 1e-15 * S.op.r_near


def test_setup_arrays_match_oracle(wires):
    """Near list and stencils bit-exact; L_direct, L_d and the kernel spectrum to FP64 rounding."""
    from paper_2210_04891_gb300 import native as N
    m, O, S, P = wires
    op = S.op
    ptr = P.export(N.EXPORT_NEAR_PTR)
    col = P.export(N.EXPORT_NEAR_COL)
    assert np.array_equal(np.repeat(np.arange(m.nt), np.diff(ptr)), op.near_i)
    assert np.array_equal(col, op.near_j)
    assert np.array_equal(P.export(N.EXPORT_START), op.start)
    for what, ref in ((N.EXPORT_LDIRECT, op.L_direct), (N.EXPORT_LD, op.L_d)):
        got = P.export(what)
        assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    Nx, Ny, Nz = op.N
    ref = np.transpose(op.Hhat.real[:Nx + 1, :Ny + 1, :Nz + 1], (1, 2, 0)) / (8 * Nx * Ny * Nz)
    assert np.abs(P.export(N.EXPORT_HHAT) - ref).max() < 1e-13 * np.abs(ref).max()


def test_projection_blocks_rebuild_oracle_B(wires):
    """The per-(node, triangle) projection blocks, scattered to branches with
    the triangles' edge signs, reproduce the oracle's projection matrix B
    (Eq. Projection) to FP64 rounding; each (node, triangle) pair appears once,
    nodes ascending per triangle."""
    import scipy.sparse as sp
    from paper_2210_04891_gb300 import native as N
    m, O, S, P = wires
    op = S.op
    ptr = P.export(N.EXPORT_PROJ_PTR)
    node = P.export(N.EXPORT_PROJ_NODE)
    W = P.export(N.EXPORT_PROJ_W)
    assert ptr[0] == 0 and ptr[-1] == node.size == W.shape[0]
    tri = np.repeat(np.arange(m.nt), np.diff(ptr))
    for t in range(m.nt):
        row = node[ptr[t]:ptr[t + 1]]
        assert np.all(np.diff(row) > 0)
        # exactly the union of the triangle's 7 stencils
        s = op.start[t]
        want = set()
        for q in range(s.shape[0]):
            for i in range(op.p.order):
                for j in range(op.p.order):
                    for k in range(op.p.order):
                        want.add(((s[q, 0] + i) * op.N[1] + s[q, 1] + j) * op.N[2] + s[q, 2] + k)
        assert set(row.tolist()) == want
    rows, cols, vals = [], [], []
    for kk in range(3):
        ok = op.tb[tri, kk] >= 0
        for d in range(3):
            rows.append(d * op.ng + node[ok])
            cols.append(op.tb[tri, kk][ok])
            vals.append(op.ts[tri, kk][ok] * W[ok, d, kk])
    B = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=op.B.shape)
    assert abs(B - op.B).max() < 1e-14 * abs(op.B).max()


@pytest.mark.parametrize("nbatch", [1, 3, 4])
def test_convolve_matches_oracle(wires, nbatch):
    from paper_2210_04891_gb300 import native as N
    m, O, S, P = wires
    Nx, Ny, Nz = S.op.N
    rng = np.random.default_rng(nbatch)
    g = rng.standard_normal((nbatch, Nx, Ny, Nz)) + 1j * rng.standard_normal((nbatch, Nx, Ny, Nz))
    ref = np.stack([S.op.convolve(g[b]) for b in range(nbatch)])
    g64 = api.pfft_convolve(P, torch.from_numpy(g).cuda(), N.PREC_FP64).cpu().numpy()
    g32 = api.pfft_convolve(P, torch.from_numpy(g.astype(np.complex64)).cuda(), N.PREC_MIXED).cpu().numpy()
    assert np.abs(g64 - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(g32 - ref).max() < 1e-6 * np.abs(ref).max()
    assert elementwise_rel(g64, ref) < 1e-11
    assert elementwise_rel(g32, ref) < 1e-4


@pytest.mark.parametrize("nrhs", [1, 3, 5])
def test_loop_matvec_fp64(wires, nrhs):
    m, O, S, P = wires
    x = synth.complex_gaussian(O.nl, nrhs, seed=11 + nrhs)
    om = 2 * np.pi * np.logspace(8, 10, nrhs)
    ref = np.stack([S.matvec(x[r], om[r]) for r in range(nrhs)])
    y = api.pfft_matvec(P, torch.from_numpy(x).cuda(), om, SPACE_LOOP, PREC_FP64).cpu().numpy()
    assert rel(y, ref).max() < 1e-10


def test_loop_matvec_mixed(wires):
    m, O, S, P = wires
    x = synth.complex_gaussian(O.nl, 4, seed=21)
    om = 2 * np.pi * np.array([1e8, 1e9, 3e9, 1e10])
    ref = np.stack([S.matvec(x[r], om[r]) for r in range(4)])
    y = api.pfft_matvec(P, torch.from_numpy(x).cuda(), om, SPACE_LOOP, PREC_MIXED).cpu().numpy()
    assert rel(y, ref).max() < 1e-5


@pytest.mark.parametrize("nrhs,prec,tol", [(20, PREC_FP64, 1e-10), (20, PREC_MIXED, 1e-5),
                                           (130, PREC_MIXED, 1e-5), (2, PREC_MIXED, 1e-5),
                                           (1, PREC_MIXED, 1e-5), (7, PREC_MIXED, 1e-5),
                                           (96, PREC_MIXED, 1e-5), (100, PREC_MIXED, 1e-5),
                                           (129, PREC_MIXED, 1e-5), (129, PREC_FP64, 1e-10)])
def test_loop_matvec_batched(wires, nrhs, prec, tol):
    """Ragged lane tails (20, 7), one ragged 128-wide slab (96, 100), more than one slab
    (130, 129); in the mixed form even counts from 96 up take the tensor-core near
    field, the others the CUDA-core gather."""
    m, O, S, P = wires
    x = synth.complex_gaussian(O.nl, nrhs, seed=100 + nrhs)
    om = 2 * np.pi * np.logspace(7, 10, nrhs)
    ref = np.stack([S.matvec(x[r], om[r]) for r in range(nrhs)])
    y = api.pfft_matvec(P, torch.from_numpy(x).cuda(), om, SPACE_LOOP, prec).cpu().numpy()
    assert rel(y, ref).max() < tol
    assert elementwise_rel(y, ref) < 100 * tol


def test_branch_matvec(wires):
    m, O, S, P = wires
    a = synth.complex_gaussian(O.nb, 2, seed=31)
    om = 2 * np.pi * np.array([2e9, 7e9])
    ref = np.stack([S.branch_product(a[r], om[r]) for r in range(2)])
    # branch space: near field, interpolated far field and the Z_s Gram term, before A
    y = api.pfft_matvec(P, torch.from_numpy(a).cuda(), om, SPACE_BRANCH, PREC_FP64).cpu().numpy()
    assert rel(y, ref).max() < 1e-10
    assert elementwise_rel(y, ref) < 1e-8
    y32 = api.pfft_matvec(P, torch.from_numpy(a).cuda(), om, SPACE_BRANCH, PREC_MIXED).cpu().numpy()
    assert rel(y32, ref).max() < 1e-5
    assert elementwise_rel(y32, ref) < 1e-3


def test_deterministic(wires):
    m, O, S, P = wires
    x = torch.from_numpy(synth.complex_gaussian(O.nl, 2, seed=41)).cuda()
    om = 2 * np.pi * np.array([1e9, 1e9])
    y1 = api.pfft_matvec(P, x, om, SPACE_LOOP, PREC_MIXED)
    y2 = api.pfft_matvec(P, x, om, SPACE_LOOP, PREC_MIXED)
    assert torch.equal(y1, y2)


def test_vs_dense_mom():
    m = synth.tiny_bar()
    params = dict(grid=(16, 8, 8), order=3, near_factor=5.0, near_min_diam=2.0, n_touch=16, h0=0.0)
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, params)
    D = DenseMoM(m)
    x = synth.complex_gaussian(L.nl, 2, seed=51)
    om = 2 * np.pi * np.array([1e9, 1e10])
    ref = np.stack([D.matvec(x[r], om[r]) for r in range(2)])
    y = api.pfft_matvec(P, torch.from_numpy(x).cuda(), om, SPACE_LOOP, PREC_FP64).cpu().numpy()
    assert rel(y, ref).max() < 1e-4


def test_h0_independence_gpu():
    m = synth.tiny_bar()
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    base = dict(grid=(16, 8, 8), order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8)
    P0 = api.Plan(M, L, dict(base, h0=0.0))
    P1 = api.Plan(M, L, dict(base, h0=2.5e6))
    x = torch.from_numpy(synth.complex_gaussian(L.nl, 1, seed=61)).cuda()
    y0 = api.pfft_matvec(P0, x, [6e9], SPACE_LOOP, PREC_FP64).cpu().numpy()
    y1 = api.pfft_matvec(P1, x, [6e9], SPACE_LOOP, PREC_FP64).cpu().numpy()
    assert rel(y1, y0).max() < 1e-9


def test_bar_1500_full_size():
    """The 1000 x 20 x 10 um bar (1,508 triangles, grid 64 x 16 x 16) at its bench settings."""
    w = synth.bar_1500()
    m = w["mesh"]
    params = dict(grid=w["grid"], order=3, near_factor=4.0, near_min_diam=2.0, n_touch=16, h0=0.0)
    O, S, P = setup(m, params)
    x = synth.complex_gaussian(O.nl, 2, seed=71)
    om = 2 * np.pi * np.array([1e9, 1e9])
    ref = np.stack([S.matvec(x[r], om[r]) for r in range(2)])
    y64 = api.pfft_matvec(P, torch.from_numpy(x).cuda(), om, SPACE_LOOP, PREC_FP64).cpu().numpy()
    y32 = api.pfft_matvec(P, torch.from_numpy(x).cuda(), om, SPACE_LOOP, PREC_MIXED).cpu().numpy()
    assert rel(y64, ref).max() < 1e-10
    assert rel(y32, ref).max() < 1e-5

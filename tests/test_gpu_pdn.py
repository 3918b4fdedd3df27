"""GPU parity on the PDN-like plane pair (two planes joined by via pairs).

Small structure (tiny_pdn, ~5k triangles, grid 32 x 32 x 16): rows of the
product against the oracle pFFT built with its near list restricted to the
triangles of the sampled rows (oracle/pfft.py): 32 random branches (branch
space) and 10 loops of at most 8 branches (loop space), FP64 within 1e-10 and
mixed within 1e-5 (relative 2-norm over the sampled rows).

Full size (pdn_500k: ~517k triangles, grid 256 x 256 x 32, whose padded
512 x 64 (y, z) plane takes the y-pencil / z-row route, 8 frequencies x 4
ports = 32 right-hand sides).  The oracle cannot build this operator, so:
* the grid convolution at that size against direct sums over all 2.1M nodes
  at sampled output nodes (the oracle's kernel, oracle/lossy.py at k = 0);
* the FP64 operator is complex symmetric, u^T Z v = v^T Z u;
* the mixed form agrees with the FP64 form within the mixed bound;
* sampled rows against the oracle pFFT on the whole structure with its near
  list restricted to the sampled rows' triangles and B applied triangle by
  triangle: 24 branch rows and 12 loop rows for two right-hand sides of the
  32-right-hand-side launch (CUDA-core near field) and of a 96-right-hand-side
  launch (tensor-core near field in the mixed form), FP64 1e-10 and mixed
  1e-5, with element-wise checks beside the 2-norm.
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.lossy import lossy_kernel
from oracle.pfft import PfftSystem, PfftParams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, native as N, SPACE_LOOP, SPACE_BRANCH, PREC_FP64, PREC_MIXED  # noqa: E402

TINY = dict(grid=(32, 32, 16), order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=0.0)


def sampled_rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_tiny_pdn_rows_match_oracle():
    m = synth.tiny_pdn()
    O = build_loops(m)
    A = O.A.tocsr()
    ln = np.diff(A.indptr)
    rng = np.random.default_rng(5)
    loops = np.sort(rng.choice(np.nonzero(ln[:O.nl - O.n_ports] <= 8)[0], 10, replace=False))
    loop_br = np.concatenate([A.indices[A.indptr[l]:A.indptr[l + 1]] for l in loops])
    branches = np.sort(rng.choice(O.nb, 32, replace=False))
    tris = np.unique(O.br_tri[np.concatenate([branches, loop_br])].ravel())
    S = PfftSystem(m, O, PfftParams(grid=TINY["grid"], order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8),
                   targets=tris)
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, TINY)
    om = 2 * np.pi * np.array([1e6, 1e8, 1e9, 1e9])
    x = synth.complex_gaussian(O.nl, om.size, seed=41)
    a = synth.complex_gaussian(O.nb, om.size, seed=42)
    for prec, tol in ((PREC_FP64, 1e-10), (PREC_MIXED, 1e-5)):
        yl = api.pfft_matvec(P, torch.from_numpy(x).cuda(), om, SPACE_LOOP, prec).cpu().numpy()
        yb = api.pfft_matvec(P, torch.from_numpy(a).cuda(), om, SPACE_BRANCH, prec).cpu().numpy()
        for r in range(om.size):
            assert sampled_rel(yl[r, loops], S.matvec(x[r], om[r])[loops]) < tol, (prec, r)
            assert sampled_rel(yb[r, branches], S.branch_product(a[r], om[r])[branches]) < tol, (prec, r)


@pytest.fixture(scope="module")
def pdn():
    w = synth.pdn_500k()
    m = w["mesh"]
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, dict(grid=w["grid"], order=3, near_factor=4.0, near_min_diam=2.0, n_touch=16, h0=0.0))
    om = np.repeat(2 * np.pi * w["freqs"], len(m.ports))
    return w, L, P, om


def test_pdn_convolution_sampled_against_direct_sums(pdn):
    w, L, P, om = pdn
    grid = tuple(w["grid"])
    h = np.array(P.info()["grid_h"])
    rng = np.random.default_rng(3)
    g = rng.standard_normal((3,) + grid) + 1j * rng.standard_normal((3,) + grid)
    g64 = api.pfft_convolve(P, torch.from_numpy(g).cuda(), PREC_FP64).cpu().numpy()
    g32 = api.pfft_convolve(P, torch.from_numpy(g.astype(np.complex64)).cuda(), PREC_MIXED).cpu().numpy()
    idx = np.stack(np.meshgrid(*[np.arange(n) for n in grid], indexing="ij"), axis=-1).reshape(-1, 3)
    nodes = np.array([[0, 0, 0], [255, 255, 31], [128, 77, 16], [3, 250, 0], [200, 5, 30], [64, 191, 9]])
    for b in range(3):
        flat = g[b].reshape(-1)
        ref = np.array([np.dot(lossy_kernel(n - idx, h, 0.0, 0.0), flat) for n in nodes])
        got64 = np.array([g64[b][tuple(n)] for n in nodes])
        got32 = np.array([g32[b][tuple(n)] for n in nodes])
        scale = np.abs(ref).max()
        assert np.abs(got64 - ref).max() < 1e-11 * scale
        assert np.abs(got32 - ref).max() < 2e-6 * scale


def test_pdn_fp64_operator_is_complex_symmetric(pdn):
    w, L, P, om = pdn
    uv = torch.from_numpy(synth.complex_gaussian(L.nl, 2, seed=19)).cuda()
    u = uv.cpu().numpy()
    for f in (1e6, 1e9):
        z = api.pfft_matvec(P, uv, 2 * np.pi * np.array([f, f]), SPACE_LOOP, PREC_FP64).cpu().numpy()
        lhs, rhs = np.sum(u[0] * z[1]), np.sum(u[1] * z[0])
        assert abs(lhs - rhs) < 1e-11 * np.linalg.norm(u[0]) * np.linalg.norm(z[1])


def test_pdn_mixed_matches_fp64(pdn):
    w, L, P, om = pdn
    x = torch.from_numpy(synth.complex_gaussian(L.nl, len(om), seed=7)).cuda()
    y64 = api.pfft_matvec(P, x, om, SPACE_LOOP, PREC_FP64).cpu().numpy()
    y32 = api.pfft_matvec(P, x, om, SPACE_LOOP, PREC_MIXED).cpu().numpy()
    err = np.linalg.norm(y32 - y64, axis=1) / np.linalg.norm(y64, axis=1)
    assert err.max() < 1e-5, err


@pytest.fixture(scope="module")
def pdn_sampled_oracle(pdn):
    # the oracle pFFT on the full plane pair with its near list restricted to the
    # triangles of 24 random branches and 12 loops (10 of at most 6 branches, 2 of
    # 40 to 80), applying B and B^T triangle by triangle (no stored B)
    w, L, P, om = pdn
    m = w["mesh"]
    O = build_loops(m)
    A = O.A.tocsr()
    ln = np.diff(A.indptr)[:O.nl - O.n_ports]
    rng = np.random.default_rng(13)
    loops = np.sort(np.concatenate([rng.choice(np.nonzero(ln <= 6)[0], 10, replace=False),
                                    rng.choice(np.nonzero((ln >= 40) & (ln <= 80))[0], 2, replace=False)]))
    loop_br = np.concatenate([A.indices[A.indptr[l]:A.indptr[l + 1]] for l in loops])
    branches = np.sort(rng.choice(O.nb, 24, replace=False))
    tris = np.unique(O.br_tri[np.concatenate([branches, loop_br])].ravel())
    S = PfftSystem(m, O, PfftParams(grid=w["grid"], order=3, near_factor=4.0, near_min_diam=2.0, n_touch=16,
                                    h0=0.0), targets=tris, lean=True)
    return O, S, loops, branches


def elementwise_rel(a, b, floor=1e-3):
    # largest relative error over the entries above floor times the largest entry
    big = np.abs(b) > floor * np.abs(b).max()
    return float((np.abs(a - b)[big] / np.abs(b)[big]).max())


@pytest.mark.parametrize("nrep", [1, 3])
def test_pdn_sampled_rows_match_oracle(pdn, pdn_sampled_oracle, nrep):
    # 32 right-hand sides (CUDA-core near gather) and 96 (tensor-core near field in
    # the mixed form): the GPU's branch-space rows and loop-space rows for two of
    # them against the oracle, FP64 within 1e-10 and mixed within 1e-5 (relative
    # 2-norm over the sampled rows) and element by element within 100 times that;
    # the loop rows are A's rows applied to the oracle's exact branch rows
    w, L, P, om = pdn
    O, S, loops, branches = pdn_sampled_oracle
    oms = np.tile(om, nrep)
    R = oms.size
    x = synth.complex_gaussian(O.nl, R, seed=71)
    A = O.A.tocsr()[:, :O.nb]
    alpha = np.ascontiguousarray(np.asarray(A.T @ x.T).T)  # the loop currents' branch currents
    sampled = (0, R - 1) if nrep == 1 else (5, R - 6)
    refs = {}
    for r in sampled:
        bp = S.branch_product(alpha[r], oms[r])
        refs[r] = (bp[branches], (A[loops] @ bp))
    xt, at = torch.from_numpy(x).cuda(), torch.from_numpy(alpha).cuda()
    for prec, tol in ((PREC_FP64, 1e-10), (PREC_MIXED, 1e-5)):
        yl = api.pfft_matvec(P, xt, oms, SPACE_LOOP, prec).cpu().numpy()
        yb = api.pfft_matvec(P, at, oms, SPACE_BRANCH, prec).cpu().numpy()
        for r in sampled:
            rb, rl = refs[r]
            assert sampled_rel(yb[r, branches], rb) < tol, (prec, r, "branch")
            assert sampled_rel(yl[r, loops], rl) < tol, (prec, r, "loop")
            assert elementwise_rel(yb[r, branches], rb) < 100 * tol, (prec, r)
            assert elementwise_rel(yl[r, loops], rl) < 100 * tol, (prec, r)

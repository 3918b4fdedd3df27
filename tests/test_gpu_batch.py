"""Batched uneven geometries: sie_batch_matvec / sie_batch_solve.

Every plan's product in a batch is the same sequence of kernels as its own
pfft_matvec, only on the plan's batch stream (eager) or inside one captured
CUDA graph (replayed), so results must equal pfft_matvec bit for bit; a graph is
captured again when an input address, a right-hand-side count, the space, the
precision or a plan's scratch changes, and not when only omega changes.  The
batch solve equals each plan's own solve.  A meander against the oracle pFFT
(oracle/pfft.py) pins the meander geometry itself: FP64 within 1e-10, mixed
within 1e-5.  The full workload (32 meanders, 5k-60k triangles each, 32
frequencies) runs in one batch: graph replays equal the eager products, the
mixed form stays within 1e-5 of FP64, and a batched solve converges with
positive R and L on every trace.  The batched solve under graph replay (one
replay per Arnoldi step of all plans, sie_batch_solve_graph) equals each plan's
own solve bit for bit, on the small batch and on the full workload.
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.pfft import PfftSystem, PfftParams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, SieError, SPACE_LOOP, SPACE_BRANCH, PREC_FP64, PREC_MIXED  # noqa: E402

PRM = dict(order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=0.0)


def make_plan(w):
    m = w["mesh"]
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    return api.Plan(M, L, dict(PRM, grid=w["grid"]))


@pytest.fixture(scope="module")
def small():
    ws = [synth.meander(k, n_tri=1500) for k in range(3)]
    plans = [make_plan(w) for w in ws]
    return ws, plans


def inputs(plans, nrhs, space, seed):
    xs, oms = [], []
    for i, (p, r) in enumerate(zip(plans, nrhs)):
        n = p.nl if space == SPACE_LOOP else p.nb
        xs.append(torch.from_numpy(synth.complex_gaussian(n, r, seed=seed + i)).cuda())
        oms.append(2 * np.pi * np.logspace(7, 9.5, r))
    return xs, oms


@pytest.mark.parametrize("space", [SPACE_LOOP, SPACE_BRANCH], ids=["loop", "branch"])
@pytest.mark.parametrize("prec", [PREC_FP64, PREC_MIXED], ids=["fp64", "mixed"])
def test_batch_equals_individual(small, space, prec):
    ws, plans = small
    B = api.Batch(plans)
    xs, oms = inputs(plans, [4, 6, 3], space, 10)
    ref = [api.pfft_matvec(p, x, o, space, prec) for p, x, o in zip(plans, xs, oms)]
    eager = B.matvec(xs, oms, space, prec, graph=False)
    outs = [torch.empty_like(x) for x in xs]
    g1 = B.matvec(xs, oms, space, prec, graph=True, outs=outs)
    g1 = [t.clone() for t in g1]
    g2 = B.matvec(xs, oms, space, prec, graph=True, outs=outs)
    for r, e, a, b in zip(ref, eager, g1, g2):
        assert torch.equal(r, e) and torch.equal(r, a) and torch.equal(r, b)
    st = B.stats()
    assert st["captures"] == 1 and st["replays"] == 2


def test_graph_recapture_rules(small):
    ws, plans = small
    B = api.Batch(plans)
    xs, oms = inputs(plans, [2, 2, 2], SPACE_LOOP, 20)
    outs = [torch.empty_like(x) for x in xs]
    B.matvec(xs, oms, graph=True, outs=outs)
    # new frequencies only: replayed with the new coefficients, no new capture
    oms2 = [o * 3.0 for o in oms]
    got = [t.clone() for t in B.matvec(xs, oms2, graph=True, outs=outs)]
    ref = [api.pfft_matvec(p, x, o) for p, x, o in zip(plans, xs, oms2)]
    assert all(torch.equal(a, b) for a, b in zip(got, ref))
    assert B.stats()["captures"] == 1
    # a plan's scratch grows (a larger batch through pfft_matvec): captured again
    big = torch.from_numpy(synth.complex_gaussian(plans[1].nl, 9, seed=3)).cuda()
    api.pfft_matvec(plans[1], big, 2 * np.pi * np.full(9, 1e8))
    got = [t.clone() for t in B.matvec(xs, oms2, graph=True, outs=outs)]
    assert all(torch.equal(a, b) for a, b in zip(got, ref))
    assert B.stats()["captures"] == 2
    # other output buffers: captured again
    B.matvec(xs, oms2, graph=True)
    assert B.stats()["captures"] == 3


def test_batch_rejects_bad_input(small):
    ws, plans = small
    with pytest.raises(SieError):
        api.Batch([plans[0], plans[0]])
    B = api.Batch(plans[:2])
    xs, oms = inputs(plans[:2], [2, 2], SPACE_LOOP, 30)
    with pytest.raises(SieError):   # x and y overlap
        B.matvec(xs, oms, graph=False, outs=xs)


def test_batch_solve_equals_individual(small):
    ws, plans = small
    freqs = [np.array([1e8, 2e9]), np.array([5e8]), np.array([1e7, 1e9, 4e9])]
    B = api.Batch(plans)
    got = B.solve(freqs, tol=1e-8, restart=100, max_iter=400)
    for p, f, (Z, st) in zip(plans, freqs, got):
        Z0, st0 = api.sie_solve(p, f, tol=1e-8, restart=100, max_iter=400)
        assert st["converged"] and st0["converged"]
        assert np.array_equal(Z, Z0)


@pytest.mark.parametrize("prec,refine", [(PREC_FP64, False), (PREC_MIXED, True)], ids=["fp64", "mixed_refined"])
def test_batch_solve_graph_equals_individual(small, prec, refine):
    # every plan's GMRES stepped in lockstep by graph replay: the same kernels in the
    # same order as the plan's own solve, so Z and the iteration counts are equal
    ws, plans = small
    freqs = [np.array([1e8, 2e9]), np.array([5e8]), np.array([1e7, 1e9, 4e9])]
    B = api.Batch(plans)
    r0 = B.stats()["replays"]
    got = B.solve(freqs, tol=1e-8, restart=100, max_iter=400, prec=prec, refine=refine, graph=True)
    assert B.stats()["replays"] > r0
    for p, f, (Z, st) in zip(plans, freqs, got):
        Z0, st0 = api.sie_solve(p, f, tol=1e-8, restart=100, max_iter=400, prec=prec, refine=refine)
        assert st["converged"] and st0["converged"]
        assert st["iterations_max"] == st0["iterations_max"] and st["matvecs"] == st0["matvecs"]
        assert np.array_equal(Z, Z0)


def test_meander_matches_oracle():
    w = synth.meander(5, n_tri=400)
    m = w["mesh"]
    O = build_loops(m)
    S = PfftSystem(m, O, PfftParams(grid=w["grid"], order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8))
    P = make_plan(w)
    om = 2 * np.pi * np.array([1e7, 1e9, 5e9])
    x = synth.complex_gaussian(O.nl, om.size, seed=51)
    ref = np.stack([S.matvec(x[r], om[r]) for r in range(om.size)])
    for prec, tol in ((PREC_FP64, 1e-10), (PREC_MIXED, 1e-5)):
        y = api.pfft_matvec(P, torch.from_numpy(x).cuda(), om, SPACE_LOOP, prec).cpu().numpy()
        err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() < tol, (prec, err)


@pytest.fixture(scope="module")
def full():
    ws = synth.meanders_32()
    plans = [make_plan(w) for w in ws]
    return ws, plans


def test_full_batch_graph_and_precision(full):
    ws, plans = full
    B = api.Batch(plans)
    xs, oms = inputs(plans, [32] * len(plans), SPACE_LOOP, 100)
    oms = [2 * np.pi * w["freqs"] for w in ws]
    e64 = B.matvec(xs, oms, SPACE_LOOP, PREC_FP64, graph=False)
    outs = [torch.empty_like(x) for x in xs]
    B.matvec(xs, oms, SPACE_LOOP, PREC_MIXED, graph=True, outs=outs)
    g32 = B.matvec(xs, oms, SPACE_LOOP, PREC_MIXED, graph=True, outs=outs)
    for i in (0, 7, 31):
        assert torch.equal(g32[i], api.pfft_matvec(plans[i], xs[i], oms[i], SPACE_LOOP, PREC_MIXED))
    for a, b in zip(g32, e64):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        err = np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
        assert err.max() < 1e-5


def test_full_batch_solve(full):
    ws, plans = full
    B = api.Batch(plans)
    freqs = [np.array([1e8, 5e9])] * len(plans)
    res = B.solve(freqs, tol=1e-6, restart=200, max_iter=1000, prec=PREC_MIXED)
    for (Z, st), f in zip(res, freqs):
        assert st["converged"]
        z = Z[:, 0, 0]
        assert np.all(z.real > 0) and np.all(z.imag / (2 * np.pi * f) > 0)


def test_full_batch_solve_graph(full):
    # the 32-meander workload: one graph replay per Arnoldi step of all plans, equal
    # to the plans' solves on host threads
    ws, plans = full
    B = api.Batch(plans)
    freqs = [np.array([1e8, 5e9])] * len(plans)
    a = B.solve(freqs, tol=1e-6, restart=200, max_iter=1000, prec=PREC_MIXED, refine=True, graph=True)
    b = B.solve(freqs, tol=1e-6, restart=200, max_iter=1000, prec=PREC_MIXED, refine=True)
    for (Za, sa), (Zb, sb) in zip(a, b):
        assert sa["converged"] and sb["converged"]
        assert np.array_equal(Za, Zb)

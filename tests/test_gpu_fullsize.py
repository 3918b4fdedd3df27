"""The bench workload at full size: 8 bond wires (40,192 triangles, 20,096 loops,
grid 128 x 64 x 32), 16 frequencies x 8 ports = 128 right-hand sides, in the
launch configuration bench.py times.  The oracle cannot build this operator in
seconds, so the checks are properties that hold at any size:

* the FP64 operator is complex symmetric (reciprocity of A Z_b A^T with
  symmetric near blocks, I = B^T and an even kernel): u^T Z v = v^T Z u;
* the mixed form (tensor-core near field at 128 right-hand sides) agrees with
  the FP64 form within the mixed parity bound;
* the tensor-core near field (even count from 96) and the CUDA-core FP32 gather (odd
  count) agree on the same vectors;
* the preconditioned solve gives a reciprocal port impedance, Z = Z^T.

And against the oracle on sampled outputs: the oracle pFFT (oracle/pfft.py),
built with its near list restricted to the triangles of sampled branches, gives
those rows of the product exactly (the grid part is computed in full).  Rows of
24 random branches (branch space) and of 12 loops (loop space, 10 of at most 6
branches and 2 of 40 to 80) for 3 of the 128 right-hand sides, FP64 within
1e-10 and mixed within 1e-5 of the oracle (relative 2-norm over the sampled
rows), in the 128-right-hand-side launch the benchmark times.  The same loop
rows of the lossy-kernel product (kernel exp(-jkR)/R, one complex spectrum and
one set of complex near blocks per frequency) against the oracle's lossy pFFT
restricted in the same way, FP64 1e-10 and mixed 1e-5.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, SPACE_LOOP, SPACE_BRANCH, PREC_FP64, PREC_MIXED  # noqa: E402

SAMPLED_RHS = (0, 77, 127)


@pytest.fixture(scope="module")
def bondwires():
    w = synth.bondwires_40k()
    m = w["mesh"]
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, dict(grid=w["grid"], order=3, near_factor=4.0, near_min_diam=2.0, n_touch=16, h0=0.0))
    om = np.repeat(2 * np.pi * w["freqs"], len(m.ports))
    x = torch.from_numpy(synth.complex_gaussian(L.nl, len(om), seed=7)).cuda()
    return w, L, P, om, x


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def test_fp64_operator_is_complex_symmetric(bondwires):
    w, L, P, om, x = bondwires
    uv = torch.from_numpy(synth.complex_gaussian(L.nl, 4, seed=17)).cuda()
    for f in (1e6, 1e10):
        o = 2 * np.pi * np.array([f] * 4)
        z = api.pfft_matvec(P, uv, o, SPACE_LOOP, PREC_FP64).cpu().numpy()
        u = uv.cpu().numpy()
        for a, b in ((0, 1), (2, 3)):
            lhs, rhs = np.sum(u[a] * z[b]), np.sum(u[b] * z[a])
            assert abs(lhs - rhs) < 1e-11 * np.linalg.norm(u[a]) * np.linalg.norm(z[b])


def test_mixed_matches_fp64_at_bench_size(bondwires):
    w, L, P, om, x = bondwires
    y64 = api.pfft_matvec(P, x, om, SPACE_LOOP, PREC_FP64).cpu().numpy()
    y32 = api.pfft_matvec(P, x, om, SPACE_LOOP, PREC_MIXED).cpu().numpy()
    assert rel(y32, y64).max() < 1e-5


def test_tensor_core_and_cuda_core_near_fields_agree(bondwires):
    """Both FP32 near fields within the mixed bound of FP64 on the same vectors
    (tf32 split products, 2^-21 per product, and FP32 FMAs round differently)."""
    w, L, P, om, x = bondwires
    y64 = api.pfft_matvec(P, x[:127].contiguous(), om[:127], SPACE_LOOP, PREC_FP64).cpu().numpy()
    y128 = api.pfft_matvec(P, x, om, SPACE_LOOP, PREC_MIXED).cpu().numpy()          # tensor cores
    y127 = api.pfft_matvec(P, x[:127].contiguous(), om[:127], SPACE_LOOP, PREC_MIXED).cpu().numpy()
    assert rel(y128[:127], y64).max() < 1e-5
    assert rel(y127, y64).max() < 1e-5
    assert rel(y127, y128[:127]).max() < 1e-5


def test_port_impedance_is_reciprocal(bondwires):
    w, L, P, om, x = bondwires
    freqs = np.array([1e8, 1e10])
    Z, st = api.sie_solve(P, freqs, tol=1e-8, restart=100, max_iter=400, prec=PREC_MIXED, refine=True)
    assert st["converged"]
    assert np.abs(Z - np.transpose(Z, (0, 2, 1))).max() < 1e-6 * np.abs(Z).max()
    R = Z.real
    assert np.all(np.diagonal(R, axis1=1, axis2=2) > 0)


@pytest.fixture(scope="module")
def sampled_oracle(bondwires):
    from oracle.graph import build_loops
    from oracle.pfft import PfftSystem, PfftParams
    w, L, P, om, x = bondwires
    m = w["mesh"]
    O = build_loops(m)
    A = O.A.tocsr()
    ln = np.diff(A.indptr)
    rng = np.random.default_rng(11)
    loops = np.sort(np.concatenate([rng.choice(np.nonzero(ln <= 6)[0], 10, replace=False),
                                    rng.choice(np.nonzero((ln >= 40) & (ln <= 80))[0], 2, replace=False)]))
    assert np.all(loops < O.nl - O.n_ports)          # no port link among the columns
    loop_br = np.concatenate([A.indices[A.indptr[l]:A.indptr[l + 1]] for l in loops])
    branches = np.sort(rng.choice(O.nb, 24, replace=False))
    tris = np.unique(O.br_tri[np.concatenate([branches, loop_br])].ravel())
    S = PfftSystem(m, O, PfftParams(grid=w["grid"], order=3, near_factor=4.0, near_min_diam=2.0, n_touch=16,
                                    h0=0.0), targets=tris)
    return O, S, loops, branches


def sampled_rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def elementwise_rel(a, b, floor=1e-2):
    # largest relative error over the entries above floor times the largest entry
    big = np.abs(b) > floor * np.abs(b).max()
    return float((np.abs(a - b)[big] / np.abs(b)[big]).max())


def test_sampled_rows_match_oracle_at_bench_size(bondwires, sampled_oracle):
    w, L, P, om, x = bondwires
    O, S, loops, branches = sampled_oracle
    xa = synth.complex_gaussian(O.nb, len(om), seed=23)
    alpha = torch.from_numpy(xa).cuda()
    xn = x.cpu().numpy()
    for prec, tol in ((PREC_FP64, 1e-10), (PREC_MIXED, 1e-5)):
        yl = api.pfft_matvec(P, x, om, SPACE_LOOP, prec).cpu().numpy()
        yb = api.pfft_matvec(P, alpha, om, SPACE_BRANCH, prec).cpu().numpy()
        for r in SAMPLED_RHS:
            ref_l = S.matvec(xn[r], om[r])[loops]
            ref_b = S.branch_product(xa[r], om[r])[branches]
            assert sampled_rel(yl[r, loops], ref_l) < tol, (prec, r)
            assert sampled_rel(yb[r, branches], ref_b) < tol, (prec, r)
            # element by element (entries above 1% of the largest) within 100 times that
            assert elementwise_rel(yl[r, loops], ref_l) < 100 * tol, (prec, r)
            assert elementwise_rel(yb[r, branches], ref_b) < 100 * tol, (prec, r)


def test_lossy_sampled_rows_match_oracle_at_bench_size(bondwires, sampled_oracle):
    # the lossy-kernel product (per-frequency complex spectra and near blocks, 16
    # frequencies in one 128-right-hand-side launch) against the oracle's lossy pFFT
    # restricted to the same sampled rows, at 1 MHz, 100 MHz and 10 GHz
    from oracle.lossy import LossyPfftSystem
    from oracle.pfft import PfftParams
    from paper_2210_04891_gb300 import native as N
    w, L, P, om, x = bondwires
    O, S, loops, branches = sampled_oracle
    m = w["mesh"]
    M = api.Mesh.from_synth(m)
    Ll = api.Loops(M, m.ports)
    Pl = api.Plan(M, Ll, dict(grid=w["grid"], order=3, near_factor=4.0, near_min_diam=2.0, n_touch=16, h0=0.0,
                              kernel=N.KERNEL_LOSSY))
    targets = np.unique(np.concatenate([S.op.targets]))
    SL = LossyPfftSystem(m, O, PfftParams(grid=w["grid"], order=3, near_factor=4.0, near_min_diam=2.0, n_touch=16,
                                          h0=0.0), targets=targets)
    xn = x.cpu().numpy()
    sampled = (0, 63, 127)
    refs = {r: SL.matvec(xn[r], om[r])[loops] for r in sampled}
    for prec, tol in ((PREC_FP64, 1e-10), (PREC_MIXED, 1e-5)):
        yl = api.pfft_matvec(Pl, x, om, SPACE_LOOP, prec).cpu().numpy()
        for r in sampled:
            assert sampled_rel(yl[r, loops], refs[r]) < tol, (prec, r)

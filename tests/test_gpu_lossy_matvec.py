"""GPU parity of the lossy-kernel product and solve (pfft_params.kernel =
SIE_KERNEL_LOSSY) against the oracle's lossy pFFT (oracle/lossy.py).

The lossy variant puts exp(-jkR)/R, k = (1 - j)/delta, in place of the static
kernel of Eq. StaticGF in all four steps of Sec. IV-B: per-frequency complex
spectra in the grid convolution and per-frequency complex near blocks.  Bars:
FP64 1e-10 and mixed 1e-5 relative 2-norm per right-hand side against the
oracle on the same seeded inputs, with several frequencies in one call (each
right-hand side its own spectrum and near blocks), in loop and branch space,
on a grid whose (y, z) plane fits one CTA and on one that does not; the
preconditioner's complex diagonal against the oracle's sparse LU of P; the
solve against the oracle's GMRES and the dense lossy LU.
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.pfft import PfftParams
from oracle.lossy import LossyPfftSystem, dense_Lt_lossy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, native as N, SPACE_LOOP, SPACE_BRANCH, PREC_FP64, PREC_MIXED  # noqa: E402


def rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


PARAMS = dict(grid=(16, 8, 4), order=3, near_factor=4.0, near_min_diam=2.0, n_touch=16, h0=0.0,
              kernel=N.KERNEL_LOSSY)


def build(m, params):
    O = build_loops(m)
    S = LossyPfftSystem(m, O, PfftParams(grid=params["grid"], order=params["order"],
                                         near_factor=params["near_factor"], near_min_diam=params["near_min_diam"],
                                         n_touch=params["n_touch"]))
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, params)
    return O, S, P


@pytest.fixture(scope="module")
def wires():
    m = synth.tiny_wires()
    return (m,) + build(m, PARAMS)


# five right-hand sides over three frequencies (|k| d from about 0.3 to 3 on these panels)
OMEGAS = 2 * np.pi * np.array([1e8, 1e8, 5e8, 2e9, 2e9])


@pytest.mark.parametrize("prec,tol", [(PREC_FP64, 1e-10), (PREC_MIXED, 1e-5)])
def test_lossy_loop_matvec_matches_oracle(wires, prec, tol):
    m, O, S, P = wires
    x = synth.complex_gaussian(O.nl, len(OMEGAS), seed=21)
    ref = np.stack([S.matvec(x[r], OMEGAS[r]) for r in range(len(OMEGAS))])
    got = api.pfft_matvec(P, torch.from_numpy(x).cuda(), OMEGAS, SPACE_LOOP, prec).cpu().numpy()
    assert rel(got, ref).max() < tol
    # element by element on the entries above a thousandth of the largest
    big = np.abs(ref) > 1e-3 * np.abs(ref).max()
    assert (np.abs(got - ref)[big] / np.abs(ref)[big]).max() < 100 * tol


@pytest.mark.parametrize("prec,tol", [(PREC_FP64, 1e-10), (PREC_MIXED, 1e-5)])
def test_lossy_branch_matvec_matches_oracle(wires, prec, tol):
    m, O, S, P = wires
    om = OMEGAS[[0, 2, 4]]
    a = synth.complex_gaussian(O.nb, 3, seed=22)
    ref = np.stack([S.branch_product(a[r], om[r]) for r in range(3)])
    got = api.pfft_matvec(P, torch.from_numpy(a).cuda(), om, SPACE_BRANCH, prec).cpu().numpy()
    assert rel(got, ref).max() < tol


def test_lossy_differs_from_static(wires):
    # the lossy product is not the static one at these frequencies (a plan that
    # ignored the kernel choice would pass nothing above)
    m, O, S, P = wires
    Ms = api.Mesh.from_synth(m)
    Ls = api.Loops(Ms, m.ports)
    Ps = api.Plan(Ms, Ls, dict(PARAMS, kernel=N.KERNEL_STATIC))
    x = torch.from_numpy(synth.complex_gaussian(O.nl, 2, seed=23)).cuda()
    om = OMEGAS[[2, 3]]
    a = api.pfft_matvec(P, x, om, SPACE_LOOP, PREC_FP64).cpu().numpy()
    b = api.pfft_matvec(Ps, x, om, SPACE_LOOP, PREC_FP64).cpu().numpy()
    assert rel(a, b).min() > 1e-3


@pytest.mark.parametrize("prec,tol", [(PREC_FP64, 1e-10), (PREC_MIXED, 1e-5)])
def test_lossy_large_plane_matches_oracle(prec, tol):
    # 4 x 256 x 16: the padded (y, z) plane (512 x 32) does not fit one CTA, so the
    # convolution runs as y pencils and z rows, each row reading its grid's spectrum
    m = synth.tiny_bar()
    O, S, P = build(m, dict(PARAMS, grid=(4, 256, 16), near_factor=1.0, near_min_diam=1.0, n_touch=8))
    om = 2 * np.pi * np.array([3e8, 1e9, 1e9])
    x = synth.complex_gaussian(O.nl, 3, seed=24)
    ref = np.stack([S.matvec(x[r], om[r]) for r in range(3)])
    got = api.pfft_matvec(P, torch.from_numpy(x).cuda(), om, SPACE_LOOP, prec).cpu().numpy()
    assert rel(got, ref).max() < tol


def test_lossy_slot_cache_eviction(wires):
    # 70 distinct frequencies in calls of 10 fill the 64 slots and replace the least
    # recently used; every result equals the one of a plan that never evicted
    m, O, S, P = wires
    x = torch.from_numpy(synth.complex_gaussian(O.nl, 10, seed=25)).cuda()
    oms = 2 * np.pi * np.geomspace(1e7, 3e9, 70)
    first = api.pfft_matvec(P, x, oms[:10], SPACE_LOOP, PREC_FP64)
    for c in range(1, 7):
        api.pfft_matvec(P, x, oms[10 * c:10 * c + 10], SPACE_LOOP, PREC_FP64)
    again = api.pfft_matvec(P, x, oms[:10], SPACE_LOOP, PREC_FP64)   # rebuilt after eviction
    assert torch.equal(first, again)
    with pytest.raises(N.SieError) as e:
        xx = torch.from_numpy(synth.complex_gaussian(O.nl, 65, seed=26)).cuda()
        api.pfft_matvec(P, xx, 2 * np.pi * np.geomspace(1e7, 3e9, 65), SPACE_LOOP, PREC_FP64)
    assert e.value.code == -1


def test_lossy_rejects_mixed_conductivity():
    m = synth.tiny_wires()
    m.sigma = np.array([4.1e7, 5.8e7])
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    with pytest.raises(N.SieError):
        api.Plan(M, L, PARAMS)


def test_lossy_precond_matches_oracle(wires):
    from oracle.gmres import Precond
    m, O, S, P = wires
    om = OMEGAS[[0, 3]]
    y = synth.complex_gaussian(O.nl, 2, seed=27)
    z = api.pfft_precond_apply(P, torch.from_numpy(y).cuda(), om).cpu().numpy()
    for r in range(2):
        ref = Precond(O, S.diag_Zb(om[r])).solve(y[r])
        assert np.linalg.norm(z[r] - ref) < 1e-9 * np.linalg.norm(ref)


def test_lossy_solve_matches_oracle(wires):
    # GMRES on the lossy loop system: the port impedance against the oracle's GMRES
    # on its lossy pFFT product with its P, and against the dense lossy LU within
    # the pFFT approximation; reciprocity Z = Z^T
    from oracle.gmres import Precond, gmres
    m, O, S, P = wires
    freqs = [1e8, 1e9]
    Z, st = api.sie_solve(P, freqs, tol=1e-10, restart=100, prec=PREC_FP64)
    assert st["converged"]
    npo = O.n_ports
    Lt0 = None
    for fi, f in enumerate(freqs):
        w = 2 * np.pi * f
        pc = Precond(O, S.diag_Zb(w))
        Y = np.zeros((npo, npo), complex)
        for p in range(npo):
            b = np.zeros(O.nl, complex)
            b[O.port_loop(p)] = 1.0
            xs, _, _ = gmres(lambda v: S.matvec(v, w), b, pc, tol=1e-12, restart=200)
            for q in range(npo):
                Y[q, p] = xs[O.port_loop(q)]
        Zo = np.linalg.inv(Y)
        assert np.abs(Z[fi] - Zo).max() < 1e-7 * np.abs(Zo).max()
        assert np.abs(Z[fi] - Z[fi].T).max() < 1e-8 * np.abs(Z[fi]).max()
        # dense lossy definition
        from oracle.mom import dense_Lt, branch_zs
        if Lt0 is None:
            Lt0 = dense_Lt(m, O)
        Lt = dense_Lt_lossy(m, O, w, float(m.sigma[0]), static_Lt=Lt0)
        A = O.A.toarray()[:, :O.nb]
        G = S.G.toarray()
        Zb = branch_zs(m, O, w)[:, None] * G + (1j * w * 4e-7 * np.pi / (4 * np.pi)) * Lt
        I = np.linalg.solve(A @ Zb @ A.T, np.stack([np.eye(O.nl)[O.port_loop(p)] for p in range(npo)], axis=1))
        Yd = np.array([[I[O.port_loop(q), p] for p in range(npo)] for q in range(npo)])
        Zd = np.linalg.inv(Yd)
        assert np.abs(Z[fi] - Zd).max() < 1e-3 * np.abs(Zd).max()


def test_batch_rejects_lossy_plans(wires):
    m, O, S, P = wires
    with pytest.raises(N.SieError):
        api.Batch([P])

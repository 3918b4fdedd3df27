"""Pins of the lossy grid kernel and its convolution (oracle/lossy.py).

* the FFT product equals the direct sum over node pairs (Toeplitz embedding);
* as w -> 0 the lossy kernel tends to the static 1/R one (closed-form limit);
* kernel values: |K| = exp(-r/delta)/r and arg K = -r/delta (mod 2 pi);
* the operator is complex symmetric (K(d) = K(-d)): <u, K v> = <v, K u>
  without conjugation, and it is not Hermitian;
* a planted mistake (a conjugated k, i.e. a growing exponential) fails the
  value pin.
"""
import numpy as np
import pytest

from oracle.lossy import (MU0, skin_wavenumber, lossy_kernel, padded_kernel, convolve_lossy,
                          convolve_lossy_direct)

H = np.array([1.5e-6, 2.0e-6, 0.7e-6])
SIG = 5.8e7


def rand_grid(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("f", [1e6, 1e9, 2e10])
def test_fft_product_equals_direct_sum(f):
    k = skin_wavenumber(2 * np.pi * f, SIG)
    q = rand_grid((6, 4, 4), 1)
    a = convolve_lossy(q, H, k, h0=0.3)
    b = convolve_lossy_direct(q, H, k, h0=0.3)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_static_limit():
    """w -> 0: exp(-jkR) = 1 - jkR + ..., so the relative change is O(|k| R_max)."""
    k = skin_wavenumber(2 * np.pi * 1e-3, SIG)     # delta ~ 2 m against a ~10 um grid
    q = rand_grid((6, 4, 4), 2)
    a = convolve_lossy_direct(q, H, k)
    idx = np.stack(np.meshgrid(np.arange(6), np.arange(4), np.arange(4), indexing="ij"), -1).reshape(-1, 3)
    d = idx[:, None, :] - idx[None, :, :]
    r = np.linalg.norm(d * H, axis=-1)
    Hs = np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), 0.0)
    b = (Hs @ q.reshape(-1)).reshape(q.shape)
    rmax = np.linalg.norm(np.array([5, 3, 3]) * H)
    assert np.abs(a - b).max() < 2 * abs(k) * rmax * np.abs(b).max()
    assert np.abs(a - b).max() > 0.0


def test_kernel_values_closed_form():
    w = 2 * np.pi * 3e9
    delta = np.sqrt(2.0 / (w * MU0 * SIG))
    assert abs(delta - 1.0 / np.sqrt(np.pi * 3e9 * MU0 * SIG)) < 1e-15   # the 1/sqrt(pi f mu sigma) form
    assert 1.20e-6 < delta < 1.21e-6                                      # Cu at 3 GHz
    d = np.array([[1, 0, 0], [2, 3, 1], [0, 0, 5]])
    r = np.linalg.norm(d * H, axis=-1)
    K = lossy_kernel(d, H, skin_wavenumber(w, SIG))
    assert np.allclose(np.abs(K), np.exp(-r / delta) / r, rtol=1e-13)
    assert np.allclose(np.angle(K), np.angle(np.exp(-1j * r / delta)), atol=1e-12)
    assert lossy_kernel(np.zeros(3, int), H, 1.0, h0=0.25) == 0.25
    # a conjugated wavenumber grows instead of decaying: the value pin catches it
    Kbad = lossy_kernel(d, H, np.conj(skin_wavenumber(w, SIG)))
    assert not np.allclose(np.abs(Kbad), np.exp(-r / delta) / r, rtol=1e-3)


def test_complex_symmetric_not_hermitian():
    k = skin_wavenumber(2 * np.pi * 1e9, SIG)
    u, v = rand_grid((5, 4, 3), 3), rand_grid((5, 4, 3), 4)
    Kv, Ku = convolve_lossy(v, H, k), convolve_lossy(u, H, k)
    assert abs(np.sum(u * Kv) - np.sum(v * Ku)) < 1e-12 * abs(np.sum(u * Kv))
    assert abs(np.vdot(u, Kv) - np.conj(np.vdot(v, Ku))) > 1e-3 * abs(np.vdot(u, Kv))


def test_padded_kernel_layout_matches_static_convention():
    """Same offsets, wrap and zeroed +-N planes as the static kernel table."""
    k = skin_wavenumber(2 * np.pi * 1e-3, SIG)
    N = np.array([4, 4, 2])

    Kp = padded_kernel(N, H, k)
    ax = [np.where(np.arange(m) < m // 2, np.arange(m), np.arange(m) - m) for m in 2 * N]
    for a, m in enumerate(2 * N):
        sl = [slice(None)] * 3
        sl[a] = m // 2
        assert np.all(Kp[tuple(sl)] == 0)
    dx, dy, dz = np.meshgrid(*ax, indexing="ij")
    r = np.linalg.norm(np.stack([dx, dy, dz], -1) * H, axis=-1)
    live = (r > 0) & (Kp != 0)
    # exp(-jkr)/r = 1/r - jk + O(k^2 r): within 2|k| of 1/r at the signed offsets
    assert np.abs(Kp[live] - 1 / r[live]).max() < 2 * abs(k)


# ---------------------------------------------------------------- the lossy product (remainder blocks, pre-correction)

from oracle.lossy import (smooth_remainder, remainder_blocks, inv_skin_depth, LossyPfftSystem,  # noqa: E402
                          dense_Lt_lossy)
from oracle.quadrature import radon7, subdivided, collapsed_gauss  # noqa: E402
from oracle.integrals import tri_geometry, pair_blocks  # noqa: E402
import synth  # noqa: E402
from oracle.graph import build_loops  # noqa: E402
from oracle.pfft import PfftParams  # noqa: E402
from oracle.mom import assemble_from_blocks, dense_Lt  # noqa: E402


def test_smooth_remainder_closed_form():
    # against the plain complex exponential where it is accurate, against the Taylor
    # series -jk + (-jk)^2 R/2 + (-jk)^3 R^2/6 where R/delta is tiny, and its limit at 0
    inv_delta = 1.0 / 2.0e-6
    k = (1 - 1j) * inv_delta
    R = np.array([1e-7, 5e-7, 2e-6, 1e-5, 4e-5])
    direct = (np.exp(-1j * k * R) - 1.0) / R
    assert np.abs(smooth_remainder(R, inv_delta) - direct).max() < 1e-12 * np.abs(direct).max()
    r = np.array([1e-13, 1e-12, 1e-11])
    ser = -1j * k + (-1j * k) ** 2 * r / 2 + (-1j * k) ** 3 * r ** 2 / 6
    assert np.abs(smooth_remainder(r, inv_delta) - ser).max() < 1e-13 * abs(k)
    assert smooth_remainder(np.array([0.0]), inv_delta)[0] == -(1 + 1j) * inv_delta


def _pairs(m):
    g = tri_geometry(m.xyz, m.tri)
    out = {"self": (0, 0)}
    for j in range(1, m.nt):
        s = len(set(m.tri[0]) & set(m.tri[j]))
        if s == 2:
            out.setdefault("edge", (0, j))
        elif s == 1:
            out.setdefault("vertex", (0, j))
        elif np.linalg.norm(g["centroid"][0] - g["centroid"][j]) < 2 * g["diam"].max():
            out.setdefault("separated", (0, j))
    return g, out


@pytest.mark.parametrize("kd", [0.05, 0.3, 1.0])
def test_remainder_rule_converged(kd):
    # the Radon 7 x 7 product against the same integrand under a 448 x 448 point rule
    # (64 sub-triangles): the error relative to the whole lossy block stays below
    # 1e-3 (|k| d)^2 for self, edge-, vertex-adjacent and separated pairs
    m = synth.tiny_bar()
    g, pairs = _pairs(m)
    d = g["diam"].max()
    inv_delta = kd / d / np.sqrt(2.0)           # |k| = sqrt(2) / delta
    P, A = g["p"], g["area"]
    for name, (i, j) in pairs.items():
        a = remainder_blocks(P[[i]], A[[i]], P[[j]], A[[j]], inv_delta)[0]
        b = remainder_blocks(P[[i]], A[[i]], P[[j]], A[[j]], inv_delta, rule=subdivided(radon7(), 3))[0]
        full = pair_blocks(P[[i]], A[[i]], P[[j]], A[[j]], collapsed_gauss(16))[0] + b
        assert np.abs(a - b).max() < 1e-3 * kd ** 2 * np.abs(full).max(), name


def test_remainder_first_order_term():
    # |k| d << 1: (exp(-jkR) - 1)/R = -jk + O(k^2 R), so the block tends to
    # -jk (int_T f_k) . (int_S f_l) with int_T f_k dS = (r_c - v_k)/2
    m = synth.tiny_bar()
    g, pairs = _pairs(m)
    inv_delta = 1e-4 / g["diam"].max()
    k = (1 - 1j) * inv_delta
    P, A, C = g["p"], g["area"], g["centroid"]
    for name, (i, j) in pairs.items():
        blk = remainder_blocks(P[[i]], A[[i]], P[[j]], A[[j]], inv_delta)[0]
        fi = (C[i][None, :] - P[i]) / 2.0
        fj = (C[j][None, :] - P[j]) / 2.0
        ref = -1j * k * fi @ fj.T
        assert np.abs(blk - ref).max() < 2e-4 * np.abs(ref).max(), name


def test_far_pair_lossy_limit():
    # a pair at fixed distance D (|k| D ~ 1.4): as the triangles shrink, the whole lossy
    # block (static closed form plus remainder) tends to (int f_k).(int f_l) exp(-jkD)/D
    # with int_T f_k dS = (r_c - v_k)/2, the error falling with the triangle size
    inv_delta = 1.0 / 20e-6
    k = (1 - 1j) * inv_delta
    D = 20e-6
    errs = []
    for s in (2e-6, 1e-6, 0.5e-6):
        tA = np.array([[[0.0, 0.0, 0.0], [s, 0.0, 0.0], [0.0, s, 0.0]]])
        tB = tA + np.array([D, 0.0, 0.0])
        aA = np.array([0.5 * s * s])
        blk = (pair_blocks(tA, aA, tB, aA, radon7())[0]
               + remainder_blocks(tA, aA, tB, aA, inv_delta)[0])
        fa = (tA[0].mean(axis=0)[None, :] - tA[0]) / 2.0
        ref = fa @ fa.T * np.exp(-1j * k * D) / D
        errs.append(np.abs(blk - ref).max() / np.abs(ref).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.3 * errs[0] and errs[2] < 0.05


@pytest.fixture(scope="module")
def wires_lossy():
    m = synth.tiny_wires()
    L = build_loops(m)
    return m, L


def test_all_near_lossy_equals_direct():
    # every pair near: the grid part cancels exactly and the lossy pFFT product is the
    # direct product of the lossy blocks (a wrong sign, a conjugated kernel or a
    # transposed grid block would leave a grid-sized residue)
    m = synth.tiny_bar()
    L = build_loops(m)
    S = LossyPfftSystem(m, L, PfftParams(grid=(8, 4, 4), near_factor=1e3))
    om = 2 * np.pi * 2e8
    op = S.op(om)
    assert op.s.near_i.shape[0] == m.nt * m.nt
    Ldense = (assemble_from_blocks(m, L, op.s.near_i, op.s.near_j, op.L_direct.real)
              + 1j * assemble_from_blocks(m, L, op.s.near_i, op.s.near_j, op.L_direct.imag))
    a = synth.complex_gaussian(L.nb, 1, seed=5)[0]
    got = op.Lt_apply(a)
    ref = Ldense @ a
    assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref)
    # the complex grid blocks (real and imaginary tables through the C loop) against
    # the numpy double sum with the complex table, on every 41st pair
    sel = slice(None, None, 41)
    Hs = op.s.Hpad
    op.s.Hpad = op.Hpad
    try:
        ref_g = op.s.grid_blocks(op.s.near_i[sel], op.s.near_j[sel], native=False)
    finally:
        op.s.Hpad = Hs
    assert np.abs(op.L_grid[sel] - ref_g).max() < 1e-12 * np.abs(ref_g).max()


def test_lossy_matvec_static_limit(wires_lossy):
    # w -> 0 with the Z_s and c_L scaling divided out: the lossy inductive product
    # tends to the static one, the difference of order |k| times the mesh extent
    m, L = wires_lossy
    S = LossyPfftSystem(m, L, PfftParams(grid=(16, 8, 4)))
    a = synth.complex_gaussian(L.nb, 1, seed=6)[0]
    om = 2 * np.pi * 1.0
    lossy = S.op(om).Lt_apply(a)
    static = S.base.op.Lt_apply(a)
    ext = np.linalg.norm(m.xyz.max(axis=0) - m.xyz.min(axis=0))
    kext = np.sqrt(2) * inv_skin_depth(om, S.sigma) * ext
    assert np.linalg.norm(lossy - static) < 2 * kext * np.linalg.norm(static)
    assert np.linalg.norm(lossy - static) > 1e-3 * kext * np.linalg.norm(static)


def test_lossy_pfft_converges_to_dense(wires_lossy):
    # the lossy pFFT product against the dense lossy product of every pair (static
    # closed form + remainder): the gap falls as the near radius grows
    m, L = wires_lossy
    om = 2 * np.pi * 1e8
    Ld = dense_Lt_lossy(m, L, om, float(m.sigma[0]))
    a = synth.complex_gaussian(L.nb, 1, seed=8)[0]
    ref = Ld @ a
    errs = []
    for nf in (2.0, 4.0):
        S = LossyPfftSystem(m, L, PfftParams(grid=(16, 8, 4), near_factor=nf, near_min_diam=nf / 2))
        errs.append(np.linalg.norm(S.op(om).Lt_apply(a) - ref) / np.linalg.norm(ref))
    assert errs[1] < errs[0] and errs[1] < 1e-3

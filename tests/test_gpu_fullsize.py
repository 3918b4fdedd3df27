"""The bench workload at full size: 8 bond wires (40,192 triangles, 20,096 loops,
grid 128 x 64 x 32), 16 frequencies x 8 ports = 128 right-hand sides, in the
launch configuration bench.py times.  The oracle cannot build this operator in
seconds, so the checks are properties that hold at any size:

* the FP64 operator is complex symmetric (reciprocity of A Z_b A^T with
  symmetric near blocks, I = B^T and an even kernel): u^T Z v = v^T Z u;
* the mixed form (tensor-core near field at 128 right-hand sides) agrees with
  the FP64 form within the mixed parity bound;
* the tensor-core near field (even count) and the CUDA-core FP32 gather (odd
  count) agree on the same vectors;
* the preconditioned solve gives a reciprocal port impedance, Z = Z^T.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, SPACE_LOOP, PREC_FP64, PREC_MIXED  # noqa: E402


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

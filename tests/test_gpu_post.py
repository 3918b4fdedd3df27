"""GPU parity of the post-processing of loop currents (Sec. V, Eqs. CurT and VolT).

sie_postprocess turns loop currents into branch currents A^T x, branch voltage
drops Z_b A^T x (the branch-space pFFT product) and panel potentials (the
tree-path sums of the drops from each panel's node to its conductor's reference
node).  Against oracle/post.py on the same loop basis: currents exact up to
FP64 rounding, drops and potentials within the matvec bounds (FP64 1e-10,
mixed 1e-5).  On a solution of the pFFT loop system the drops derive from the
potentials on every branch, links included (Kirchhoff's voltage law), and the
driven port's source contact sits 1 V from its sink.
"""
import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from oracle.pfft import PfftSystem, PfftParams
from oracle.post import branch_currents, panel_potentials

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, native as N, SieError, SPACE_LOOP, PREC_FP64, PREC_MIXED  # noqa: E402

P_WIRES = dict(grid=(16, 8, 4), order=3, near_factor=5.0, near_min_diam=2.0, n_touch=16, h0=0.0)
OM = 2 * np.pi * np.array([1e6, 1e8, 1e9, 3e9])


def system(ports):
    m = synth.tiny_wires()
    O = build_loops(m, ports=ports)
    S = PfftSystem(m, O, PfftParams(grid=P_WIRES["grid"], order=3, near_factor=5.0, near_min_diam=2.0,
                                    n_touch=16))
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, ports)
    return m, O, S, api.Plan(M, L, P_WIRES)


@pytest.fixture(scope="module")
def wires():
    m = synth.tiny_wires()
    return system(m.ports)


def sinks_of(O):
    return [O.tail[O.nb + p] for p in range(O.n_ports)]


def oracle_post(O, S, x, om):
    a = np.stack([branch_currents(O, x[r]) for r in range(len(om))])
    v = np.stack([S.branch_product(a[r], om[r]) for r in range(len(om))])
    phi = np.stack([panel_potentials(O, v[r], sinks_of(O)) for r in range(len(om))])
    return a, v, phi


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("prec,tol", [(PREC_FP64, 1e-10), (PREC_MIXED, 1e-5)], ids=["fp64", "mixed"])
def test_postprocess_matches_oracle(wires, prec, tol):
    m, O, S, P = wires
    x = synth.complex_gaussian(O.nl, OM.size, seed=91)
    a0, v0, p0 = oracle_post(O, S, x, OM)
    a, v, phi = (t.cpu().numpy() for t in api.postprocess(P, torch.from_numpy(x).cuda(), OM, prec))
    assert rel(a, a0) < 1e-14          # exact sums of at most a few loop currents
    assert rel(v, v0) < tol
    for r in range(OM.size):
        assert rel(phi[r], p0[r]) < tol
    # the drops are the branch-space product itself
    vb = api.pfft_matvec(P, torch.from_numpy(a).cuda(), OM, N.SPACE_BRANCH, prec).cpu().numpy()
    assert np.array_equal(vb, v)


def test_partial_outputs_and_errors(wires):
    m, O, S, P = wires
    x = torch.from_numpy(synth.complex_gaussian(O.nl, 2, seed=92)).cuda()
    a, v, phi = api.postprocess(P, x, OM[:2])
    a1, v1, p1 = api.postprocess(P, x, None, currents=True, voltages=False, potentials=False)
    assert v1 is None and p1 is None and torch.equal(a1, a)
    a2, v2, p2 = api.postprocess(P, x, OM[:2], currents=False, voltages=False, potentials=True)
    assert a2 is None and v2 is None and torch.equal(p2, phi)
    # one right-hand side at a time gives the same rows
    _, _, p3 = api.postprocess(P, x[1:].contiguous(), OM[1:2])
    assert torch.equal(p3[0], phi[1])
    with pytest.raises(ValueError):
        api.postprocess(P, x, None)
    lib = N.lib()
    nt = m.nt
    buf = torch.empty((2, nt), dtype=torch.complex128, device="cuda")
    import ctypes
    with pytest.raises(SieError):      # potentials without omega: rejected by the library too
        N.check(lib.sie_postprocess(P.h, ctypes.c_void_p(x.data_ptr()), 2, None, PREC_FP64, None, None,
                                    ctypes.c_void_p(buf.data_ptr()), None))
    with pytest.raises(SieError):
        N.check(lib.sie_postprocess(P.h, ctypes.c_void_p(x.data_ptr()), 0, None, PREC_FP64,
                                    ctypes.c_void_p(buf.data_ptr()), None, None, None))
    with pytest.raises(SieError):
        N.check(lib.sie_postprocess(P.h, ctypes.c_void_p(x.data_ptr()), 2, None, 7,
                                    ctypes.c_void_p(buf.data_ptr()), None, None, None))


def test_kirchhoff_on_a_solution(wires):
    """x solves the pFFT loop system with 1 V in port 0 (oracle matrix, columns of
    its matvec): the GPU drops then equal phi(tail) - phi(head) on every branch."""
    m, O, S, P = wires
    w = OM[2]
    Zl = np.stack([S.matvec(e, w) for e in np.eye(O.nl)], axis=1)
    V = np.zeros(O.nl, complex)
    V[O.port_loop(0)] = 1.0
    x = np.linalg.solve(Zl, V)[None, :]
    for prec, tol in [(PREC_FP64, 1e-9), (PREC_MIXED, 1e-5)]:
        a, v, phi = (t.cpu().numpy()[0] for t in api.postprocess(P, torch.from_numpy(x).cuda(), [w], prec))
        node_phi = np.full(O.n_nodes, np.nan + 0j)
        node_phi[O.node_of_tri] = phi
        assert not np.isnan(node_phi.real).any()
        d = node_phi[O.tail[:O.nb]] - node_phi[O.head[:O.nb]]
        assert np.abs(d - v).max() < tol * np.abs(v).max()
        sinks = sinks_of(O)
        srcs = [O.head[O.nb + p] for p in range(O.n_ports)]
        assert node_phi[sinks[0]] == 0 and node_phi[sinks[1]] == 0
        assert abs(abs(node_phi[srcs[0]]) - 1.0) < 10 * tol
        assert abs(node_phi[srcs[1]]) < 10 * tol


def test_conductor_without_port_uses_its_tree_root():
    m = synth.tiny_wires()
    m, O, S, P = system(m.ports[:1])
    assert O.n_comp == 2 and O.n_ports == 1
    x = synth.complex_gaussian(O.nl, 2, seed=93)
    _, _, p0 = oracle_post(O, S, x, OM[:2])
    _, _, phi = (t.cpu().numpy() if t is not None else None
                 for t in api.postprocess(P, torch.from_numpy(x).cuda(), OM[:2], PREC_FP64))
    assert rel(phi, p0) < 1e-10
    root = int(np.nonzero((O.parent < 0) & (O.comp_of_node == O.comp_of_node[O.node_of_tri[-1]]))[0][0])
    on_root = np.nonzero(O.node_of_tri == root)[0]
    assert on_root.size and np.all(phi[:, on_root] == 0)

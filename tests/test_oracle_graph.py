"""Pins of the oracle's circuit graph and loop basis (Sec. II-D, III).

Exact integer checks: loop count b - n + s + p (Sec. III-A, III-C), KCL
M A^T = 0 (the loop currents conserve charge, Sec. II-A), rank A = l
(independent and complete loops, Sec. III-A), entries +-1 (Sec. III-B), the
Euler characteristic of closed surfaces, and the prism of Fig. 1 (8 triangles,
12 edges) with its five fundamental loops, read from a golden fixture.
"""
import json
import os

import numpy as np
import pytest

import synth
from synth.meshes import Mesh
from oracle.graph import build_loops, mesh_edges, BadPort, NonManifold

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def prism_mesh():
    """Triangular prism: two triangular caps, three rectangular sides split in two."""
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0.5, 0.8, 0], [0, 0, 2], [1, 0, 2], [0.5, 0.8, 2]], float)
    tri = np.array([[0, 2, 1], [3, 4, 5], [0, 1, 4], [0, 4, 3], [1, 2, 5], [1, 5, 4],
                    [2, 0, 3], [2, 3, 5]], np.int32)
    return Mesh(xyz=xyz, tri=tri, cond=np.zeros(8, np.int32), sigma=np.array([5.8e7]))


def check_invariants(mesh, loops):
    M = loops.incidence()
    A = loops.A
    assert set(np.unique(A.data)) <= {-1.0, 1.0}
    assert abs(M @ A.T).max() == 0.0
    assert np.linalg.matrix_rank(A.toarray()) == loops.nl
    n, b, s, p = loops.n_nodes, loops.nb, loops.n_comp, loops.n_ports
    assert loops.nl == b - n + s + p
    # every link appears in exactly its own loop
    for l, e in enumerate(loops.link_branch):
        col = A[:, e].toarray().ravel()
        assert col[l] == 1.0 and np.count_nonzero(col) == 1


def test_prism_fig1_golden():
    with open(os.path.join(GOLD, "prism_fig1.json")) as f:
        gold = json.load(f)
    m = prism_mesh()
    edges, _ = mesh_edges(m.tri)
    L = build_loops(m, ports=[])
    assert m.nt == gold["triangles"]
    assert edges.shape[0] == gold["edges"]
    assert L.nb == gold["edges"]
    assert L.nl == gold["loops_without_source"]
    check_invariants(m, L)
    # a source between two nodes adds one link and one loop (Sec. III-C)
    L2 = build_loops(m, ports=[(np.array([0]), np.array([1]))])
    assert L2.nl == gold["loops_without_source"] + 1
    check_invariants(m, L2)


def test_euler_and_loop_ratio():
    m = synth.tiny_bar()
    edges, _ = mesh_edges(m.tri)
    assert m.nv - edges.shape[0] + m.nt == 2
    # closed surface: b = 1.5 n, so loops ~ n/2 (Sec. III-B)
    L = build_loops(m, ports=[])
    assert L.nb == 3 * m.nt // 2
    assert L.nl == m.nt // 2 + 1
    check_invariants(m, L)


@pytest.mark.parametrize("make", [synth.tiny_bar, synth.tiny_wires, synth.tiny_two_bars])
def test_invariants_with_ports(make):
    m = make()
    L = build_loops(m)
    check_invariants(m, L)
    assert L.n_comp == m.ncond
    # port loops come last and each holds its port link
    for p in range(L.n_ports):
        assert L.link_branch[L.port_loop(p)] == L.nb + p


def test_root_choice_changes_tree_not_counts():
    m = synth.tiny_wires()
    a = build_loops(m, root="lowest")
    b = build_loops(m, root="highest")
    assert a.nl == b.nl and a.nb == b.nb
    assert (a.A != b.A).nnz > 0
    check_invariants(m, b)


def test_bad_ports():
    m = synth.tiny_two_bars()
    src0 = m.ports[0][0]
    snk1 = m.ports[1][1]
    with pytest.raises(BadPort):
        build_loops(m, ports=[(src0, snk1)])
    with pytest.raises(BadPort):
        build_loops(m, ports=[(src0, src0)])


def test_non_manifold_rejected():
    m = prism_mesh()
    xyz = np.vstack([m.xyz, [[0.5, -1.0, 1.0]]])
    tri = np.vstack([m.tri, [[0, 1, 6]]]).astype(np.int32)   # third triangle on edge (0,1)
    mm = Mesh(xyz=xyz, tri=tri, cond=np.zeros(9, np.int32), sigma=np.array([1.0]))
    with pytest.raises(NonManifold):
        build_loops(mm, ports=[])


def test_loops_per_triangle_pdn_table():
    # Sec. III-B: on a closed surface every triangle has three edges shared by two,
    # so b = 1.5 n and l = b - n + s + p = n/2 + s + p; the paper's PDN table (Sec. V-D)
    # prints loops close to half the triangles for every array size
    with open(os.path.join(GOLD, "pdn_table2.json")) as f:
        gold = json.load(f)
    for nt, nl in zip(gold["triangles"], gold["loops"]):
        assert 0.5 <= nl / nt < 0.55
    # the oracle's graph on a closed two-plane structure joined by vias, with ports:
    # contracting the contacts removes their internal edges, so l falls just below n/2
    m = synth.tiny_pdn()
    L = build_loops(m)
    assert L.nl == L.nb - L.n_nodes + L.n_comp + L.n_ports
    assert 0.49 <= L.nl / m.nt < 0.55
    check_invariants(m, L)

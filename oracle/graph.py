"""Circuit graph, spanning tree and fundamental loops of a triangle mesh.

Sec. II-D / Table I: each triangle is a circuit node and each edge shared by two
triangles is a branch, oriented T+ -> T- with T+ the lower triangle index (the
modified RWG function of Eq. (RWG) carries its current from T+ to T-).
Sec. III-A: a spanning tree per connected part; its branches are twigs, the
others links; there are n - s twigs and b - n + s links for s separate parts.
Sec. III-B: one fundamental loop per link (the link plus the tree path joining
its ends); A (l x b, entries +-1) maps branch voltages to loop voltages
(Eq. VolT), A^T loop currents to branch currents (Eq. CurT).
Sec. III-C: each voltage source adds one link and one loop, b - n + s + p loops.

Readings where the paper is silent:
  * a port's source and sink faces are contracted into one node each (an
    equipotential electrode); edges inside a contact carry no branch;
  * the tree is the breadth-first tree of each connected part, rooted at the
    part's lowest node id, neighbours taken in ascending branch id;
  * port p's link runs from its sink node to its source node (the source
    lifts the source face to +1 V), so loop current = current through the
    conductor from source to sink; port links are numbered after all branches
    and their loops come last;
  * an edge shared by more than two triangles is rejected (non-manifold).
Parity: exact integers; pinned by loop count = b - n + s + p, M A^T = 0,
rank A = l and the Euler characteristic (tests/test_oracle_graph.py).
"""
from __future__ import annotations

from collections import deque
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


class NonManifold(ValueError):
    pass


class BadPort(ValueError):
    pass


@dataclass
class Loops:
    nt: int
    node_of_tri: np.ndarray     # int64 [nt] -> node id
    n_nodes: int
    br_tri: np.ndarray          # int64 [nb, 2]  (T+, T-)
    br_local: np.ndarray        # int64 [nb, 2]  local edge index (opposite vertex) in T+, T-
    br_edge: np.ndarray         # int64 [nb]     edge id
    tail: np.ndarray            # int64 [nb + p] node of branch tail
    head: np.ndarray            # int64 [nb + p]
    n_comp: int
    comp_of_node: np.ndarray
    parent: np.ndarray          # int64 [n_nodes], -1 at roots
    parent_branch: np.ndarray   # int64 [n_nodes], -1 at roots
    is_twig: np.ndarray         # bool [nb + p]
    link_branch: np.ndarray     # int64 [nl]  branch id of each loop's link
    A: sp.csr_matrix            # [nl, nb + p], entries +-1
    n_ports: int

    @property
    def nb(self):
        return int(self.br_tri.shape[0])

    @property
    def nl(self):
        return int(self.link_branch.shape[0])

    def port_loop(self, p):
        return self.nl - self.n_ports + p

    def incidence(self):
        """M [n_nodes, nb + p]: +1 at a branch's tail, -1 at its head."""
        nbp = self.tail.shape[0]
        rows = np.concatenate([self.tail, self.head])
        cols = np.concatenate([np.arange(nbp), np.arange(nbp)])
        vals = np.concatenate([np.ones(nbp), -np.ones(nbp)])
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n_nodes, nbp))


def mesh_edges(tri):
    """Unique undirected edges.

    Returns (edges [ne,2] sorted (vmin, vmax) in lexicographic order,
    tri_edge [nt,3] edge id of the edge opposite each local vertex)."""
    tri = np.asarray(tri, dtype=np.int64)
    nt = tri.shape[0]
    e = np.stack([np.stack([tri[:, (k + 1) % 3], tri[:, (k + 2) % 3]], axis=1) for k in range(3)],
                 axis=1)                       # [nt, 3, 2], edge opposite vertex k
    e = np.sort(e, axis=2).reshape(-1, 2)
    edges, inv = np.unique(e, axis=0, return_inverse=True)
    return edges, inv.reshape(nt, 3)


def build_loops(mesh, ports=None, root="lowest"):
    """Graph, BFS tree, fundamental loops and A for `mesh` with its ports.

    root="lowest" (the default reading) roots each part at its lowest node id;
    root="highest" picks the highest id, used to check that port impedance
    does not depend on the tree."""
    if ports is None:
        ports = mesh.ports
    nt = mesh.nt
    edges, tri_edge = mesh_edges(mesh.tri)
    ne = edges.shape[0]

    # contact contraction by union-find over triangles
    parent_uf = np.arange(nt)

    def find(a):
        while parent_uf[a] != a:
            parent_uf[a] = parent_uf[parent_uf[a]]
            a = parent_uf[a]
        return a

    for src, snk in ports:
        for group in (src, snk):
            group = np.asarray(group, dtype=np.int64)
            if group.size == 0:
                raise BadPort("empty contact set")
            r0 = find(int(group.min()))
            for t in group:
                r = find(int(t))
                if r != r0:
                    lo, hi = min(r, r0), max(r, r0)
                    parent_uf[hi] = lo
                    r0 = lo
    rep = np.array([find(t) for t in range(nt)])
    reps = np.unique(rep)
    node_of_tri = np.searchsorted(reps, rep)
    n_nodes = reps.shape[0]

    # branches: edges with exactly two triangles on different nodes
    owners = [[] for _ in range(ne)]
    for t in range(nt):
        for k in range(3):
            owners[tri_edge[t, k]].append((t, k))
    br_tri, br_local, br_edge = [], [], []
    for e in range(ne):
        o = owners[e]
        if len(o) > 2:
            raise NonManifold(f"edge {e} shared by {len(o)} triangles")
        if len(o) < 2:
            continue
        (ta, ka), (tb, kb) = sorted(o)
        if node_of_tri[ta] == node_of_tri[tb]:
            continue
        br_tri.append((ta, tb))
        br_local.append((ka, kb))
        br_edge.append(e)
    br_tri = np.array(br_tri, dtype=np.int64).reshape(-1, 2)
    br_local = np.array(br_local, dtype=np.int64).reshape(-1, 2)
    br_edge = np.array(br_edge, dtype=np.int64)
    nb = br_tri.shape[0]
    P = len(ports)
    tail = np.concatenate([node_of_tri[br_tri[:, 0]],
                           [node_of_tri[int(np.min(snk))] for _, snk in ports]]).astype(np.int64)
    head = np.concatenate([node_of_tri[br_tri[:, 1]],
                           [node_of_tri[int(np.min(src))] for src, _ in ports]]).astype(np.int64)

    # adjacency over real branches, ascending branch id
    adj = [[] for _ in range(n_nodes)]
    for b in range(nb):
        adj[tail[b]].append((b, head[b]))
        adj[head[b]].append((b, tail[b]))

    parent = np.full(n_nodes, -1, dtype=np.int64)
    parent_branch = np.full(n_nodes, -1, dtype=np.int64)
    depth = np.zeros(n_nodes, dtype=np.int64)
    comp = np.full(n_nodes, -1, dtype=np.int64)
    n_comp = 0
    order = range(n_nodes) if root == "lowest" else range(n_nodes - 1, -1, -1)
    for root in order:
        if comp[root] >= 0:
            continue
        comp[root] = n_comp
        q = deque([root])
        while q:
            u = q.popleft()
            for b, w in adj[u]:
                if comp[w] < 0:
                    comp[w] = n_comp
                    parent[w] = u
                    parent_branch[w] = b
                    depth[w] = depth[u] + 1
                    q.append(w)
        n_comp += 1

    for p, (src, snk) in enumerate(ports):
        a, b = tail[nb + p], head[nb + p]
        if a == b:
            raise BadPort(f"port {p}: source and sink are the same node")
        if comp[a] != comp[b]:
            raise BadPort(f"port {p}: source and sink on separate conductors")

    is_twig = np.zeros(nb + P, dtype=bool)
    is_twig[parent_branch[parent_branch >= 0]] = True
    link_branch = np.concatenate([np.nonzero(~is_twig[:nb])[0], nb + np.arange(P)])

    rows, cols, vals = [], [], []
    for l, e in enumerate(link_branch):
        u, w = tail[e], head[e]
        rows.append(l)
        cols.append(e)
        vals.append(1.0)
        # tree path w -> u: climb from both ends to their common ancestor
        x, y = w, u
        up_w, up_u = [], []
        while depth[x] > depth[y]:
            up_w.append(x)
            x = parent[x]
        while depth[y] > depth[x]:
            up_u.append(y)
            y = parent[y]
        while x != y:
            up_w.append(x)
            up_u.append(y)
            x, y = parent[x], parent[y]
        for z in up_w:                    # traversed child -> parent
            t = parent_branch[z]
            rows.append(l)
            cols.append(t)
            vals.append(1.0 if tail[t] == z else -1.0)
        for z in up_u:                    # traversed parent -> child
            t = parent_branch[z]
            rows.append(l)
            cols.append(t)
            vals.append(1.0 if head[t] == z else -1.0)
    nl = link_branch.shape[0]
    A = sp.csr_matrix((vals, (rows, cols)), shape=(nl, nb + P))
    return Loops(nt=nt, node_of_tri=node_of_tri, n_nodes=n_nodes, br_tri=br_tri,
                 br_local=br_local, br_edge=br_edge, tail=tail, head=head, n_comp=n_comp,
                 comp_of_node=comp, parent=parent, parent_branch=parent_branch,
                 is_twig=is_twig, link_branch=link_branch, A=A, n_ports=P)

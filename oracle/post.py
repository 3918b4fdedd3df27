"""Post-processing of a loop-space solution (oracle, test infrastructure only).

Plain FP64 CPU code used by the tests; the GPU library never imports it.

From loop currents I_l (Eq. LoopVandI) the paper derives, for its current and
potential plots (Sec. V): branch currents alpha = A^T I_l (Eq. CurT, port links
excluded), branch voltage drops V_b = Z_b alpha from tail to head (Eq. VolT,
the branch-space product), and node (panel) potentials.  Reading: a node's
potential is the sum of the branch voltage drops along the spanning tree from
the node to its conductor's reference node, the sink contact of the first port
on that conductor (the tree root if it has none), so that V_b = phi(tail) -
phi(head) on every tree branch, and on every branch when I_l solves the loop
system.  Panel potentials repeat their node's value (contact triangles share
their contact's node).
"""
from __future__ import annotations

from collections import deque

import numpy as np


def branch_currents(loops, x):
    """alpha = A^T x over the mesh branches (Eq. CurT)."""
    nb = loops.nb
    return (loops.A[:, :nb].T @ np.asarray(x)).astype(complex)


def reference_nodes(loops, port_sink_nodes):
    """Reference node of each component: the first port's sink node on it, else
    its tree root."""
    ref = np.full(loops.n_comp, -1, dtype=np.int64)
    for v in port_sink_nodes:
        c = loops.comp_of_node[v]
        if ref[c] < 0:
            ref[c] = v
    roots = np.nonzero(loops.parent < 0)[0]
    for r in roots:
        c = loops.comp_of_node[r]
        if ref[c] < 0:
            ref[c] = r
    return ref


def node_potentials(loops, v_branch, port_sink_nodes):
    """phi[n_nodes]: walk each tree from its reference node, phi(head) = phi(tail) - V_b."""
    n = loops.n_nodes
    phi = np.full(n, np.nan + 0j)
    # tree adjacency
    adj = [[] for _ in range(n)]
    for v in range(n):
        b = loops.parent_branch[v]
        if b >= 0:
            u = loops.parent[v]
            adj[u].append((v, b))
            adj[v].append((u, b))
    for ref in reference_nodes(loops, port_sink_nodes):
        phi[ref] = 0.0
        q = deque([ref])
        while q:
            u = q.popleft()
            for w, b in adj[u]:
                if np.isnan(phi[w].real):
                    # V_b = phi(tail) - phi(head)
                    phi[w] = phi[u] - v_branch[b] if loops.tail[b] == u else phi[u] + v_branch[b]
                    q.append(w)
    return phi


def panel_potentials(loops, v_branch, port_sink_nodes):
    return node_potentials(loops, v_branch, port_sink_nodes)[loops.node_of_tri]

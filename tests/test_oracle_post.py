"""Pins of the post-processing oracle (oracle/post.py) on solved excitations.

Kirchhoff's laws fix the results: for a solution of the loop system with a unit
source in one port, the branch currents balance at every node except the two
contacts (which carry the port current, equal to the port loop current); the
voltage drops derive from the potentials on every mesh branch (not only the
tree ones); the driven port's source contact sits at the source voltage above its
sink (reference 0); an undriven port is a short between its contacts.
"""
import numpy as np
import pytest

import synth
from oracle.mom import DenseMoM
from oracle.post import branch_currents, node_potentials


@pytest.fixture(scope="module")
def solved():
    m = synth.tiny_wires()
    D = DenseMoM(m)
    O = D.loops
    w = 2 * np.pi * 1e9
    V = np.zeros(O.nl, complex)
    V[O.port_loop(0)] = 1.0            # 1 V in port 0's loop
    x = np.linalg.solve(D.Zl(w), V)
    a = branch_currents(O, x)
    vb = D.Zb(w) @ a
    sinks = [O.tail[O.nb + p] for p in range(O.n_ports)]
    srcs = [O.head[O.nb + p] for p in range(O.n_ports)]
    phi = node_potentials(O, vb, sinks)
    return m, O, x, a, vb, phi, sinks, srcs


def test_kcl_at_nodes(solved):
    m, O, x, a, vb, phi, sinks, srcs = solved
    M = O.incidence()[:, :O.nb]
    net = M @ a                                      # out of tails, into heads
    scale = np.abs(a).max()
    contacts = set(sinks) | set(srcs)
    for v in range(O.n_nodes):
        if v not in contacts:
            assert abs(net[v]) < 1e-9 * scale
    I_port = x[O.port_loop(0)]
    assert abs(abs(net[srcs[0]]) - abs(I_port)) < 1e-9 * scale


def test_voltage_drops_derive_from_potentials_on_every_branch(solved):
    m, O, x, a, vb, phi, sinks, srcs = solved
    d = phi[O.tail[:O.nb]] - phi[O.head[:O.nb]]
    assert np.abs(d - vb).max() < 1e-9 * np.abs(vb).max()


def test_contact_potentials(solved):
    m, O, x, a, vb, phi, sinks, srcs = solved
    assert phi[sinks[0]] == 0 and phi[sinks[1]] == 0
    # the driven port: source contact at the source voltage relative to its sink
    assert abs(abs(phi[srcs[0]] - phi[sinks[0]]) - 1.0) < 1e-9
    # the undriven port is a short (no source, no impedance in its link): no drop across it
    assert abs(phi[srcs[1]] - phi[sinks[1]]) < 1e-9

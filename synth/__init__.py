"""Seeded synthetic inputs (meshes, ports, frequencies, vectors) shared by the
oracle, the tests and the bench.  No arithmetic of the method lives here."""
from .meshes import Mesh, box_mesh, wire_array_mesh, merge, plane_pair_mesh, meander_mesh  # noqa: F401
from .workloads import (bar_1500, bondwires_40k, pdn_500k, tiny_bar, tiny_pdn, tiny_wires, tiny_two_bars,  # noqa: F401
                        complex_gaussian, meander, meanders_32, grid_for, learned_geometry,
                        WORKLOADS)

"""The synthetic geometries are valid conductor surfaces: every edge shared by
exactly two triangles, consistently oriented (each directed edge once), Euler
characteristic 2 - 2 genus with the expected genus (0 for a trace, one handle
per via for the plane pair), outward normals (positive enclosed volume), and
port contacts on the intended faces.  No GPU needed."""
import numpy as np
import pytest

import synth
from synth.meshes import meander_mesh, plane_pair_mesh


def topology(m):
    e = np.concatenate([m.tri[:, [0, 1]], m.tri[:, [1, 2]], m.tri[:, [2, 0]]])
    und, cnt = np.unique(np.sort(e, axis=1), axis=0, return_counts=True)
    directed = np.unique(e, axis=0).shape[0] == e.shape[0]
    chi = m.nv - und.shape[0] + m.nt
    p = m.xyz[m.tri]
    vol = np.einsum("ij,ij->i", p[:, 0], np.cross(p[:, 1], p[:, 2])).sum() / 6.0
    return set(cnt.tolist()), directed, chi, vol


@pytest.mark.parametrize("n_seg", [3, 4, 8, 12])
def test_meander_is_a_closed_oriented_sphere(n_seg):
    m = meander_mesh(n_seg, 20e-6, 10e-6, 300e-6, kw=2, seed=n_seg)
    counts, directed, chi, vol = topology(m)
    assert counts == {2} and directed and chi == 2 and vol > 0
    (src, snk), = m.ports
    assert len(src) == len(snk) > 0 and not set(src) & set(snk)
    c = m.xyz[m.tri].mean(axis=1)
    # the source end face lies on x = 0, the sink end face on x = 0 or x = max
    assert np.allclose(c[src, 0], 0.0)
    assert np.allclose(c[snk, 0], 0.0) or np.allclose(c[snk, 0], m.xyz[:, 0].max())


def test_plane_pair_has_one_handle_per_via():
    m = plane_pair_mesh(L=0.6e-3, n=24, m_gap=3, n_pairs=2, via_k=1, n_ports=2, pad_k=2, site=6, seed=3)
    counts, directed, chi, vol = topology(m)
    assert counts == {2} and directed and vol > 0
    assert (2 - chi) // 2 == 2 * 2 - 1          # two planes joined by 4 vias: genus 3
    top = m.xyz[:, 2].max()
    c = m.xyz[m.tri].mean(axis=1)
    for src, snk in m.ports:
        assert np.allclose(c[src, 2], top) and np.allclose(c[snk, 2], 0.0)
        assert np.allclose(np.sort(c[src, :2], axis=0), np.sort(c[snk, :2], axis=0), atol=0.2 * 25e-6)


def test_meander_workload_sizes():
    ws = synth.meanders_32(n=6)
    for w in ws:
        assert 4e3 <= w["mesh"].nt <= 7e4
        assert all(4 <= g <= 256 and g & (g - 1) == 0 for g in w["grid"])
        assert len(w["freqs"]) == 32


@pytest.mark.parametrize("name,nt,nl,nports,grid,nf,f0,f1,genus", [
    ("bar_1000x20x10um_1.5k", 1508, None, 1, (64, 16, 16), 1, 1e9, 1e9, 0),
    ("bondwires_8x2mm_40k", 40192, 20096, 8, (128, 64, 32), 16, 1e6, 1e10, 0),
    ("pdn_2x10mm_500k", 516800, 258373, 4, (256, 256, 32), 8, 1e6, 1e9, 399),
])
def test_named_workloads_follow_their_recipe(name, nt, nl, nports, grid, nf, f0, f1, genus):
    # the sizes the input recipe states and the bench lines are quoted on: triangles,
    # loops (from the host loop basis), ports, grid, log-spaced frequencies, and the
    # surface topology (every wire and the bar closed genus 0; the plane pair one
    # closed surface with a handle per via but one)
    from paper_2210_04891_gb300 import api
    w = synth.WORKLOADS[name]()
    m = w["mesh"]
    assert m.nt == nt and len(m.ports) == nports and tuple(w["grid"]) == grid
    f = np.asarray(w["freqs"])
    assert f.size == nf and np.isclose(f[0], f0) and np.isclose(f[-1], f1)
    if nf > 2:
        assert np.allclose(np.diff(np.log(f)), np.log(f1 / f0) / (nf - 1))
    counts, directed, chi, vol = topology(m)
    assert counts == {2} and directed and vol > 0
    ncomp = 8 if name.startswith("bondwires") else 1
    assert (2 * ncomp - chi) // 2 == genus
    if nl is not None:
        L = api.Loops(api.Mesh.from_synth(m), m.ports)
        assert L.nl == nl

"""sie_mesh_load_file: the library's own text mesh format round-trips a mesh
exactly (the loop basis built from the file equals the one built from the
arrays, and plan-free host results agree bit for bit), comments and free
whitespace are accepted, and every malformed file is rejected with
SIE_ERR_ARG.  No GPU needed."""
import numpy as np
import pytest

import synth
from paper_2210_04891_gb300 import api
from paper_2210_04891_gb300.native import SieError


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2210_04891_gb300.build import build
    build()


def same_loops(a, b):
    ea, eb = a.export(), b.export()
    assert a.stats == b.stats
    for x, y in zip(ea, eb):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("make", [synth.tiny_wires, synth.tiny_two_bars])
def test_round_trip(tmp_path, make):
    m = make()
    path = tmp_path / "m.sie"
    api.write_mesh_file(path, m.xyz, m.tri, m.cond, m.sigma)
    F = api.Mesh.from_file(path)
    assert F.nt == m.nt and F.ncond == m.sigma.shape[0]
    same_loops(api.Loops(F, m.ports), api.Loops(api.Mesh.from_synth(m), m.ports))
    # 17 significant digits give the same doubles back
    toks = " ".join(line.split("#", 1)[0] for line in open(path)).split()
    k = 5 + m.sigma.shape[0]
    xyz = np.array(toks[k:k + 3 * m.xyz.shape[0]], float)
    assert np.array_equal(xyz.reshape(-1, 3), m.xyz)


def test_comments_and_whitespace(tmp_path):
    path = tmp_path / "tet.sie"
    # a tetrahedron: 4 vertices, 4 outward triangles, one conductor
    path.write_text("# a comment line\n  sie_mesh   1  # trailing comment\n4 4\t1\n5.8e7\n"
                    "0 0 0  1e-6 0 0\n0 1e-6 0 0 0 1e-6\n"
                    "0 2 1 0\n0 1 3 0   # face\n0 3 2 0\n1 2 3 0\n")
    F = api.Mesh.from_file(path)
    L = api.Loops(F, [])
    assert L.stats["n_nodes"] == 4 and L.nb == 6 and L.nl == 3


BAD = {
    "magic": "sie_mesh_x 1\n3 1 1\n1\n0 0 0 1 0 0 0 1 0\n0 1 2 0\n",
    "version": "sie_mesh 2\n3 1 1\n1\n0 0 0 1 0 0 0 1 0\n0 1 2 0\n",
    "short": "sie_mesh 1\n3 1 1\n1\n0 0 0 1 0 0 0 1\n",
    "trailing": "sie_mesh 1\n3 1 1\n1\n0 0 0 1 0 0 0 1 0\n0 1 2 0 7\n",
    "number": "sie_mesh 1\n3 1 1\n1\n0 0 0 1 0 0 0 1x 0\n0 1 2 0\n",
    "index": "sie_mesh 1\n3 1 1\n1\n0 0 0 1 0 0 0 1 0\n0 1 3 0\n",
    "cond": "sie_mesh 1\n3 1 1\n1\n0 0 0 1 0 0 0 1 0\n0 1 2 1\n",
    "sigma": "sie_mesh 1\n3 1 1\n-1\n0 0 0 1 0 0 0 1 0\n0 1 2 0\n",
    "degenerate": "sie_mesh 1\n3 1 1\n1\n0 0 0 1 0 0 2 0 0\n0 1 2 0\n",
    "sizes": "sie_mesh 1\n-3 1 1\n1\n",
    "empty": "",
}


@pytest.mark.parametrize("case", sorted(BAD))
def test_malformed_files_are_rejected(tmp_path, case):
    path = tmp_path / (case + ".sie")
    path.write_text(BAD[case])
    with pytest.raises(SieError) as e:
        api.Mesh.from_file(path, nt=1, ncond=1)
    assert e.value.code == -1          # SIE_ERR_ARG


def test_missing_file(tmp_path):
    with pytest.raises(SieError):
        api.Mesh.from_file(tmp_path / "nope.sie", nt=1, ncond=1)

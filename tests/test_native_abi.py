"""The C-ABI library loads and exports every symbol include/sie.h declares; the
host-side loop basis (Sec. II-D, III) is identical to the oracle's; argument
errors come back as the documented codes.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from oracle.graph import build_loops
from paper_2210_04891_gb300 import api, native
from paper_2210_04891_gb300.native import SieError

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2210_04891_gb300.build import build
    build()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "sie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", src)) - {"if", "sizeof"})


def test_exports_every_declared_symbol():
    lib = native.lib()
    decl = declared_symbols()
    assert set(decl) == set(native.EXPORTS), decl
    for name in decl:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("make", [synth.tiny_bar, synth.tiny_wires, synth.tiny_two_bars,
                                  lambda: synth.bar_1500()["mesh"]])
def test_loop_basis_matches_oracle(make):
    m = make()
    L = api.Loops(api.Mesh.from_synth(m), m.ports)
    O = build_loops(m)
    rp, col, val, br = L.export()
    assert L.nl == O.nl and L.nb == O.nb
    assert L.stats["n_comp"] == O.n_comp and L.stats["n_nodes"] == O.n_nodes
    assert np.array_equal(br, O.br_tri)
    A = O.A.tocsr()
    for l in range(O.nl):
        a = sorted(zip(A.indices[A.indptr[l]:A.indptr[l + 1]].tolist(),
                       A.data[A.indptr[l]:A.indptr[l + 1]].astype(int).tolist()))
        b = sorted(zip(col[rp[l]:rp[l + 1]].tolist(), val[rp[l]:rp[l + 1]].astype(int).tolist()))
        assert a == b, l
    assert L.stats["n_loops"] == L.stats["n_branches"] - L.stats["n_nodes"] + L.stats["n_comp"] + L.stats["n_ports"]


def test_error_codes():
    m = synth.tiny_two_bars()
    M = api.Mesh.from_synth(m)
    with pytest.raises(SieError) as e:
        api.Loops(M, [(m.ports[0][0], m.ports[1][1])])
    assert e.value.code == -3
    with pytest.raises(SieError) as e:
        api.Loops(M, [(m.ports[0][0], m.ports[0][0])])
    assert e.value.code == -3
    bad = m.tri.copy()
    bad[0, 0] = m.nv + 5
    with pytest.raises(SieError) as e:
        api.Mesh(m.xyz, bad, m.cond, m.sigma)
    assert e.value.code == -1
    with pytest.raises(SieError) as e:
        api.Mesh(m.xyz, m.tri, m.cond, -m.sigma)
    assert e.value.code == -1
    # non-manifold: a third triangle on an existing edge
    xyz = np.vstack([m.xyz, [[0.0, -5e-5, 5e-6]]])
    t0 = m.tri[0]
    tri = np.vstack([m.tri, [[t0[0], t0[1], m.nv]]]).astype(np.int32)
    cond = np.concatenate([m.cond, [0]]).astype(np.int32)
    with pytest.raises(SieError) as e:
        api.Loops(api.Mesh(xyz, tri, cond, m.sigma), [])
    assert e.value.code == -2

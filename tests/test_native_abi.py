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


@pytest.mark.parametrize("name", ["bondwires_8x2mm_40k", "pdn_2x10mm_500k"])
def test_loop_basis_matches_oracle_at_full_size(name):
    # the bond-wire array (40,192 triangles, 20,096 loops) and the plane pair with its vias
    # (516,800 triangles, 258,373 loops): integer work, so bit for bit: branch list, component
    # and node counts, and every signed entry of A (compared as sorted CSR matrices)
    import scipy.sparse as sp
    m = synth.WORKLOADS[name]()["mesh"]
    L = api.Loops(api.Mesh.from_synth(m), m.ports)
    O = build_loops(m)
    assert (L.nl, L.nb) == (O.nl, O.nb)
    assert L.stats["n_comp"] == O.n_comp and L.stats["n_nodes"] == O.n_nodes
    rp, col, val, br = L.export()
    assert np.array_equal(br, O.br_tri)
    G = sp.csr_matrix((np.asarray(val, dtype=np.int64), np.asarray(col), np.asarray(rp)), shape=O.A.shape)
    A = sp.csr_matrix(O.A, dtype=np.int64)
    G.sort_indices()
    A.sort_indices()
    assert np.array_equal(G.indptr, A.indptr)
    assert np.array_equal(G.indices, A.indices)
    assert np.array_equal(G.data, A.data)
    assert set(np.unique(G.data).tolist()) <= {-1, 1}


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


# entry points whose first argument is a handle (plan, batch or network):
# a NULL handle comes back as SIE_ERR_ARG naming the call, before any CUDA call
HANDLE_CALLS = ["pfft_matvec", "pfft_precond_apply", "pfft_precond_info", "sie_solve", "pfft_convolve",
                "pfft_convolve_lossy", "pfft_convolve_noalloc", "sie_postprocess", "pfft_plan_info",
                "pfft_plan_export", "pfft_profile_enable", "pfft_profile_read", "pfft_plan_set_surface_model",
                "sie_batch_matvec", "sie_batch_solve", "sie_batch_stats", "sie_mlp_get_params",
                "sie_mlp_set_params", "sie_mlp_forward", "sie_mlp_grad", "sie_mlp_train",
                "pfft_branch_features", "pfft_branch_probe_target", "pfft_plan_set_learned",
                "sie_selftest_bounded_wait", "sie_loops_export", "pfft_plan_create", "pfft_autotune"]


def neutral_args(fn):
    """NULL for pointers, 1 for integers, 1.0 for reals: only the handle is wrong."""
    out = []
    for t in fn.argtypes:
        if t in (ctypes.c_double, ctypes.c_float):
            out.append(t(1.0))
        elif t in (ctypes.c_int8, ctypes.c_int16, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int):
            out.append(t(1))
        else:
            out.append(None)
    return out


@pytest.mark.parametrize("name", HANDLE_CALLS)
def test_null_handle_is_an_argument_error(name):
    lib = native.lib()
    fn = getattr(lib, name)
    assert fn.argtypes is not None, name
    assert fn(*neutral_args(fn)) == -1
    assert lib.sie_last_error().decode().startswith(name)


def test_destroy_and_counts_accept_null():
    lib = native.lib()
    for name in ("pfft_plan_destroy", "sie_batch_destroy", "sie_mlp_destroy", "sie_mesh_destroy",
                 "sie_loops_destroy"):
        getattr(lib, name)(None)
    assert lib.pfft_plan_launches(None) == 0
    assert lib.sie_mlp_param_count(None) == 0
    out = ctypes.c_void_p(1)
    assert lib.sie_batch_create(None, 0, ctypes.byref(out)) == -1 and not out.value
    assert lib.sie_mlp_create(24, 0, ctypes.byref(out)) == -1 and not out.value

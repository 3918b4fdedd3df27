"""Failure detection without a GPU fault.

The tensor-core near field waits on mbarriers with a time limit; a wait that
runs out sets the plan's device error flag and returns, and the call reports
SIE_ERR_TIMEOUT.  The self-test drives that path to its end: a wait on a
barrier nothing completes.  Checked: the code and message, that the flag is
cleared, and that the plan and the CUDA context stay usable (the next product
equals the one taken before, bit for bit).
"""
import time

import numpy as np
import pytest

import synth
from oracle.graph import build_loops

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2210_04891_gb300 import api, native as N, PREC_FP64  # noqa: E402

PRM = dict(grid=(16, 8, 4), order=3, near_factor=4.0, near_min_diam=2.0, n_touch=8, h0=0.0)


def test_bounded_wait_times_out_and_context_survives():
    m = synth.tiny_wires()
    O = build_loops(m)
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, PRM)
    om = 2 * np.pi * np.array([1e9, 3e9])
    x = torch.from_numpy(synth.complex_gaussian(O.nl, 2, seed=41)).cuda()
    y0 = api.pfft_matvec(P, x, om, prec=PREC_FP64)
    torch.cuda.synchronize()

    t0 = time.perf_counter()
    rc = api.selftest_bounded_wait(P, limit_ms=5.0)
    dt = time.perf_counter() - t0
    assert rc == -8, N.lib().sie_last_error().decode()
    assert "bounded device-side wait" in N.lib().sie_last_error().decode()
    assert dt < 5.0       # the wait ended on its own limit

    # the flag was cleared: a normal call succeeds and gives the same product
    y1 = api.pfft_matvec(P, x, om, prec=PREC_FP64)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)
    # a second run of the self-test reports the timeout again (the flag was reset, not stuck)
    assert api.selftest_bounded_wait(P, limit_ms=1.0) == -8
    y2 = api.pfft_matvec(P, x, om, prec=PREC_FP64)
    assert torch.equal(y0, y2)


def test_selftest_rejects_bad_limits():
    m = synth.tiny_wires()
    M = api.Mesh.from_synth(m)
    L = api.Loops(M, m.ports)
    P = api.Plan(M, L, PRM)
    for bad in (0.0, -1.0, 5000.0):
        assert api.selftest_bounded_wait(P, limit_ms=bad) == -1

"""Host logic of bench.py's roofline figures, checked against counts worked out by hand.

The bench reports each stage's achieved rate as an algorithmic amount per launch
divided by the launch's CUDA-event time; these tests pin the amounts (and the
derived FP32 peak) for the bond-wire workload, so that a dropped term or a wrong
factor in the bookkeeping shows here rather than as a plausible fraction.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

# bond-wire array: 128 right-hand sides, grid 128 x 64 x 32 padded to 256 x 128 x 64
BOND = dict(R=128, cb=8, rec=48, Ng=128 * 64 * 32, Nx=128, My=128, Mz=64, nt=40192, nl=20096,
            n_near=11808648, n_pair=2302016, n_active=151040)


def test_fp32_peak_of_a_gb300():
    # 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz
    assert bench.alu_peak_tflops(2070.0, 152) == pytest.approx(80.54784, rel=1e-12)


def test_plane_flops_of_the_bond_wire_plane():
    # one x-frequency plane, data 64 x 32 in a padded 128 x 64 plane, 5 n log2 n per FFT line:
    #   forward z on the 64 data rows (length 64):       64 * 5 * 64 * 6  = 122,880
    #   forward y on the 64 columns (length 128):        64 * 5 * 128 * 7 = 286,720
    #   real kernel product, 2 flop per point:            128 * 64 * 2     =  16,384
    #   inverse y on the 64 columns:                                         286,720
    #   inverse z on the 64 kept rows:                                       122,880
    assert bench.plane_flops(64, 32, 128, 64) == 835584


def test_plane_stage_per_launch():
    bound, flop, unit = bench.stage_work("fft_yz", BOND)
    # 3 components x 128 right-hand sides x 256 x-frequency planes x 835,584
    assert (bound, unit) == ("alu", "flop")
    assert flop == 3 * 128 * 256 * 835584 == 82141249536
    # HBM basis: each grid's x-transformed copy (2 N_g values) read and written, 8 B complex
    assert bench.stage_bytes("fft_yz", BOND) == 3 * 128 * (2 * 262144) * 2 * 8 == 3221225472


def test_pencil_stages_move_three_grid_units():
    # forward: N_g values read, 2 N_g written; inverse the reverse; 8 B complex, 384 grids
    assert bench.stage_work("fft_x_fwd", BOND) == ("hbm", 384 * 3 * 262144 * 8, "B")
    assert bench.stage_work("fft_x_inv", BOND) == ("hbm", 384 * 3 * 262144 * 8, "B")


def test_near_field_route_by_rhs_count():
    # even R from 96 in the mixed form: tensor cores over the near pairs only
    assert bench.stage_work("near", BOND) == ("tensor", 36 * 128 * 11808648, "flop")
    # below 96, or odd: the CUDA-core gather, which also applies the far-field blocks
    for R in (32, 95, 127):
        c = dict(BOND, R=R)
        assert bench.stage_work("near", c) == ("alu", 36 * R * (11808648 + 2302016), "flop")


def test_loop_maps_and_preconditioner_bytes():
    # loop currents in (16 B) and three local currents per triangle out (8 B) ...
    assert bench.stage_work("loop_to_branch", BOND) == ("hbm", 128 * 20096 * 16 + 128 * 40192 * 3 * 8, "B")
    # ... triangle outputs in (16 B double-float) and loop voltages out (16 B)
    assert bench.stage_work("branch_to_loop", BOND) == ("hbm", 128 * 40192 * 3 * 16 + 128 * 20096 * 16, "B")
    assert bench.stage_work("precond_apply", BOND) == ("hbm", 2 * 128 * 20096 * 16, "B")
    assert bench.stage_work("no_such_stage", BOND) is None
    assert bench.stage_bytes("project", BOND) is None


def test_measured_traffic_scales_to_a_bench_launch():
    # the plane kernel's ncu traffic was taken on 48 grids; a bench launch has 384
    tb, grids = bench.MEASURED_TRAFFIC["fft_yz"]
    assert grids == 48
    assert tb * 384 / grids == pytest.approx(2.79048e9, rel=1e-6)

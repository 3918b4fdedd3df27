"""ctypes loader of the oracle's plain C loops (oracle/c/oracle_kernels.c).

Test infrastructure only.  `build()` compiles the C file with gcc (-O2,
OpenMP, no floating-point contraction, so results do not depend on the host
architecture's fused multiply-add); the library sits beside the source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c", "oracle_kernels.c")
LIB = os.path.join(HERE, "c", "liboracle_kernels.so")
_lib = None


def build(force=False):
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               SRC, "-o", LIB + ".tmp", "-lm"])
        os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int64
        _lib.orc_pair_blocks.argtypes = [I, P, P, P, P, I, P, P, P]
        _lib.orc_grid_blocks.argtypes = [I, P, P, I, I, I, P, P, P, P, I, I, I, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def pair_blocks(pT, aT, pS, aS, rule):
    pT = np.ascontiguousarray(pT, dtype=np.float64)
    pS = np.ascontiguousarray(pS, dtype=np.float64)
    aT = np.ascontiguousarray(aT, dtype=np.float64)
    aS = np.ascontiguousarray(aS, dtype=np.float64)
    bary = np.ascontiguousarray(rule[0], dtype=np.float64)
    w = np.ascontiguousarray(rule[1], dtype=np.float64)
    m = pT.shape[0]
    out = np.empty((m, 3, 3))
    lib().orc_pair_blocks(m, _p(pT), _p(aT), _p(pS), _p(aS), w.shape[0], _p(bary), _p(w), _p(out))
    return out


def grid_blocks(ti, tj, start, lw, mom, Hpad):
    ti = np.ascontiguousarray(ti, dtype=np.int64)
    tj = np.ascontiguousarray(tj, dtype=np.int64)
    start = np.ascontiguousarray(start, dtype=np.int64)
    lw = np.ascontiguousarray(np.stack(lw), dtype=np.float64)
    mom = np.ascontiguousarray(mom, dtype=np.float64)
    Hpad = np.ascontiguousarray(Hpad, dtype=np.float64)
    nt, Q = start.shape[:2]
    O = lw.shape[-1]
    out = np.empty((ti.shape[0], 3, 3))
    lib().orc_grid_blocks(ti.shape[0], _p(ti), _p(tj), nt, Q, O, _p(start), _p(lw), _p(mom),
                          _p(Hpad), Hpad.shape[0], Hpad.shape[1], Hpad.shape[2], _p(out))
    return out

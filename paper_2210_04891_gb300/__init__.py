"""GB300 (sm_103a) pFFT matvec and preconditioned loop-basis GMRES of the MQS
surface integral equation of arXiv 2210.04891.

The compute path is libsie.so (include/sie.h): host C++ for the mesh graph and
loop basis, hand-written CUDA for the plan setup and every step of the matvec,
preconditioner and solve.  `paper_2210_04891_gb300.api` is the thin Python
binding.
"""
from .native import (SieError, SPACE_LOOP, SPACE_BRANCH, PREC_FP64, PREC_MIXED, PREC_DF,  # noqa: F401
                     REFINE_OFF, REFINE_FP64, REFINE_DF)

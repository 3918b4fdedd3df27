"""Plain, slow FP64 CPU oracle of the MQS surface-integral-equation method.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's CPU
baseline leg may import anything from this package; the product path never
does, and nothing here imports the product package.  The only code shared with
the GPU path is the seeded input generator package `synth`, which holds none of
the method's arithmetic.

Modules
  quadrature  triangle quadrature rules (Radon 7-point, collapsed Gauss product)
  graph       circuit graph of a mesh, spanning tree, fundamental loops, A (Sec. II-D, III)
  integrals   Gram and 1/R panel integrals of the modified RWG functions (Eq. Zb)
  mom         dense method of moments and port impedance extraction (O1)
  pfft        plain pre-corrected FFT product in the paper's four steps (Sec. IV-B, O2)
  gmres       plain restarted left-preconditioned GMRES with P = A Z_b^N A^T (Sec. IV-A)

Parity status of each function is stated in its docstring; every function here
is pinned by a `-m "not gpu"` test against closed forms, invariants or brute
force (tests/test_oracle_*.py).
"""

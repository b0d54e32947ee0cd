"""Plain FP64 CPU oracle for the spectral-element screened-Poisson solver.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the C-ABI library and
its Python binding) imports, links or runs this package. Only the tests, the
smoke check and the benchmark's CPU-baseline leg use it, to check the GPU
results against a slow, obviously correct restatement of the method of
Remacle, Gandham & Warburton, "GPU accelerated spectral finite elements on
all-hex meshes":

  gll.py       GLL nodes/weights, Lagrange basis, derivative matrix (Sec. 2.1, 2.4)
  numbering.py global numbering of GLL nodes, scatter/gather (Sec. 2.2, Eq. scatter/gather)
  geometry.py  trilinear map, Jacobian, geometric factors and weights (Sec. 2.3-2.4)
  operator.py  matrix-free residual (Eq. R, Algorithm 2) and explicit assembly
  schwarz.py   overlapping-patch fine preconditioner (Sec. 4.2, Eq. subd, Eq. z)
  coarse.py    coarse-grid correction (Sec. 4.1, Eq. coarse)
  amg.py       aggregation AMG used as the coarse solve (Sec. 4.1.1)
  pcg.py       preconditioned conjugate gradients (Algorithm 1)
  problem.py   one object tying the pieces together

Parity status of each function is stated in its module docstring. The AMG
aggregation rule is a reading (the paper does not define it; the oracle and
the GPU library implement the same written rule independently); it is pinned
to that written rule by cases worked out by hand (tests/test_oracle_amg_rules.py).
"""

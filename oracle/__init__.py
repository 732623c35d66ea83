"""FP64 CPU oracle for the SAA risk + gradient path of arXiv 2305.20053.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline / reference legs of `bench.py` may import this package.  The
product path (the CUDA library and its Python binding) never imports it and
shares no code, table or constant generator with it.

Everything here is plain numpy/scipy in float64, written to be checked against
the paper by eye:

  philox.py  counter-based Philox4x32-10 and Box-Muller normals (published
             definition of the generator; Salmon et al., SC'11)
  field.py   Matern random field by its Karhunen-Loeve expansion (Sec. 2,
             prior C = (-gamma Lap + delta I)^-2), control sources (Sec. 4.2),
             target state
  pde.py     finite-difference semilinear elliptic state equation (Sec. 4.2,
             Eq. for -div(e^m grad u) + r u^3 = sum z_i f_i), Newton with a
             banded Cholesky direct solve, QoI, adjoint gradient (Sec. 2.3)
  risk.py    mean + variance and the smoothed-CVaR risk measures (Sec. 2.1,
             2.2) and their gradients (Sec. 2.3, chain rule)
  dino.py    reduced-basis neural operator (Sec. 3.3): KL projection, POD,
             MLP forward, forward-mode control Jacobian, DINO loss in the
             reduced space (Sec. 3.4), backward pass, Adam, Jacobian data

Parity status: every function is pinned by a `-m "not gpu"` test in
tests/test_oracle_*.py against closed forms, brute force, finite differences,
a dense eigendecomposition or published known-answer vectors.
"""

"""CPU FP64 oracle for the semilinear lens-inversion inner loop.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously
correct restatement of what the GPU path computes, written from the paper
(Rogers & Fiege 2011, Sections 2.1-2.6): explicit sparse L, explicit B,
diagonal W, explicit H, dense Cholesky per lambda, and the L-curve corner by
spline curvature.  It shares no code with the CUDA library and neither side
imports the other; only the seeded input generators in ``synth`` serve both.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product path never calls it.

Modules: ``lens`` (ray trace), ``operators`` (L with bilinear, nearest-
neighbour or bicubic interpolation; B, W, H), ``solve``
(Cholesky solve, chi^2, regularisation measure, forward batch), ``lcurve``
(corner), ``data`` (synthetic observations), ``mlp`` (surrogate network
forward/backward/Adam), ``cg`` (matrix-free FP64 CGLS, used where a dense
F = B L does not fit), ``iterlc`` (fixed-iteration CGLS, the L-curve over
its iterations and the Monte Carlo degrees of freedom).

Every function is pinned by tests against something other than itself
(closed forms, invariants, brute force, library routines; see the
``tests/test_oracle_*.py`` docstrings).  The paper's printed E1/E3/E5
numbers are not pins: their inputs are not available.
"""

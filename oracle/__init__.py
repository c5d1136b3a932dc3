"""CPU FP64 oracle for the interior-point solver of dynamical optimal transport.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the discrete problem of Facca, Todeschi, Natale, Benzi,
"Efficient preconditioners for solving dynamical optimal transport via
interior point methods" (arXiv 2209.00315).  Only the test-suite, the
``smoke()`` check of the build entry point and the CPU-baseline leg of the
benchmark may import it.  The CUDA library never calls it, and it shares no
code with the CUDA library: the two only share the seeded input generators of
``ot_inputs``.

Modules
  mesh       generic triangle meshes, the midpoint 4-split, TPFA geometry (Sec. 2.1)
  operators  sparse matrices of Sec. 2.1-3 and of the projected / BB systems (Sec. 4.3),
             and one BB or SIMPLE application with exact inner solves
  ipm        residual F, Jacobian, exact Newton directions, the IPM loop, cost and dual value
  adjoint    gradient of the cost with respect to rho_in, rho_f (transposed-Jacobian solve)

Parity unpinned: nothing here fixes the number of Krylov or multigrid
iterations of the accelerated path; those are compared only qualitatively
with Table 3 of the paper.
"""

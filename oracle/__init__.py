"""Plain, slow, FP64 CPU oracle for the randomized Nystrom PCG hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import anything from here.  The
product path (the CUDA library and its Python binding) never imports,
calls or links this package, and this package shares no code with it: the
two meet only in the seeded input generators of
``paper_2110_02820_gb300.workloads``, which hold none of the method's
arithmetic.

Contents, each following the paper (Frangella, Tropp & Udell, "Randomized
Nystrom Preconditioning", arXiv 2110.02820) step by step:

* ``operators``  the matvec oracles x -> A x (Sec. 1.1): dense A, the ridge
  Gram operator X^T X (Sec. 1.3, Eq. (1.6)) and the Gaussian kernel
  (Sec. 6.3);
* ``nystrom``    Algorithm 1 (randomized Nystrom approximation), the
  preconditioner of Eq. (5.3), Algorithm 4 (randomized power error
  estimate), Algorithm 5 (adaptive rank doubling, Strategy 1) and the
  ratio rule of Strategy 2 (Sec. 5.4.2), Algorithm 2 (sketch-and-solve);
* ``pcg``        Algorithm 3 (Nystrom PCG), its independent-batch form,
  block Nystrom PCG for several right-hand sides of one shift (Sec. 5.2),
  and FP64-residual iterative refinement around a float32 inner solve;
* ``path``       the regularization path with warm starts and factor reuse
  of the paper's path experiments (Sec. 6.2);
* ``krr``        the KRR validation loss and its gradient by implicit
  differentiation (adjoint solve).

The random test matrix Omega and the power-step start vectors are inputs:
the parity tests draw them from ``workloads`` and pass the same arrays to
both sides.

Parity pins: every function here is checked by the ``-m "not gpu"`` tests
against closed forms, invariants, library routines or brute force on tiny
inputs.  Functions with no such pin say "parity unpinned" in their docstring.
"""

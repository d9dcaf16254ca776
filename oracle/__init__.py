"""CPU oracle for the fast Basic SSA hot path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously correct FP64 implementation of what
the paper's method computes.  It exists to check the CUDA library against;
it is never part of the product path.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import it.  It shares no code with the CUDA path (no
kernels, headers, tables or helpers); the only thing both sides consume is
the seeded input generator module ``paper_0911_4498_gb300.synth``.

Modules (each function cites the part of the paper it follows):
  dft          -- naive DFT and an own iterative radix-2 FFT (section 4.1).
  trajectory   -- explicit trajectory matrix, explicit X v / X^T u, naive
                  diagonal averaging (sections 2.1, 2.4).
  fast_hankel  -- Algorithms 2, 3 and 4 on the oracle's own FFT (sections
                  4.3 and 5).
  jacobi       -- one-sided Jacobi SVD of an explicit matrix (plain C).
  lanczos      -- Golub-Kahan-Lanczos bidiagonalisation (Algorithm 1) with
                  full reorthogonalisation by modified Gram-Schmidt applied
                  twice, thick restart and the residual test from relation (2)
                  (section 3).
  ssa          -- decompose / reconstruct front-ends, sign rule, L > K case.
  rng          -- splitmix64 in counter mode for the Lanczos starting vector.
"""

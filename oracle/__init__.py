"""CPU oracle for the cavity Helmholtz frequency-response solve (test infrastructure).

Plain, slow, obviously-correct complex128 numpy/scipy code that states what the GPU
path computes. It is TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference leg may import it. The product library
never imports it and shares no code with it; both take their inputs from the seeded
generators in ``helm_inputs``.

Modules (paper sections they follow):
  mesh     -- box lattice and boundary quads (Sec. 3.2: FE discretisation of the cavity)
  fem      -- Q1 element matrices by Gauss quadrature, assembly of K - k^2 M + i k rho c B(beta),
              symmetric Dirichlet elimination of the sun-roof pressure (Sec. 3.2, Helmholtz eq.)
  krylov   -- restarted GMRES(m) with complex Givens, COCG (Sec. 4: Krylov solve, complex FP64)
  ras      -- restricted additive Schwarz with exact local solves (Sec. 4: overlapping Schwarz DD)
  adjoint  -- listener objective and its gradient by an adjoint solve

Parity status per function is stated in each module header.
"""

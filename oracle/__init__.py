"""Plain FP64 CPU oracle for the Stokes-preconditioned Newton hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may use it. It shares no code with the CUDA library; the only
module both sides read is ``seeded_inputs`` (random numbers, no arithmetic
of the method).

Contents
  couette.py  the BEFE step, its tangent and adjoint for plane Couette flow
              (direct DFTs, explicit Chebyshev matrices, dense LU of the full
              coupled per-mode Chebyshev-tau Stokes system).
  newton.py   Newton-GMRES (modified Gram-Schmidt Arnoldi, no restarts) with
              a hookstep trust region, written for any state vector type.
"""

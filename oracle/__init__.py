"""FP64 CPU oracle for the monolithic ALE cylinder solver (test infrastructure).

This package is test infrastructure only.  It is imported by the tests, by
``__graft_entry__.smoke()`` and by the bench's CPU-baseline leg; the product
path never imports it and shares no code with it.

What it computes, and where in the paper each part is defined:
  * ``fem``     - Q2/Q1 bases, Gauss quadrature, the element residual of the
                  nonlinear functional NL(U) (Eq. nonlinear_functional,
                  Eq. weak_system), and the element Jacobian as the Gateaux
                  derivative of NL (Section 3.2) taken by complex-step
                  differentiation, so it is exact to rounding by definition.
  * ``solver``  - degrees of freedom, Dirichlet handling (Eq. flowBC,
                  Eq. psBC), the force-position constraint x = X - (1/k) int lambda
                  (Eq. lambda_coupling, Eq. coupling_constraint) written as two
                  border unknowns delta, BDF1/BDF2 time stepping and the
                  Newton-Raphson iteration (Eq. NR_iteration) with a library
                  sparse LU (SuperLU via scipy) as the linear solve.
  * ``mms``     - manufactured solutions (Section 5.1) and closed-form exact
                  patch solutions used to pin the oracle.

Parity status of each function is listed in the module headers; every
function here is pinned by a ``-m "not gpu"`` test (see tests/test_oracle_*.py).
"""

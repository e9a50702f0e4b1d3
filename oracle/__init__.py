"""CPU oracle for the space-time Galerkin BEM of the 2D heat equation (FP64).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path
(no kernels, helpers, tables or constants); both sides read their inputs from
the neutral ``workloads`` module only.

What it computes, all in plain float64 numpy/scipy:

* ``geometry``   -- boundary mesh Gamma_h, the half-segment dual pieces and the
                    pair classes used by the quadrature rule;
* ``special``    -- exponential integrals E1, E2 and the entire function Ein;
* ``quadrature`` -- Gauss-Legendre, geometrically graded and Duffy rules;
* ``timeint``    -- exact double time integrals of the heat kernels over a
                    pair of uniform time steps (closed form or Peano form);
* ``assembly``   -- block-Toeplitz lag blocks of V_h, K_h and D_h, the mass
                    matrix M_h of the right-hand side and the lumped mixed mass
                    of the preconditioner (Section 1 eq. (4); Section 2 Theorem);
* ``rhs``        -- the manufactured Dirichlet datum, f = (1/2 M_h + K_h) g and
                    the exact Neumann datum w = d_n u;
* ``solve``      -- block-Toeplitz products, exact block forward substitution in
                    time and a right-preconditioned GMRES;
* ``initial``    -- the initial-data operator M_h^0 on a triangulation of
                    Omega (eq. (4)) and the data of the Section 4 example;
* ``evaluate``   -- u in Q by the representation formula (eq. (2)) from the
                    discrete Cauchy data and initial datum;
* ``nonuniform``  -- V_h, K_h, D_h blocks on non-uniform time grids (block
                    lower triangular, not Toeplitz), their solve and data;
* ``gradient``   -- shape (vertex) and alpha derivatives of V_h, K_h, M_h and
                    g, the adjoint (backward-in-time) solve and the gradient of
                    ||w_h - w_target||^2.

Parity status of each function (what pins it) is listed in the module
docstrings; functions without an independent pin say "parity unpinned".
"""
from .rules import Rules, DEFAULT_RULES  # noqa: F401

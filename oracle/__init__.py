"""Plain FP64 CPU oracle for the weighted-upwind vector kinetic lattice Boltzmann
(WU-VKLB) method of Brown, Chaudhry and Shadid.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) imports, calls or links anything in this directory.  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may use it.

The oracle is deliberately slow and literal: numpy arrays in float64, one step of
the flow chart (Sec. 3.5, Fig. 5) at a time, with no blocking or fusion.  The
weighted flux splitting (Sec. 3.1, Eqs. (25)-(27)) is evaluated as the matrix
function  F+ = alpha(A) F  with  A = dF/dU  obtained by complex-step
differentiation and  alpha(A) = E (E + I)^-1,  E = expm(k A / max|lambda|).  This
is the basis-free form of  sum_j alpha(lambda_j) phi_j r_j  (Eqs. (16), (25),
(26)); it needs no eigenvectors and so shares nothing with the closed-form
eigen-structures of the CUDA path.  A second, literal eigen-decomposition route
(numpy.linalg.eig, Eqs. (15)-(18), (25)-(26)) exists for cross-checks.

Modules
-------
systems   flux functions F^(d)(U) of the shallow-water (Eq. 52), Euler (Eq. 54)
          and GLM-cleaned ideal-MHD (Eq. 58) systems, plus scalar advection.
splitting complex-step Jacobian, weighted / discontinuous / centered splittings.
vklb      equilibria (Eqs. 22-24, 41), collision (Eq. 42), streaming (Eq. 43),
          periodic and characteristic boundary conditions (Eqs. 33-37), CFL
          lattice speed (Eq. 29), the time loop of Fig. 5.
riemann   exact Riemann solutions (shallow water, Euler) used to pin the oracle.

Parity status per function is listed in each module header.  Every function has
a pin in ``tests/test_oracle_*.py`` except the Orszag-Tang solution profile
(parity unpinned: the paper compares it with an external code's output that is
not available; only the invariants and the two-route splitting check pin the
MHD-GLM oracle).
"""

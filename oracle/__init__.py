"""Plain FP64 CPU oracle for the controllability CG method (CMCG) of Grote, Nataf, Tang and
Tournier, "Parallel Controllability Methods for the Helmholtz Equation".

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  The CUDA path never calls it, shares no code
with it, and fails loudly when its own extension is missing.

Every function is written for a reader checking it against the paper by eye: plain numpy /
scipy.sparse on whole arrays, float64 and complex128 throughout, no blocking, no fusion.

Modules
  grid     the finite-difference discretisation (mass-lumped vertex-centred analogue of the
           paper's P1/Q1 FE with mass lumping, Sec. 4.1 and 4.3): weights W, boundary areas A,
           stiffness K, mass M, damping B, load F, period length and time step.
  wave     the leapfrog period map (velocity-Verlet form), its literal transpose, the energy
           functional J (Eq. cost_functional_J).
  riesz    the Riesz map of Eq. CMCG_PRECONDITIONIER: g~0 = K^+ g0 by a sparse direct solve.
  cmcg     the CMCG Algorithm of Sec. 2.3, steps (1)-(6), with the compatibility-condition
           shift removal of Sec. 2.1.
  direct   the plain definition of the method's fixed point: a direct sparse solve of the
           time-discrete Helmholtz system (K - wt^2 M - i wh B) U = F.
  first_order
           the first-order formulation of Sec. 3 on a staggered grid (v on nodes, p on links):
           its leapfrog period, literal transpose, J^, CMCG without a Riesz solve, and the two
           recoveries (Eq. mix_solution, Eq. TH_FILTERED_MIXED_SOLUTION).

Parity status of each function is stated in its module header.
"""

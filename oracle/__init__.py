"""Plain FP64 CPU oracle of the FR right-hand side (test infrastructure only).

This package is the independent reference that the CUDA library is checked
against.  Only the test-suite, the smoke check and the benchmark's CPU-baseline
leg may import it; the product path never does.  It shares no code with the
CUDA library: the only common inputs come from ``fr_inputs`` (meshes and
analytic fields, no method arithmetic).

Contents (each module cites the part of the paper it follows):

* ``polys``     Gauss-Legendre rules, Legendre/Jacobi polynomials, Lagrange
* ``elements``  point sets, nodal basis (Sec. 2), operators M0..M6 (App. A)
* ``geometry``  element mappings and metric terms (Sec. 2)
* ``physics``   Euler/NS fluxes (Sec. 4), Rusanov (App. B), LDG (Sec. 4.3),
                boundary ghosts (App. C)
* ``steppers`` forward Euler and DOPRI5 (Sec. 3 lists them beside RK4)
* ``system``    pairing, the RHS of Eq. negdivconf, classical RK4
* ``adjoint``   discrete adjoint of RHS and RK4 (not in the paper)

Pins (tests/test_oracle_*.py, ``-m "not gpu"``) tie every function to something
other than itself: closed forms, library routines, exact rational integration,
invariants (freestream, conservation, Kronecker property), FR-DG equivalence
to a weak-form DG residual, and the p+1 convergence order on the isentropic
vortex.  Parity with the paper's own printed numbers is unpinned wherever the
paper's meshes are missing (Couette tables) and for the triangle solution
points (Williams-Shunn coordinates are not printed).
"""

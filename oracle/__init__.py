"""CPU oracle for the eMG DG Euler hot path (arXiv 1807.01151) -- TEST INFRASTRUCTURE.

Plain, slow, obviously-correct FP64 numpy implementation of what the GPU path
computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it; the product library never
does, and this package never imports the product.  The only code the two sides
share is the seeded input generators in ``workloads/``.

Modules and the passages they follow:

* ``geometry``  reference maps, Gauss-Legendre rules, face matching, |E|, x_c, L,
                |dE|, h = 2d|E|/|dE|                          (Sec. 3.2, Eq. x3d)
* ``basis``     Cartesian normalised monomials + modified Gram-Schmidt
                                                             (Sec. 3.2, Eqs. basis2/basis)
* ``euler``     Euler flux and EOS (Eq. euler), Roe flux (Sec. 3.1), slip-wall and
                Riemann-invariant far-field ghost states (Sec. 3.3)
* ``dg``        residual R_p (Eq. euler3); Jacobian blocks as the derivative of R_p
                by complex-step differentiation (Eqs. jac1/jac2, Sec. 3.3)
* ``emg``       PRK smoother (Eq. prk_scalar), Arnoldi + phi_1 (Eqs. vm, final),
                EXP1 (Eq. EXP1), FAS V-cycle (Sec. 2.3), dtau and CFL_n
                (Eqs. x3d, cfl)

Pins (tests/test_oracle_*.py, all ``-m "not gpu"``): basis Gram matrix = I and
monomial reproduction; faceted-annulus area in closed form; Roe consistency,
antisymmetry, Roe-matrix property and |A| from the Lagrange form of the matrix
function; flux Jacobian against the closed form of the Appendix (Eq. dfdu);
free-stream preservation; discrete conservation; order p+1 on a manufactured
solution; Jacobian blocks against central finite differences and dense brute force;
PRK amplification polynomial; Krylov phi_1 against dense expm, linear-ODE
exactness and the dt limits; the EXP1 step on tiny p = 0 meshes (Krylov space
exhausted) against the dense phi_1(DT J_0) DT R~_0 from its Taylor series and from
A^-1 (e^A - I) N; restriction/prolongation identities; h_2D = 4A/P and
Eq. x2d; CFL_n sequence; converged state symmetry and path independence.

Parity unpinned: the paper's own iteration counts and CPU times (its figures are
not available), and the choice of the small-matrix exponential routine (Pade
scaling-and-squaring instead of the Chebyshev rational approximation named in
Sec. 2.2; both equal phi_1 to rounding).
"""

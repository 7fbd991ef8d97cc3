"""FP64 CPU oracle for the rank-structured 3D Coulomb convolution.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports, links or calls this
package; only the tests, the smoke check and the benchmark's CPU-baseline leg
do.  It is a plain, slow, direct-summation restatement of what the method
computes, in float64 with numpy/scipy library primitives (matmul, erf, erfc,
Gauss-Legendre nodes) and no blocking, fusion or FFT.

Modules and the passages they follow (Khoromskaia & Khoromskij, arXiv:1504.06289):

* ``sinc``            sinc-quadrature Gaussian sum for 1/r (Appendix 3, Eq. sinc_Newt).
* ``kernel_vectors``  Galerkin cell integrals p_q of the Newton kernel
                      (Appendix 3, Eq. galten and the vectors p_q^(l)); the 2n
                      master kernel of Sec. 5.1 (Eq. refTensor).
* ``cp``              grid sampling of Gaussians (Sec. 3.1, Eq. disc_GTO), CP
                      convolution by 1D convolutions (Sec. 2.5, Eq. conv), the
                      convolution matrices U^T (p_q * U) (Sec. 3.2,
                      Eq. Factor_Mk_Conv), the scalar product (Sec. 2.5, Eq. scal)
                      giving E_H, and its adjoint.
* ``coulomb``         Coulomb matrix J_{mu nu} = <G_mu . G_nu, V_H> (Sec. 3.1).
* ``lattice``         assembled lattice sums (Sec. 5.1, Eqs. CoulombLattice,
                      CoulombLatTensCan), their evaluation on a sub-grid, and the
                      interaction energy of the lattice charges (Sec. 5.3,
                      Eqs. EnergyLatSum, EnergyLattice).
* ``tei``             two-electron integrals by 1D density fitting and a
                      truncated Cholesky factorisation of the TEI matrix, and
                      J(D) for a density matrix (Sec. 3.2).
* ``nuclear``         nuclear potential of a molecule by windowed shifts of the
                      master kernel and its Galerkin matrix (Sec. 3.3).
* ``closed_forms``    analytic Gaussian Coulomb results used only to pin the
                      oracle (not part of the method).

Parity status: every function here is pinned by a ``-m "not gpu"`` test against
something other than itself (closed forms, mpmath, brute force, invariants);
see tests/test_oracle_*.py.
"""

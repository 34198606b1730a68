"""Plain FP64 CPU oracle for spin-adapted two-site DMRG (test infrastructure only).

This package exists to check the CUDA library.  Only tests/, the smoke() entry of
__graft_entry__ and the cpu_baseline / reference legs of bench.py may import it; the
library itself never does.  It shares no code with the library: it restates the
paper (Wouters, Poelmans, Ayers, Van Neck, CheMPS2, Comput. Phys. Commun.) in the
most direct form available:

  * su2.py   - Clebsch-Gordan coefficients and Wigner 6-j symbols (Racah formulas),
               used by Eq. 22 (Wigner-Eckart factorisation) and Eqs. 25-26.
  * fci.py   - full configuration interaction in the determinant basis: the plain
               definition of the Hamiltonian of Sec. 4.1 (physics notation), the
               one-body folding of Eq. 11, and S^2 for spin checks.
  * mps.py   - reduced MPS tensors (Eq. 22), the symmetry sectors of Sec. 3, the
               initial equal distribution of D (Sec. 4.3), the reduced two-site
               object (Eq. 25) and its back-transform (Eq. 26), the block SVD and
               truncation (Eqs. 27-28, discarded weight Eq. 15), and the expansion of
               the reduced two-site basis into determinants, from which the effective
               Hamiltonian of Eq. 9 is formed as P^T H P (its plain definition).
  * dmrg.py  - the two-site sweep of Secs. 2.3-2.4 and 4.3 with that dense H_eff.

Parity unpinned: none of the energy or matvec functions; individual singular
vectors and operator blocks are gauge dependent and are never compared.
"""

"""Pins for the oracle's excited-state Hamiltonian H_m = H_0 + sum_k eta_{k+1} |Psi_k><Psi_k|
(Sec. 4.3): at full D the two-site basis spans every state of the symmetry sector, so

* where the two-site basis spans the sector (the middle pair of the Hubbard chain L=6 at
  full D), the projection of the ground state has unit norm and the spectrum of the
  projected effective Hamiltonian is FCI's with E_0 moved to E_0 + eta;
* the projection of a converged state onto its own two-site basis is its two-site vector;
* the sweep on H_1 (then H_2) converges to FCI's second (third) root, with S fixed."""
import numpy as np
import pytest

from oracle import dmrg
from oracle import mps as M
from oracle.fci import fci_ground_state
from tests.test_oracle_mps import canonical_mps, move_center_right, problem

CASES = [("hubbard", 6, 6, 0, 0), ("random", 5, 4, 0, 1), ("random", 5, 5, 1, 0)]


@pytest.mark.parametrize("case", CASES)
def test_excited_states_at_full_d_equal_fci_roots(case):
    kind, L, N, tS, IG = case
    irreps, h, V, prob = problem(*case)
    E, _, _ = fci_ground_state(h, V, N, tS, irreps, IG, nroots=3)
    assert E[1] - E[0] > 1e-6 and E[2] - E[1] > 1e-6
    m0 = canonical_mps(irreps, N, tS, IG, 400, 5)
    e0, _ = dmrg.sweep(prob, m0, 400, 2)
    assert abs(e0 - E[0]) < 1e-10
    eta = 2.0 * (E[2] - E[0]) + 1.0
    # the ground state's projection onto its own basis, and the shifted spectrum
    # sweeps on H_1 and H_2
    m1 = canonical_mps(irreps, N, tS, IG, 400, 9)
    e1, _ = dmrg.sweep(prob, m1, 400, 2, lower=[(m0, eta)])
    assert abs(e1 - E[1]) < 1e-9
    m2 = canonical_mps(irreps, N, tS, IG, 400, 10)
    e2, _ = dmrg.sweep(prob, m2, 400, 2, lower=[(m0, eta), (m1, eta)])
    assert abs(e2 - E[2]) < 1e-9


def test_projection_of_own_state_is_the_two_site_vector():
    irreps, h, V, prob = problem("random", 5, 4, 0, 1)
    m = canonical_mps(irreps, 4, 0, 1, 400, 5)
    dmrg.sweep(prob, m, 400, 1)
    for i in range(4):
        H, G, proj = dmrg.effective_hamiltonian(prob, m, i)
        x = proj.flatten(M.tt_to_x(m, i))
        v = dmrg.projected_state(prob, proj, dmrg.determinant_components(prob, m))
        assert abs(abs(v @ x) / np.linalg.norm(x) - 1.0) < 1e-10
        if i < 3:
            move_center_right(m, i)


def test_shifted_spectrum_at_the_middle_pair():
    # Hubbard L=6: at the middle pair both environments of a full-D state hold every state
    # of their two orbitals, so the two-site basis spans the sector whatever the state
    irreps, h, V, prob = problem("hubbard", 6, 6, 0, 0)
    E, _, _ = fci_ground_state(h, V, 6, 0, irreps, 0, nroots=3)
    m0 = canonical_mps(irreps, 6, 0, 0, 400, 5)
    dmrg.sweep(prob, m0, 400, 2)
    eta = 2.0 * (E[2] - E[0]) + 1.0
    m = canonical_mps(irreps, 6, 0, 0, 400, 8)
    for i in range(2):
        move_center_right(m, i)
    H, G, proj = dmrg.effective_hamiltonian(prob, m, 2)
    v = dmrg.projected_state(prob, proj, dmrg.determinant_components(prob, m0))
    assert abs(v @ v - 1.0) < 1e-10
    Hm, _, _ = dmrg.excited_hamiltonian(prob, m, 2, [(m0, eta)])
    w = np.linalg.eigvalsh(Hm)
    assert abs(w[0] - E[1]) < 1e-9 and abs(w[1] - E[2]) < 1e-9
    assert np.any(np.abs(w - (E[0] + eta)) < 1e-9)

"""Pins for the oracle's reduced density matrices (oracle/rdm.py).

* a brute-force Fock-space evaluation of the definitions with Jordan-Wigner matrices,
  which shares nothing with the string machinery of oracle/fci.py;
* the closed shell of the U = 0 Hubbard chain: gamma = 2 P_occ and
  Gamma_ijkl = gamma_ik gamma_jl - gamma_il gamma_jk / 2 (Wick's theorem);
* the energy of Sec. 4.1 rebuilt from (gamma, Gamma) equals the FCI eigenvalue, and the
  traces tr gamma = N, sum_j Gamma_ijkj = (N - 1) gamma_ik;
* Hellmann-Feynman: central differences of the FCI eigenvalue under symmetric changes
  of h and V equal the RDM contractions;
* the spin-summed RDMs of every Sz component of an MPS multiplet agree."""
import itertools

import numpy as np

from oracle import mps as om
from oracle.fci import fci_ground_state
from oracle.rdm import energy, mps_state, rdm_from_vector, sym8
from tests.test_oracle_fci import jw_ops
from workloads import hubbard_chain, random_integrals, round_robin_irreps, uniform_pm1


def brute_rdm(h, V, N):
    """RDMs of the lowest N-electron state of the Fock-space Hamiltonian, from the
    Jordan-Wigner matrices of every spin orbital (interleaved up / down order)."""
    L = h.shape[0]
    cr = jw_ops(L)
    an = [o.T for o in cr]
    H = np.zeros_like(cr[0])
    for p, q in itertools.product(range(L), repeat=2):
        for s in range(2):
            H += h[p, q] * cr[2 * p + s] @ an[2 * q + s]
    for i, j, k, l in itertools.product(range(L), repeat=4):
        if V[i, j, k, l] != 0.0:
            for s, t in itertools.product(range(2), repeat=2):
                H += 0.5 * V[i, j, k, l] * cr[2 * i + s] @ cr[2 * j + t] @ an[2 * l + t] @ an[2 * k + s]
    nop = np.diag(sum(cr[k] @ an[k] for k in range(2 * L)))
    sel = np.flatnonzero(np.abs(nop - N) < 1e-9)
    w, U = np.linalg.eigh(H[np.ix_(sel, sel)])
    assert w[1] - w[0] > 1e-6, "ground state must be non-degenerate"
    psi = np.zeros(H.shape[0])
    psi[sel] = U[:, 0]
    gamma = np.zeros((L, L))
    Gamma = np.zeros((L,) * 4)
    for i, k in itertools.product(range(L), repeat=2):
        gamma[i, k] = sum(psi @ (cr[2 * i + s] @ (an[2 * k + s] @ psi)) for s in range(2))
    for i, j, k, l in itertools.product(range(L), repeat=4):
        Gamma[i, j, k, l] = sum(psi @ (cr[2 * i + s] @ (cr[2 * j + t] @ (an[2 * l + t] @ (an[2 * k + s] @ psi))))
                                for s, t in itertools.product(range(2), repeat=2))
    return w[0], gamma, Gamma


def test_matches_bruteforce_fock_space():
    # half-filled Hubbard chain: non-degenerate singlet ground state (Lieb-Mattis)
    L, N = 4, 4
    h, V = hubbard_chain(L, 1.0, 4.0)
    e_ref, g_ref, G_ref = brute_rdm(h, V, N)
    E, vecs, space = fci_ground_state(h, V, N, 0, [0] * L, 0)
    assert abs(E[0] - e_ref) < 1e-10
    gamma, Gamma = rdm_from_vector(space, vecs[0])
    assert np.abs(gamma - g_ref).max() < 1e-10
    assert np.abs(Gamma - G_ref).max() < 1e-10


def test_closed_shell_wick():
    L, N = 6, 6
    h, V = hubbard_chain(L, 1.0, 0.0)
    E, vecs, space = fci_ground_state(h, V, N, 0, [0] * L, 0)
    gamma, Gamma = rdm_from_vector(space, vecs[0])
    eps, phi = np.linalg.eigh(h)
    P = phi[:, : N // 2] @ phi[:, : N // 2].T
    g0 = 2.0 * P
    G0 = np.einsum("ik,jl->ijkl", g0, g0) - 0.5 * np.einsum("il,jk->ijkl", g0, g0)
    assert np.abs(gamma - g0).max() < 1e-10
    assert np.abs(Gamma - G0).max() < 1e-10


def test_energy_traces_and_symmetry_random():
    L = 6
    irreps = round_robin_irreps(L)
    h, V = random_integrals(irreps, 17)
    for N, two_S in ((6, 0), (5, 1), (6, 2)):
        E, vecs, space = fci_ground_state(h, V, N, two_S, irreps, 0, ecore=0.3)
        gamma, Gamma = rdm_from_vector(space, vecs[0])
        assert abs(energy(gamma, Gamma, h, V, 0.3) - E[0]) < 1e-10
        assert abs(np.trace(gamma) - N) < 1e-11
        assert np.abs(np.einsum("ijkj->ik", Gamma) - (N - 1) * gamma).max() < 1e-10
        assert abs(np.einsum("ijij->", Gamma) - N * (N - 1)) < 1e-9
        assert np.abs(gamma - gamma.T).max() < 1e-12
        # particle exchange and Hermiticity (real state)
        assert np.abs(Gamma - Gamma.transpose(1, 0, 3, 2)).max() < 1e-11
        assert np.abs(Gamma - Gamma.transpose(2, 3, 0, 1)).max() < 1e-11
        # the symmetrised part carries the whole energy
        assert abs(energy(gamma, sym8(Gamma), h, V, 0.3) - E[0]) < 1e-10


def test_sym8_projection():
    rng = np.random.default_rng(3)
    G = rng.normal(size=(3,) * 4)
    S = sym8(G)
    assert np.abs(sym8(S) - S).max() < 1e-14
    for i, j, k, l in itertools.product(range(3), repeat=4):
        imgs = [G[i, j, k, l], G[j, i, l, k], G[k, l, i, j], G[l, k, j, i],
                G[k, j, i, l], G[i, l, k, j], G[l, i, j, k], G[j, k, l, i]]
        assert abs(S[i, j, k, l] - np.mean(imgs)) < 1e-14
    V = random_integrals([0, 0, 0], 2, n_irrep=1)[1]
    assert np.abs(sym8(V) - V).max() < 1e-14


def test_hellmann_feynman_central_differences():
    L, N = 5, 4
    irreps = [0] * L
    h, V = random_integrals(irreps, 23, n_irrep=1)
    E, vecs, space = fci_ground_state(h, V, N, 0, irreps, 0)
    gamma, Gamma = rdm_from_vector(space, vecs[0])
    Gs = sym8(Gamma)
    d = 1e-4
    for (i, k) in ((0, 0), (1, 3), (2, 4)):
        dh = np.zeros_like(h)
        dh[i, k] += d
        if i != k:
            dh[k, i] += d
        ep = fci_ground_state(h + dh, V, N, 0, irreps, 0)[0][0]
        em = fci_ground_state(h - dh, V, N, 0, irreps, 0)[0][0]
        assert abs((ep - em) / (2 * d) - np.sum(gamma * dh) / d) < 1e-7
    for idx in ((0, 1, 2, 3), (1, 1, 0, 4), (2, 2, 2, 2), (0, 3, 0, 3)):
        dV = np.zeros_like(V)
        i, j, k, l = idx
        for img in ((i, j, k, l), (j, i, l, k), (k, l, i, j), (l, k, j, i),
                    (k, j, i, l), (i, l, k, j), (l, i, j, k), (j, k, l, i)):
            dV[img] = d
        ep = fci_ground_state(h, V + dV, N, 0, irreps, 0)[0][0]
        em = fci_ground_state(h, V - dV, N, 0, irreps, 0)[0][0]
        fd = (ep - em) / (2 * d)
        assert abs(fd - 0.5 * np.sum(Gs * dV) / d) < 1e-7
        assert abs(fd - 0.5 * np.sum(Gamma * dV) / d) < 1e-7


def test_mps_multiplet_components_agree():
    irreps = round_robin_irreps(5)
    m = om.random_mps(irreps, 5, 1, 0, 12, uniform_pm1(7, 10 ** 6))
    g0, G0 = rdm_from_vector(*mps_state(m, 0))
    g1, G1 = rdm_from_vector(*mps_state(m, 1))
    assert np.abs(g0 - g1).max() < 1e-12
    assert np.abs(G0 - G1).max() < 1e-12
    assert abs(np.trace(g1) - 5) < 1e-12

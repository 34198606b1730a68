"""Pins for the oracle FCI solver: closed forms and a brute-force Fock-space build.

The brute-force reference writes every a+_{p s} as a Jordan-Wigner matrix on the
4^L Fock space and sums the Hamiltonian of Sec. 4.1 term by term, sharing nothing
with the string machinery of oracle/fci.py."""
import itertools
import math

import numpy as np
import pytest

from oracle.fci import fold, fci_ground_state
from workloads import hubbard_chain, random_integrals, round_robin_irreps


def jw_ops(L):
    """Creation matrices for spin orbitals 2p (up), 2p+1 (down), interleaved order."""
    n = 2 * L
    c = np.array([[0.0, 0.0], [1.0, 0.0]])  # |1><0|
    Z = np.diag([1.0, -1.0])
    I = np.eye(2)
    ops = []
    for k in range(n):
        m = np.array([[1.0]])
        for j in range(n):
            m = np.kron(m, Z if j < k else (c if j == k else I))
        ops.append(m)
    return ops


def brute_hamiltonian(h, V):
    L = h.shape[0]
    cr = jw_ops(L)
    an = [o.T for o in cr]
    H = np.zeros_like(cr[0])
    for p, q in itertools.product(range(L), repeat=2):
        for s in range(2):
            H += h[p, q] * cr[2 * p + s] @ an[2 * q + s]
    for i, j, k, l in itertools.product(range(L), repeat=4):
        if V[i, j, k, l] == 0.0:
            continue
        for s, t in itertools.product(range(2), repeat=2):
            H += 0.5 * V[i, j, k, l] * cr[2 * i + s] @ cr[2 * j + t] @ an[2 * l + t] @ an[2 * k + s]
    Nop = sum(cr[k] @ an[k] for k in range(2 * L))
    Sz = 0.5 * sum(cr[2 * p] @ an[2 * p] - cr[2 * p + 1] @ an[2 * p + 1] for p in range(L))
    Sp = sum(cr[2 * p] @ an[2 * p + 1] for p in range(L))
    S2 = Sp.T @ Sp + Sz @ Sz + Sz
    return H, Nop, Sz, S2


def brute_lowest(h, V, irreps, N, two_S, I_G):
    L = h.shape[0]
    H, Nop, Sz, S2 = brute_hamiltonian(h, V)
    dim = H.shape[0]
    # occupation of each basis state (bit k of the index, mode 0 = most significant)
    irr = np.zeros(dim, dtype=int)
    for b in range(dim):
        ir = 0
        for k in range(2 * L):
            if (b >> (2 * L - 1 - k)) & 1:
                ir ^= irreps[k // 2]
        irr[b] = ir
    sel = np.flatnonzero((np.abs(np.diag(Nop) - N) < 1e-9) & (np.abs(np.diag(Sz) - two_S / 2) < 1e-9)
                         & (irr == I_G))
    if sel.size == 0:
        return None
    Hs = H[np.ix_(sel, sel)]
    S2s = S2[np.ix_(sel, sel)]
    w, U = np.linalg.eigh(Hs)
    S = two_S / 2
    for a in range(w.size):
        s2 = U[:, a] @ S2s @ U[:, a]
        if abs(s2 - S * (S + 1)) < 1e-6:
            return w[a]
    return None


@pytest.mark.parametrize("L,seed", [(2, 1), (3, 2), (4, 3)])
def test_fci_matches_bruteforce_all_sectors(L, seed):
    irreps = round_robin_irreps(L, 4)
    h, V = random_integrals(irreps, seed, n_irrep=4)
    for N in range(1, 2 * L):
        for two_S in range(N % 2, min(N, 2 * L - N) + 1, 2):
            for I_G in range(4):
                ref = brute_lowest(h, V, irreps, N, two_S, I_G)
                if ref is None:
                    continue
                E, vecs, space = fci_ground_state(h, V, N, two_S, irreps, I_G)
                assert abs(E[0] - ref) < 1e-10, (N, two_S, I_G)
                assert abs(space.s2(vecs[0]) - two_S / 2 * (two_S / 2 + 1)) < 1e-9


def test_hubbard_dimer_closed_form():
    # two sites, two electrons, singlet: E = (U - sqrt(U^2 + 16 t^2)) / 2
    for U in (0.0, 1.0, 4.0, 10.0):
        h, V = hubbard_chain(2, 1.0, U)
        E, _, _ = fci_ground_state(h, V, 2, 0, [0, 0], 0)
        assert abs(E[0] - (U - math.sqrt(U * U + 16.0)) / 2) < 1e-12


def test_hubbard_u0_closed_form_and_spin():
    # open chain orbital energies -2t cos(k pi / (L+1)); closed shell of N/2 lowest
    L, N = 8, 8
    h, V = hubbard_chain(L, 1.0, 0.0)
    E, vecs, space = fci_ground_state(h, V, N, 0, [0] * L, 0)
    exact = 2 * sum(-2.0 * math.cos(k * math.pi / (L + 1)) for k in range(1, N // 2 + 1))
    assert abs(E[0] - exact) < 1e-12
    assert abs(E[0] - (-9.517540966287)) < 1e-11
    assert abs(space.s2(vecs[0])) < 1e-10


def test_v0_random_h_is_orbital_energy_sum():
    L, N = 8, 6
    irreps = round_robin_irreps(L)
    h, _ = random_integrals(irreps, 5)
    V = np.zeros((L,) * 4)
    E, _, _ = fci_ground_state(h, V, N, 0, irreps, 0)
    eps = np.linalg.eigvalsh(h)
    assert abs(E[0] - 2 * np.sort(eps)[: N // 2].sum()) < 1e-11


def test_folding_is_exact_in_the_n_electron_space():
    L = 6
    irreps = round_robin_irreps(L)
    h, V = random_integrals(irreps, 9)
    for N, two_S in ((6, 0), (5, 1), (4, 2)):
        E1, _, _ = fci_ground_state(h, V, N, two_S, irreps, 0)
        g = fold(h, V, N)
        E2, _, _ = fci_ground_state(np.zeros_like(h), g, N, two_S, irreps, 0)
        assert abs(E1[0] - E2[0]) < 1e-11


def test_hubbard8_u4_singlet():
    h, V = hubbard_chain(8, 1.0, 4.0)
    E, vecs, space = fci_ground_state(h, V, 8, 0, [0] * 8, 0)
    assert space.mask.sum() == 4900
    assert abs(space.s2(vecs[0])) < 1e-10
    # Lieb-Mattis: the absolute ground state of the half-filled chain is a singlet
    E1, _, _ = fci_ground_state(h, V, 8, 2, [0] * 8, 0)
    assert E[0] < E1[0]

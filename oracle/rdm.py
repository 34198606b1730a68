"""Spin-summed one- and two-particle reduced density matrices (oracle, FP64).

Test infrastructure only: the library never imports this module.

Definitions (Sec. 4.3, the spin-summed 2-RDM Gamma^A and the 1-RDM as its partial trace),
in the index order of the Hamiltonian of Sec. 4.1 (physics notation):
    gamma_ik   = sum_s  <a+_is a_ks>               = <E_ik>
    Gamma_ijkl = sum_st <a+_is a+_jt a_lt a_ks>    = <E_ik E_jl> - delta_jk <E_il>
with E_pq = sum_s a+_ps a_qs.  For a normalised state
    <H> = E_c + sum_ik h_ik gamma_ik + 1/2 sum_ijkl V_ijkl Gamma_ijkl,
which is linear in (h, V) at a fixed state: dE/dh_ik = gamma_ik and
dE/dV_ijkl = Gamma_ijkl / 2.  For an exact eigenstate these are also the derivatives
of the eigenvalue (Hellmann-Feynman), which is what DMRG-SCF consumes (Sec. 4.4).
Sec. 4.1 requires V to be invariant under eight index permutations; an energy
written with such a V sees only the part of Gamma with the same invariance, the
projection `sym8`.

The state is a determinant vector C[alpha string, beta string] of oracle/fci.py;
`mps_state` expands an oracle MPS into that basis through the reduced two-site
projector of oracle/mps.py (the expansion behind the dense H_eff of Eq. 9).
"""
import numpy as np

from .fci import FCISpace
from .mps import TwoSiteProjector, tt_to_x

# the eight index permutations of Sec. 4.1 (ijkl itself first), as einsum inputs
SYM8 = ("ijkl", "jilk", "klij", "lkji", "kjil", "ilkj", "lijk", "jkli")


def rdm_from_vector(space, C):
    """(gamma, Gamma) of the state C (normalised here) from the definitions above:
    <E_ik E_jl> = <E_ki C, E_jl C> since E_ik^T = E_ki for real determinant vectors."""
    L = space.L
    C = np.asarray(C, dtype=float)
    C = C / np.sqrt(np.vdot(C, C))
    Ev = np.empty((L * L, C.size))
    for p in range(L):
        for q in range(L):
            Ev[p * L + q] = space.E(p, q, C).ravel()
    gamma = (Ev @ C.ravel()).reshape(L, L)
    G = Ev @ Ev.T  # G[(p q), (r s)] = <E_pq C, E_rs C>
    Gamma = np.empty((L,) * 4)
    for i in range(L):
        for j in range(L):
            for k in range(L):
                for l in range(L):
                    Gamma[i, j, k, l] = G[k * L + i, j * L + l] - (gamma[i, l] if j == k else 0.0)
    return gamma, Gamma


def sym8(G):
    """Average of G over the eight permutations that leave a valid V invariant."""
    return sum(np.einsum(s + "->ijkl", G) for s in SYM8) / 8.0


def energy(gamma, Gamma, h, V, ecore=0.0):
    """E_c + sum h gamma + 1/2 sum V Gamma."""
    return ecore + float(np.sum(h * gamma)) + 0.5 * float(np.sum(V * Gamma))


def mps_state(m, f=None):
    """Determinant vector (FCISpace, C) of an oracle MPS, component Sz = (2f - 2S)/2
    of its spin multiplet (default f = 2S: Sz = S)."""
    tS = m.two_S
    spaces = []
    for ff in range(tS + 1):
        tm = 2 * ff - tS
        spaces.append(FCISpace(m.L, (m.N + tm) // 2, (m.N - tm) // 2, m.irreps, m.I_G))
    f = tS if f is None else f
    proj = TwoSiteProjector(m, 0, spaces)
    v = proj.P[f] @ proj.flatten(tt_to_x(m, 0))
    return spaces[f], v.reshape(spaces[f].shape)

"""Pins for the oracle's reduced MPS, Eqs. 25-28 and the projected H_eff.

Independent references: FCI (exact at full D), a Jordan-Wigner brute-force Fock
Hamiltonian (sharing no code with oracle/fci.py), S^2 of the expanded state, and the
orthogonality relations of the recoupling."""
import numpy as np
import pytest

from oracle import dmrg
from oracle import mps as M
from oracle.fci import fci_ground_state
from tests.test_oracle_fci import brute_hamiltonian, jw_ops
from workloads import hubbard_chain, random_integrals, round_robin_irreps, uniform_pm1


def canonical_mps(irreps, N, two_S, I_G, D, seed):
    m = M.random_mps(irreps, N, two_S, I_G, D, uniform_pm1(seed, 10 ** 6))
    return M.right_canonicalize(m)


def move_center_right(m, i):
    x = M.tt_to_x(m, i)
    M.svd_truncate(m, i, x, 10 ** 9, "right")


CASES = [
    ("hubbard", 6, 6, 0, 0),
    ("random", 6, 6, 2, 0),
    ("random", 6, 5, 1, 3),
    ("random", 7, 6, 0, 1),
]


def problem(kind, L, N, two_S, I_G, seed=11):
    if kind == "hubbard":
        irreps = [0] * L
        h, V = hubbard_chain(L, 1.0, 4.0)
    else:
        irreps = round_robin_irreps(L)
        h, V = random_integrals(irreps, seed)
    return irreps, h, V, dmrg.Problem(h, V, irreps, N, two_S, I_G)


@pytest.mark.parametrize("case", CASES)
def test_projector_is_isometry_and_heff_symmetric(case):
    kind, L, N, tS, IG = case
    irreps, h, V, prob = problem(*case)
    m = canonical_mps(irreps, N, tS, IG, 40, 3)
    for i in range(L - 1):
        H, G, proj = dmrg.effective_hamiltonian(prob, m, i)
        assert np.abs(G - np.eye(proj.n)).max() < 1e-12
        x = proj.flatten(M.tt_to_x(m, i))
        assert abs(x @ x - 1.0) < 1e-12
        if i < L - 2:
            move_center_right(m, i)


@pytest.mark.parametrize("case", CASES)
def test_full_d_dmrg_equals_fci(case):
    kind, L, N, tS, IG = case
    irreps, h, V, prob = problem(*case)
    m = canonical_mps(irreps, N, tS, IG, 400, 5)
    emin, es = dmrg.sweep(prob, m, 400, 2)
    E, _, _ = fci_ground_state(h, V, N, tS, irreps, IG)
    assert abs(emin - E[0]) < 1e-10
    assert abs(es[-1] - E[0]) < 1e-10


def test_truncated_dmrg_is_variational_and_reports_weights():
    irreps, h, V, prob = problem("random", 7, 6, 0, 1)
    E, _, _ = fci_ground_state(h, V, 6, 0, irreps, 1)
    m = canonical_mps(irreps, 6, 0, 1, 6, 7)
    emin, es = dmrg.sweep(prob, m, 6, 2)
    assert emin >= E[0] - 1e-10
    # truncation: kappa normalised, w_disc in [0, 1)
    x = M.tt_to_x(m, 2)
    w, kept, groups = M.svd_truncate(m, 2, x, 3, "right")
    norm2 = sum((g[0][0] + 1) * np.sum(g[6] ** 2) for g in groups)
    kept_w = sum((groups[gi][0][0] + 1) * groups[gi][6][a] ** 2 for _, gi, a in kept) / norm2
    assert abs(kept_w + w - 1.0) < 1e-12
    assert 0.0 <= w < 1.0


@pytest.mark.parametrize("case", CASES)
def test_s_tt_round_trip(case):
    kind, L, N, tS, IG = case
    irreps, h, V, prob = problem(*case)
    m = canonical_mps(irreps, N, tS, IG, 40, 9)
    i = L // 2 - 1
    for k in range(i):
        move_center_right(m, k)
    x = M.tt_to_x(m, i)
    # Eq. 26 then Eq. 25 (through an exact SVD that keeps every lambda) is identity
    m2 = m.copy()
    w, _, _ = M.svd_truncate(m2, i, {k: v.copy() for k, v in x.items()}, 10 ** 9, "right")
    assert w < 1e-28
    x2 = M.tt_to_x(m2, i)
    for key in x:
        assert np.abs(x[key] - x2.get(key, 0.0)).max() < 1e-12


def jw_state_from_dets(C, space, L):
    """Psi in the Jordan-Wigner basis: apply a+_{p up} (p ascending) then a+_{p dn}
    to the vacuum for every determinant (alpha-then-beta creator order)."""
    cr = jw_ops(L)
    dim = cr[0].shape[0]
    vac = np.zeros(dim); vac[0] = 1.0
    psi = np.zeros(dim)
    for ia, a in enumerate(space.A.strs):
        for ib, b in enumerate(space.B.strs):
            c = C[ia, ib]
            if c == 0.0:
                continue
            v = vac.copy()
            for p in reversed(range(L)):
                if (b >> p) & 1:
                    v = cr[2 * p + 1] @ v
            for p in reversed(range(L)):
                if (a >> p) & 1:
                    v = cr[2 * p] @ v
            psi += c * v
    return psi


@pytest.mark.parametrize("case", [("random", 4, 4, 0, 0), ("random", 4, 3, 1, 1), ("hubbard", 4, 4, 2, 0)])
def test_energy_and_spin_against_jordan_wigner(case):
    kind, L, N, tS, IG = case
    irreps, h, V, prob = problem(kind, L, N, tS, IG, seed=21)
    m = canonical_mps(irreps, N, tS, IG, 30, 13)
    Hb, Nop, Sz, S2 = brute_hamiltonian(h, V)
    i = 1
    H, G, proj = dmrg.effective_hamiltonian(prob, m, i)
    x = proj.flatten(M.tt_to_x(m, i))
    e_red = x @ H @ x
    e_bf, n_bf, s2_bf = 0.0, 0.0, 0.0
    for f, P in enumerate(proj.P):
        space = prob.spaces[f]
        C = (P @ x).reshape(space.shape)
        psi = jw_state_from_dets(C, space, L)
        e_bf += psi @ Hb @ psi
        n_bf += psi @ psi
        s2_bf += psi @ S2 @ psi
        assert abs(psi @ Nop @ psi - N * (psi @ psi)) < 1e-10
    assert abs(n_bf - 1.0) < 1e-12
    assert abs(e_red - e_bf) < 1e-11
    S = tS / 2
    assert abs(s2_bf - S * (S + 1)) < 1e-10

"""Pins for three oracle functions that the energy pins cannot see:

* the selection rule of `mps.svd_truncate` ("the D largest values of lambda are kept",
  Sec. 4.2, Eqs. 27-28) and its discarded weight (Eq. 15), against the dense Schmidt
  spectrum of the same state expanded into a Jordan-Wigner Fock space and grouped into
  SU(2) multiplets by its Sz sectors;
* the noise branch of `dmrg.micro_iteration` (Sec. 4.2: noise bounded by
  0.5 gamma w_disc added just before the decomposition) on the Hubbard dimer, whose
  ground state, post-noise vector, Schmidt values and discarded weight are written
  here in closed form;
* `mps.distribute` (Sec. 4.3: D spread equally over the sectors of a bond, none above
  its FCI dimension) against hand-worked tables and the max-min fairness that defines an
  equal spread under caps.
"""
import itertools

import numpy as np
import pytest

from oracle import dmrg
from oracle import mps as M
from workloads import hubbard_chain, random_integrals, round_robin_irreps, uniform_pm1


# ------------------------------------------------------------ dense Schmidt spectrum

def det_to_fock(C, space, L):
    """Determinant coefficients (alpha strings x beta strings, creators ordered all alpha
    ascending, then all beta ascending) -> vector over the 4^L interleaved Jordan-Wigner
    basis (mode 2p = orbital p up, 2p+1 = down; mode 0 is the most significant bit).
    A creator on mode k picks up (-1)^(occupied modes before k)."""
    nm = 2 * L
    psi = np.zeros(4 ** L)
    for ia, a in enumerate(space.A.strs):
        for ib, b in enumerate(space.B.strs):
            c = C[ia, ib]
            if c == 0.0:
                continue
            modes = [2 * p for p in range(L) if (a >> p) & 1] + [2 * p + 1 for p in range(L) if (b >> p) & 1]
            state, sign = 0, 1.0
            for k in reversed(modes):  # the rightmost creator acts first
                bit = 1 << (nm - 1 - k)
                assert not state & bit
                before = state >> (nm - k)  # modes 0 .. k-1
                if bin(before).count("1") % 2:
                    sign = -sign
                state |= bit
            psi[state] += sign * c
    return psi


def left_labels(nl, irreps):
    """(N, 2Sz, irrep) of every basis state of the first nl orbitals."""
    out = []
    for idx in range(4 ** nl):
        n = tsz = ir = 0
        for p in range(nl):
            up = (idx >> (2 * nl - 1 - 2 * p)) & 1
            dn = (idx >> (2 * nl - 2 - 2 * p)) & 1
            n += up + dn
            tsz += up - dn
            if up + dn == 1:
                ir ^= irreps[p]
        out.append((n, tsz, ir))
    return out


def dense_multiplets(psi_ext, nl, irreps):
    """SU(2) multiplets (value, 2j, N, irrep) of the Schmidt decomposition of a state that
    is a singlet of (orbitals x the embedding spin), cut after nl orbitals.  A left
    multiplet of spin j appears once in every Sz sector -j..j of its (N, irrep) with the
    same Schmidt value; the spin-j ones are those of sector Sz=j not already present in
    Sz=j+1."""
    lab = left_labels(nl, irreps)
    vals = {}
    for key in set(lab):
        rows = [i for i, l in enumerate(lab) if l == key]
        s = np.linalg.svd(psi_ext[rows, :], compute_uv=False)
        vals[key] = sorted(s[s > 1e-12].tolist(), reverse=True)
    out = []
    for (n, tsz, ir), v in vals.items():
        if tsz < 0:
            continue
        above = list(vals.get((n, tsz + 2, ir), []))
        for x in v:
            j = min(range(len(above)), key=lambda k: abs(above[k] - x), default=None)
            if j is not None and abs(above[j] - x) < 1e-9:
                above.pop(j)
            else:
                out.append((x, tsz, n, ir))
        assert not above, "a higher-Sz value without its Sz=j partner"
    return sorted(out, reverse=True)


def ext_matrix(prob, m, i, x):
    """Psi_ext = sum_f |Psi_f>|f> as a matrix (first i+1 orbitals) x (rest, f)."""
    proj = M.TwoSiteProjector(m, i, prob.spaces)
    v = proj.flatten(x)
    L, nl = m.L, i + 1
    cols = []
    for f, P in enumerate(proj.P):
        space = prob.spaces[f]
        C = np.zeros(space.shape).ravel()
        C[prob.idx[f]] = (P @ v)[prob.idx[f]]
        psi = det_to_fock(C.reshape(space.shape), space, L)
        cols.append(psi.reshape(4 ** nl, 4 ** (L - nl)))
    return np.concatenate(cols, axis=1), proj


@pytest.mark.parametrize("N,two_S,I_G", [(6, 0, 0), (6, 2, 0), (5, 1, 3)])
def test_truncation_keeps_the_d_largest_multiplets(N, two_S, I_G):
    L, i = 6, 2
    irreps = round_robin_irreps(L)
    h, V = random_integrals(irreps, 31)
    prob = dmrg.Problem(h, V, irreps, N, two_S, I_G)
    m = M.right_canonicalize(M.random_mps(irreps, N, two_S, I_G, 400, uniform_pm1(17, 10 ** 6)))
    for k in range(i):
        M.svd_truncate(m, k, M.tt_to_x(m, k), 10 ** 9, "right")
    proj = M.TwoSiteProjector(m, i, prob.spaces)
    v = np.random.default_rng(N + two_S).normal(size=proj.n)
    x = proj.unflatten(v / np.linalg.norm(v))
    A, _ = ext_matrix(prob, m, i, x)
    assert abs(np.sum(A * A) - 1.0) < 1e-12
    dense = dense_multiplets(A, i + 1, irreps)
    # full spectrum: reduced singular values normalised as in Eq. 28 = dense multiplets
    _, _, groups = M.svd_truncate(m.copy(), i, {k: b.copy() for k, b in x.items()}, 10 ** 9, "right")
    norm2 = sum((g[0][0] + 1) * float(np.sum(g[6] ** 2)) for g in groups)
    red = sorted([(lam / np.sqrt(norm2), g[0][0], g[0][1], g[0][2]) for g in groups for lam in g[6]
                  if lam / np.sqrt(norm2) > 1e-12], reverse=True)
    assert len(red) == len(dense)
    for a, b in zip(red, dense):
        assert abs(a[0] - b[0]) < 1e-10 and a[1:] == b[1:]
    # selection and discarded weight for every D; one D must separate "largest lambda"
    # from "largest (2j+1) lambda^2" so that the rule is actually exercised
    separates = False
    for D in range(1, len(dense) + 1):
        keep = dense[:D]
        w_exp = sum((t + 1) * x0 ** 2 for x0, t, _, _ in dense[D:])
        by_weight = sorted(dense, key=lambda r: -(r[1] + 1) * r[0] ** 2)[:D]
        separates |= sorted(by_weight) != sorted(keep)
        w, kept, groups = M.svd_truncate(m.copy(), i, {k: b.copy() for k, b in x.items()}, D, "right")
        got = sorted([(-c[0] / np.sqrt(norm2), groups[c[1]][0][0], groups[c[1]][0][1], groups[c[1]][0][2])
                      for c in kept], reverse=True)
        assert len(got) == len(keep)
        for a, b in zip(got, keep):
            assert abs(a[0] - b[0]) < 1e-10 and a[1:] == b[1:]
        assert abs(w - w_exp) < 1e-12
    assert separates


# ------------------------------------------------------------ noise: Hubbard dimer

def dimer_mps(eps):
    """L=2, N=2, S=0 MPS with bond-1 sectors (0,0,0), (1,1,0), (0,2,0), each of
    dimension 1; its two-site vector is |20> plus O(eps) of the other states."""
    dims = [{(0, 0, 0): 1}, {(0, 0, 0): 1, (1, 1, 0): 1, (0, 2, 0): 1}, {(0, 2, 0): 1}]
    m = M.MPS([0, 0], 2, 0, 0, dims)
    m.T[0] = {(0, (0, 0, 0), (0, 0, 0)): np.array([[eps]]), (1, (0, 0, 0), (1, 1, 0)): np.array([[eps]]),
              (2, (0, 0, 0), (0, 2, 0)): np.array([[1.0]])}
    m.T[1] = {(2, (0, 0, 0), (0, 2, 0)): np.array([[1.0]]), (1, (1, 1, 0), (0, 2, 0)): np.array([[1.0]]),
              (0, (0, 2, 0), (0, 2, 0)): np.array([[1.0]])}
    return m


@pytest.mark.parametrize("gamma,w_prev", [(1.0, 1.0), (4.0, 0.25)])
def test_noise_branch_on_the_hubbard_dimer(gamma, w_prev):
    """Hubbard dimer (t=1, U=4): E0 = (U - sqrt(U^2 + 16 t^2)) / 2 with amplitudes
    |c_S| : |c_D| = 2t : |E0| on the covalent singlet and (|20> + |02>)/sqrt(2).  Noise r =
    e_{|20>} of amplitude a = 0.5 gamma w_prev gives |20> -> |c_D|/sqrt(2) + a (the
    oracle fixes the sign of the eigenvector by its overlap with the starting vector,
    which is |20> here).  At bond 1 the three reduced Schmidt values are |c_20|, |c_02|
    (spin 0) and |c_S| / sqrt(2) (spin 1/2, two components).  a = 0.5 puts kappa_20
    between kappa_S and sqrt(2) kappa_S: keeping D = 1 by lambda keeps |20>, by
    (2j+1) lambda^2 it would keep the singlet."""
    t, U = 1.0, 4.0
    E0 = (U - np.sqrt(U * U + 16 * t * t)) / 2
    cS = 2 * t / np.sqrt(4 * t * t + E0 * E0)
    cD = abs(E0) / np.sqrt(4 * t * t + E0 * E0)
    a = 0.5 * gamma * w_prev
    c20, c02 = cD / np.sqrt(2) + a, cD / np.sqrt(2)
    nrm2 = c20 ** 2 + c02 ** 2 + cS ** 2
    h, V = hubbard_chain(2, t, U)
    prob = dmrg.Problem(h, V, [0, 0], 2, 0, 0)
    blocks = M.two_site_blocks(dimer_mps(1e-3), 0)
    k20 = blocks.index(((0, 0, 0), 2, 0, 0, (0, 2, 0)))
    k02 = blocks.index(((0, 0, 0), 0, 2, 0, (0, 2, 0)))
    kS = blocks.index(((0, 0, 0), 1, 1, 0, (0, 2, 0)))
    r = np.zeros(len(blocks))
    r[k20] = 1.0
    # D = 3 keeps everything: T[0] T[1] is the normalised post-noise vector
    m = dimer_mps(1e-3)
    e, w = dmrg.micro_iteration(prob, m, 0, 3, "right", noise=gamma, noise_values=r, w_prev=w_prev)
    assert abs(e - E0) < 1e-12 and w < 1e-28
    xv = np.array([M.tt_to_x(m, 0)[b][0, 0] for b in blocks])
    assert abs(xv[k20] - c20 / np.sqrt(nrm2)) < 1e-12
    assert abs(abs(xv[k02]) - c02 / np.sqrt(nrm2)) < 1e-12
    assert abs(abs(xv[kS]) - cS / np.sqrt(nrm2)) < 1e-12
    # D = 1: the largest kappa (|20>) is kept, the rest is the discarded weight of Eq. 15
    m = dimer_mps(1e-3)
    e, w = dmrg.micro_iteration(prob, m, 0, 1, "right", noise=gamma, noise_values=r, w_prev=w_prev)
    kS_red, k20_red = cS / np.sqrt(2), c20
    assert k20_red > kS_red and c20 ** 2 < 2 * kS_red ** 2  # the case separates the two rules
    assert abs(w - (c02 ** 2 + cS ** 2) / nrm2) < 1e-12
    assert m.dims[1] == {(0, 2, 0): 1}
    x1 = M.tt_to_x(m, 0)
    assert abs(x1[blocks[k20]][0, 0] - c20 / np.sqrt(nrm2)) < 1e-12
    # without noise the same call keeps the singlet (largest lambda of the ground state)
    m = dimer_mps(1e-3)
    e, w = dmrg.micro_iteration(prob, m, 0, 1, "right")
    assert m.dims[1] == {(1, 1, 0): 1}
    assert abs(w - cD ** 2) < 1e-12


# ------------------------------------------------------------ initial distribution

# Hubbard chain L=4, N=4, S=0, C1, bond 2: FCI-capped reduced dimensions worked by hand.
# Two orbitals hold 1 (N=0), 2 doublets (N=1), 3 singlets + 1 triplet (N=2), 2 doublets
# (N=3), 1 singlet (N=4); a left sector pairs with the right sector of the same spin and
# complementary N, so the cap is min(left, right) of those counts.
HUB4_BOND2 = {(0, 0, 0): 1, (1, 1, 0): 2, (0, 2, 0): 3, (2, 2, 0): 1, (1, 3, 0): 2, (0, 4, 0): 1}
# D -> allocation in sector order (N, 2j, I), each worked by hand from "equal share to
# every open sector, capped, repeated on the remainder"
HUB4_TABLE = {
    4: [1, 1, 1, 1, 0, 0],    # share 4 // 6 = 0 -> one each, in order, until D is used
    8: [1, 2, 2, 1, 1, 1],    # one each (2 left), then one to the first two open sectors
    9: [1, 2, 2, 1, 2, 1],    # one each (3 left), then one to each of the 3 open sectors
    12: [1, 2, 3, 1, 2, 1],   # two each capped (9 used), then (0,2,0) reaches its cap
    40: [1, 2, 3, 1, 2, 1],   # every sector at its FCI dimension
}


def test_fci_caps_of_a_small_bond_worked_by_hand():
    assert M.fci_bond_dims([0] * 4, 4, 0, 0, 2) == HUB4_BOND2


@pytest.mark.parametrize("D", sorted(HUB4_TABLE))
def test_distribute_hand_table(D):
    order = M.sector_order(HUB4_BOND2)
    assert order == [(0, 0, 0), (1, 1, 0), (0, 2, 0), (2, 2, 0), (1, 3, 0), (0, 4, 0)]
    got = M.distribute(HUB4_BOND2, D)
    assert [got.get(s, 0) for s in order] == HUB4_TABLE[D]


def test_distribute_is_an_equal_spread_under_caps():
    """Max-min fairness: the total is min(D, sum of caps), no sector exceeds its cap, and
    a sector below its cap holds at least as much as any other sector minus one."""
    rng = np.random.default_rng(5)
    for _ in range(300):
        ns = int(rng.integers(1, 9))
        caps = {(int(t), int(n), 0): int(c) for t, n, c in zip(range(ns), range(ns),
                                                              rng.integers(1, 12, size=ns))}
        D = int(rng.integers(1, 60))
        a = M.distribute(caps, D)
        assert sum(a.values()) == min(D, sum(caps.values()))
        for s, v in a.items():
            assert 1 <= v <= caps[s]
        for s, c in caps.items():
            if a.get(s, 0) < c:
                assert all(v <= a.get(s, 0) + 1 for v in a.values())

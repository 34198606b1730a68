"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (FP64 path): matvec relative error <= 1e-12 element by element (the
relative error of a sum of ~1e3 rounded products of O(1) terms is ~1e-15; 1e-12 leaves
room for cancellation), Davidson eigenvalue within 1e-9 of the dense eigenvalue
(residual tolerance 1e-10), sweep energies within 1e-8 Eh of the oracle DMRG."""
import json
import os

import numpy as np
import pytest

from oracle import dmrg as odmrg
from oracle import mps as om
from oracle.fci import fci_ground_state
from tests.mps_io import lib_x_to_oracle, mps_to_bytes, oracle_x_to_lib, truncation_bound, widest_cut
from workloads import (hubbard_chain, make_problem, random_integrals, round_robin_irreps,
                       uniform_pm1)

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "energies.json")


@pytest.fixture(scope="module")
def Context():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1312_2415_gb300 import Context as C
    return C


def setup(kind, L, N, tS, IG, D, seed, center):
    if kind == "hubbard":
        irr = [0] * L
        h, V = hubbard_chain(L, 1.0, 4.0)
    else:
        irr = round_robin_irreps(L)
        h, V = random_integrals(irr, 11)
    m = om.right_canonicalize(om.random_mps(irr, N, tS, IG, D, uniform_pm1(seed, 10 ** 6)))
    for k in range(center):
        om.svd_truncate(m, k, om.tt_to_x(m, k), 10 ** 9, "right")
    prob = odmrg.Problem(h, V, irr, N, tS, IG)
    return irr, h, V, m, prob


CASES = [("hubbard", 8, 8, 0, 0, 40), ("random", 6, 6, 2, 0, 40), ("random", 6, 5, 1, 3, 40),
         ("random", 7, 6, 0, 1, 40), ("random", 8, 8, 0, 0, 60), ("hubbard", 7, 7, 1, 0, 30)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}L{c[1]}N{c[2]}S{c[3]}I{c[4]}")
def test_matvec_diag_and_eq25_match_oracle(Context, case):
    kind, L, N, tS, IG, D = case
    for i in sorted({0, L // 2 - 1, L - 2}):
        irr, h, V, m, prob = setup(kind, L, N, tS, IG, D, 3, i)
        H, G, proj = odmrg.effective_hamiltonian(prob, m, i)
        ctx = Context(L, irr, N, tS, IG)
        ctx.set_integrals(h, V)
        ctx.set_mps(mps_to_bytes(m))
        n, table = ctx.layout(i)
        assert n == proj.n
        # Eq. 25
        x = ctx.tt_to_x(i)
        xo = oracle_x_to_lib(om.tt_to_x(m, i), table, n)
        assert np.abs(x - xo).max() <= 1e-13 * max(1.0, np.abs(xo).max())
        # H_eff x for random x, element by element
        rng = np.random.default_rng(i)
        v = rng.normal(size=n)
        y = ctx.matvec(i, v)
        yo = oracle_x_to_lib(proj.unflatten(H @ proj.flatten(lib_x_to_oracle(v, table))), table, n)
        assert np.abs(y - yo).max() <= 1e-12 * np.abs(yo).max()
        # diagonal (Davidson preconditioner)
        d = ctx.diag(i)
        do = oracle_x_to_lib(proj.unflatten(np.diag(H).copy()), table, n)
        assert np.abs(d - do).max() <= 1e-12 * np.abs(do).max()
        # lowest eigenpair
        x0 = ctx.tt_to_x(i)
        e, it, ok = ctx.davidson(i, x0)
        w, U = np.linalg.eigh(H)
        assert ok and abs(e - w[0]) < 1e-9
        u = proj.flatten(lib_x_to_oracle(x0, table))
        assert abs(abs(u @ U[:, 0]) - 1.0) < 1e-8


@pytest.mark.parametrize("case", CASES[:4], ids=lambda c: f"{c[0]}L{c[1]}N{c[2]}S{c[3]}I{c[4]}")
@pytest.mark.parametrize("direction", [1, -1])
def test_truncation_matches_oracle(Context, case, direction):
    """Eqs. 26-28: the discarded weight and the truncated two-site tensor (gauge
    invariant) agree with the oracle.  A cut of the ground state at the widest gap of its
    reduced spectrum between D = 2 and 6 forces a real truncation; a random unit vector (full rank,
    no values near the library's zero threshold) is decomposed without a cut.  The
    tolerance is the Davis-Kahan bound of the library's Gram route (tests/mps_io), asserted
    to be small itself."""
    kind, L, N, tS, IG, D = case
    i = L // 2 - 1
    irr, h, V, m, prob = setup(kind, L, N, tS, IG, D, 7, i)
    H, _, proj = odmrg.effective_hamiltonian(prob, m, i)
    w, U = np.linalg.eigh(H)
    vec = proj.unflatten(U[:, 0])
    ctx = Context(L, irr, N, tS, IG)
    ctx.set_integrals(h, V)
    ctx.set_mps(mps_to_bytes(m))
    n, table = ctx.layout(i)
    x = oracle_x_to_lib(vec, table, n)
    # the cut between D = 2 and 6 with the widest gap of the reduced spectrum (stated
    # minimum: 1e-4 of lambda_max^2)
    _, _, full = om.svd_truncate(m.copy(), i, {k: v.copy() for k, v in vec.items()}, 10 ** 9, "right")
    cut, rel_gap = widest_cut(full, 4, 2)
    assert rel_gap > 1e-4, rel_gap
    rnd = np.random.default_rng(direction + 31).normal(size=n)
    rnd /= np.linalg.norm(rnd)
    for Dt, xv in ((cut, x), (10 ** 6, rnd)):
        m2 = m.copy()
        wd_o, kept, groups = om.svd_truncate(m2, i, lib_x_to_oracle(xv, table), Dt,
                                             "right" if direction > 0 else "left")
        ctx.set_mps(mps_to_bytes(m))
        wd = ctx.truncate(i, direction, Dt, xv)
        assert abs(wd - wd_o) < 1e-12
        xl = ctx.tt_to_x(i)
        xo = oracle_x_to_lib(om.tt_to_x(m2, i), table, n)
        # Davis-Kahan bound of the library's Gram route plus the weight of values it
        # treats as zero (tests/mps_io.truncation_bound), asserted small itself
        tol = truncation_bound(groups, Dt)
        assert tol < 1e-9, (Dt, tol)
        assert np.abs(xl - xo).max() < tol


@pytest.mark.parametrize("case", [("hubbard", 6, 6, 0, 0, 8, 3), ("random", 6, 6, 2, 0, 6, 3),
                                  ("random", 7, 6, 0, 1, 200, 2), ("random", 6, 5, 1, 3, 5, 2)])
def test_sweeps_match_oracle_dmrg(Context, case):
    kind, L, N, tS, IG, D, nsw = case
    irr, h, V, m, prob = setup(kind, L, N, tS, IG, D, 5, 0)
    data = mps_to_bytes(m)
    eo, es = odmrg.sweep(prob, m.copy(), D, nsw)
    ctx = Context(L, irr, N, tS, IG)
    ctx.set_integrals(h, V, econst=0.25)
    ctx.set_schedule([D], [0.0], [nsw], [0.0], 1e-10, 200)
    ctx.set_mps(data)
    emin, elast = ctx.solve()
    assert abs(emin - 0.25 - eo) < 1e-8
    assert abs(elast - 0.25 - es[-1]) < 1e-8


def test_hubbard8_d64_six_sweeps_golden(Context):
    """Hubbard L=8, N=8, S=0, U=4, D=64, 6 macro-iterations, Davidson tol 1e-10,
    against the oracle's value stored by tests/golden/make_golden.py; also bounded by
    FCI (variational)."""
    gold = json.load(open(GOLDEN))
    cfg, h, V = make_problem("hubbard8")
    irr = cfg["group_irreps"]
    m = om.right_canonicalize(om.random_mps(irr, 8, 0, 0, 64, uniform_pm1(2415001, 10 ** 6)))
    ctx = Context(8, irr, 8, 0, 0)
    ctx.set_integrals(h, V)
    ctx.set_schedule([64], [0.0], [6], [0.0], 1e-10, 200)
    ctx.set_mps(mps_to_bytes(m))
    emin, elast = ctx.solve()
    assert abs(emin - gold["hubbard8_dmrg_d64"]["e_min"]) < 1e-8
    assert emin >= gold["hubbard8_fci"]["e"] - 1e-10


def test_full_d_equals_fci_and_u0_closed_form(Context):
    for U, want in ((4.0, None), (0.0, 2 * sum(-2 * np.cos(k * np.pi / 9) for k in range(1, 5)))):
        h, V = hubbard_chain(8, 1.0, U)
        if want is None:
            want = fci_ground_state(h, V, 8, 0, [0] * 8, 0)[0][0]
        ctx = Context(8, [0] * 8, 8, 0, 0)
        ctx.set_integrals(h, V)
        ctx.set_schedule([126], [1e-12], [4], [0.0], 1e-10, 200)
        ctx.init_mps(99)
        emin, elast = ctx.solve()
        assert abs(emin - want) < 1e-8


@pytest.mark.parametrize("case", CASES[:4], ids=lambda c: f"{c[0]}L{c[1]}N{c[2]}S{c[3]}I{c[4]}")
def test_energy_symmetric_form_matches_oracle(Context, case):
    """dmrg_energy: the sweep's FP64 energy from the block pairs of input block >= output
    block (H_eff symmetric, the others' share counted twice) equals the oracle's
    x . (P^T H P x) / x . x and the library's own x . (H x) (FP64 matvec) for a random
    vector, in both precision modes (the energy is FP64 in both).  Tolerance: 1e-12 of
    |H x| / |x|, the matvec's own bound carried through the dot product."""
    kind, L, N, tS, IG, D = case
    for i in sorted({0, L // 2 - 1, L - 2}):
        irr, h, V, m, prob = setup(kind, L, N, tS, IG, D, 3, i)
        H, _, proj = odmrg.effective_hamiltonian(prob, m, i)
        for prec in (0, 1):
            ctx = Context(L, irr, N, tS, IG, precision=prec)
            ctx.set_integrals(h, V)
            ctx.set_mps(mps_to_bytes(m))
            n, table = ctx.layout(i)
            v = np.random.default_rng(i + 17).normal(size=n)
            yo = oracle_x_to_lib(proj.unflatten(H @ proj.flatten(lib_x_to_oracle(v, table))), table, n)
            eo = (v @ yo) / (v @ v)
            bound = 1e-12 * np.linalg.norm(yo) / np.linalg.norm(v)
            e = ctx.energy(i, v)
            assert abs(e - eo) <= bound, (e, eo, bound)
            ctx.set_precision(0, 0)
            y = ctx.matvec(i, v)
            assert abs(e - (v @ y) / (v @ v)) <= bound

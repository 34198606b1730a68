"""Noise before the decomposition (Sec. 4.2) and the initial MPS (Sec. 4.3) against the
oracle.

Noise: the library adds, to the Davidson vector x of a sweep step, uniform noise of
amplitude 0.5 gamma w_prev, w_prev the largest discarded weight of the previous half
sweep, drawn from a counter-based stream (element i of the k-th noisy step since the MPS
was loaded: splitmix64 of 0x5eed0000 + k * 1000003 + i).  The test redraws those values
on the host (`workloads.counter_uniform_pm1`) and feeds them to the oracle's
`micro_iteration(noise_values=...)`.  The GPU's and the oracle's renormalised bases differ
by the signs their decompositions choose, so before each noisy step the oracle takes the
library's own MPS (dmrg_get_mps): the noise then lands on the same basis vectors.
Compared: the energy (Davidson tol 1e-12 against dense eigh: 1e-9), the discarded weight
(1e-10) and the truncated two-site vector, element by element (1e-8 of its largest
element; both are the projection of the same noisy vector onto its D largest reduced
Schmidt values)."""
import numpy as np
import pytest

from oracle import dmrg as odmrg
from oracle import mps as om
from tests.mps_io import lib_x_to_oracle, mps_from_bytes, mps_to_bytes, oracle_x_to_lib
from workloads import (counter_uniform_pm1, hubbard_chain, make_problem, random_integrals,
                       round_robin_irreps, uniform_pm1)

pytestmark = pytest.mark.gpu

NOISE_SEED, NOISE_STRIDE = 0x5EED0000, 1000003


@pytest.fixture(scope="module")
def Context():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1312_2415_gb300 import Context as C
    return C


def system(kind, L, seed=11):
    if kind == "hubbard":
        irr = [0] * L
        h, V = hubbard_chain(L, 1.0, 4.0)
    else:
        irr = round_robin_irreps(L)
        h, V = random_integrals(irr, seed)
    return irr, h, V


@pytest.mark.parametrize("case", [("hubbard", 6, 6, 0, 0, 6, 50.0), ("random", 6, 6, 2, 0, 5, 20.0),
                                  ("random", 7, 6, 0, 1, 8, 5.0)],
                         ids=lambda c: f"{c[0]}L{c[1]}N{c[2]}S{c[3]}I{c[4]}D{c[5]}")
def test_noisy_half_sweep_matches_oracle(Context, case):
    kind, L, N, tS, IG, D, gamma = case
    irr, h, V = system(kind, L)
    prob = odmrg.Problem(h, V, irr, N, tS, IG)
    m0 = om.right_canonicalize(om.random_mps(irr, N, tS, IG, D, uniform_pm1(5, 10 ** 6)))
    ctx = Context(L, irr, N, tS, IG)
    ctx.set_integrals(h, V)
    ctx.set_schedule([D], [0.0], [1], [gamma], 1e-12, 400)
    ctx.set_mps(mps_to_bytes(m0))
    # right half sweep: no previous half sweep, so no noise yet
    mo = m0.copy()
    wmax = 0.0
    for i in range(L - 1):
        e, w, it, ok = ctx.sweep_step(i, 1, D, gamma)
        eo, wo = odmrg.micro_iteration(prob, mo, i, D, "right")
        assert ok and abs(e - eo) < 1e-9 and abs(w - wo) < 1e-10
        wmax = max(wmax, wo)
    assert wmax > 1e-6, "the case must truncate for the noise to be nonzero"
    # left half sweep: noise of amplitude 0.5 gamma wmax before every decomposition
    for k, i in enumerate(range(L - 2, 0, -1)):
        mg = mps_from_bytes(ctx.get_mps(), irr)
        n, table = ctx.layout(i)
        rb = lib_x_to_oracle(counter_uniform_pm1(NOISE_SEED + k * NOISE_STRIDE, n), table)
        keys = om.two_site_blocks(mg, i)
        assert set(keys) == set(rb)
        r = np.concatenate([rb[key].ravel() for key in keys])
        e, w, it, ok = ctx.sweep_step(i, -1, D, gamma)
        clean = mg.copy()
        _, w_clean = odmrg.micro_iteration(prob, clean, i, D, "left")
        eo, wo = odmrg.micro_iteration(prob, mg, i, D, "left", noise=gamma, noise_values=r, w_prev=wmax)
        assert ok and abs(e - eo) < 1e-9
        assert abs(w - wo) < 1e-10, (i, w, wo)
        n2, table2 = ctx.layout(i)
        x = ctx.tt_to_x(i)
        xo = oracle_x_to_lib(om.tt_to_x(mg, i), table2, n2)
        assert np.abs(x - xo).max() <= 1e-8 * np.abs(xo).max()
        if k == 0:
            # the noise is visible: the noisy step differs from the noiseless one
            xc = oracle_x_to_lib(om.tt_to_x(clean, i), table2, n2)
            assert np.abs(xc - xo).max() > 1e-3 * np.abs(xo).max()


@pytest.mark.parametrize("workload,D", [("hubbard8", 24), ("random12", 120), ("random28", 2500)])
def test_initial_mps_is_the_oracles_bit_for_bit(Context, workload, D):
    """Sec. 4.3: D spread equally over the sectors of every bond (capped by the FCI
    dimension), filled from splitmix64(seed) site by site, block by block, row-major.
    Integer layout and values are compared exactly."""
    cfg, h, V = make_problem(workload)
    irr = cfg["group_irreps"]
    ctx = Context(cfg["L"], irr, cfg["N"], cfg["two_S"], cfg["irrep"])
    ctx.set_integrals(h, V)
    ctx.set_schedule([D], [0.0], [1], [0.0], 1e-10, 10)
    seed = 2415 + D
    ctx.init_mps(seed)
    got = mps_from_bytes(ctx.get_mps(), irr)
    dims = om.initial_dims(irr, cfg["N"], cfg["two_S"], cfg["irrep"], D)
    total = sum(dims[k][b[1]] * dims[k + 1][b[2]]
                for k in range(cfg["L"]) for b in om.MPS(irr, cfg["N"], cfg["two_S"], cfg["irrep"], dims).blocks(k))
    want = om.random_mps(irr, cfg["N"], cfg["two_S"], cfg["irrep"], D, uniform_pm1(seed, total))
    assert got.dims == want.dims
    for k in range(cfg["L"]):
        assert set(got.T[k]) == set(want.T[k])
        for key, blk in want.T[k].items():
            assert np.array_equal(got.T[k][key], blk)


def test_decomposed_step_equals_sweep_step(Context):
    """dmrg_tt_to_x, dmrg_davidson, dmrg_truncate and dmrg_update_operators through host
    buffers do the work of one dmrg_sweep_step: the next steps see the same operators
    (their energies agree with the one-call path and with the oracle's sweep)."""
    L, N, D = 7, 6, 12
    irr, h, V = system("random", L, 3)
    prob = odmrg.Problem(h, V, irr, N, 0, 1)
    m0 = om.right_canonicalize(om.random_mps(irr, N, 0, 1, D, uniform_pm1(9, 10 ** 6)))
    ctxs = []
    for _ in range(2):
        c = Context(L, irr, N, 0, 1)
        c.set_integrals(h, V)
        c.set_schedule([D], [0.0], [1], [0.0], 1e-12, 400)
        c.set_mps(mps_to_bytes(m0))
        ctxs.append(c)
    a, b = ctxs
    mo = m0.copy()
    for i in range(L - 1):
        ea, wa, _, oka = a.sweep_step(i, 1, D)
        x = b.tt_to_x(i)
        eb, _, okb = b.davidson(i, x)
        wb = b.truncate(i, 1, D, x)
        b.update_operators(i, 1)
        eo, wo = odmrg.micro_iteration(prob, mo, i, D, "right")
        assert oka and okb
        assert abs(ea - eo) < 1e-9 and abs(eb - eo) < 1e-9 and abs(wa - wb) < 1e-12 and abs(wa - wo) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_next_site_hint_does_not_change_results(Context, precision):
    """dmrg_set_next_site only changes when tables are built (a step at the same site
    keeps them; another site's are built while the step finishes): a sweep with hints
    gives the energies and discarded weights of the same sweep without them."""
    L, N, D = 8, 8, 20
    irr, h, V = system("random", L, 4)
    m0 = om.right_canonicalize(om.random_mps(irr, N, 0, 0, D, uniform_pm1(12, 10 ** 6)))
    out = []
    for hint in (False, True):
        c = Context(L, irr, N, 0, 0, precision=precision)
        c.set_integrals(h, V)
        c.set_schedule([D], [0.0], [1], [0.0], 1e-12, 400)
        c.set_mps(mps_to_bytes(m0))
        seq = [(i, 1) for i in range(L - 1)] + [(i, -1) for i in range(L - 2, -1, -1)] + [(0, 1), (1, 1)]
        res = []
        for k, (i, d) in enumerate(seq):
            if hint and k + 1 < len(seq):
                c.set_next_site(seq[k + 1][0])
            e, w, it, ok = c.sweep_step(i, d, D)
            res.append((e, w))
        out.append(np.array(res))
    assert np.abs(out[0] - out[1]).max() < 1e-10

"""Mixed-precision path (precision 1): block products on the tcgen05 tensor cores in
split TF32 (a = a_hi + a_lo, three products, FP32 accumulation), Davidson finished by
FP64 iterations.

Tolerances.  One split-TF32 product has a relative error of about 2^-21 (5e-7); the
accumulators are promoted to FP32 registers every two 32-wide K chunks, so the sums add
little to it (measured 5.5e-7 of max|y| at L=28, D=2500).  The matvec is held to 2e-6
relative to max|y|: four times the measured level, so that a lost promotion (1e-5
measured with 48-task runs) or a dropped split term (2^-11) fails.
Energies are FP64 Rayleigh quotients after the FP64 iterations, held to the 1e-6 Eh
target of the mixed path (and reported)."""
import numpy as np
import pytest

from oracle import dmrg as odmrg
from oracle import mps as om
from tests.mps_io import lib_x_to_oracle, mps_to_bytes, oracle_x_to_lib
from tests.test_gpu_parity import setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    import torch
    assert torch.cuda.is_available()
    from paper_1312_2415_gb300 import Context as C
    return C


CASES = [("hubbard", 8, 8, 0, 0, 40), ("random", 8, 8, 0, 0, 60), ("random", 6, 5, 1, 3, 40),
         ("random", 7, 6, 0, 1, 40)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}L{c[1]}N{c[2]}S{c[3]}I{c[4]}")
def test_tensor_core_matvec_and_energy(Context, case):
    kind, L, N, tS, IG, D = case
    i = L // 2 - 1
    irr, h, V, m, prob = setup(kind, L, N, tS, IG, D, 3, i)
    H, _, proj = odmrg.effective_hamiltonian(prob, m, i)
    ctx = Context(L, irr, N, tS, IG, precision=1)
    ctx.set_integrals(h, V)
    ctx.set_schedule([D], [0.0], [1], [0.0], 1e-10, 200)
    ctx.set_mps(mps_to_bytes(m))
    n, table = ctx.layout(i)
    v = np.random.default_rng(2).normal(size=n)
    y = ctx.matvec(i, v)
    yo = oracle_x_to_lib(proj.unflatten(H @ proj.flatten(lib_x_to_oracle(v, table))), table, n)
    err = np.abs(y - yo).max() / np.abs(yo).max()
    assert err <= 2e-6, err
    assert err > 0.0  # it really ran in reduced precision
    x = ctx.tt_to_x(i)
    e, it, ok = ctx.davidson(i, x)
    w = np.linalg.eigvalsh(H)[0]
    assert ok and abs(e - w) <= 1e-6, (e, w)
    st = ctx.stats()
    assert st["tc_matvecs"] > 0


def test_tensor_core_sweeps_match_oracle(Context):
    kind, L, N, tS, IG, D, nsw = ("random", 7, 6, 0, 1, 40, 2)
    irr, h, V, m, prob = setup(kind, L, N, tS, IG, D, 5, 0)
    eo, es = odmrg.sweep(prob, m.copy(), D, nsw)
    ctx = Context(L, irr, N, tS, IG, precision=1)
    ctx.set_integrals(h, V)
    ctx.set_schedule([D], [0.0], [nsw], [0.0], 1e-10, 200)
    ctx.set_mps(mps_to_bytes(m))
    emin, elast = ctx.solve()
    assert abs(emin - eo) <= 1e-6

"""Synthetic ab initio system L=12, N=12, S=0, Ag, D2h irreps round-robin, random
integrals (seed 2415012), D_SU(2)=500: the FP64 sweep energy is a variational upper
bound of the oracle's FCI energy (107120 determinants, tests/golden/energies.json),
and the mixed-precision sweep (split-TF32 tensor-core matvecs, Davidson finished in
FP64) reaches the FP64 sweep's energy to 1e-6 Eh from the same initial MPS."""
import json
import os

import pytest

from workloads import make_problem

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "energies.json")))


@pytest.fixture(scope="module")
def Context():
    import torch
    assert torch.cuda.is_available()
    from paper_1312_2415_gb300 import Context as C
    return C


def _solve(Context, precision):
    cfg, h, V = make_problem("random12")
    ctx = Context(cfg["L"], cfg["group_irreps"], cfg["N"], cfg["two_S"], cfg["irrep"], group=7,
                  precision=precision)
    ctx.set_integrals(h, V)
    ctx.set_schedule([cfg["D"]], [1e-10], [4], [0.0], 1e-9, 200)
    ctx.set_precision(precision, 0)
    ctx.init_mps(cfg["seed"])
    return ctx.solve()


def test_random12_d500_variational_and_mixed(Context):
    e_fci = GOLD["random12_fci"]["e"]
    e64, _ = _solve(Context, 0)
    assert e64 >= e_fci - 1e-10, (e64, e_fci)
    assert e64 - e_fci < 1e-2, (e64, e_fci)  # D=500 is far from the FCI-capped 1676
    e32, _ = _solve(Context, 1)
    assert abs(e32 - e64) <= 1e-6, (e32, e64)

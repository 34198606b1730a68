"""Sec. 4.3 / Eq. 16 on the GPU path: a convergence scheme with increasing D on the
Hubbard chain L=8 (t=1, U=4, N=8, S=0) records per instruction the energy and the
largest discarded weight of its last macro-iteration; every energy lies above the
oracle's FCI energy and the extrapolation E_exact of Eq. 16 lands closer to it than the
largest-D energy."""
import json
import os

import pytest

from workloads import hubbard_chain

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "energies.json")))


def test_energy_extrapolation_towards_fci():
    import torch
    assert torch.cuda.is_available()
    from paper_1312_2415_gb300 import Context, extrapolate
    e_fci = GOLD["hubbard8_fci"]["e"]
    h, V = hubbard_chain(8, 1.0, 4.0)
    ctx = Context(8, [0] * 8, 8, 0, 0)
    ctx.set_integrals(h, V)
    Ds = [8, 10, 12, 14]  # below the chain's Schmidt rank: energies 3e-3 .. 4e-5 Eh above FCI
    ctx.set_schedule(Ds, [1e-9] * 4, [6] * 4, [0.0] * 4, 1e-10, 200)
    ctx.init_mps(5)
    ctx.solve()
    D, E, W = ctx.solve_history()
    assert list(D) == Ds
    assert all(e >= e_fci - 1e-10 for e in E)
    assert all(W[k] > W[k + 1] for k in range(3))
    e0, c1 = extrapolate(W, E)
    assert c1 > 0.0
    assert abs(e0 - e_fci) < 0.1 * abs(E[-1] - e_fci), (e0, E[-1], e_fci)

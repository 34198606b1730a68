"""Degenerate and extreme cases of the method against the oracle's FCI (exact D):

* the smallest chain (L=2, a single site pair) with 2, 3 and 4 electrons, against the
  Hubbard dimer's closed form and FCI;
* N = 2 (the smallest N the folding of Eq. 11 allows) and N = 2L (one determinant: the
  bonds are one-dimensional, D = 1 is exact);
* the largest spin of a sector (S = N/2) and an empty target sector (rejected);
* D = 1 (a product of one multiplet per bond): variational, above FCI."""
import math

import numpy as np
import pytest

from oracle.fci import fci_ground_state
from workloads import hubbard_chain, random_integrals, round_robin_irreps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1312_2415_gb300 import Context as C
    return C


def _solve(Context, L, irr, N, tS, IG, h, V, D=64, precision=0):
    ctx = Context(L, irr, N, tS, IG)
    ctx.set_integrals(h, V)
    ctx.set_schedule([D], [1e-12], [4], [0.0], 1e-11, 200)
    ctx.set_precision(precision, 0)
    ctx.init_mps(5)
    return ctx.solve()[0]


@pytest.mark.parametrize("precision", [0, 1])
def test_dimer(Context, precision):
    for U in (0.0, 4.0):
        h, V = hubbard_chain(2, 1.0, U)
        e = _solve(Context, 2, [0, 0], 2, 0, 0, h, V, precision=precision)
        assert abs(e - (U - math.sqrt(U * U + 16.0)) / 2) < 1e-9
    h, V = hubbard_chain(2, 1.0, 4.0)
    for N, tS in ((3, 1), (4, 0)):
        ref = fci_ground_state(h, V, N, tS, [0, 0], 0)[0][0]
        assert abs(_solve(Context, 2, [0, 0], N, tS, 0, h, V, precision=precision) - ref) < 1e-9


def test_two_electrons_and_full_filling(Context):
    L = 5
    irr = round_robin_irreps(L)
    h, V = random_integrals(irr, 7)
    for N, tS, IG in ((2, 0, 0), (2, 2, 3), (2 * L, 0, 0)):
        ref = fci_ground_state(h, V, N, tS, irr, IG)[0][0]
        D = 1 if N == 2 * L else 64
        assert abs(_solve(Context, L, irr, N, tS, IG, h, V, D=D) - ref) < 1e-9


def test_highest_spin_and_empty_sector(Context):
    from paper_1312_2415_gb300 import DMRGError
    L = 4
    h, V = hubbard_chain(L, 1.0, 4.0)
    ref = fci_ground_state(h, V, 4, 4, [0] * L, 0)[0][0]
    assert abs(_solve(Context, L, [0] * L, 4, 4, 0, h, V) - ref) < 1e-9
    # D2h orbitals 0..3 with one electron: no state of irrep 4 exists
    irr = [0, 1, 2, 3]
    h2, V2 = random_integrals(irr, 3)
    ctx = Context(L, irr, 1 + 1, 0, 4, group=7)
    ctx.set_integrals(h2, V2)
    ctx.set_schedule([16], [0.0], [1], [0.0], 1e-10, 50)
    with pytest.raises(DMRGError):
        ctx.init_mps(1)


def test_d1_is_variational(Context):
    L, N = 6, 6
    h, V = hubbard_chain(L, 1.0, 4.0)
    ref = fci_ground_state(h, V, N, 0, [0] * L, 0)[0][0]
    e = _solve(Context, L, [0] * L, N, 0, 0, h, V, D=1)
    assert e >= ref - 1e-10
    assert np.isfinite(e)

"""Eqs. 26-28 on blocks above the shared-memory eigensolver's limit (Gram matrices of
105-210 rows at the middle of a Hubbard chain L=12, D=1500), which the library
diagonalises with the one-sided block Jacobi: the discarded weight (Eq. 15) and the
truncated two-site tensor (gauge invariant) against the oracle's numpy SVD of the
same blocks, in both sweep directions, with and without a cut (the cut placed at the
widest gap of the reduced spectrum near D = 700, so that the truncation is well
defined; the tolerance is the Davis-Kahan bound of the Gram route, asserted small)."""
import numpy as np
import pytest

from oracle import mps as om
from tests.mps_io import lib_x_to_oracle, mps_to_bytes, oracle_x_to_lib, truncation_bound, widest_cut
from workloads import hubbard_chain, uniform_pm1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    import torch
    assert torch.cuda.is_available()
    from paper_1312_2415_gb300 import Context as C
    return C


@pytest.fixture(scope="module")
def state():
    L, N, D = 12, 12, 1500
    i = L // 2 - 1
    irr = [0] * L
    h, V = hubbard_chain(L, 1.0, 4.0)
    m = om.right_canonicalize(om.random_mps(irr, N, 0, 0, D, uniform_pm1(12, 10 ** 7)))
    for k in range(i):
        om.svd_truncate(m, k, om.tt_to_x(m, k), 10 ** 9, "right")
    return L, N, irr, h, V, m, i


@pytest.mark.parametrize("direction", [1, -1])
def test_large_block_truncation_matches_oracle(Context, state, direction):
    L, N, irr, h, V, m, i = state
    ctx = Context(L, irr, N, 0, 0)
    ctx.set_integrals(h, V)
    ctx.set_mps(mps_to_bytes(m))
    n, table = ctx.layout(i)
    x = np.random.default_rng(direction + 5).normal(size=n)
    x /= np.linalg.norm(x)
    # the cut near D = 700 with the widest gap in the reduced spectrum (stated minimum:
    # 1e-6 of lambda_max^2, which bounds the Davis-Kahan term by ~1.4e-8)
    _, _, full = om.svd_truncate(m.copy(), i, lib_x_to_oracle(x, table), 10 ** 9, "right")
    cut, rel_gap = widest_cut(full, 700, 40)
    assert rel_gap > 1e-6, rel_gap
    for Dt in (cut, 10 ** 6):
        m2 = m.copy()
        wd_o, kept, groups = om.svd_truncate(m2, i, lib_x_to_oracle(x, table), Dt,
                                             "right" if direction > 0 else "left")
        ctx.set_mps(mps_to_bytes(m))
        wd = ctx.truncate(i, direction, Dt, x)
        assert abs(wd - wd_o) < 1e-12, (Dt, wd, wd_o)
        xl = ctx.tt_to_x(i)
        xo = oracle_x_to_lib(om.tt_to_x(m2, i), table, n)
        tol = truncation_bound(groups, Dt)
        assert tol < 2e-8, (Dt, tol)  # the bound itself is small: the comparison is meaningful
        assert np.abs(xl - xo).max() < tol, (Dt, np.abs(xl - xo).max(), tol)

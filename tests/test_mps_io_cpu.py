"""The helpers every GPU parity test relies on to move states between the oracle and the
library (tests/mps_io.py), checked on the CPU: the serialised MPS (the dmrg_set_mps /
dmrg_get_mps format) round-trips an oracle MPS exactly, including sectors, dimensions
and every block; the two-site block table maps oracle blocks to the library's flat
vector and back without loss, and a block missing from one side is zero on the other;
the truncation tolerance shrinks as the gap at the cut opens; the cut search finds the
largest gap of the reduced spectrum."""
import struct

import numpy as np

from oracle import mps as om
from tests.mps_io import (layout_keys, lib_x_to_oracle, mps_from_bytes, mps_to_bytes, oracle_x_to_lib,
                          truncation_bound, widest_cut)
from workloads import round_robin_irreps, uniform_pm1


def _random_state():
    irr = round_robin_irreps(6)
    return om.right_canonicalize(om.random_mps(irr, 6, 2, 1, 20, uniform_pm1(9, 10 ** 5)))


def test_mps_bytes_round_trip():
    m = _random_state()
    data = mps_to_bytes(m)
    magic, ver, L, N, two_S, I_G = struct.unpack_from("<6i", data, 0)
    assert (magic, ver, L, N, two_S, I_G) == (0x444D5247, 1, m.L, m.N, m.two_S, m.I_G)
    m2 = mps_from_bytes(data, m.irreps)
    assert m2.dims == m.dims
    for k in range(m.L):
        assert set(m2.T[k]) == set(m.T[k])
        for key, blk in m.T[k].items():
            assert np.array_equal(m2.T[k][key], blk)
    assert mps_to_bytes(m2) == data


def _table(m, i):
    """A block table in the library's row format (tjL nL iL ls1 ls2 tj tjR nR iR dL dR off)
    for the oracle's two-site blocks, in an order other than the oracle's."""
    rows, off = [], 0
    for key in reversed(om.two_site_blocks(m, i)):
        lsec, ls1, ls2, tj, rsec = key
        dL, dR = m.dims[i][lsec], m.dims[i + 2][rsec]
        rows.append([*lsec, ls1, ls2, tj, *rsec, dL, dR, off])
        off += dL * dR
    return np.array(rows, dtype=np.int64), off


def test_two_site_layout_round_trip():
    m = _random_state()
    i = 2
    table, n = _table(m, i)
    x = om.tt_to_x(m, i)
    assert set(layout_keys(table)) == set(x)
    v = oracle_x_to_lib(x, table, n)
    assert v.shape == (n,) and np.count_nonzero(v) > 0
    back = lib_x_to_oracle(v, table)
    for key, blk in x.items():
        assert np.array_equal(back[key], blk)
    # every element of the flat vector belongs to exactly one block
    w = np.arange(n, dtype=np.float64)
    assert np.array_equal(oracle_x_to_lib(lib_x_to_oracle(w, table), table, n), w)
    # a block the oracle does not hold is zero in the library's vector
    drop = next(iter(x))
    v2 = oracle_x_to_lib({k: b for k, b in x.items() if k != drop}, table, n)
    assert np.all(lib_x_to_oracle(v2, table)[drop] == 0.0)


def test_truncation_bound_and_cut():
    # groups in the layout truncation_bound reads: g[0][0] = 2j of the sector, g[6] = values
    def groups(vals):
        return [((0,), None, None, None, None, None, np.array(vals))]
    wide = groups([1.0, 0.9, 0.8, 0.1, 0.05])
    narrow = groups([1.0, 0.9, 0.8, 0.79, 0.05])
    assert truncation_bound(wide, 3) < truncation_bound(narrow, 3)
    # well separated cut: the bound is at the level of rounding
    assert truncation_bound(wide, 3) < 1e-11
    # values below 3e-8 of the largest that the oracle keeps widen the bound by their weight
    tiny = groups([1.0, 0.5, 1e-9, 1e-10])
    assert truncation_bound(tiny, 4) >= 2.0 * 1e-9
    d, gap = widest_cut(groups([1.0, 0.99, 0.5, 0.49, 0.48, 0.1]), 3, 2)
    assert d == 2 and abs(gap - (0.99 ** 2 - 0.5 ** 2)) < 1e-15

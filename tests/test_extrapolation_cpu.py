"""Eq. 16 extrapolation E(D) = E_exact + C1 w_disc(D): the oracle's least-squares fit
pinned by exact lines, two-point interpolation and the normal equations, and the
library's host-only dmrg_extrapolate against it (no GPU needed)."""
import numpy as np
import pytest

from oracle import dmrg as odmrg


def test_oracle_recovers_exact_line():
    w = np.array([3e-4, 1e-4, 4e-5, 1e-5])
    e0, c1 = odmrg.extrapolate(w, -7.5 + 120.0 * w)
    assert abs(e0 + 7.5) < 1e-13 and abs(c1 - 120.0) < 1e-9


def test_oracle_two_points_interpolate():
    e0, c1 = odmrg.extrapolate([2e-4, 5e-5], [-1.0, -1.3])
    assert abs(e0 + c1 * 2e-4 + 1.0) < 1e-13 and abs(e0 + c1 * 5e-5 + 1.3) < 1e-13


def test_oracle_normal_equations():
    rng = np.random.default_rng(16)
    w = rng.uniform(1e-6, 1e-3, size=7)
    e = -3.0 + 50.0 * w + rng.normal(scale=1e-4, size=7)
    e0, c1 = odmrg.extrapolate(w, e)
    r = e - (e0 + c1 * w)
    assert abs(r.sum()) < 1e-12 and abs((r * w).sum()) < 1e-15


def test_library_matches_oracle():
    try:
        from paper_1312_2415_gb300 import extrapolate
        lib_extrapolate = extrapolate
        lib_extrapolate([1e-4, 2e-4], [0.0, 1.0])
    except OSError:
        pytest.skip("library not built")
    rng = np.random.default_rng(3)
    for _ in range(5):
        w = rng.uniform(1e-7, 1e-3, size=5)
        e = -40.0 + rng.normal(scale=1.0) * w * 1e3 + rng.normal(scale=1e-5, size=5)
        a = lib_extrapolate(w, e)
        b = odmrg.extrapolate(w, e)
        assert abs(a[0] - b[0]) < 1e-12 and abs(a[1] - b[1]) < 1e-9 * max(1.0, abs(b[1]))

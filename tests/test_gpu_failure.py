"""Failure detection, made on the host (no GPU fault, trap or hang is provoked):

* Davidson stopped by its iteration cap reports DMRG_ENOTCONV and still returns its best
  pair: a unit vector whose Rayleigh quotient is the returned energy, above the exact
  lowest eigenvalue of the oracle's H_eff; a sweep step at the cap completes the step;
* a cap on the library's device memory turns the allocation of the mixed-precision
  tables into DMRG_ENOMEM; what the failing call allocated is released (the library's
  device bytes return to their value before the call) and, with the cap removed, the
  same call succeeds and gives the right product.
"""
import numpy as np
import pytest

from oracle import dmrg as odmrg
from oracle import mps as om
from tests.mps_io import lib_x_to_oracle, mps_to_bytes
from workloads import hubbard_chain, random_integrals, round_robin_irreps, uniform_pm1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1312_2415_gb300 as pkg
    return torch, pkg


def test_davidson_cap_returns_enotconv_with_its_best_pair(lib):
    torch, pkg = lib
    L, N, i = 7, 6, 2
    irr = round_robin_irreps(L)
    h, V = random_integrals(irr, 11)
    m = om.right_canonicalize(om.random_mps(irr, N, 0, 1, 30, uniform_pm1(3, 10 ** 6)))
    for k in range(i):
        om.svd_truncate(m, k, om.tt_to_x(m, k), 10 ** 9, "right")
    prob = odmrg.Problem(h, V, irr, N, 0, 1)
    H, _, proj = odmrg.effective_hamiltonian(prob, m, i)
    e_exact = np.linalg.eigvalsh(H)[0]
    ctx = pkg.Context(L, irr, N, 0, 1)
    ctx.set_integrals(h, V)
    ctx.set_schedule([30], [0.0], [1], [0.0], 1e-14, 2)
    ctx.set_mps(mps_to_bytes(m))
    n, table = ctx.layout(i)
    x = ctx.tt_to_x(i)
    e, it, ok = ctx.davidson(i, x)
    assert not ok and it == 2
    assert "iteration cap" in ctx.lib.dmrg_last_error(ctx.h).decode()
    assert abs(np.linalg.norm(x) - 1.0) < 1e-12
    v = proj.flatten(lib_x_to_oracle(x, table))
    assert abs(v @ H @ v - e) < 1e-10
    assert e >= e_exact - 1e-12 and e - e_exact > 1e-8  # not converged, but a bound
    # a sweep step at the cap is completed (decomposition and update done)
    ew, w, it, ok = ctx.sweep_step(i, 1, 30)
    assert not ok and np.isfinite(ew) and ew >= e_exact - 1e-12
    n2, _ = ctx.layout(i + 1)
    assert n2 > 0 and np.isfinite(ctx.tt_to_x(i + 1)).all()


def test_device_memory_cap_gives_enomem_without_leaking(lib):
    torch, pkg = lib
    L, N, i = 12, 12, 5
    irr = round_robin_irreps(L)
    h, V = random_integrals(irr, 7)
    ctx = pkg.Context(L, irr, N, 0, 0)
    ctx.set_integrals(h, V)
    ctx.set_schedule([200], [0.0], [1], [0.0], 1e-10, 20)
    ctx.init_mps(3)
    ctx.canonicalize(i)
    n, _ = ctx.layout(i)
    x = torch.tensor(np.random.default_rng(1).normal(size=n), device="cuda")
    y64, y = torch.empty_like(x), torch.empty_like(x)
    ctx.set_precision(0, 0)
    ctx.matvec(i, x, y64)  # environments and the FP64 tables of the site are built
    torch.cuda.synchronize()
    before = pkg.device_memory_in_use()
    assert before > 0
    ctx.set_precision(1, 0)  # the next matvec builds the tensor-core tables
    try:
        pkg.set_device_memory_cap(before + (64 << 10))
        with pytest.raises(pkg.DMRGError) as err:
            ctx.matvec(i, x, y)
        assert err.value.code == -4
        torch.cuda.synchronize()
        assert pkg.device_memory_in_use() == before
    finally:
        pkg.set_device_memory_cap(0)
    ctx.matvec(i, x, y)
    torch.cuda.synchronize()
    assert pkg.device_memory_in_use() > before
    err = ((y - y64).abs().max() / y64.abs().max()).item()
    assert err < 2e-6, err


def test_tensor_core_wait_timeout_is_reported_and_recovered(lib):
    """The fused kernel's bounded waits: with the test hook on, every CTA gives up on a
    barrier that nothing completes (a few thousand polls), frees its tensor memory and
    returns; the call reports DMRG_ECUDA.  With the hook off the next matvec gives the
    right product (tensor memory and the context are usable)."""
    torch, pkg = lib
    # blocks large enough for the fused kernel (output tiles of at most 4 x 4 go to the
    # CUDA-core path, which has no waits): a Hubbard chain (C1, few and large sectors)
    L, N, i = 12, 12, 5
    irr = [0] * L
    h, V = hubbard_chain(L, 1.0, 4.0)
    ctx = pkg.Context(L, irr, N, 0, 0, precision=1)
    ctx.set_integrals(h, V)
    ctx.set_schedule([400], [0.0], [1], [0.0], 1e-10, 20)
    ctx.init_mps(7)
    ctx.canonicalize(i)
    n, _ = ctx.layout(i)
    x = torch.tensor(np.random.default_rng(3).normal(size=n), device="cuda")
    y, y64 = torch.empty_like(x), torch.empty_like(x)
    ctx.set_precision(0, 0)
    ctx.matvec(i, x, y64)
    ctx.set_precision(1, 0)
    ctx.matvec(i, x, y)  # tables built, kernel run once normally
    try:
        pkg.test_tc_timeout(1)
        with pytest.raises(pkg.DMRGError) as err:
            ctx.matvec(i, x, y)
        assert err.value.code == -5 and "timed out" in str(err.value)
    finally:
        pkg.test_tc_timeout(0)
    for _ in range(2):
        y.fill_(0.0)
        ctx.matvec(i, x, y)
        torch.cuda.synchronize()
        assert ((y - y64).abs().max() / y64.abs().max()).item() < 2e-6

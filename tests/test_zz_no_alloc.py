"""The allocation-free matvec entry point (dmrg_heff_matvec_noalloc).

It has no counterpart in the paper: it serves callers that must not allocate device
memory while they apply H_eff (for example code being captured into a CUDA graph, or
running under a fixed memory budget).  It must give the same y = H_eff x as the
allocating entry point dmrg_heff_matvec, call after call, although every call reuses
one fixed scratch array inside the library.  This file is collected last so that a
run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matvec_matches_allocating_entry_point():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    from paper_1312_2415_gb300 import Context
    from workloads import random_integrals, round_robin_irreps
    L, N, site = 8, 8, 3
    irr = round_robin_irreps(L)
    h, V = random_integrals(irr, 17)
    ctx = Context(L, irr, N, 0, 0)
    ctx.set_integrals(h, V)
    ctx.set_schedule([80], [0.0], [1], [0.0], 1e-10, 50)
    ctx.init_mps(4242)
    ctx.canonicalize(site)
    n, _ = ctx.layout(site)
    rng = np.random.default_rng(5)
    xs = [rng.normal(size=n), rng.normal(size=n)]
    # the allocating entry point (host buffers); it also prepares the site's tables
    refs = [ctx.matvec(site, x) for x in xs]
    stream = torch.cuda.current_stream().cuda_stream
    y = torch.full((n,), 1e300, dtype=torch.float64, device="cuda")  # stale garbage
    for x, ref in zip(xs, refs):
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        ctx.matvec_noalloc(site, xd.data_ptr(), y.data_ptr(), stream)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        # same tables and the same summation order: agreement to rounding (1e-12 relative,
        # the matvec tolerance of the parity tests)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_noalloc_matvec_rejects_unprepared_site():
    import torch
    from paper_1312_2415_gb300 import Context, DMRGError
    from workloads import hubbard_chain
    ctx = Context(6, [0] * 6, 6, 0, 0)
    h, V = hubbard_chain(6)
    ctx.set_integrals(h, V)
    ctx.init_mps(1)
    ctx.canonicalize(2)
    n, _ = ctx.layout(2)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(DMRGError) as e:
        ctx.matvec_noalloc(2, x.data_ptr(), y.data_ptr(), 0)
    assert e.value.code == -1

"""The allocation-free matvec entry point (dmrg_heff_matvec_noalloc).

It has no counterpart in the paper: it serves callers that cannot allocate device
memory when they apply H_eff (a process that reserved its device memory up front and
must not grow it, or a host framework whose allocator owns the GPU).  It must give the
FP64 y = H_eff x of the allocating entry point dmrg_heff_matvec, call after call,
although every call reuses one fixed scratch array inside the library.  This file is collected last so that a
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


def _context(L, N, D, seed, site, precision=0):
    from paper_1312_2415_gb300 import Context
    from workloads import random_integrals, round_robin_irreps
    irr = round_robin_irreps(L)
    h, V = random_integrals(irr, seed)
    ctx = Context(L, irr, N, 0, 0, precision=precision)
    ctx.set_integrals(h, V)
    ctx.set_schedule([D], [0.0], [1], [0.0], 1e-10, 50)
    ctx.init_mps(seed)
    ctx.canonicalize(site)
    return ctx


def test_noalloc_matvec_runs_fp64_tables_in_a_mixed_precision_context():
    """For a precision-1 context the allocation-free matvec is the FP64 product (the
    header says so), not the split-TF32 one of dmrg_heff_matvec."""
    import torch
    site = 3
    ctx = _context(8, 8, 60, 23, site, precision=1)
    n, _ = ctx.layout(site)
    x = torch.tensor(np.random.default_rng(8).normal(size=n), dtype=torch.float64, device="cuda")
    y32, y64, y = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
    ctx.matvec(site, x, y32)   # tensor-core product; prepares the site's tables
    ctx.set_precision(0, 0)
    ctx.matvec(site, x, y64)   # FP64 product of the same tables
    ctx.set_precision(1, 0)
    ctx.matvec_noalloc(site, x.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    scale = y64.abs().max().item()
    assert (y - y64).abs().max().item() <= 1e-12 * scale
    assert (y32 - y64).abs().max().item() > 0.0


def test_noalloc_on_a_side_stream_then_a_call_that_frees_its_tables():
    """The work is queued on the caller's stream and the call returns at once; the next
    context call (here a canonicalisation that releases the site's tables) must not
    free what that work still reads."""
    import torch
    site = 3
    ctx = _context(8, 8, 80, 31, site)
    n, _ = ctx.layout(site)
    xs = [np.random.default_rng(k).normal(size=n) for k in range(4)]
    refs = [ctx.matvec(site, x) for x in xs]
    side = torch.cuda.Stream()
    xd = [torch.tensor(x, dtype=torch.float64, device="cuda") for x in xs]
    ys = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in xs]
    torch.cuda.synchronize()
    for x, y in zip(xd, ys):
        ctx.matvec_noalloc(site, x.data_ptr(), y.data_ptr(), side.cuda_stream)
    ctx.canonicalize(site + 1)  # no synchronisation in between
    torch.cuda.synchronize()
    for y, ref in zip(ys, refs):
        got = y.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_noalloc_rejects_a_problem_above_its_fixed_scratch():
    import torch
    from paper_1312_2415_gb300 import DMRGError
    site = 7
    ctx = _context(16, 16, 1000, 2415016, site)
    n, _ = ctx.layout(site)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.matvec(site, x, y)  # tables prepared; their scratch exceeds the 64 MiB array
    with pytest.raises(DMRGError) as e:
        ctx.matvec_noalloc(site, x.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -1 and "64 MiB" in str(e.value)

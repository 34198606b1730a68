"""Batched mixed-precision matvecs (dmrg_batch_*): the H_eff x of several independent
instances of uneven size (Hubbard and random-integral systems, S = 0 and 1, different
D) run as one grouped launch per phase replayed from a CUDA graph, element by element
against each instance's FP64 matvec (2e-5 of max|y|, the bound of the single-instance
mixed tests) and against its own single-instance mixed matvec; a replay gives the same
result; a context that rebuilds its tables invalidates the batch."""
import numpy as np
import pytest

from workloads import hubbard_chain, random_integrals, round_robin_irreps

pytestmark = pytest.mark.gpu

CASES = [("h", 8, 8, 0, 40), ("r", 8, 8, 2, 50), ("h", 10, 10, 0, 120), ("r", 10, 10, 0, 150),
         ("h", 12, 12, 2, 300), ("r", 9, 8, 0, 60)]


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available()
    from paper_1312_2415_gb300 import Batch, Context, DMRGError
    return torch, Batch, Context, DMRGError


def _instances(Context):
    ctxs, sites = [], []
    for kind, L, N, tS, D in CASES:
        if kind == "h":
            irr = [0] * L
            h, V = hubbard_chain(L, 1.0, 4.0)
        else:
            irr = round_robin_irreps(L)
            h, V = random_integrals(irr, 7)
        c = Context(L, irr, N, tS, 0)
        c.set_integrals(h, V)
        c.set_schedule([D], [0.0], [1], [0.0], 1e-10, 40)
        c.init_mps(3)
        i = L // 2 - 1
        c.canonicalize(i)
        ctxs.append(c)
        sites.append(i)
    return ctxs, sites


def test_batched_matvec_matches_each_instance(mods):
    torch, Batch, Context, DMRGError = mods
    ctxs, sites = _instances(Context)
    xs, ref64, ref32 = [], [], []
    for k, (c, i) in enumerate(zip(ctxs, sites)):
        n, _ = c.layout(i)
        x = torch.tensor(np.random.default_rng(k).normal(size=n), device="cuda")
        y = torch.empty_like(x)
        c.set_precision(0, 0)
        c.matvec(i, x, y)
        ref64.append(y.clone())
        c.set_precision(1, 0)
        c.matvec(i, x, y)
        ref32.append(y.clone())
        xs.append(x)
    b = Batch(ctxs, sites, autotune=True)
    info = b.info()
    assert info["packs_per_unit"] > 0 and info["tasks_per_unit"] > 0
    ys = [torch.empty_like(x) for x in xs]
    for rep in range(2):  # a graph replay gives the same products
        b.run(xs, ys)
        torch.cuda.synchronize()
        for y, y64, y32 in zip(ys, ref64, ref32):
            err = ((y - y64).abs().max() / y64.abs().max()).item()
            assert 0.0 < err <= 2e-5, err
            assert ((y - y32).abs().max() / y64.abs().max()).item() <= 2e-5
    # a context that rebuilds its tables invalidates the batch
    ctxs[0].truncate(sites[0], 1, CASES[0][4], xs[0])
    with pytest.raises(DMRGError):
        b.run(xs, ys)
    b.close()

"""Batched mixed-precision matvecs (dmrg_batch_*): the H_eff x of several independent
instances of uneven size (Hubbard and random-integral systems, S = 0 and 1, different
D) run as one grouped launch per phase replayed from a CUDA graph.  Every instance the
oracle can project densely (L <= 9) is compared element by element with the oracle's
P^T H P x on the library's own state (2e-6 of max|y|, the mixed-precision bound of the
single-instance tests); every instance is also compared with its FP64 and its own
single-instance mixed matvec.  A replay gives the same result; a context that rebuilds
its tables invalidates the batch."""
import numpy as np
import pytest

from oracle import dmrg as odmrg
from tests.mps_io import lib_x_to_oracle, mps_from_bytes, oracle_x_to_lib
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


def _instances(Context, systems=None):
    ctxs, sites = [], []
    for kind, L, N, tS, D in CASES:
        if kind == "h":
            irr = [0] * L
            h, V = hubbard_chain(L, 1.0, 4.0)
        else:
            irr = round_robin_irreps(L)
            h, V = random_integrals(irr, 7)
        if systems is not None:
            systems.append((irr, h, V, N, tS))
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
    systems = []
    ctxs, sites = _instances(Context, systems)
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
    assert info["row_tile"] in (64, 128) and info["x_chunk"] in (32, 64)
    ys = [torch.empty_like(x) for x in xs]
    for rep in range(2):  # a graph replay gives the same products
        b.run(xs, ys)
        torch.cuda.synchronize()
        for y, y64, y32 in zip(ys, ref64, ref32):
            err = ((y - y64).abs().max() / y64.abs().max()).item()
            assert 0.0 < err <= 2e-6, err
            assert ((y - y32).abs().max() / y64.abs().max()).item() <= 2e-6
    # the oracle: P^T H P x on each small instance's own (canonicalised) state
    checked = 0
    for c, i, x, y, (irr, h, V, N, tS) in zip(ctxs, sites, xs, ys, systems):
        if len(irr) > 9:
            continue
        m = mps_from_bytes(c.get_mps(), irr)
        prob = odmrg.Problem(h, V, irr, N, tS, 0)
        H, _, proj = odmrg.effective_hamiltonian(prob, m, i)
        n, table = c.layout(i)
        xv = x.cpu().numpy()
        yo = oracle_x_to_lib(proj.unflatten(H @ proj.flatten(lib_x_to_oracle(xv, table))), table, n)
        err = np.abs(y.cpu().numpy() - yo).max() / np.abs(yo).max()
        assert 0.0 < err <= 2e-6, err
        checked += 1
    assert checked == 3
    # a context that rebuilds its tables invalidates the batch
    ctxs[0].truncate(sites[0], 1, CASES[0][4], xs[0])
    with pytest.raises(DMRGError):
        b.run(xs, ys)
    b.close()


def test_batched_davidson_matches_each_instance(mods):
    """dmrg_batch_davidson: the instances' Davidsons in lockstep (one batched matvec and
    one launch per vector operation per iteration).  Its FP64-finished energies equal the
    lowest eigenvalue of the oracle's P^T H P on every instance the oracle projects
    (L <= 9) and each context's own FP64 Davidson on all, within 1e-6 Eh (the mixed
    path's target); the Ritz vectors have unit norm and a non-negative overlap with their
    start vectors; the tensor-core Ritz values sit within the split-TF32 bias (1e-5 of
    |E|) of them."""
    torch, Batch, Context, DMRGError = mods
    systems = []
    ctxs, sites = _instances(Context, systems)
    starts, ref = [], []
    for c, i, (irr, h, V, N, tS), (_, _, _, _, D) in zip(ctxs, sites, systems, CASES):
        x0 = c.tt_to_x(i)
        starts.append(torch.tensor(x0, device="cuda"))
        c.set_precision(0, 0)
        c.set_schedule([D], [0.0], [1], [0.0], 1e-9, 300)
        x = x0.copy()
        e, it, ok = c.davidson(i, x)
        assert ok
        ref.append(e)
        if len(irr) <= 9:
            m = mps_from_bytes(c.get_mps(), irr)
            H, _, _ = odmrg.effective_hamiltonian(odmrg.Problem(h, V, irr, N, tS, 0), m, i)
            assert abs(np.linalg.eigvalsh(H)[0] - e) < 1e-9
    b = Batch(ctxs, sites, autotune=False)
    xs = [s.clone() for s in starts]
    e64, iters, conv = b.davidson(xs, tol=1e-4, max_iter=200, fp64_energy=True)
    assert conv.all() and (iters >= 1).all()
    for e, r, x, s in zip(e64, ref, xs, starts):
        assert abs(e - r) < 1e-6, (e, r)
        assert abs(torch.linalg.norm(x).item() - 1.0) < 1e-12
        assert (x @ s).item() >= 0.0
    xs = [s.clone() for s in starts]
    etc, _, conv = b.davidson(xs, tol=1e-4, max_iter=200, fp64_energy=False)
    assert conv.all()
    for e, r in zip(etc, ref):
        assert abs(e - r) < 1e-5 * abs(r) + 1e-8, (e, r)
    # the batched matvec computes every instance again afterwards (the Davidson's
    # per-instance skip flags are restored)
    ys = [torch.empty_like(x) for x in xs]
    b.run(xs, ys)
    torch.cuda.synchronize()
    for c, i, x, y in zip(ctxs, sites, xs, ys):
        c.set_precision(0, 0)
        y64 = torch.empty_like(x)
        c.matvec(i, x, y64)
        assert ((y - y64).abs().max() / y64.abs().max()).item() <= 2e-6
    b.close()

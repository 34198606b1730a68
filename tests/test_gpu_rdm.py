"""GPU checks of dmrg_rdm: the spin-summed 1- and 2-RDMs as the adjoint of the H_eff
matvec (Eq. 9) with respect to the integrals of the operator recursion (Sec. 2.5).

* parity with the oracle (oracle/rdm.py on the determinant expansion of the same MPS),
  element by element, for random states of Hubbard and D2h random-integral problems
  with S = 0, 1/2, 1: FP64 sums of O(1e4) products of O(1) numbers, 1e-11 absolute;
* at the differentiation workload's size (L=16, N=16, S=0, D2h, D=1000), where no
  determinant expansion exists: the energy of Sec. 4.1 rebuilt from the RDMs equals the
  Rayleigh quotient of the library's own matvec, tr gamma = N, 0 <= occupations <= 2,
  and central differences (step 1e-5) of that Rayleigh quotient at the fixed state under
  symmetric changes of h and V equal the RDM contractions;
* the torch.autograd.Function: at a D where DMRG is exact, the gradients equal the
  oracle's FCI RDMs and central differences of re-solved energies (Hellmann-Feynman)."""
import numpy as np
import pytest

from oracle import mps as om
from oracle.fci import fci_ground_state
from oracle.rdm import energy, mps_state, rdm_from_vector, sym8
from tests.mps_io import mps_to_bytes
from workloads import hubbard_chain, make_problem, random_integrals, round_robin_irreps, uniform_pm1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1312_2415_gb300 import Context as C
    return C


def _problem(kind, L):
    if kind == "hubbard":
        irr = [0] * L
        h, V = hubbard_chain(L, 1.0, 4.0)
    else:
        irr = round_robin_irreps(L)
        h, V = random_integrals(irr, 11)
    return irr, h, V


CASES = [("hubbard", 8, 8, 0, 0, 40), ("random", 6, 6, 2, 0, 40), ("random", 6, 5, 1, 3, 40),
         ("random", 7, 6, 0, 1, 40), ("random", 8, 8, 0, 0, 60), ("hubbard", 7, 7, 1, 0, 30)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}L{c[1]}N{c[2]}S{c[3]}I{c[4]}D{c[5]}")
def test_rdm_matches_oracle(Context, case):
    import torch
    kind, L, N, tS, IG, D = case
    irr, h, V = _problem(kind, L)
    m = om.right_canonicalize(om.random_mps(irr, N, tS, IG, D, uniform_pm1(5, 10 ** 6)))
    g0, G0 = rdm_from_vector(*mps_state(m))
    G0s = sym8(G0)
    ctx = Context(L, irr, N, tS, IG)
    ctx.set_integrals(h, V)
    ctx.set_mps(mps_to_bytes(m))
    g1, G1 = ctx.rdm()  # host buffers
    assert np.abs(g1 - g0).max() < 1e-11
    assert np.abs(G1 - G0s).max() < 1e-11
    # device buffers on the current stream, from the state the first call left behind
    gd = torch.empty((L, L), dtype=torch.float64, device="cuda")
    Gd = torch.empty((L,) * 4, dtype=torch.float64, device="cuda")
    ctx.rdm(gd, Gd)
    torch.cuda.synchronize()
    assert np.abs(gd.cpu().numpy() - g0).max() < 1e-11
    assert np.abs(Gd.cpu().numpy() - G0s).max() < 1e-11
    assert abs(energy(g1, G1, h, V) - energy(g0, G0, h, V)) < 1e-10


def _rayleigh(ctx, site):
    import torch
    n, _ = ctx.layout(site)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.tt_to_x(site, x)
    y = torch.empty_like(x)
    ctx.matvec(site, x, y)
    return float((x @ y) / (x @ x))


def _sym_h(rng, irr):
    L = len(irr)
    a = rng.normal(size=(L, L))
    a = a + a.T
    ir = np.asarray(irr)
    return a * (ir[:, None] == ir[None, :])


def _sym_v(rng, irr):
    L = len(irr)
    a = rng.normal(size=(L,) * 4)
    a = sum(np.einsum(s + "->ijkl", a) for s in ("ijkl", "jilk", "klij", "lkji", "kjil", "ilkj", "lijk", "jkli"))
    ir = np.asarray(irr)
    ok = (ir[:, None, None, None] ^ ir[None, :, None, None] ^ ir[None, None, :, None] ^ ir[None, None, None, :]) == 0
    return a * ok


def test_rdm_differentiation_workload_properties(Context):
    cfg, h, V = make_problem("random16")
    L, N, irr = cfg["L"], cfg["N"], cfg["group_irreps"]
    ctx = Context(L, irr, N, cfg["two_S"], cfg["irrep"], group=7)
    ctx.set_integrals(h, V)
    ctx.set_schedule([cfg["D"]], [0.0], [1], [0.0], 1e-10, 50)
    ctx.init_mps(cfg["seed"])
    gamma, Gamma = ctx.rdm()
    site = L - 2  # dmrg_rdm leaves the centre here
    e0 = _rayleigh(ctx, site)
    assert abs(energy(gamma, Gamma, h, V) - e0) < 1e-9 * max(1.0, abs(e0))
    assert abs(np.trace(gamma) - N) < 1e-9
    occ = np.linalg.eigvalsh(gamma)
    assert occ.min() > -1e-9 and occ.max() < 2 + 1e-9
    assert abs(np.einsum("ijij->", Gamma) - N * (N - 1)) < 1e-7
    rng = np.random.default_rng(16)
    d = 1e-5
    for _ in range(2):
        dh, dV = _sym_h(rng, irr), _sym_v(rng, irr)
        for kind in ("h", "V"):
            hp, hm = (h + d * dh, h - d * dh) if kind == "h" else (h, h)
            Vp, Vm = (V, V) if kind == "h" else (V + d * dV, V - d * dV)
            ctx.set_integrals(hp, Vp)
            ep = _rayleigh(ctx, site)
            ctx.set_integrals(hm, Vm)
            em = _rayleigh(ctx, site)
            fd = (ep - em) / (2 * d)
            an = np.sum(gamma * dh) if kind == "h" else 0.5 * np.sum(Gamma * dV)
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (kind, fd, an)
    ctx.set_integrals(h, V)


def test_autograd_gradients_hellmann_feynman(Context):
    import torch
    from paper_1312_2415_gb300.autograd import dmrg_energy
    L, N = 6, 6
    irr = round_robin_irreps(L)
    h0, V0 = random_integrals(irr, 31)
    ctx = Context(L, irr, N, 0, 0)
    ctx.set_integrals(h0, V0)
    ctx.set_schedule([100], [1e-11], [8], [0.0], 1e-11, 200)
    ctx.init_mps(3)
    h = torch.tensor(h0, requires_grad=True)
    V = torch.tensor(V0, requires_grad=True)
    E = dmrg_energy(h, V, ctx)
    E.backward()
    Ef, vecs, space = fci_ground_state(h0, V0, N, 0, irr, 0)
    assert abs(E.item() - Ef[0]) < 1e-9
    gf, Gf = rdm_from_vector(space, vecs[0])
    assert np.abs(h.grad.numpy() - gf).max() < 1e-7
    assert np.abs(V.grad.numpy() - 0.5 * sym8(Gf)).max() < 1e-7
    rng = np.random.default_rng(6)
    d = 1e-5
    for dh, dV in ((_sym_h(rng, irr), 0 * V0), (0 * h0, _sym_v(rng, irr))):
        ep = dmrg_energy(torch.tensor(h0 + d * dh), torch.tensor(V0 + d * dV), ctx).item()
        em = dmrg_energy(torch.tensor(h0 - d * dh), torch.tensor(V0 - d * dV), ctx).item()
        an = float(np.sum(h.grad.numpy() * dh) + np.sum(V.grad.numpy() * dV))
        assert abs((ep - em) / (2 * d) - an) < 1e-5 * max(1.0, abs(an))

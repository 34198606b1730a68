"""GPU checks of the excited-state Hamiltonian H_m = H_0 + sum_k eta_{k+1} |Psi_k><Psi_k|
(Sec. 4.3; dmrg_push_excitation).

* matvec parity with the oracle's projected effective Hamiltonian (H_eff of Eq. 9 plus
  eta v v^T, v the determinant-space projection of the lower state onto the two-site
  basis), element by element at three site pairs, S = 0, 1/2 and a non-trivial irrep:
  FP64, 1e-12 of max |y|;
* solves: at D where DMRG is exact, the second and third states equal the oracle FCI's
  second and third roots of the same (N, S, irrep) sector to 1e-8, on the FP64 path and
  on the mixed-precision path (split-TF32 tensor cores + FP64 Davidson finish)."""
import numpy as np
import pytest

from oracle import dmrg as odmrg
from oracle import mps as om
from oracle.fci import fci_ground_state
from tests.mps_io import mps_to_bytes, oracle_x_to_lib
from tests.test_gpu_parity import setup
from workloads import hubbard_chain, random_integrals, round_robin_irreps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1312_2415_gb300 import Context as C
    return C


CASES = [("hubbard", 8, 8, 0, 0, 40), ("random", 6, 5, 1, 3, 40), ("random", 7, 6, 0, 1, 40)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}L{c[1]}N{c[2]}S{c[3]}I{c[4]}")
def test_projected_matvec_matches_oracle(Context, case):
    kind, L, N, tS, IG, D = case
    eta = 3.7
    for i in sorted({0, L // 2 - 1, L - 2}):
        irr, h, V, m, prob = setup(kind, L, N, tS, IG, D, 3, i)
        m0 = setup(kind, L, N, tS, IG, D, 9, 0)[3]
        Hm, _, proj = odmrg.excited_hamiltonian(prob, m, i, [(m0, eta)])
        ctx = Context(L, irr, N, tS, IG)
        ctx.set_integrals(h, V)
        ctx.set_mps(mps_to_bytes(m0))
        ctx.push_excitation(eta)
        assert ctx.excitation_count() == 1
        ctx.set_mps(mps_to_bytes(m))
        n, table = ctx.layout(i)
        rng = np.random.default_rng(i)
        xo = {k: rng.normal(size=v.shape) for k, v in om.tt_to_x(m, i).items()}
        x = oracle_x_to_lib(xo, table, n)
        y = ctx.matvec(i, x)
        yo = oracle_x_to_lib(proj.unflatten(Hm @ proj.flatten(xo)), table, n)
        assert np.abs(y - yo).max() <= 1e-12 * np.abs(yo).max()
        ctx.clear_excitations()
        H0, _, _ = odmrg.effective_hamiltonian(prob, m, i)
        y0 = oracle_x_to_lib(proj.unflatten(H0 @ proj.flatten(xo)), table, n)
        assert np.abs(ctx.matvec(i, x) - y0).max() <= 1e-12 * np.abs(y0).max()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind", ["hubbard", "random"])
def test_excited_states_equal_fci_roots(Context, kind, precision):
    L, N = 8, 8
    irr = [0] * L if kind == "hubbard" else round_robin_irreps(L)
    h, V = hubbard_chain(L, 1.0, 4.0) if kind == "hubbard" else random_integrals(irr, 11)
    E, _, _ = fci_ground_state(h, V, N, 0, irr, 0, nroots=3)
    assert E[1] - E[0] > 1e-6 and E[2] - E[1] > 1e-6
    ctx = Context(L, irr, N, 0, 0)
    ctx.set_integrals(h, V)
    ctx.set_schedule([200], [1e-11], [6], [0.0], 1e-10, 200)
    ctx.set_precision(precision, 0)
    ctx.init_mps(1)
    eta = 2.0 * (E[2] - E[0]) + 1.0
    e0, _ = ctx.solve()
    ctx.push_excitation(eta)
    ctx.init_mps(2)
    e1, _ = ctx.solve()
    ctx.push_excitation(eta)
    ctx.init_mps(3)
    e2, _ = ctx.solve()
    assert abs(e0 - E[0]) < 1e-8
    assert abs(e1 - E[1]) < 1e-8
    assert abs(e2 - E[2]) < 1e-8

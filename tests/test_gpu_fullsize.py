"""Matvec checks at full size: the L=28, N=12, D2h random-integral system at D=2500
(middle site pair, the benchmark's launch configuration), where the oracle's dense
projected H_eff is out of reach, and large-sector Hubbard chains whose blocks exceed
one tensor-core tile (K > 32, stacks and blocks above 128 rows, outputs above 64
columns).  Properties that hold at any size are checked on the FP64 path:
  * Hermiticity of H_eff (Eq. 9 is a projection of a Hermitian operator):
    <u, H v> = <H u, v> to 1e-12 relative;
  * sampled diagonal entries (H e_i)_i equal the separately computed diagonal (the
    Davidson preconditioner) to 1e-12 relative;
and the mixed-precision (split-TF32 tensor-core) matvec is compared with the FP64 one
element by element (2e-6 of max|y|, the bound of the small-case parity tests)."""
import numpy as np
import pytest

from workloads import hubbard_chain, make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Context():
    import torch
    assert torch.cuda.is_available()
    from paper_1312_2415_gb300 import Context as C
    return C


def _ctx(Context, L, irreps, N, two_S, IG, h, V, D, seed, group):
    ctx = Context(L, irreps, N, two_S, IG, group=group)
    ctx.set_integrals(h, V)
    ctx.set_schedule([D], [0.0], [1], [0.0], 1e-10, 50)
    ctx.init_mps(seed)
    return ctx


def _matvec(ctx, precision, site, v):
    import torch
    ctx.set_precision(precision, 0)
    x = torch.from_numpy(v).cuda()
    y = torch.empty_like(x)
    ctx.matvec(site, x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _mixed_vs_fp64(ctx, site, rng):
    n, _ = ctx.layout(site)
    v = rng.normal(size=n)
    y64 = _matvec(ctx, 0, site, v)
    y32 = _matvec(ctx, 1, site, v)
    err = np.abs(y32 - y64).max() / np.abs(y64).max()
    assert 0.0 < err <= 2e-6, err
    return n, err


def test_bench_workload_fp64_properties_and_mixed(Context):
    import torch
    cfg, h, V = make_problem("random28")
    L = cfg["L"]
    site = L // 2 - 1
    ctx = _ctx(Context, L, cfg["group_irreps"], cfg["N"], cfg["two_S"], cfg["irrep"], h, V, cfg["D"],
               cfg["seed"], 7)
    ctx.canonicalize(site)
    n, _ = ctx.layout(site)
    rng = np.random.default_rng(28)
    u, v = rng.normal(size=n), rng.normal(size=n)
    hu, hv = _matvec(ctx, 0, site, u), _matvec(ctx, 0, site, v)
    assert abs(u @ hv - hu @ v) <= 1e-12 * np.linalg.norm(u) * np.linalg.norm(hv)
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.diag(site, d)
    d = d.cpu().numpy()
    for i in rng.choice(n, size=3, replace=False):
        e = np.zeros(n)
        e[i] = 1.0
        assert abs(_matvec(ctx, 0, site, e)[i] - d[i]) <= 1e-12 * max(1.0, abs(d[i]))
    _mixed_vs_fp64(ctx, site, rng)


@pytest.mark.parametrize("L,D", [(12, 3000), (14, 4000)])
def test_large_sector_mixed_matvec(Context, L, D):
    h, V = hubbard_chain(L, 1.0, 4.0)
    ctx = _ctx(Context, L, [0] * L, L, 0, 0, h, V, D, 5, 0)
    site = L // 2 - 1
    ctx.canonicalize(site)
    _mixed_vs_fp64(ctx, site, np.random.default_rng(L))

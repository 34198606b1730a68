"""Synthetic Hamiltonians and seeded random streams.

Workloads (the paper's molecular integrals are not available, so these stand in):
  * open Hubbard chain: h[i,i+1] = h[i+1,i] = -t, V[i,i,i,i] = U, point group C1;
  * random ab initio-like integrals with abelian point-group structure:
      h symmetric, off-diagonal N(0, 0.5) where irrep(i) == irrep(j), diagonal a
      linear ramp from -2 to 0;
      V[i,j,k,l] = sum_P Lp[P][i,k] * Lp[P][j,l]   (physics notation; the factor
      matrices are symmetric with N(0, 0.3) entries where irrep(i) ^ irrep(j)
      equals the irrep P mod n_irrep of the factor, rank 3L).
Irreps are integers 0..7 whose direct product is XOR (real abelian groups).
"""
import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(seed, n):
    """First n outputs of Vigna's splitmix64 generator started at state `seed`.

    state += 0x9E3779B97F4A7C15; z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) * 0x94D049BB133111EB;
    return z ^ (z >> 31).
    """
    out = np.empty(n, dtype=np.uint64)
    s = seed & MASK64
    with np.errstate(over="ignore"):
        idx = np.arange(1, n + 1, dtype=np.uint64)
        z = (np.uint64(s) + idx * np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        out[:] = z ^ (z >> np.uint64(31))
    return out


def uniform_pm1(seed, n):
    """n doubles uniform in [-1, 1): top 53 bits of splitmix64 mapped affinely."""
    u = splitmix64(seed, n) >> np.uint64(11)
    return u.astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0


def counter_uniform_pm1(seed, n, start=0):
    """Counter-based stream: element i is splitmix64's first output from state
    seed + start + i (one mix per element, no sequential state), mapped to [-1, 1) by
    its top 53 bits.  This is the stream a device kernel draws with one thread per
    element; here it is an input generator for tests."""
    with np.errstate(over="ignore"):
        idx = np.arange(n, dtype=np.uint64) + np.uint64((seed + start) & MASK64)
        z = idx + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0


def hubbard_chain(L, t=1.0, U=4.0):
    h = np.zeros((L, L))
    for i in range(L - 1):
        h[i, i + 1] = h[i + 1, i] = -t
    V = np.zeros((L, L, L, L))
    for i in range(L):
        V[i, i, i, i] = U
    return h, V


def round_robin_irreps(L, n_irrep=8):
    return [i % n_irrep for i in range(L)]


def irreps_from_counts(counts):
    return [ir for ir, c in enumerate(counts) for _ in range(c)]


def random_integrals(irreps, seed, n_irrep=8, sigma_h=0.5, sigma_l=0.3, rank=None):
    L = len(irreps)
    rng = np.random.default_rng(seed)
    irr = np.asarray(irreps)
    same = irr[:, None] == irr[None, :]
    off = rng.normal(0.0, sigma_h, size=(L, L))
    off = np.triu(off, 1)
    off = off + off.T
    h = np.where(same, off, 0.0)
    np.fill_diagonal(h, [-2.0 + 2.0 * i / max(L - 1, 1) for i in range(L)])
    if rank is None:
        rank = 3 * L
    pair_irrep = irr[:, None] ^ irr[None, :]
    V = np.zeros((L, L, L, L))
    for P in range(rank):
        g = rng.normal(0.0, sigma_l, size=(L, L))
        g = np.triu(g) + np.triu(g, 1).T
        Lp = np.where(pair_irrep == (P % n_irrep), g, 0.0)
        V += np.einsum("ik,jl->ijkl", Lp, Lp)
    return h, V


# Named workloads. Sizes follow the configurations the library is measured on.
CONFIGS = {
    "hubbard8": dict(kind="hubbard", L=8, N=8, two_S=0, irrep=0, group_irreps=[0] * 8,
                     t=1.0, U=4.0, D=64, sweeps=6, davidson_tol=1e-10),
    "random12": dict(kind="random", L=12, N=12, two_S=0, irrep=0,
                     group_irreps=round_robin_irreps(12), seed=2415012, D=500),
    "random16": dict(kind="random", L=16, N=16, two_S=0, irrep=0,
                     group_irreps=round_robin_irreps(16), seed=2415016, D=1000),
    "random28": dict(kind="random", L=28, N=12, two_S=0, irrep=0,
                     group_irreps=irreps_from_counts([8, 3, 3, 2, 6, 2, 2, 2]),
                     seed=2415028, D=2500),
}


def make_problem(name_or_cfg):
    cfg = CONFIGS[name_or_cfg] if isinstance(name_or_cfg, str) else name_or_cfg
    if cfg["kind"] == "hubbard":
        h, V = hubbard_chain(cfg["L"], cfg.get("t", 1.0), cfg.get("U", 4.0))
    else:
        h, V = random_integrals(cfg["group_irreps"], cfg["seed"])
    return cfg, h, V

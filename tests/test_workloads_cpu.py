"""The synthetic inputs (workloads/): the seeded streams against the published splitmix64
test vectors, the counter-based stream against its definition, and the random
ab initio-like integrals against the properties their recipe states (symmetric h with
point-group zeros and the -2..0 diagonal ramp; V = sum_P L^P (x) L^P in physics notation,
eightfold symmetric and zero unless the four irreps multiply to the totally symmetric
one; rank 3L); the Hubbard chain; the L=28 irrep counts."""
import numpy as np

from workloads import hubbard_chain, make_problem, random_integrals, round_robin_irreps
from workloads.synthetic import counter_uniform_pm1, irreps_from_counts, splitmix64, uniform_pm1


def test_splitmix64_published_vectors():
    # Vigna's splitmix64: state 0 and state 1234567, first three outputs
    assert [int(v) for v in splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(v) for v in splitmix64(1234567, 3)] == [6457827717110365317, 3203168211198807973,
                                                         9817491932198370423]


def test_uniform_streams():
    u = uniform_pm1(7, 10000)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.05
    # element i of the counter-based stream is the first draw of the sequential stream
    # started at seed + start + i
    c = counter_uniform_pm1(11, 50, start=3)
    assert np.array_equal(c, np.array([uniform_pm1(11 + 3 + i, 1)[0] for i in range(50)]))


def test_random_integrals_recipe():
    irr = round_robin_irreps(10)
    h, V = random_integrals(irr, 5)
    L = len(irr)
    ir = np.asarray(irr)
    assert np.array_equal(h, h.T)
    assert np.all(h[ir[:, None] != ir[None, :]] == 0.0)
    assert np.allclose(np.diag(h), [-2.0 + 2.0 * i / (L - 1) for i in range(L)])
    # physics notation V_ijkl = (ik|jl): the eightfold symmetry (ik|jl) = (ki|jl) = (ik|lj)
    # = (ki|lj) = (jl|ik) = (lj|ik) = (jl|ki) = (lj|ki), as permutations of (i, j, k, l)
    for perm in ("kjil", "ilkj", "klij", "jilk", "lijk", "jkli", "lkji"):
        assert np.allclose(V, np.einsum("ijkl->" + perm, V)), perm
    # and not more: a generic V is not symmetric under i <-> j alone
    assert not np.allclose(V, np.einsum("ijkl->jikl", V))
    # point group: zero unless irr_i ^ irr_j ^ irr_k ^ irr_l == 0
    prod = ir[:, None, None, None] ^ ir[None, :, None, None] ^ ir[None, None, :, None] ^ ir[None, None, None, :]
    assert np.all(V[prod != 0] == 0.0) and np.any(V[prod == 0] != 0.0)
    # V as a matrix on pairs (ik),(jl) is a sum of 3L symmetric rank-one terms: positive
    # semidefinite with rank <= 3L
    M = V.transpose(0, 2, 1, 3).reshape(L * L, L * L)
    w = np.linalg.eigvalsh((M + M.T) / 2)
    assert w.min() > -1e-10 * w.max() and np.sum(w > 1e-10 * w.max()) <= 3 * L


def test_hubbard_chain_and_problem_sizes():
    h, V = hubbard_chain(6, 1.0, 4.0)
    assert np.allclose(h, h.T) and h[0, 1] == -1.0 and h[0, 2] == 0.0 and np.all(np.diag(h) == 0.0)
    assert V[2, 2, 2, 2] == 4.0 and np.count_nonzero(V) == 6
    counts = [8, 3, 3, 2, 6, 2, 2, 2]
    irr = irreps_from_counts(counts)
    assert len(irr) == 28 and [irr.count(k) for k in range(8)] == counts
    cfg, h28, V28 = make_problem("random28")
    assert cfg["L"] == 28 and cfg["N"] == 12 and cfg["D"] == 2500 and cfg["group_irreps"] == irr
    assert h28.shape == (28, 28) and V28.shape == (28,) * 4

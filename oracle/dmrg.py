"""Two-site spin-adapted DMRG sweep for the oracle (plain dense algebra).

Each micro-iteration follows Secs. 2.3, 2.4 and 3.3:
  x = Eq. 25 from T[i] T[i+1]  ->  H_eff x = lambda x (Eq. 9) with H_eff = P^T H P,
  its plain definition (P: reduced two-site basis -> determinants, H: Sec. 4.1)
  ->  Eqs. 26-28 block SVD and truncation to D  ->  new T[i], T[i+1].
A macro-iteration is a sweep to the right followed by a sweep to the left (Sec. 4.2);
Solve reports the minimum energy over all micro-iterations (Sec. 4.3).
The lowest eigenpair of the dense H_eff is taken from numpy.linalg.eigh.
Excited states (Sec. 4.3): the Hamiltonian H_m = H_0 + sum_k eta_{k+1} |Psi_k><Psi_k| of
the m-th state adds eta v v^T per lower state to H_eff, v the projection of Psi_k onto
the current two-site basis (`excited_hamiltonian`).
"""
import numpy as np
from .fci import FCISpace
from .mps import TwoSiteProjector, tt_to_x, svd_truncate


class Problem:
    def __init__(self, h, V, irreps, N, two_S, I_G, ecore=0.0):
        self.h, self.V = np.asarray(h, float), np.asarray(V, float)
        self.irreps, self.N, self.two_S, self.I_G = list(irreps), N, two_S, I_G
        self.ecore = ecore
        self.L = len(irreps)
        self.spaces, self.idx, self.H = [], [], []
        for f in range(two_S + 1):
            tm = 2 * f - two_S
            na, nb = (N + tm) // 2, (N - tm) // 2
            sp = FCISpace(self.L, na, nb, irreps, I_G)
            idx = np.flatnonzero(sp.mask.ravel())
            self.spaces.append(sp)
            self.idx.append(idx)
            self.H.append(sp.hamiltonian_matrix(self.h, self.V, idx, ecore))


def effective_hamiltonian(prob, m, i):
    """Dense H_eff for sites (i, i+1) and the projector used to build it."""
    proj = TwoSiteProjector(m, i, prob.spaces)
    H = np.zeros((proj.n, proj.n))
    G = np.zeros((proj.n, proj.n))
    for f, P in enumerate(proj.P):
        Pr = P[prob.idx[f]]
        H += Pr.T @ (prob.H[f] @ Pr)
        G += Pr.T @ Pr
    return 0.5 * (H + H.T), G, proj


def matvec(prob, m, i, x):
    H, _, proj = effective_hamiltonian(prob, m, i)
    v = proj.flatten(x)
    return proj.unflatten(H @ v)


def determinant_components(prob, m):
    """The state of an MPS in the determinant basis, one vector per Sz component f
    (restricted to the symmetry sector), from the two-site expansion at sites (0, 1)."""
    proj = TwoSiteProjector(m, 0, prob.spaces)
    x = proj.flatten(tt_to_x(m, 0))
    return [P[prob.idx[f]] @ x for f, P in enumerate(proj.P)]


def projected_state(prob, proj, psi):
    """v = P^T |psi> / |psi| in the reduced two-site basis of `proj` (norm summed over the
    Sz components, the inner product in which P^T P = 1)."""
    nrm = np.sqrt(sum(float(c @ c) for c in psi))
    return sum(P[prob.idx[f]].T @ psi[f] for f, P in enumerate(proj.P)) / nrm


def excited_hamiltonian(prob, m, i, lower):
    """Effective Hamiltonian of H_m = H_0 + sum_k eta_{k+1} |Psi_k><Psi_k| (Sec. 4.3,
    excited states): H_eff of Eq. 9 plus eta v v^T for every lower state, v its
    projection onto the two-site basis.  lower = [(MPS of Psi_k, eta_{k+1}), ...]."""
    H, G, proj = effective_hamiltonian(prob, m, i)
    for mk, eta in lower:
        v = projected_state(prob, proj, determinant_components(prob, mk))
        H = H + eta * np.outer(v, v)
    return H, G, proj


def micro_iteration(prob, m, i, D, direction, noise=0.0, noise_values=None, w_prev=0.0, lower=()):
    H, _, proj = excited_hamiltonian(prob, m, i, lower) if lower else effective_hamiltonian(prob, m, i)
    w, U = np.linalg.eigh(H)
    e = float(w[0])
    v = U[:, 0]
    x0 = proj.flatten(tt_to_x(m, i))
    if np.dot(v, x0) < 0:
        v = -v
    if noise > 0.0 and noise_values is not None:
        v = v + 0.5 * noise * w_prev * np.asarray(noise_values[:v.size])
        v = v / np.linalg.norm(v)
    w_disc, _, _ = svd_truncate(m, i, proj.unflatten(v), D, direction)
    return e, w_disc


def sweep(prob, m, D, n_macro, log=None, lower=()):
    """Right sweep then left sweep per macro-iteration; returns (min energy, list of
    per-micro-iteration energies).  `lower`: projected lower states (excited_hamiltonian)."""
    energies = []
    L = m.L
    for it in range(n_macro):
        for i in range(0, L - 1):
            e, wd = micro_iteration(prob, m, i, D, "right", lower=lower)
            energies.append(e)
        for i in range(L - 2, -1, -1):
            e, wd = micro_iteration(prob, m, i, D, "left", lower=lower)
            energies.append(e)
        if log is not None:
            log(it, energies[-1])
    return min(energies), energies


def extrapolate(w_disc, energy):
    """Eq. 16: the linear relation E(D) = E_exact + C1 w_disc(D) fitted by least squares
    to the (w_disc, E) pairs of several D; returns (E_exact, C1)."""
    w = np.asarray(w_disc, dtype=np.float64)
    A = np.stack([np.ones_like(w), w], axis=1)
    (e0, c1), *_ = np.linalg.lstsq(A, np.asarray(energy, dtype=np.float64), rcond=None)
    return float(e0), float(c1)

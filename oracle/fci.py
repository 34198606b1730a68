"""Full configuration interaction in the determinant basis (oracle, FP64).

The Hamiltonian is the plain second-quantised definition of Sec. 4.1 with
(ij|V|kl) = V_ijkl in physics notation:
    H = E_c + sum_{ik,s} h_ik a+_{is} a_{ks}
            + 1/2 sum_{ijkl,s,t} V_ijkl a+_{is} a+_{jt} a_{lt} a_{ks}.
Determinants are pairs (alpha string, beta string) of occupation bit masks with the
creation operators ordered all-alpha (orbital 0 first) then all-beta.  With the
spin-free generators E_pq = sum_s a+_{ps} a_{qs} the two-body part is
1/2 sum V_pqrs (E_pr E_qs - delta_qr E_ps).  Eq. 11's folding of h into V is in
`fold`.  Eigenpairs come from numpy / scipy library routines.
"""
import itertools
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def fold(h, V, N):
    """Eq. 11: (ij|h|kl) = V_ijkl + [h_ik delta_jl + h_jl delta_ik] / (N - 1)."""
    L = h.shape[0]
    if N < 2:
        raise ValueError("folding needs N >= 2")
    g = V.copy()
    eye = np.eye(L)
    g += (np.einsum("ik,jl->ijkl", h, eye) + np.einsum("jl,ik->ijkl", h, eye)) / (N - 1)
    return g


def strings(L, n):
    return [sum(1 << b for b in c) for c in itertools.combinations(range(L), n)]


def popcount(x):
    return bin(x).count("1")


class StringSpace:
    """Occupation strings of one spin with n electrons in L orbitals."""

    def __init__(self, L, n, irreps):
        self.L, self.n = L, n
        self.strs = strings(L, n) if 0 <= n <= L else []
        self.index = {s: i for i, s in enumerate(self.strs)}
        self.irrep = np.array([_str_irrep(s, irreps) for s in self.strs], dtype=np.int64)
        self._E = {}

    def E(self, p, q):
        """Sparse matrix of a+_p a_q on this string space (same spin)."""
        key = (p, q)
        if key not in self._E:
            rows, cols, vals = [], [], []
            for i, s in enumerate(self.strs):
                if not (s >> q) & 1:
                    continue
                t = s & ~(1 << q)
                if (t >> p) & 1:
                    continue
                sign = (-1) ** popcount(s & ((1 << q) - 1))
                sign *= (-1) ** popcount(t & ((1 << p) - 1))
                u = t | (1 << p)
                rows.append(self.index[u]); cols.append(i); vals.append(sign)
            m = len(self.strs)
            self._E[key] = sp.csr_matrix((vals, (rows, cols)), shape=(m, m))
        return self._E[key]


def _str_irrep(s, irreps):
    ir = 0
    for b in range(len(irreps)):
        if (s >> b) & 1:
            ir ^= irreps[b]
    return ir


class FCISpace:
    """Determinants with n_alpha, n_beta electrons; vectors are C[alpha, beta]."""

    def __init__(self, L, n_alpha, n_beta, irreps, target_irrep=None):
        self.L = L
        self.irreps = list(irreps)
        self.A = StringSpace(L, n_alpha, irreps)
        self.B = StringSpace(L, n_beta, irreps)
        self.shape = (len(self.A.strs), len(self.B.strs))
        if target_irrep is None:
            self.mask = np.ones(self.shape, dtype=bool)
        else:
            self.mask = (self.A.irrep[:, None] ^ self.B.irrep[None, :]) == target_irrep

    def E(self, p, q, C):
        return self.A.E(p, q) @ C + (self.B.E(p, q) @ C.T).T

    def sigma(self, h, V, C, ecore=0.0):
        """H C with H of Sec. 4.1 (h one-body, V two-body in physics notation)."""
        L = self.L
        # one-body part, including the -1/2 sum_q V_pqqs E_ps from E_pr E_qs reordering
        h_eff = h - 0.5 * np.einsum("pqqs->ps", V)
        out = ecore * C
        for p in range(L):
            for q in range(L):
                if h_eff[p, q] != 0.0:
                    out = out + h_eff[p, q] * self.E(p, q, C)
        D = np.empty((L * L,) + C.shape)
        for q in range(L):
            for s in range(L):
                D[q * L + s] = self.E(q, s, C)
        # W_pr = 1/2 sum_qs V_pqrs D_qs
        Vm = V.transpose(0, 2, 1, 3).reshape(L * L, L * L)  # [(p r), (q s)]
        W = 0.5 * (Vm @ D.reshape(L * L, -1)).reshape((L * L,) + C.shape)
        for p in range(L):
            for r in range(L):
                if np.any(W[p * L + r]):
                    out = out + self.E(p, r, W[p * L + r])
        return out

    def E_matrix(self, p, q):
        """Sparse E_pq on the whole (alpha, beta) string product space."""
        nA, nB = self.shape
        return (sp.kron(self.A.E(p, q), sp.identity(nB), format="csr")
                + sp.kron(sp.identity(nA), self.B.E(p, q), format="csr"))

    def hamiltonian_matrix(self, h, V, idx, ecore=0.0):
        """Sparse H (same operator as `sigma`) on the determinants `idx`.  The
        products E_pr E_qs are formed on the whole string space (intermediate
        determinants may lie in other irreps) and restricted at the end."""
        L = self.L
        nA, nB = self.shape
        Em = {(p, q): self.E_matrix(p, q) for p in range(L) for q in range(L)}
        h_eff = h - 0.5 * np.einsum("pqqs->ps", V)
        H = ecore * sp.identity(nA * nB, format="csr")
        for (p, q), M in Em.items():
            if h_eff[p, q] != 0.0:
                H = H + h_eff[p, q] * M
        for p in range(L):
            for r in range(L):
                W = None
                for q in range(L):
                    for s in range(L):
                        v = V[p, q, r, s]
                        if v != 0.0:
                            W = 0.5 * v * Em[(q, s)] if W is None else W + 0.5 * v * Em[(q, s)]
                if W is not None:
                    H = H + Em[(p, r)] @ W
        H = H.tocsr()
        return H[idx][:, idx]

    def s2_matrix(self, idx):
        """Sparse S^2 on the determinants `idx`: S^2 = Sz^2 + Sz + S- S+, with
        S+ = sum_p a+_{p,up} a_{p,dn} (the beta annihilator passes all alpha
        creators, sign (-1)^n_alpha)."""
        nA, nB = self.shape
        n = idx.size
        sz = 0.5 * (self.A.n - self.B.n)
        S2 = (sz * sz + sz) * sp.identity(nA * nB, format="csr")
        if self.B.n > 0 and self.A.n < self.L:
            A1 = StringSpace(self.L, self.A.n + 1, self.irreps)
            B1 = StringSpace(self.L, self.B.n - 1, self.irreps)
            Sp = None
            for p in range(self.L):
                cA = _ladder(self.A, A1, p, create=True)
                aB = _ladder(self.B, B1, p, create=False)
                term = (-1) ** self.A.n * sp.kron(cA, aB, format="csr")
                Sp = term if Sp is None else Sp + term
            S2 = S2 + (Sp.T @ Sp)
        S2 = S2.tocsr()
        return S2[idx][:, idx]

    def s2_apply(self, C):
        """S^2 C = (Sz^2 + Sz) C + S- S+ C with S+ C = (-1)^n_a sum_p c+_p C a_p^T
        (alpha creation on the rows, beta annihilation on the columns)."""
        sz = 0.5 * (self.A.n - self.B.n)
        out = (sz * sz + sz) * C
        if self.B.n > 0 and self.A.n < self.L:
            if not hasattr(self, "_lad"):
                A1 = StringSpace(self.L, self.A.n + 1, self.irreps)
                B1 = StringSpace(self.L, self.B.n - 1, self.irreps)
                self._lad = [(_ladder(self.A, A1, p, True), _ladder(self.B, B1, p, False))
                             for p in range(self.L)]
            sg = (-1) ** self.A.n
            Sp = sum(cA @ C @ aB.T for cA, aB in self._lad) * sg
            out = out + sg * sum(cA.T @ Sp @ aB for cA, aB in self._lad)
        return out

    def s_plus(self, other, C):
        """S+ = sum_p a+_{p,up} a_{p,down}: maps this space's vector into `other`
        (n_alpha + 1, n_beta - 1).  Beta annihilation passes all alpha creators."""
        out = np.zeros(other.shape)
        na = self.A.n
        for p in range(self.L):
            for ib, b in enumerate(self.B.strs):
                if not (b >> p) & 1:
                    continue
                b2 = b & ~(1 << p)
                sb = (-1) ** (na + popcount(b & ((1 << p) - 1)))
                jb = other.B.index[b2]
                for ia, a in enumerate(self.A.strs):
                    if (a >> p) & 1 or C[ia, ib] == 0.0:
                        continue
                    sa = (-1) ** popcount(a & ((1 << p) - 1))
                    out[other.A.index[a | (1 << p)], jb] += sa * sb * C[ia, ib]
        return out

    def s2(self, C):
        """<C|S^2|C> / <C|C> using S^2 = Sz^2 + Sz + S- S+."""
        sz = 0.5 * (self.A.n - self.B.n)
        val = (sz * sz + sz) * np.vdot(C, C)
        if self.B.n > 0 and self.A.n < self.L:
            other = FCISpace(self.L, self.A.n + 1, self.B.n - 1, self.irreps)
            Sp = self.s_plus(other, C)
            val += np.vdot(Sp, Sp)
        return val / np.vdot(C, C)


def fci_ground_state(h, V, N, two_S, irreps, target_irrep, ecore=0.0, nroots=1,
                     dense_max=6000, tol=1e-12, spin_penalty=None):
    """Lowest eigenpair(s) of H in the sector (N, S, irrep) with Sz = S.

    States with total spin above S share the Sz = S sector; an S^2 penalty shift
    (removed afterwards) pushes them up.  Returns (energies, vectors, space)."""
    L = h.shape[0]
    na, nb = (N + two_S) // 2, (N - two_S) // 2
    space = FCISpace(L, na, nb, irreps, target_irrep)
    idx = np.flatnonzero(space.mask.ravel())
    n = idx.size
    shape = space.shape
    S = two_S / 2.0
    if spin_penalty is None:
        spin_penalty = 4.0 * (np.abs(h).sum() + np.abs(V).sum() / L + 1.0)
    other = FCISpace(L, na + 1, nb - 1, irreps) if (nb > 0 and na < L) else None

    def embed(x):
        C = np.zeros(shape[0] * shape[1]); C[idx] = x
        return C.reshape(shape)

    if n <= dense_max:
        Hs = space.hamiltonian_matrix(h, V, idx, ecore)
        S2 = space.s2_matrix(idx)
        Hm = (Hs + spin_penalty * (S2 - S * (S + 1) * sp.identity(n))).toarray()
        Hm = 0.5 * (Hm + Hm.T)
        w, U = np.linalg.eigh(Hm)
        U = U[:, :nroots]
    else:
        def matvec(x):
            C = embed(x)
            y = space.sigma(h, V, C, ecore) + spin_penalty * (space.s2_apply(C) - S * (S + 1) * C)
            return y.ravel()[idx]
        op = spla.LinearOperator((n, n), matvec=matvec, dtype=np.float64)
        w, U = spla.eigsh(op, k=nroots, which="SA", tol=tol)
        order = np.argsort(w); U = U[:, order]
    vecs = [embed(U[:, r]) for r in range(nroots)]
    energies = []
    for C in vecs:
        HC = space.sigma(h, V, C, ecore)
        energies.append(float(np.vdot(C, HC) / np.vdot(C, C)))
    return np.array(energies), vecs, space


def _s_minus(src, dst, C):
    """S- = (S+)^T from src (n_a+1, n_b-1) back to dst, as the transpose of s_plus."""
    out = np.zeros(dst.shape)
    na = dst.A.n
    for p in range(dst.L):
        for ib, b in enumerate(dst.B.strs):
            if not (b >> p) & 1:
                continue
            b2 = b & ~(1 << p)
            sb = (-1) ** (na + popcount(b & ((1 << p) - 1)))
            jb = src.B.index[b2]
            for ia, a in enumerate(dst.A.strs):
                if (a >> p) & 1:
                    continue
                sa = (-1) ** popcount(a & ((1 << p) - 1))
                out[ia, ib] += sa * sb * C[src.A.index[a | (1 << p)], jb]
    return out


def _ladder(src, dst, p, create):
    """Sparse a+_p (create) or a_p on one spin's strings, src -> dst space."""
    rows, cols, vals = [], [], []
    for i, s in enumerate(src.strs):
        occ = (s >> p) & 1
        if create == bool(occ):
            continue
        t = s | (1 << p) if create else s & ~(1 << p)
        rows.append(dst.index[t]); cols.append(i)
        vals.append((-1) ** popcount(s & ((1 << p) - 1)))
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(dst.strs), len(src.strs)))

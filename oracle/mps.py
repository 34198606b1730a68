"""Reduced spin-adapted MPS for the oracle (plain loops, FP64).

Conventions (each a reading of the paper where it leaves the choice open):
  * Sec. 3.2 local states of orbital k: index 0 = empty (s=0, N=0, I=0),
    1 = singly occupied (s=1/2, N=1, I=I_k), 2 = doubly occupied (s=0, N=2, I=0);
    m-resolved |up> = a+_{k,up}|0>, |dn> = a+_{k,dn}|0>, |2> = a+_{k,up} a+_{k,dn}|0>.
    A product state is ordered by orbital index (orbital 0's creators leftmost).
  * Eq. 22: A[k] = <jL mL s ms | jR mR> T[k]; bond 0 is (0,0,I0), bond L is the
    target (S, N, I) (singlet embedding).  The last bond's m is an extra index of the
    state, so Psi_ext = sum_m |Psi_m>|m> (norm = sum over the multiplet).
  * Sectors are (tj, N, I) with tj = 2j.
  * Eq. 25 coefficients S^j are those of |(jL (s1 s2) j) jR>, and the vector the
    effective Hamiltonian acts on is x = sqrt(2 jR + 1) S, for which the Euclidean
    norm is the norm of Psi_ext (so H_eff is symmetric).
"""
import numpy as np
from .su2 import cg, sixj, triangle


def local_states(Ik):
    return [(0, 0, 0), (1, 1, Ik), (0, 2, 0)]  # (2s, N, I) for ls = 0, 1, 2


# m-resolved site states: (ls, 2ms) -> occupation code (bit0 = up, bit1 = down)
SITE_CODE = {(0, 0): 0, (1, 1): 1, (1, -1): 2, (2, 0): 3}


def block_multiplets(irreps):
    """Number of (2j, N, I) multiplets of the product space of the given orbitals."""
    d = {(0, 0, 0): 1}
    for Ik in irreps:
        nd = {}
        for (tj, N, I), m in d.items():
            for (ts, n, Il) in local_states(Ik):
                for tjp in range(abs(tj - ts), tj + ts + 1, 2):
                    key = (tjp, N + n, I ^ Il)
                    nd[key] = nd.get(key, 0) + m
        d = nd
    return d


def fci_bond_dims(irreps, N, two_S, I_G, k):
    """FCI-capped reduced dimension of each sector at bond k (after k orbitals)."""
    left = block_multiplets(irreps[:k])
    right = block_multiplets(irreps[k:])
    out = {}
    for (tj, n, I), m in left.items():
        r = 0
        for (tjr, nr, Ir), mr in right.items():
            if nr == N - n and Ir == (I_G ^ I) and triangle(tj, tjr, two_S):
                r += mr
        if r:
            out[(tj, n, I)] = min(m, r)
    return out


def sector_order(keys):
    return sorted(keys, key=lambda s: (s[1], s[0], s[2]))


def distribute(fci, D):
    """Sec. 4.3: D spread equally over the sectors, none above its FCI dimension
    (water-filling in sector order until D is used or every sector is full)."""
    keys = sector_order(fci)
    alloc = {k: 0 for k in keys}
    left = D
    while left > 0:
        open_ = [k for k in keys if alloc[k] < fci[k]]
        if not open_:
            break
        share = max(1, left // len(open_))
        for k in open_:
            add = min(share, fci[k] - alloc[k], left)
            alloc[k] += add
            left -= add
            if left == 0:
                break
    return {k: v for k, v in alloc.items() if v > 0}


class MPS:
    """Reduced tensors T[k][(ls, left_sector, right_sector)] of shape (dL, dR)."""

    def __init__(self, irreps, N, two_S, I_G, dims):
        self.irreps = list(irreps)
        self.L = len(irreps)
        self.N, self.two_S, self.I_G = N, two_S, I_G
        self.dims = [dict(d) for d in dims]  # len L+1, sector -> dim
        self.T = [dict() for _ in range(self.L)]

    def blocks(self, k):
        """All allowed (ls, lsec, rsec) for site k given current bond dims."""
        out = []
        for lsec in sector_order(self.dims[k]):
            for ls, (ts, n, Il) in enumerate(local_states(self.irreps[k])):
                for rsec in sector_order(self.dims[k + 1]):
                    if rsec[1] == lsec[1] + n and rsec[2] == (lsec[2] ^ Il) \
                            and triangle(lsec[0], ts, rsec[0]):
                        out.append((ls, lsec, rsec))
        return out

    def copy(self):
        m = MPS(self.irreps, self.N, self.two_S, self.I_G, self.dims)
        m.T = [{k: v.copy() for k, v in t.items()} for t in self.T]
        return m


def initial_dims(irreps, N, two_S, I_G, D):
    L = len(irreps)
    return [distribute(fci_bond_dims(irreps, N, two_S, I_G, k), D) for k in range(L + 1)]


def random_mps(irreps, N, two_S, I_G, D, values):
    """Initial MPS of Sec. 4.3 filled from the stream `values` (consumed in order:
    site, then block order, then row-major)."""
    m = MPS(irreps, N, two_S, I_G, initial_dims(irreps, N, two_S, I_G, D))
    pos = 0
    for k in range(m.L):
        for key in m.blocks(k):
            dL, dR = m.dims[k][key[1]], m.dims[k + 1][key[2]]
            n = dL * dR
            m.T[k][key] = np.asarray(values[pos:pos + n], dtype=np.float64).reshape(dL, dR)
            pos += n
    return m


def _ts(m, k, ls):
    return local_states(m.irreps[k])[ls][0]


def right_normalize_site(m, k, rank_tol=1e-13):
    """Make T[k] right-normalised (reduced form of Eq. 6:
    sum (2jR+1)/(2jL+1) T T^T = 1 per left sector) by an SVD per left sector; the
    remaining factor is pushed into T[k-1] (or returned for k == 0)."""
    new = {}
    carry = {}
    newdims = {}
    for lsec in sector_order(m.dims[k]):
        keys = [key for key in m.T[k] if key[1] == lsec]
        if not keys:
            continue
        w = [np.sqrt((key[2][0] + 1) / (lsec[0] + 1)) for key in keys]
        M = np.concatenate([m.T[k][key] * wi for key, wi in zip(keys, w)], axis=1)
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        r = int(np.sum(s > rank_tol * max(s[0], 1e-300))) if s.size else 0
        if r == 0:
            continue
        newdims[lsec] = r
        carry[lsec] = U[:, :r] * s[:r]
        off = 0
        for key, wi in zip(keys, w):
            dR = m.T[k][key].shape[1]
            new[key] = Vt[:r, off:off + dR] / wi
            off += dR
    m.T[k] = new
    if k == 0:
        return carry
    m.dims[k] = newdims
    prev = {}
    for key, blk in m.T[k - 1].items():
        if key[2] in carry:
            prev[key] = blk @ carry[key[2]]
    m.T[k - 1] = prev
    return None


def right_canonicalize(m):
    """Right-normalise sites L-1..1 and normalise the state (Psi_ext has norm 1)."""
    for k in range(m.L - 1, 0, -1):
        right_normalize_site(m, k)
    nrm2 = sum((key[2][0] + 1) * np.sum(b * b) for key, b in m.T[0].items())
    for key in m.T[0]:
        m.T[0][key] = m.T[0][key] / np.sqrt(nrm2)
    return m


# ---------------------------------------------------------------- two-site object

def two_site_blocks(m, i):
    """Blocks of x for sites (i, i+1): key (lsec, ls1, ls2, tj, rsec)."""
    out = []
    loc1, loc2 = local_states(m.irreps[i]), local_states(m.irreps[i + 1])
    for lsec in sector_order(m.dims[i]):
        for ls1, (t1, n1, I1) in enumerate(loc1):
            for ls2, (t2, n2, I2) in enumerate(loc2):
                for rsec in sector_order(m.dims[i + 2]):
                    if rsec[1] != lsec[1] + n1 + n2 or rsec[2] != (lsec[2] ^ I1 ^ I2):
                        continue
                    for tj in range(abs(t1 - t2), t1 + t2 + 1, 2):
                        if triangle(lsec[0], tj, rsec[0]):
                            out.append((lsec, ls1, ls2, tj, rsec))
    return out


def tt_to_x(m, i):
    """Eq. 25, then x = sqrt(2jR+1) S."""
    loc1, loc2 = local_states(m.irreps[i]), local_states(m.irreps[i + 1])
    x = {}
    for key in two_site_blocks(m, i):
        lsec, ls1, ls2, tj, rsec = key
        t1, t2 = loc1[ls1][0], loc2[ls2][0]
        tjL, tjR = lsec[0], rsec[0]
        acc = np.zeros((m.dims[i][lsec], m.dims[i + 2][rsec]))
        for msec in m.dims[i + 1]:
            k1, k2 = (ls1, lsec, msec), (ls2, msec, rsec)
            if k1 not in m.T[i] or k2 not in m.T[i + 1]:
                continue
            tjM = msec[0]
            c = (np.sqrt(tj + 1) * _phase(tjL + tjR + t1 + t2) * np.sqrt(tjM + 1)
                 * sixj(tjL, tjR, tj, t2, t1, tjM))
            if c != 0.0:
                acc += c * (m.T[i][k1] @ m.T[i + 1][k2])
        x[key] = np.sqrt(tjR + 1) * acc
    return x


def x_to_tt(m, i, x, mid_sectors):
    """Eq. 26 with S = x / sqrt(2jR+1): TT[(ls1, ls2, lsec, msec, rsec)]."""
    loc1, loc2 = local_states(m.irreps[i]), local_states(m.irreps[i + 1])
    tt = {}
    for (lsec, ls1, ls2, tj, rsec), blk in x.items():
        t1, n1, I1 = loc1[ls1]
        t2 = loc2[ls2][0]
        tjL, tjR = lsec[0], rsec[0]
        nM, IM = lsec[1] + n1, lsec[2] ^ I1
        for tjM in range(abs(tjL - t1), tjL + t1 + 1, 2):
            msec = (tjM, nM, IM)
            if msec not in mid_sectors or not triangle(tjM, t2, tjR):
                continue
            c = (np.sqrt(tjM + 1) * _phase(tjL + tjR + t1 + t2)
                 * sixj(tjL, tjR, tj, t2, t1, tjM) * np.sqrt(tj + 1))
            if c == 0.0:
                continue
            key = (ls1, ls2, lsec, msec, rsec)
            tt[key] = tt.get(key, 0.0) + c * blk / np.sqrt(tjR + 1)
    return tt


def _phase(two_x):
    # (-1)^(jL + jR + s1 + s2) with the exponent given doubled (always even here)
    assert two_x % 2 == 0
    return -1.0 if (two_x // 2) % 2 else 1.0


def mid_sector_candidates(m, i):
    loc1 = local_states(m.irreps[i])
    cands = set()
    for lsec in m.dims[i]:
        for (t1, n1, I1) in loc1:
            for tjM in range(abs(lsec[0] - t1), lsec[0] + t1 + 1, 2):
                cands.add((tjM, lsec[1] + n1, lsec[2] ^ I1))
    return cands


def svd_truncate(m, i, x, D, direction, zero_tol=1e-13):
    """Eqs. 26-28 and Eq. 15: back-transform, SVD per (jM, NM, IM) of TT with the
    columns weighted by sqrt((2jR+1)/(2jM+1)), keep the D largest lambda (ties:
    larger lambda first, then sector order, then index), kappa normalised with
    sum (2jM+1) lambda^2; writes T[i], T[i+1] (direction 'right': A[i]=U,
    A[i+1]=kappa V; 'left': A[i]=U kappa, A[i+1]=V).  Returns discarded weight
    sum over dropped (2jM+1) kappa^2."""
    L = m.L
    fci_mid = fci_bond_dims(m.irreps, m.N, m.two_S, m.I_G, i + 1)
    cands = [s for s in sector_order(mid_sector_candidates(m, i)) if s in fci_mid]
    tt = x_to_tt(m, i, x, set(cands))
    groups = []
    for msec in cands:
        rows = sorted({(k[2], k[0]) for k in tt if k[3] == msec},
                      key=lambda r: ((r[0][1], r[0][0], r[0][2]), r[1]))
        cols = sorted({(k[4], k[1]) for k in tt if k[3] == msec},
                      key=lambda c: ((c[0][1], c[0][0], c[0][2]), c[1]))
        if not rows or not cols:
            continue
        rdim = [m.dims[i][r[0]] for r in rows]
        cdim = [m.dims[i + 2][c[0]] for c in cols]
        M = np.zeros((sum(rdim), sum(cdim)))
        roff = np.concatenate([[0], np.cumsum(rdim)])
        coff = np.concatenate([[0], np.cumsum(cdim)])
        for a, (lsec, ls1) in enumerate(rows):
            for b, (rsec, ls2) in enumerate(cols):
                key = (ls1, ls2, lsec, msec, rsec)
                if key in tt:
                    w = np.sqrt((rsec[0] + 1) / (msec[0] + 1))
                    M[roff[a]:roff[a + 1], coff[b]:coff[b + 1]] = tt[key] * w
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        groups.append((msec, rows, cols, roff, coff, U, s, Vt))
    # global selection of the D largest lambda
    cand = []
    for gi, g in enumerate(groups):
        for a, lam in enumerate(g[6]):
            cand.append((-lam, gi, a))
    cand.sort()
    norm2 = sum((g[0][0] + 1) * float(np.sum(g[6] ** 2)) for g in groups)
    smax = -cand[0][0] if cand else 0.0
    kept = [c for c in cand[:D] if -c[0] > zero_tol * smax]
    keep_set = {(c[1], c[2]) for c in kept}
    w_disc = 0.0
    for gi, g in enumerate(groups):
        for a, lam in enumerate(g[6]):
            if (gi, a) not in keep_set:
                w_disc += (g[0][0] + 1) * lam * lam / norm2
    newdims = {}
    Ti, Tj = {}, {}
    for gi, (msec, rows, cols, roff, coff, U, s, Vt) in enumerate(groups):
        sel = [a for a in range(s.size) if (gi, a) in keep_set]
        if not sel:
            continue
        newdims[msec] = len(sel)
        kappa = s[sel] / np.sqrt(norm2)
        Us, Vs = U[:, sel], Vt[sel, :]
        if direction == "left":
            Us = Us * kappa
        else:
            Vs = kappa[:, None] * Vs
        for a, (lsec, ls1) in enumerate(rows):
            Ti[(ls1, lsec, msec)] = Us[roff[a]:roff[a + 1], :].copy()
        for b, (rsec, ls2) in enumerate(cols):
            w = np.sqrt((msec[0] + 1) / (rsec[0] + 1))
            Tj[(ls2, msec, rsec)] = w * Vs[:, coff[b]:coff[b + 1]]
    m.dims[i + 1] = newdims
    m.T[i] = Ti
    m.T[i + 1] = Tj
    return w_disc, kept, groups


# ----------------------------------------------------- expansion into determinants

def left_basis(m, k):
    """States |jL mL alpha> of orbitals 0..k-1 as arrays [d, 2j+1, n_cfg] over the
    list of occupation codes (base-4 digit per orbital: bit0 up, bit1 down)."""
    basis = {(0, 0, 0): (np.ones((1, 1, 1)), [0])}
    for site in range(k):
        loc = local_states(m.irreps[site])
        nb = {}
        for (ls, lsec, rsec), T in m.T[site].items():
            if lsec not in basis:
                continue
            vec, cfgs = basis[lsec]
            ts = loc[ls][0]
            tjL, tjR = lsec[0], rsec[0]
            if rsec not in nb:
                nb[rsec] = {}
            acc = nb[rsec]
            for imR, tmR in enumerate(range(-tjR, tjR + 1, 2)):
                for imL, tmL in enumerate(range(-tjL, tjL + 1, 2)):
                    tms = tmR - tmL
                    if abs(tms) > ts:
                        continue
                    c = cg(tjL, tmL, ts, tms, tjR, tmR)
                    if c == 0.0:
                        continue
                    code = SITE_CODE[(ls, tms)]
                    newcfg = tuple(cf + code * 4 ** site for cf in cfgs)
                    contrib = c * np.einsum("ab,ac->bc", T, vec[:, imL, :])
                    for jc, cf in enumerate(newcfg):
                        key = (imR, cf)
                        acc[key] = acc.get(key, 0.0) + contrib[:, jc]
        basis = {}
        for rsec, acc in nb.items():
            cfgs = sorted({cf for (_, cf) in acc})
            pos = {cf: j for j, cf in enumerate(cfgs)}
            d = m.T[site][next(kk for kk in m.T[site] if kk[2] == rsec)].shape[1]
            arr = np.zeros((d, rsec[0] + 1, len(cfgs)))
            for (imR, cf), v in acc.items():
                arr[:, imR, pos[cf]] += v
            basis[rsec] = (arr, cfgs)
    return basis


def right_basis(m, k):
    """Functions phi_{jR mR alpha} of orbitals k..L-1 and the final index f, as
    arrays [d, 2j+1, n_cfg, 2S+1]; the orbital k digit is the lowest."""
    tS = m.two_S
    fin = (tS, m.N, m.I_G)
    arr0 = np.zeros((1, tS + 1, 1, tS + 1))
    for f in range(tS + 1):
        arr0[0, f, 0, f] = 1.0
    basis = {fin: (arr0, [0])}
    for site in range(m.L - 1, k - 1, -1):
        loc = local_states(m.irreps[site])
        nb = {}
        for (ls, lsec, rsec), T in m.T[site].items():
            if rsec not in basis:
                continue
            vec, cfgs = basis[rsec]
            ts = loc[ls][0]
            tjL, tjR = lsec[0], rsec[0]
            acc = nb.setdefault(lsec, {})
            for imL, tmL in enumerate(range(-tjL, tjL + 1, 2)):
                for imR, tmR in enumerate(range(-tjR, tjR + 1, 2)):
                    tms = tmR - tmL
                    if abs(tms) > ts:
                        continue
                    c = cg(tjL, tmL, ts, tms, tjR, tmR)
                    if c == 0.0:
                        continue
                    code = SITE_CODE[(ls, tms)]
                    contrib = c * np.einsum("ab,bcf->acf", T, vec[:, imR, :, :])
                    for jc, cf in enumerate(cfgs):
                        key = (imL, code + 4 * cf)
                        acc[key] = acc.get(key, 0.0) + contrib[:, jc, :]
        basis = {}
        for lsec, acc in nb.items():
            cfgs = sorted({cf for (_, cf) in acc})
            pos = {cf: j for j, cf in enumerate(cfgs)}
            d = m.T[site][next(kk for kk in m.T[site] if kk[1] == lsec)].shape[0]
            arr = np.zeros((d, lsec[0] + 1, len(cfgs), tS + 1))
            for (imL, cf), v in acc.items():
                arr[:, imL, pos[cf], :] += v
            basis[lsec] = (arr, cfgs)
    return basis


def _config_to_det(code, L):
    """Interleaved occupation code -> (alpha bits, beta bits, sign of reordering to
    all-alpha-then-all-beta creators)."""
    a = b = 0
    ups = []
    dns = []
    for k in range(L):
        d = (code >> (2 * k)) & 3
        if d & 1:
            a |= 1 << k
        if d & 2:
            b |= 1 << k
        ups.append(d & 1)
        dns.append((d >> 1) & 1)
    # move each down creator (orbital k) right past the up creators of orbitals > k
    n = 0
    for k in range(L):
        if dns[k]:
            n += sum(ups[k + 1:])
    return a, b, (-1.0 if n % 2 else 1.0)


class TwoSiteProjector:
    """P mapping x (the reduced two-site vector) to Psi_ext in the determinant basis,
    one matrix per final index f (Sz = (2f - 2S)/2)."""

    def __init__(self, m, i, spaces):
        self.m, self.i = m, i
        self.blocks = two_site_blocks(m, i)
        lb = left_basis(m, i)
        rb = right_basis(m, i + 2)
        loc1, loc2 = local_states(m.irreps[i]), local_states(m.irreps[i + 1])
        L = m.L
        tS = m.two_S
        offs = [0]
        for key in self.blocks:
            offs.append(offs[-1] + m.dims[i][key[0]] * m.dims[i + 2][key[4]])
        self.offs = offs
        self.n = offs[-1]
        self.P = []
        det_cache = {}

        def rows_for(lcfg, rcfg, code12, space, nB):
            key = (id(lcfg), id(rcfg), code12, id(space))
            if key in det_cache:
                return det_cache[key]
            rows = np.full((len(lcfg), len(rcfg)), -1, dtype=np.int64)
            sg = np.zeros((len(lcfg), len(rcfg)))
            for jl, cl in enumerate(lcfg):
                for jr, cr in enumerate(rcfg):
                    code = cl + code12 * 4 ** i + cr * 4 ** (i + 2)
                    a, b, sgn = _config_to_det(code, L)
                    ia = space.A.index.get(a)
                    ib = space.B.index.get(b)
                    if ia is None or ib is None:
                        continue
                    rows[jl, jr] = ia * nB + ib
                    sg[jl, jr] = sgn
            det_cache[key] = (rows, sg)
            return rows, sg

        for f in range(tS + 1):
            space = spaces[f]
            nA, nB = space.shape
            P = np.zeros((nA * nB, self.n))
            for bi, (lsec, ls1, ls2, tj, rsec) in enumerate(self.blocks):
                if lsec not in lb or rsec not in rb:
                    continue
                lv, lcfg = lb[lsec]
                rv, rcfg = rb[rsec]
                t1, t2 = loc1[ls1][0], loc2[ls2][0]
                tjL, tjR = lsec[0], rsec[0]
                cols = np.arange(offs[bi], offs[bi + 1])
                for imR, tmR in enumerate(range(-tjR, tjR + 1, 2)):
                    for imL, tmL in enumerate(range(-tjL, tjL + 1, 2)):
                        tmj = tmR - tmL
                        c2 = cg(tjL, tmL, tj, tmj, tjR, tmR)
                        if c2 == 0.0:
                            continue
                        for tm1 in range(-t1, t1 + 1, 2):
                            tm2 = tmj - tm1
                            if abs(tm2) > t2:
                                continue
                            c1 = cg(t1, tm1, t2, tm2, tj, tmj)
                            if c1 == 0.0:
                                continue
                            code12 = SITE_CODE[(ls1, tm1)] + 4 * SITE_CODE[(ls2, tm2)]
                            coef = c1 * c2 / np.sqrt(tjR + 1)
                            rows, sg = rows_for(lcfg, rcfg, code12, space, nB)
                            ok = rows >= 0
                            if not np.any(ok):
                                continue
                            # contrib[jl, jr, aL, aR] = lv[aL, imL, jl] rv[aR, imR, jr, f]
                            contrib = np.einsum("aj,bk->jkab", lv[:, imL, :], rv[:, imR, :, f])
                            contrib = contrib * (sg * coef)[:, :, None, None]
                            r = rows[ok]
                            P[r[:, None], cols[None, :]] += contrib[ok].reshape(r.size, -1)
            self.P.append(P)

    def flatten(self, x):
        return np.concatenate([x[key].ravel() for key in self.blocks]) if self.blocks else np.zeros(0)

    def unflatten(self, v):
        out = {}
        for bi, key in enumerate(self.blocks):
            dL, dR = self.m.dims[self.i][key[0]], self.m.dims[self.i + 2][key[4]]
            out[key] = v[self.offs[bi]:self.offs[bi + 1]].reshape(dL, dR)
        return out

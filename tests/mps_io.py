"""Serialise an oracle MPS into the library's dmrg_set_mps format and map the
library's two-site block table onto the oracle's block keys (test helpers)."""
import struct

import numpy as np

from oracle.mps import sector_order


def mps_to_bytes(m):
    out = [struct.pack("<6i", 0x444D5247, 1, m.L, m.N, m.two_S, m.I_G)]
    orders = []
    for k in range(m.L + 1):
        secs = sector_order(m.dims[k])
        orders.append({s: i for i, s in enumerate(secs)})
        out.append(struct.pack("<i", len(secs)))
        for s in secs:
            out.append(struct.pack("<4i", s[0], s[1], s[2], m.dims[k][s]))
    for k in range(m.L):
        blocks = [(key, blk) for key, blk in m.T[k].items()
                  if key[1] in orders[k] and key[2] in orders[k + 1]]
        out.append(struct.pack("<i", len(blocks)))
        for (ls, lsec, rsec), blk in blocks:
            out.append(struct.pack("<3i", ls, orders[k][lsec], orders[k + 1][rsec]))
            out.append(np.ascontiguousarray(blk, dtype="<f8").tobytes())
    return b"".join(out)


def layout_keys(table):
    """Oracle block keys (lsec, ls1, ls2, tj, rsec) of the library's block table rows."""
    keys = []
    for row in table:
        tjL, nL, iL, ls1, ls2, tj, tjR, nR, iR, dL, dR, off = (int(v) for v in row)
        keys.append(((tjL, nL, iL), ls1, ls2, tj, (tjR, nR, iR)))
    return keys


def oracle_x_to_lib(x_blocks, table, n):
    v = np.zeros(n)
    for key, row in zip(layout_keys(table), table):
        dL, dR, off = int(row[9]), int(row[10]), int(row[11])
        if key in x_blocks:
            v[off:off + dL * dR] = x_blocks[key].ravel()
    return v


def lib_x_to_oracle(v, table):
    out = {}
    for key, row in zip(layout_keys(table), table):
        dL, dR, off = int(row[9]), int(row[10]), int(row[11])
        out[key] = v[off:off + dL * dR].reshape(dL, dR).copy()
    return out


def mps_from_bytes(data, irreps):
    """The library's serialised MPS (dmrg_get_mps) as an oracle MPS object."""
    from oracle.mps import MPS
    pos = 0

    def take(fmt):
        nonlocal pos
        v = struct.unpack_from(fmt, data, pos)
        pos += struct.calcsize(fmt)
        return v

    magic, ver, L, N, two_S, I_G = take("<6i")
    assert magic == 0x444D5247 and ver == 1 and L == len(irreps)
    secs, dims = [], []
    for _ in range(L + 1):
        (ns,) = take("<i")
        s = [take("<4i") for _ in range(ns)]
        secs.append([(t[0], t[1], t[2]) for t in s])
        dims.append({(t[0], t[1], t[2]): t[3] for t in s})
    m = MPS(irreps, N, two_S, I_G, dims)
    for k in range(L):
        (nb,) = take("<i")
        for _ in range(nb):
            ls, li, ri = take("<3i")
            lsec, rsec = secs[k][li], secs[k + 1][ri]
            dL, dR = dims[k][lsec], dims[k + 1][rsec]
            blk = np.frombuffer(data, dtype="<f8", count=dL * dR, offset=pos).reshape(dL, dR).copy()
            pos += 8 * dL * dR
            m.T[k][(ls, lsec, rsec)] = blk
    assert pos == len(data)
    return m


def truncation_bound(groups, D):
    """Element-wise tolerance of the library's truncated two-site tensor against the
    oracle's for a cut keeping D reduced values: the library decomposes through Gram
    matrices (M M^T or M^T M) formed with an error ~ eps |M|^2, so the kept subspace moves
    by ~ eps lambda_max^2 / gap with gap = lambda_D^2 - lambda_{D+1}^2 (Davis-Kahan), and
    it treats values below 3e-8 lambda_max as zero (their weight bounds the rest)."""
    import numpy as np
    vals = sorted(((float(v), g[0][0] + 1) for g in groups for v in g[6]), reverse=True)
    lam = np.array([v for v, _ in vals])
    kept = min(D, int(np.sum(lam > 3e-8 * lam[0])))
    gap = lam[kept - 1] ** 2 - lam[kept] ** 2 if kept < lam.size else lam[0] ** 2
    # values the oracle keeps (among the first D) but the library treats as zero
    tiny = np.sqrt(sum(w * v * v for v, w in vals[:D] if v <= 3e-8 * lam[0]))
    return 1e-12 + 64 * 2.2e-16 * lam[0] ** 2 / max(gap, 1e-300) + 2.0 * tiny


def widest_cut(groups, D, window):
    """The cut within D +- window with the largest gap lambda_D^2 - lambda_{D+1}^2 of the
    reduced spectrum (so that the truncation is well defined)."""
    import numpy as np
    lam = np.sort(np.concatenate([g[6] for g in groups]))[::-1]
    best, best_gap = D, -1.0
    for d in range(max(1, D - window), min(lam.size - 1, D + window) + 1):
        g = lam[d - 1] ** 2 - lam[d] ** 2
        if g > best_gap:
            best, best_gap = d, g
    return best, best_gap / lam[0] ** 2

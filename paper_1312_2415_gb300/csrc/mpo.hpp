// Renormalized and complementary operators of the two-site spin-adapted DMRG
// (Sec. 2.5) organised as a chain of site recursions.
//
// A bipartition of the orbitals at bond k (left block = orbitals 0..k-1) writes the
// folded Hamiltonian of Eq. 11 as H = sum_b sum_q L_{b,q} R_{b,q}.  The left factors
// are bare operators on the left block (identity, block Hamiltonian, b+_p, b_p, the
// pair operators A, Abar, B of spin 0 and 1) and complementary operators that carry
// the integrals for one index outside the block (Rc_r, the three-operator sums of
// Eq. 12, and its conjugate).  Their partners R on the right block follow from the
// same recursion read backwards.  Every factor is an irreducible tensor operator
// (b+ and b of Eqs. 23-24 are doublets), so only reduced blocks are stored.
//
// The recursions are written in m-resolved second quantisation (spin projections
// explicit, Jordan-Wigner order = orbital order, left block first) and reduced
// numerically: each (source op, target op, rule) carries a "pattern" of site
// matrices indexed by the two operators' components, from which the planner derives
// the 6-j/9-j recoupling factors as explicit Clebsch-Gordan sums.
#pragma once
#include <cstdint>
#include <unordered_map>
#include <vector>

namespace dmrg {

enum OpType : int { OP_I = 0, OP_H, OP_CRE, OP_ANN, OP_A, OP_AD, OP_B, OP_RC, OP_RCD };

struct OpKey {
  int type = 0, p = 0, q = 0, tk = 0;
  bool operator==(const OpKey& o) const {
    return type == o.type && p == o.p && q == o.q && tk == o.tk;
  }
  uint64_t code() const {
    return (uint64_t)type | ((uint64_t)(p + 1) << 8) | ((uint64_t)(q + 1) << 24) |
           ((uint64_t)tk << 40);
  }
};

struct OpInfo {
  OpKey key;
  int tk, dn, ir, parity;
};

// Operator set of the bipartition at bond k of an L-orbital chain.
struct OpSet {
  std::vector<OpInfo> ops;
  std::unordered_map<uint64_t, int> index;
  int find(const OpKey& k) const {
    auto it = index.find(k.code());
    return it == index.end() ? -1 : it->second;
  }
};
OpSet make_op_set(int k, int L, const std::vector<int>& orb_ir);

// Site pattern: for component indices (qa, qb) a 4x4 matrix on the m-resolved site
// basis {|0>, |up>, |dn>, |2>} (row = bra).  w[((qa*(tkb+1))+qb)*16 + bra*4 + ket].
struct Pattern {
  int tka = 0, tkb = 0, pa = 0, pO = 0;
  std::vector<double> w;
  double at(int qa, int qb, int bra, int ket) const {
    return w[((size_t)(qa * (tkb + 1) + qb)) * 16 + bra * 4 + ket];
  }
};

struct PatternTable {
  std::vector<Pattern> pats;
  std::unordered_map<uint64_t, std::vector<int>> by_hash;
  int intern(const Pattern& p);
};

// One term of the recursion at a site: L_b(bond k+1) += scalar * [L_a(bond k) x pattern].
// scalar = gc * g[gi] for a term that carries one folded integral, gc for gi < 0.
struct WEntry {
  int a, b, pattern;
  double scalar;
  int64_t gi;
  double gc;
};

// Integrals after the folding of Eq. 11: g[((p*L+q)*L+r)*L+s] = (pq|h|rs).  With
// keep_zero set, the recursion keeps the terms of integrals that vanish but are allowed
// by the point group (ir = orbital irreps), so that derivatives with respect to every
// allowed integral can be taken on it.
struct Integrals {
  int L = 0;
  std::vector<double> g;
  bool keep_zero = false;
  std::vector<int> ir;
  int64_t idx(int p, int q, int r, int s) const { return (((int64_t)p * L + q) * L + r) * L + s; }
  double at(int p, int q, int r, int s) const { return g[(size_t)idx(p, q, r, s)]; }
  bool use(int p, int q, int r, int s) const {
    return at(p, q, r, s) != 0.0 || (keep_zero && (ir[p] ^ ir[q] ^ ir[r] ^ ir[s]) == 0);
  }
};

// Recursion entries of site k, mapping bond-k operators to bond-(k+1) operators.
std::vector<WEntry> build_site_recursion(int k, const OpSet& from, const OpSet& to,
                                         const Integrals& g, PatternTable& pt);

}  // namespace dmrg

// Site recursions of the renormalized / complementary operators (see mpo.hpp).
//
// Elementary m-resolved operators (left block, Jordan-Wigner order):
//   C(p,s) = a+_{ps}, A(p,s) = a_{ps}, CC = a+_{ps} a+_{qt}, AA = a_{ps} a_{qt},
//   CA = a+_{ps} a_{qt}, RC(r,s) = sum_{pqu in block} g_{pqru} a+_{ps} sum_t a+_{qt} a_{ut}
//   (Eq. 12's three-operator complementary sum) and RCD = RC^dagger.
// Multiplets (Eqs. 23-24): b+_{p,s} = a+_{ps}; b_{p,s} = (-1)^(1/2-s) a_{p,-s};
//   A^K_pq = [b+_p b+_q]^K, Abar^K_pq = [b_p b_q]^K, B^K_pt = [b+_p b_t]^K,
//   Rc_r with components a+-like, Rcbar_{r,s} = (-1)^(1/2-s) Rc^dagger_{r,-s}.
// Only p <= q pair multiplets are stored ([b_q b_p]^K = (-1)^K [b_p b_q]^K);
// A^1_pp = Abar^1_pp = 0.  The conjugation and commutation relations of Eq. 13 are
// what allow this reduced storage.
#include "mpo.hpp"

#include <array>
#include <cmath>
#include <map>
#include <stdexcept>
#include <tuple>

#include "su2.hpp"

namespace dmrg {

namespace {

using Mat4 = std::array<double, 16>;

Mat4 zero4() { Mat4 m; m.fill(0.0); return m; }
Mat4 eye4() { Mat4 m = zero4(); for (int i = 0; i < 4; ++i) m[i * 4 + i] = 1.0; return m; }
Mat4 cdag(int s) {  // a+_{s} on one orbital: |0>->|s>, |-s> -> +/-|2>
  Mat4 m = zero4();
  if (s > 0) { m[1 * 4 + 0] = 1.0; m[3 * 4 + 2] = 1.0; }
  else { m[2 * 4 + 0] = 1.0; m[3 * 4 + 1] = -1.0; }
  return m;
}
Mat4 tr(const Mat4& a) { Mat4 m; for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) m[i * 4 + j] = a[j * 4 + i]; return m; }
Mat4 cann(int s) { return tr(cdag(s)); }
Mat4 mul(const Mat4& a, const Mat4& b) {
  Mat4 m = zero4();
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k)
      if (a[i * 4 + k] != 0.0)
        for (int j = 0; j < 4; ++j) m[i * 4 + j] += a[i * 4 + k] * b[k * 4 + j];
  return m;
}
Mat4 add(const Mat4& a, const Mat4& b) { Mat4 m; for (int i = 0; i < 16; ++i) m[i] = a[i] + b[i]; return m; }
Mat4 scale(const Mat4& a, double s) { Mat4 m; for (int i = 0; i < 16; ++i) m[i] = a[i] * s; return m; }
Mat4 num() { return add(mul(cdag(1), cann(1)), mul(cdag(-1), cann(-1))); }
const int kSiteN[4] = {0, 1, 1, 2};
int mat_parity(const Mat4& a) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      if (std::fabs(a[i * 4 + j]) > 0) return (kSiteN[i] - kSiteN[j]) & 1;
  return 0;
}

enum { E_I, E_H, E_C, E_A, E_CC, E_AA, E_CA, E_RC, E_RCD };
struct Elem { int kind, p, sp, q, sq; };
int elem_parity(const Elem& e) {
  return (e.kind == E_C || e.kind == E_A || e.kind == E_RC || e.kind == E_RCD) ? 1 : 0;
}
Elem adjoint(const Elem& e) {
  switch (e.kind) {
    case E_C: return {E_A, e.p, e.sp, 0, 0};
    case E_A: return {E_C, e.p, e.sp, 0, 0};
    case E_CC: return {E_AA, e.q, e.sq, e.p, e.sp};
    case E_AA: return {E_CC, e.q, e.sq, e.p, e.sp};
    case E_CA: return {E_CA, e.q, e.sq, e.p, e.sp};
    case E_RC: return {E_RCD, e.p, e.sp, 0, 0};
    case E_RCD: return {E_RC, e.p, e.sp, 0, 0};
    default: return e;
  }
}

struct Src { OpKey a; int tqa; double c; };
inline double ph_a(int s) { return s > 0 ? -1.0 : 1.0; }  // (-1)^(1/2+s)
inline double ph_b(int m) { return m > 0 ? 1.0 : -1.0; }  // (-1)^(1/2-m)

void pair_expand(int type, int p, int m1, int q, int m2, double pre, std::vector<Src>& out) {
  // operator X_{p m1} X_{q m2} of two doublets -> pair multiplets (p <= q stored)
  if (p == q) {
    if (m1 == m2) return;
    double c = clebsch(1, m1, 1, m2, 0, 0);
    out.push_back({{type, p, p, 0}, 0, pre * c});
  } else if (p < q) {
    for (int tk = 0; tk <= 2; tk += 2) {
      double c = clebsch(1, m1, 1, m2, tk, m1 + m2);
      if (c != 0.0) out.push_back({{type, p, q, tk}, m1 + m2, pre * c});
    }
  } else {
    for (int tk = 0; tk <= 2; tk += 2) {
      double c = clebsch(1, m2, 1, m1, tk, m1 + m2);
      if (c != 0.0) out.push_back({{type, q, p, tk}, m1 + m2, -pre * c});
    }
  }
}

void expand(const Elem& e, std::vector<Src>& out) {
  out.clear();
  switch (e.kind) {
    case E_I: out.push_back({{OP_I, -1, -1, 0}, 0, 1.0}); break;
    case E_H: out.push_back({{OP_H, -1, -1, 0}, 0, 1.0}); break;
    case E_C: out.push_back({{OP_CRE, e.p, -1, 1}, e.sp, 1.0}); break;
    case E_A: out.push_back({{OP_ANN, e.p, -1, 1}, -e.sp, ph_a(e.sp)}); break;
    case E_CC: pair_expand(OP_A, e.p, e.sp, e.q, e.sq, 1.0, out); break;
    case E_AA: pair_expand(OP_AD, e.p, -e.sp, e.q, -e.sq, ph_a(e.sp) * ph_a(e.sq), out); break;
    case E_CA:
      for (int tk = 0; tk <= 2; tk += 2) {
        double c = clebsch(1, e.sp, 1, -e.sq, tk, e.sp - e.sq);
        if (c != 0.0) out.push_back({{OP_B, e.p, e.q, tk}, e.sp - e.sq, ph_a(e.sq) * c});
      }
      break;
    case E_RC: out.push_back({{OP_RC, e.p, -1, 1}, e.sp, 1.0}); break;
    case E_RCD: out.push_back({{OP_RCD, e.p, -1, 1}, -e.sp, ph_a(e.sp)}); break;
  }
}

void components(const OpKey& b, int tqb, std::vector<std::pair<Elem, double>>& out) {
  out.clear();
  switch (b.type) {
    case OP_I: out.push_back({{E_I, 0, 0, 0, 0}, 1.0}); break;
    case OP_H: out.push_back({{E_H, 0, 0, 0, 0}, 1.0}); break;
    case OP_CRE: out.push_back({{E_C, b.p, tqb, 0, 0}, 1.0}); break;
    case OP_ANN: out.push_back({{E_A, b.p, -tqb, 0, 0}, ph_b(tqb)}); break;
    case OP_A:
      for (int s = -1; s <= 1; s += 2) {
        int t = tqb - s;
        if (t != 1 && t != -1) continue;
        double c = clebsch(1, s, 1, t, b.tk, tqb);
        if (c != 0.0) out.push_back({{E_CC, b.p, s, b.q, t}, c});
      }
      break;
    case OP_AD:
      for (int m1 = -1; m1 <= 1; m1 += 2) {
        int m2 = tqb - m1;
        if (m2 != 1 && m2 != -1) continue;
        double c = clebsch(1, m1, 1, m2, b.tk, tqb);
        if (c != 0.0) out.push_back({{E_AA, b.p, -m1, b.q, -m2}, c * ph_b(m1) * ph_b(m2)});
      }
      break;
    case OP_B:
      for (int s = -1; s <= 1; s += 2) {
        int m = tqb - s;
        if (m != 1 && m != -1) continue;
        double c = clebsch(1, s, 1, m, b.tk, tqb);
        if (c != 0.0) out.push_back({{E_CA, b.p, s, b.q, -m}, c * ph_b(m)});
      }
      break;
    case OP_RC: out.push_back({{E_RC, b.p, tqb, 0, 0}, 1.0}); break;
    case OP_RCD: out.push_back({{E_RCD, b.p, -tqb, 0, 0}, ph_b(tqb)}); break;
  }
}

struct Rule {
  int rule, i0, i1;
  Elem src;
  Mat4 O;
  double scalar;
  int64_t gi = -1;   // scalar = gc * g[gi] (gi >= 0) or gc
  double gc = 1.0;
};
// rule whose scalar is c times the folded integral g(p, q, r, s)
Rule grule(int rule, int i0, int i1, const Elem& src, const Mat4& O, double c, const Integrals& g,
           int p, int q, int r, int s) {
  return {rule, i0, i1, src, O, c * g.at(p, q, r, s), g.idx(p, q, r, s), c};
}

enum {
  R_ID = 1, R_NEW, R_CC_P, R_CC_Q, R_CC_L, R_AA_P, R_AA_Q, R_AA_L, R_CA_P, R_CA_T, R_CA_L,
  R_RC_ID, R_RC_2, R_RC_3, R_RC_4, R_RC_5, R_RC_6, R_RC_7, R_RC_8,
  R_H_ID, R_H_LOC, R_H_C, R_H_A, R_H_RC, R_H_RCD, R_H_CC, R_H_AA, R_H_BN, R_H_BX,
  R_ADJ = 100
};

void rc_rules(int r, int s, int k, const Integrals& g, std::vector<Rule>& out) {
  // Rc_{r s}(block + site k) from Rc_{r s}(block) and the seven ways to place
  // orbital k among the three block indices of Eq. 12's sum.
  Mat4 I4 = eye4();
  out.push_back({R_RC_ID, -1, -1, {E_RC, r, s, 0, 0}, I4, 1.0});
  {
    Mat4 O = zero4();
    for (int t = -1; t <= 1; t += 2) O = add(O, mul(mul(cdag(s), cdag(t)), cann(t)));
    if (g.use(k, k, r, k)) out.push_back(grule(R_RC_2, -1, -1, {E_I, 0, 0, 0, 0}, O, 1.0, g, k, k, r, k));
  }
  Mat4 nk = num();
  for (int a = 0; a < k; ++a) {
    for (int b = 0; b < k; ++b) {
      const bool u3 = g.use(k, a, r, b);   // p = k: sum_t a+_{a t} a_{b t} . a+_{k s}
      const bool u4 = g.use(a, k, r, b);   // q = k: - a+_{a s} a_{b t} . a+_{k t}
      const bool u5 = g.use(a, b, r, k);   // u = k: a+_{a s} a+_{b t} . a_{k t}
      for (int t = -1; t <= 1; t += 2) {
        if (u3) out.push_back(grule(R_RC_3, a, b, {E_CA, a, t, b, t}, cdag(s), 1.0, g, k, a, r, b));
        if (u4) out.push_back(grule(R_RC_4, a, b, {E_CA, a, s, b, t}, cdag(t), -1.0, g, a, k, r, b));
        if (u5) out.push_back(grule(R_RC_5, a, b, {E_CC, a, s, b, t}, cann(t), 1.0, g, a, b, r, k));
      }
    }
    const bool u6 = g.use(k, k, r, a);     // p = q = k: a_{a t} . a+_{k s} a+_{k t}
    const bool u7 = g.use(k, a, r, k);     // p = u = k: - a+_{a t} . a+_{k s} a_{k t}
    const bool u8 = g.use(a, k, r, k);     // q = u = k: a+_{a s} . n_k
    for (int t = -1; t <= 1; t += 2) {
      if (u6) out.push_back(grule(R_RC_6, a, -1, {E_A, a, t, 0, 0}, mul(cdag(s), cdag(t)), 1.0, g, k, k, r, a));
      if (u7) out.push_back(grule(R_RC_7, a, -1, {E_C, a, t, 0, 0}, mul(cdag(s), cann(t)), -1.0, g, k, a, r, k));
    }
    if (u8) out.push_back(grule(R_RC_8, a, -1, {E_C, a, s, 0, 0}, nk, 1.0, g, a, k, r, k));
  }
}

void h_rules(int k, const Integrals& g, std::vector<Rule>& out) {
  // H(block + site k): bipartition of Eq. 11's two-body operator between the block
  // (orbitals < k) and orbital k, with all terms written block-operator first.
  Mat4 I4 = eye4();
  out.push_back({R_H_ID, -1, -1, {E_H, 0, 0, 0, 0}, I4, 1.0});
  {
    Mat4 O = zero4();
    for (int s = -1; s <= 1; s += 2)
      for (int t = -1; t <= 1; t += 2)
        O = add(O, mul(mul(cdag(s), cdag(t)), mul(cann(t), cann(s))));
    if (g.use(k, k, k, k))
      out.push_back(grule(R_H_LOC, -1, -1, {E_I, 0, 0, 0, 0}, scale(O, 0.5), 1.0, g, k, k, k, k));
  }
  for (int p = 0; p < k; ++p) {
    if (!g.use(p, k, k, k)) continue;
    for (int s = -1; s <= 1; s += 2) {
      Mat4 Oc = zero4(), Oa = zero4();
      for (int t = -1; t <= 1; t += 2) {
        Oc = add(Oc, mul(mul(cdag(t), cann(t)), cann(s)));
        Oa = add(Oa, mul(mul(cdag(s), cdag(t)), cann(t)));
      }
      out.push_back(grule(R_H_C, p, -1, {E_C, p, s, 0, 0}, Oc, 1.0, g, p, k, k, k));
      out.push_back(grule(R_H_A, p, -1, {E_A, p, s, 0, 0}, Oa, -1.0, g, p, k, k, k));
    }
  }
  for (int s = -1; s <= 1; s += 2) {
    out.push_back({R_H_RC, -1, -1, {E_RC, k, s, 0, 0}, cann(s), 1.0});
    out.push_back({R_H_RCD, -1, -1, {E_RCD, k, s, 0, 0}, cdag(s), -1.0});
  }
  Mat4 nk = num();
  for (int p = 0; p < k; ++p)
    for (int q = 0; q < k; ++q) {
      const bool ue = g.use(p, q, k, k);
      const bool un = g.use(p, k, q, k);
      const bool ux = g.use(p, k, k, q);
      for (int s = -1; s <= 1; s += 2) {
        if (un) out.push_back(grule(R_H_BN, p, q, {E_CA, p, s, q, s}, nk, 1.0, g, p, k, q, k));
        for (int t = -1; t <= 1; t += 2) {
          if (ue) {
            out.push_back(grule(R_H_CC, p, q, {E_CC, p, s, q, t}, mul(cann(t), cann(s)), 0.5, g, p, q, k, k));
            out.push_back(grule(R_H_AA, p, q, {E_AA, q, t, p, s}, mul(cdag(s), cdag(t)), 0.5, g, p, q, k, k));
          }
          if (ux) out.push_back(grule(R_H_BX, p, q, {E_CA, p, s, q, t}, mul(cdag(t), cann(s)), -1.0, g, p, k, k, q));
        }
      }
    }
}

void rules(const Elem& e, int k, const Integrals& g, std::vector<Rule>& out) {
  out.clear();
  Mat4 I4 = eye4();
  switch (e.kind) {
    case E_I: out.push_back({R_ID, -1, -1, e, I4, 1.0}); break;
    case E_H: h_rules(k, g, out); break;
    case E_C:
      if (e.p < k) out.push_back({R_ID, -1, -1, e, I4, 1.0});
      else out.push_back({R_NEW, -1, -1, {E_I, 0, 0, 0, 0}, cdag(e.sp), 1.0});
      break;
    case E_A:
      if (e.p < k) out.push_back({R_ID, -1, -1, e, I4, 1.0});
      else out.push_back({R_NEW, -1, -1, {E_I, 0, 0, 0, 0}, cann(e.sp), 1.0});
      break;
    case E_CC:
      if (e.p < k && e.q < k) out.push_back({R_ID, -1, -1, e, I4, 1.0});
      else if (e.p < k) out.push_back({R_CC_P, -1, -1, {E_C, e.p, e.sp, 0, 0}, cdag(e.sq), 1.0});
      else if (e.q < k) out.push_back({R_CC_Q, -1, -1, {E_C, e.q, e.sq, 0, 0}, cdag(e.sp), -1.0});
      else out.push_back({R_CC_L, -1, -1, {E_I, 0, 0, 0, 0}, mul(cdag(e.sp), cdag(e.sq)), 1.0});
      break;
    case E_AA:
      if (e.p < k && e.q < k) out.push_back({R_ID, -1, -1, e, I4, 1.0});
      else if (e.p < k) out.push_back({R_AA_P, -1, -1, {E_A, e.p, e.sp, 0, 0}, cann(e.sq), 1.0});
      else if (e.q < k) out.push_back({R_AA_Q, -1, -1, {E_A, e.q, e.sq, 0, 0}, cann(e.sp), -1.0});
      else out.push_back({R_AA_L, -1, -1, {E_I, 0, 0, 0, 0}, mul(cann(e.sp), cann(e.sq)), 1.0});
      break;
    case E_CA:
      if (e.p < k && e.q < k) out.push_back({R_ID, -1, -1, e, I4, 1.0});
      else if (e.p < k) out.push_back({R_CA_P, -1, -1, {E_C, e.p, e.sp, 0, 0}, cann(e.sq), 1.0});
      else if (e.q < k) out.push_back({R_CA_T, -1, -1, {E_A, e.q, e.sq, 0, 0}, cdag(e.sp), -1.0});
      else out.push_back({R_CA_L, -1, -1, {E_I, 0, 0, 0, 0}, mul(cdag(e.sp), cann(e.sq)), 1.0});
      break;
    case E_RC: rc_rules(e.p, e.sp, k, g, out); break;
    case E_RCD: {
      std::vector<Rule> tmp;
      rc_rules(e.p, e.sp, k, g, tmp);
      for (auto& r : tmp) {
        // (X . O)^dagger = (-1)^{p(X) p(O)} X^dagger . O^dagger
        double sg = (elem_parity(r.src) && mat_parity(r.O)) ? -1.0 : 1.0;
        out.push_back({r.rule + R_ADJ, r.i0, r.i1, adjoint(r.src), tr(r.O), sg * r.scalar, r.gi, sg * r.gc});
      }
      break;
    }
  }
}

uint64_t hash_pattern(const Pattern& p) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t x) { h ^= x; h *= 1099511628211ull; };
  mix((uint64_t)p.tka); mix((uint64_t)p.tkb); mix((uint64_t)p.pa); mix((uint64_t)p.pO);
  for (double v : p.w) mix((uint64_t)(int64_t)std::llround(v * 1e9));
  return h;
}

}  // namespace

OpSet make_op_set(int k, int L, const std::vector<int>& ir) {
  OpSet s;
  auto add = [&](int type, int p, int q, int tk) {
    OpInfo o;
    o.key = {type, p, q, tk};
    o.tk = tk;
    switch (type) {
      case OP_I: case OP_H: o.dn = 0; o.ir = 0; break;
      case OP_CRE: o.dn = 1; o.ir = ir[p]; break;
      case OP_ANN: o.dn = -1; o.ir = ir[p]; break;
      case OP_A: o.dn = 2; o.ir = ir[p] ^ ir[q]; break;
      case OP_AD: o.dn = -2; o.ir = ir[p] ^ ir[q]; break;
      case OP_B: o.dn = 0; o.ir = ir[p] ^ ir[q]; break;
      case OP_RC: o.dn = 1; o.ir = ir[p]; break;
      case OP_RCD: o.dn = -1; o.ir = ir[p]; break;
    }
    o.parity = o.dn & 1;
    s.index[o.key.code()] = (int)s.ops.size();
    s.ops.push_back(o);
  };
  add(OP_I, -1, -1, 0);
  if (k >= 1) {
    add(OP_H, -1, -1, 0);
    for (int p = 0; p < k; ++p) add(OP_CRE, p, -1, 1);
    for (int p = 0; p < k; ++p) add(OP_ANN, p, -1, 1);
    for (int t = OP_A; t <= OP_AD; ++t)
      for (int p = 0; p < k; ++p)
        for (int q = p; q < k; ++q)
          for (int tk = 0; tk <= 2; tk += 2)
            if (!(p == q && tk == 2)) add(t, p, q, tk);
    for (int p = 0; p < k; ++p)
      for (int q = 0; q < k; ++q)
        for (int tk = 0; tk <= 2; tk += 2) add(OP_B, p, q, tk);
    for (int r = k; r < L; ++r) add(OP_RC, r, -1, 1);
    for (int r = k; r < L; ++r) add(OP_RCD, r, -1, 1);
  }
  return s;
}

int PatternTable::intern(const Pattern& p) {
  uint64_t h = hash_pattern(p);
  auto& v = by_hash[h];
  for (int id : v) {
    const Pattern& o = pats[id];
    if (o.tka != p.tka || o.tkb != p.tkb || o.pa != p.pa || o.pO != p.pO) continue;
    bool same = true;
    for (size_t i = 0; i < p.w.size(); ++i)
      if (std::fabs(o.w[i] - p.w[i]) > 1e-12) { same = false; break; }
    if (same) return id;
  }
  pats.push_back(p);
  v.push_back((int)pats.size() - 1);
  return (int)pats.size() - 1;
}

std::vector<WEntry> build_site_recursion(int k, const OpSet& from, const OpSet& to,
                                         const Integrals& g, PatternTable& pt) {
  std::vector<WEntry> out;
  std::vector<std::pair<Elem, double>> comps;
  std::vector<Rule> rl;
  std::vector<Src> srcs;
  for (int bi = 0; bi < (int)to.ops.size(); ++bi) {
    const OpInfo& b = to.ops[bi];
    struct Acc { std::vector<double> w; double scalar; int a; int64_t gi; double gc; };
    std::map<std::tuple<int, int, int, int>, Acc> acc;
    for (int tqb = -b.tk; tqb <= b.tk; tqb += 2) {
      int qb = (tqb + b.tk) / 2;
      components(b.key, tqb, comps);
      for (auto& ce : comps) {
        rules(ce.first, k, g, rl);
        for (auto& r : rl) {
          expand(r.src, srcs);
          for (auto& s : srcs) {
            int a = from.find(s.a);
            if (a < 0) {
              // H and the complementary operators of an empty block vanish
              if (k == 0 && (s.a.type == OP_H || s.a.type == OP_RC || s.a.type == OP_RCD)) continue;
              throw std::runtime_error("recursion source outside the operator set");
            }
            const OpInfo& ai = from.ops[a];
            auto key = std::make_tuple(a, r.rule, r.i0, r.i1);
            auto it = acc.find(key);
            if (it == acc.end()) {
              Acc z;
              z.w.assign((size_t)(ai.tk + 1) * (b.tk + 1) * 16, 0.0);
              z.scalar = r.scalar;
              z.a = a;
              z.gi = r.gi;
              z.gc = r.gc;
              it = acc.emplace(key, std::move(z)).first;
            }
            int qa = (s.tqa + ai.tk) / 2;
            double c = ce.second * s.c;
            double* w = &it->second.w[((size_t)qa * (b.tk + 1) + qb) * 16];
            for (int i = 0; i < 16; ++i) w[i] += c * r.O[i];
          }
        }
      }
    }
    for (auto& kv : acc) {
      Acc& z = kv.second;
      double mx = 0.0;
      for (double& v : z.w) {
        if (std::fabs(v) < 1e-13) v = 0.0;
        mx = std::max(mx, std::fabs(v));
      }
      if (mx == 0.0 || (z.scalar == 0.0 && !g.keep_zero)) continue;
      Pattern p;
      p.tka = from.ops[z.a].tk;
      p.tkb = b.tk;
      p.pa = from.ops[z.a].parity;
      p.pO = (p.pa + b.parity) & 1;
      p.w = z.w;
      int pid = pt.intern(p);
      out.push_back({z.a, bi, pid, z.scalar, z.gi, z.gc});
    }
  }
  return out;
}

}  // namespace dmrg

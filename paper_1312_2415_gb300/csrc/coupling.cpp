#include "coupling.hpp"

#include <cmath>

#include "su2.hpp"
#include "symmetry.hpp"

namespace dmrg {

namespace {
inline uint64_t pk(uint64_t a, int b, int c, int d, int e, int f, int g) {
  auto u = [](int x) { return (uint64_t)(uint32_t)(x + 64) & 0xFFu; };
  return (a << 48) | (u(b) << 40) | (u(c) << 32) | (u(d) << 24) | (u(e) << 16) | (u(f) << 8) | u(g);
}
inline int sgn_pow(int two_x) { return ((two_x / 2) & 1) ? -1 : 1; }  // (-1)^(x) for doubled even
}  // namespace

double Coupling::left(int pat, int tjL, int ls, int tjM, int tjLp, int lsp, int tjMp) {
  uint64_t key = pk((uint64_t)pat, tjL, ls, tjM, tjLp, lsp, tjMp);
  auto it = cl_.find(key);
  if (it != cl_.end()) return it->second;
  const Pattern& P = pt_->pats[pat];
  const int ts = local_ts(ls), tsp = local_ts(lsp);
  double best = 0.0;
  int bm = 0, bq = 0;
  for (int tmM = -tjM; tmM <= tjM; tmM += 2)
    for (int tqb = -P.tkb; tqb <= P.tkb; tqb += 2) {
      double c = clebsch(tjM, tmM, P.tkb, tqb, tjMp, tmM + tqb);
      if (std::fabs(c) > std::fabs(best) + 1e-14) { best = c; bm = tmM; bq = tqb; }
    }
  double val = 0.0;
  if (best != 0.0) {
    const int tmMp = bm + bq, qb = (bq + P.tkb) / 2;
    double sum = 0.0;
    for (int tmL = -tjL; tmL <= tjL; tmL += 2) {
      int tms = bm - tmL;
      if (tms < -ts || tms > ts) continue;
      double c1 = clebsch(tjL, tmL, ts, tms, tjM, bm);
      if (c1 == 0.0) continue;
      for (int tqa = -P.tka; tqa <= P.tka; tqa += 2) {
        int tmLp = tmL + tqa;
        double c3 = clebsch(tjL, tmL, P.tka, tqa, tjLp, tmLp);
        if (c3 == 0.0) continue;
        int tmsp = tmMp - tmLp;
        if (tmsp < -tsp || tmsp > tsp) continue;
        double c2 = clebsch(tjLp, tmLp, tsp, tmsp, tjMp, tmMp);
        if (c2 == 0.0) continue;
        double w = P.at((tqa + P.tka) / 2, qb, site_s4(lsp, tmsp), site_s4(ls, tms));
        sum += c1 * c2 * c3 * w;
      }
    }
    double sg = (P.pO && (tjL & 1)) ? -1.0 : 1.0;  // operator passes the block's electrons
    val = sg * sum / best;
  }
  cl_.emplace(key, val);
  return val;
}

double Coupling::right(int pat, int ls, int tj2, int tj, int lsp, int tj2p, int tjp) {
  uint64_t key = pk((uint64_t)pat, ls, tj2, tj, lsp, tj2p, tjp);
  auto it = cr_.find(key);
  if (it != cr_.end()) return it->second;
  const Pattern& P = pt_->pats[pat];
  const int ts = local_ts(ls), tsp = local_ts(lsp), Ns = local_n(ls);
  const int pb = (P.pa + P.pO) & 1;
  double best = 0.0;
  int bm = 0, bq = 0;
  for (int tmu = -tj; tmu <= tj; tmu += 2)
    for (int tqa = -P.tka; tqa <= P.tka; tqa += 2) {
      double c = clebsch(tj, tmu, P.tka, tqa, tjp, tmu + tqa);
      if (std::fabs(c) > std::fabs(best) + 1e-14) { best = c; bm = tmu; bq = tqa; }
    }
  double val = 0.0;
  if (best != 0.0) {
    const int tmup = bm + bq;
    const int qa = (-bq + P.tka) / 2;
    const double pha = sgn_pow(P.tka + bq);
    double sum = 0.0;
    for (int tms = -ts; tms <= ts; tms += 2) {
      int tmu2 = bm - tms;
      double c1 = clebsch(ts, tms, tj2, tmu2, tj, bm);
      if (c1 == 0.0) continue;
      for (int tqb = -P.tkb; tqb <= P.tkb; tqb += 2) {
        int tnu = -tqb;
        int tmu2p = tmu2 + tnu;
        double c3 = clebsch(tj2, tmu2, P.tkb, tnu, tj2p, tmu2p);
        if (c3 == 0.0) continue;
        int tmsp = tmup - tmu2p;
        if (tmsp < -tsp || tmsp > tsp) continue;
        double c2 = clebsch(tsp, tmsp, tj2p, tmu2p, tjp, tmup);
        if (c2 == 0.0) continue;
        double w = P.at(qa, (tqb + P.tkb) / 2, site_s4(lsp, tmsp), site_s4(ls, tms));
        sum += c1 * c2 * c3 * w * sgn_pow(P.tkb - tqb);
      }
    }
    double sg = (pb && (Ns & 1)) ? -1.0 : 1.0;  // right operator passes the site's electrons
    val = sg * pha * sum / best;
  }
  cr_.emplace(key, val);
  return val;
}

double Coupling::singlet(int tk, int parity, int tjM, int tjMp) {
  uint64_t key = pk(0, tk, parity, tjM, tjMp, 0, 0);
  auto it = cs_.find(key);
  if (it != cs_.end()) return it->second;
  double sum = 0.0;
  for (int tm = -tjM; tm <= tjM; tm += 2)
    for (int tq = -tk; tq <= tk; tq += 2) {
      int tmp = tm + tq;
      if (tmp < -tjMp || tmp > tjMp) continue;
      double cb = clebsch(tjMp, tmp, tjMp, -tmp, 0, 0);
      double ck = clebsch(tjM, tm, tjM, -tm, 0, 0);
      double cl = clebsch(tjM, tm, tk, tq, tjMp, tmp);
      double cr = clebsch(tjM, -tm, tk, -tq, tjMp, -tmp);
      sum += cb * ck * cl * cr * sgn_pow(tk - tq);
    }
  if (parity && (tjM & 1)) sum = -sum;  // right factor passes the left part's electrons
  cs_.emplace(key, sum);
  return sum;
}

double Coupling::overlap(int tjL, int ls1, int ls2, int tj, int tjR, int tjM) {
  uint64_t key = pk(0, tjL, ls1, ls2, tj, tjR, tjM);
  auto it = co_.find(key);
  if (it != co_.end()) return it->second;
  const int t1 = local_ts(ls1), t2 = local_ts(ls2);
  double sum = 0.0;
  for (int tmL = -tjL; tmL <= tjL; tmL += 2)
    for (int tm1 = -t1; tm1 <= t1; tm1 += 2)
      for (int tm2 = -t2; tm2 <= t2; tm2 += 2) {
        int tmj = tm1 + tm2, tmR = tmL + tmj;
        if (tmR < -tjR || tmR > tjR) continue;
        double X = clebsch(t1, tm1, t2, tm2, tj, tmj) * clebsch(tjL, tmL, tj, tmj, tjR, tmR) *
                   clebsch(tjR, tmR, tjR, -tmR, 0, 0);
        if (X == 0.0) continue;
        int tmM = tmL + tm1;
        if (tmM < -tjM || tmM > tjM) continue;
        double Y = clebsch(tjM, tmM, tjM, -tmM, 0, 0) * clebsch(tjL, tmL, t1, tm1, tjM, tmM) *
                   clebsch(t2, tm2, tjR, -tmR, tjM, -tmM);
        sum += X * Y;
      }
  co_.emplace(key, sum);
  return sum;
}

}  // namespace dmrg

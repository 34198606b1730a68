#include "symmetry.hpp"

#include <algorithm>

#include "su2.hpp"

namespace dmrg {

int Bond::find(const Sector& s) const {
  auto it = std::lower_bound(sec.begin(), sec.end(), s);
  if (it != sec.end() && *it == s) return (int)(it - sec.begin());
  return -1;
}

int64_t Bond::total() const {
  int64_t t = 0;
  for (int d : dim) t += d;
  return t;
}

namespace {

std::map<Sector, int64_t> multiplets(const std::vector<int>& irs) {
  std::map<Sector, int64_t> d;
  d[{0, 0, 0}] = 1;
  for (int Ik : irs) {
    std::map<Sector, int64_t> nd;
    for (auto& kv : d) {
      const Sector& s = kv.first;
      for (int ls = 0; ls < 3; ++ls) {
        int ts = local_ts(ls);
        for (int tj = std::abs(s.tj - ts); tj <= s.tj + ts; tj += 2)
          nd[{tj, s.n + local_n(ls), s.ir ^ local_ir(ls, Ik)}] += kv.second;
      }
    }
    d.swap(nd);
  }
  return d;
}

}  // namespace

std::vector<std::map<Sector, int>> Symmetry::fci_dims() const {
  std::vector<std::map<Sector, int>> out(L + 1);
  for (int k = 0; k <= L; ++k) {
    std::vector<int> left(orb_ir.begin(), orb_ir.begin() + k);
    std::vector<int> right(orb_ir.begin() + k, orb_ir.end());
    auto ml = multiplets(left);
    auto mr = multiplets(right);
    for (auto& kv : ml) {
      const Sector& s = kv.first;
      int64_t r = 0;
      for (auto& kr : mr) {
        const Sector& t = kr.first;
        if (t.n == N - s.n && t.ir == (irrep ^ s.ir) && triangle(s.tj, t.tj, two_S)) r += kr.second;
      }
      if (r > 0) out[k][s] = (int)std::min<int64_t>(std::min<int64_t>(kv.second, r), 1 << 30);
    }
  }
  return out;
}

std::vector<Bond> Symmetry::initial_bonds(int D) const {
  auto fci = fci_dims();
  std::vector<Bond> bonds(L + 1);
  for (int k = 0; k <= L; ++k) {
    std::vector<Sector> keys;
    for (auto& kv : fci[k]) keys.push_back(kv.first);
    std::sort(keys.begin(), keys.end());
    std::vector<int> alloc(keys.size(), 0);
    int left = D;
    while (left > 0) {
      int n_open = 0;
      for (size_t i = 0; i < keys.size(); ++i)
        if (alloc[i] < fci[k][keys[i]]) ++n_open;
      if (n_open == 0) break;
      int share = std::max(1, left / n_open);
      for (size_t i = 0; i < keys.size() && left > 0; ++i) {
        int cap = fci[k][keys[i]];
        if (alloc[i] >= cap) continue;
        int add = std::min(std::min(share, cap - alloc[i]), left);
        alloc[i] += add;
        left -= add;
      }
    }
    for (size_t i = 0; i < keys.size(); ++i)
      if (alloc[i] > 0) {
        bonds[k].sec.push_back(keys[i]);
        bonds[k].dim.push_back(alloc[i]);
      }
  }
  return bonds;
}

}  // namespace dmrg

// Symmetry sectors of SU(2) x U(1) x P (Sec. 3): labels, bonds and the local basis.
#pragma once
#include <cstdint>
#include <map>
#include <vector>

namespace dmrg {

// (2j, N, irrep) label of a reduced multiplet (Eq. 21).
struct Sector {
  int tj, n, ir;
  bool operator<(const Sector& o) const {
    if (n != o.n) return n < o.n;
    if (tj != o.tj) return tj < o.tj;
    return ir < o.ir;
  }
  bool operator==(const Sector& o) const { return tj == o.tj && n == o.n && ir == o.ir; }
};

// Local reduced states of one orbital (Eqs. 17-20): 0 = empty, 1 = single (s=1/2),
// 2 = double.  m-resolved site basis index s4: 0 |0>, 1 |up>, 2 |dn>, 3 |up dn>.
inline int local_ts(int ls) { return ls == 1 ? 1 : 0; }
inline int local_n(int ls) { return ls; }
inline int local_ir(int ls, int orb_ir) { return ls == 1 ? orb_ir : 0; }
inline int site_s4(int ls, int tms) { return ls == 0 ? 0 : (ls == 2 ? 3 : (tms > 0 ? 1 : 2)); }

// Sectors and their reduced dimensions at one bond, kept in Sector order.
struct Bond {
  std::vector<Sector> sec;
  std::vector<int> dim;
  int find(const Sector& s) const;
  int64_t total() const;
};

struct Symmetry {
  int L = 0, N = 0, two_S = 0, irrep = 0, n_irrep = 1;
  std::vector<int> orb_ir;
  // FCI-capped reduced dimensions per bond (0..L).
  std::vector<std::map<Sector, int>> fci_dims() const;
  // Sec. 4.3: D spread equally over the sectors of every bond, none above its FCI
  // dimension (water-filling in sector order).
  std::vector<Bond> initial_bonds(int D) const;
};

}  // namespace dmrg

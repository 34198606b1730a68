// Reduced recoupling factors for the two-site effective Hamiltonian and the operator
// updates.  Each factor is the reduced matrix element of a coupled operator product
// on coupled states (the role of the paper's 6-j / 9-j symbols), evaluated as an
// explicit Clebsch-Gordan sum over projections and memoised by spin labels.
#pragma once
#include <cstdint>
#include <unordered_map>

#include "mpo.hpp"

namespace dmrg {

class Coupling {
 public:
  explicit Coupling(const PatternTable* pt) : pt_(pt) {}
  // Left growth (block x site -> new block, CG <jL mL s ms | jM mM>): reduced element
  // of L_b = [L_a x pattern] between (jL' s') jM' and (jL s) jM per unit L_a.
  double left(int pat, int tjL, int ls, int tjM, int tjLp, int lsp, int tjMp);
  // Right growth (site x block -> new block, CG <s ms j2 m2 | j m>): reduced element of
  // the partner of the pattern's source a, built from the partner of its target b.
  double right(int pat, int ls, int tj2, int tj, int lsp, int tj2p, int tjp);
  // <[jM' x jM']^0 | sum_q L_q R_q | [jM x jM]^0> for unit reduced elements.
  double singlet(int tk, int parity, int tjM, int tjMp);
  // <[(jL s1)jM x (s2 jR)jM]^0 | [(jL (s1 s2)j) jR x jR]^0>.
  double overlap(int tjL, int ls1, int ls2, int tj, int tjR, int tjM);

 private:
  const PatternTable* pt_;
  std::unordered_map<uint64_t, double> cl_, cr_, cs_, co_;
};

}  // namespace dmrg

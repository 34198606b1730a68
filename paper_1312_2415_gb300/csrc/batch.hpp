// Batched Davidson (Sec. 2.3) over independent instances, one launch per operation.
#pragma once
#include <functional>
#include <vector>

#include "device.hpp"

namespace dmrg {

struct BdInst {
  double* x;           // in: start vector; out: Ritz vector of unit norm (n doubles, device)
  const double* diag;  // H_eff diagonal (device)
  double* bx;          // the batched matvec's input for this instance (device)
  double* by;          // and its output
  int64_t n;
};
struct BdResult {
  double theta = 0.0;  // lowest Ritz value at exit
  int iters = 0;
  int converged = 0;
};
// `matvec` queues y = H_eff x on stream s for every instance (bx -> by); tile_active
// (device, one int per instance, or null) receives the instances still iterating before
// each matvec, which skips the others.  The caller restores it afterwards.
void batch_davidson(const std::vector<BdInst>& inst, double tol, int maxit, const std::function<void()>& matvec,
                    int* tile_active, Stream s, std::vector<BdResult>& out);

}  // namespace dmrg

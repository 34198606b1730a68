// Device-side plan tables shared by the FP64 and tensor-core kernels (internal).
#pragma once
#include "device.hpp"

namespace dmrg {

void note_launches(int64_t k);  // adds to the count kernel_launches() reports

struct GemmPlan {
  GemmTask* tasks = nullptr;
  GemmGroup* groups = nullptr;
  int ngroups = 0, ntiles = 0;
  int64_t ntasks = 0;
};

struct CombPlan {
  CombSrc* src = nullptr;
  CombDst* dst = nullptr;
  int ndst = 0;
};

struct DiagPlan {
  DiagTerm* t = nullptr;
  DiagOut* o = nullptr;
  int n = 0;
};

}  // namespace dmrg

// SU(2) coupling coefficients used by the planner.
// All angular momenta are doubled integers (tj = 2j, tm = 2m).
#pragma once

namespace dmrg {

// <j1 m1 j2 m2 | J M>, Condon-Shortley phases (the convention of Eq. 22).
double clebsch(int tj1, int tm1, int tj2, int tm2, int tJ, int tM);

// Wigner 6-j symbol {a b c; d e f} (Eqs. 25-26).
double wigner6j(int a, int b, int c, int d, int e, int f);

inline bool triangle(int a, int b, int c) {
  return (a + b + c) % 2 == 0 && c >= (a > b ? a - b : b - a) && c <= a + b;
}

}  // namespace dmrg

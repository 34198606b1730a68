// Racah closed forms for Clebsch-Gordan coefficients and 6-j symbols, evaluated in
// long double with a factorial table and memoised per argument tuple.
#include "su2.hpp"

#include <cmath>
#include <cstdint>
#include <mutex>
#include <unordered_map>

namespace dmrg {
namespace {

constexpr int kMaxFact = 170;

const long double* fact_table() {
  static long double f[kMaxFact + 1];
  static bool init = false;
  if (!init) {
    f[0] = 1.0L;
    for (int i = 1; i <= kMaxFact; ++i) f[i] = f[i - 1] * (long double)i;
    init = true;
  }
  return f;
}

// factorial of x2/2 for even, non-negative x2
inline long double fh(int x2) { return fact_table()[x2 / 2]; }

long double delta_sq(int a, int b, int c) {
  return fh(a + b - c) * fh(a - b + c) * fh(-a + b + c) / fh(a + b + c + 2);
}

double clebsch_raw(int tj1, int tm1, int tj2, int tm2, int tJ, int tM) {
  if (tm1 + tm2 != tM || !triangle(tj1, tj2, tJ)) return 0.0;
  if (tm1 > tj1 || -tm1 > tj1 || tm2 > tj2 || -tm2 > tj2 || tM > tJ || -tM > tJ) return 0.0;
  if (((tj1 + tm1) & 1) || ((tj2 + tm2) & 1) || ((tJ + tM) & 1)) return 0.0;
  long double pre = (long double)(tJ + 1) * delta_sq(tj1, tj2, tJ) * fh(tj1 + tm1) *
                    fh(tj1 - tm1) * fh(tj2 + tm2) * fh(tj2 - tm2) * fh(tJ + tM) * fh(tJ - tM);
  long double s = 0.0L;
  for (int k = 0; k <= tj1 + tj2 + tJ; k += 2) {
    int d[6] = {k, tj1 + tj2 - tJ - k, tj1 - tm1 - k, tj2 + tm2 - k, tJ - tj2 + tm1 + k,
                tJ - tj1 - tm2 + k};
    bool ok = true;
    long double den = 1.0L;
    for (int x : d) {
      if (x < 0) { ok = false; break; }
      den *= fh(x);
    }
    if (!ok) continue;
    s += (((k / 2) & 1) ? -1.0L : 1.0L) / den;
  }
  return (double)(s * sqrtl(pre));
}

double sixj_raw(int a, int b, int c, int d, int e, int f) {
  if (!triangle(a, b, c) || !triangle(a, e, f) || !triangle(d, b, f) || !triangle(d, e, c))
    return 0.0;
  long double pre = delta_sq(a, b, c) * delta_sq(a, e, f) * delta_sq(d, b, f) * delta_sq(d, e, c);
  int lo = a + b + c;
  if (a + e + f > lo) lo = a + e + f;
  if (d + b + f > lo) lo = d + b + f;
  if (d + e + c > lo) lo = d + e + c;
  int hi = a + b + d + e;
  if (b + c + e + f < hi) hi = b + c + e + f;
  if (a + c + d + f < hi) hi = a + c + d + f;
  long double s = 0.0L;
  for (int t = lo; t <= hi; t += 2) {
    long double den = fh(t - a - b - c) * fh(t - a - e - f) * fh(t - d - b - f) *
                      fh(t - d - e - c) * fh(a + b + d + e - t) * fh(b + c + e + f - t) *
                      fh(a + c + d + f - t);
    s += (((t / 2) & 1) ? -1.0L : 1.0L) * fh(t + 2) / den;
  }
  return (double)(s * sqrtl(pre));
}

inline uint64_t pack6(int a, int b, int c, int d, int e, int f) {
  auto u = [](int x) { return (uint64_t)(uint32_t)(x + 512) & 0x3FFu; };
  return u(a) | (u(b) << 10) | (u(c) << 20) | (u(d) << 30) | (u(e) << 40) | (u(f) << 50);
}

std::mutex g_mu;

}  // namespace

double clebsch(int tj1, int tm1, int tj2, int tm2, int tJ, int tM) {
  static std::unordered_map<uint64_t, double> cache;
  if (tm1 + tm2 != tM) return 0.0;
  uint64_t key = pack6(tj1, tm1, tj2, tm2, tJ, tM);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  double v = clebsch_raw(tj1, tm1, tj2, tm2, tJ, tM);
  std::lock_guard<std::mutex> lk(g_mu);
  cache.emplace(key, v);
  return v;
}

double wigner6j(int a, int b, int c, int d, int e, int f) {
  static std::unordered_map<uint64_t, double> cache;
  uint64_t key = pack6(a, b, c, d, e, f);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  double v = sixj_raw(a, b, c, d, e, f);
  std::lock_guard<std::mutex> lk(g_mu);
  cache.emplace(key, v);
  return v;
}

}  // namespace dmrg

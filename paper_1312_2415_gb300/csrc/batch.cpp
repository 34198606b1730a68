// Davidson's algorithm (Sec. 2.3) for the instances of a batch in lockstep: every
// iteration applies H_eff to all of them in one launch sequence (the batched tensor-core
// matvec) and runs each vector operation of the iteration as one launch over all
// instances.  Per instance it is the algorithm of Engine::davidson_core: subspace up to
// 32 vectors (fewer for an instance smaller than that), restart on the 3 lowest Ritz
// vectors, diagonal preconditioner, two classical Gram-Schmidt passes, convergence on
// ||r||_2; an instance that has converged is frozen (its operations are skipped) while
// the others go on.  All instances share the subspace size: they start together and
// restart together.
#include "batch.hpp"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace dmrg {

void batch_davidson(const std::vector<BdInst>& inst, double tol, int maxit, const std::function<void()>& matvec,
                    int* tile_active, Stream s, std::vector<BdResult>& out) {
  const int K = (int)inst.size();
  out.assign(K, BdResult{});
  if (K == 0) return;
  if (maxit < 1) throw std::invalid_argument("Davidson needs at least one iteration");
  int64_t nmin = inst[0].n, nmax = inst[0].n;
  for (const BdInst& I : inst) {
    if (I.n < 1 || !I.x || !I.diag || !I.bx || !I.by) throw std::invalid_argument("batched Davidson: empty instance");
    nmin = std::min(nmin, I.n);
    nmax = std::max(nmax, I.n);
  }
  const int mmax = (int)std::min<int64_t>(32, std::max<int64_t>(nmin, 1));
  const int nkeep = std::min(3, mmax - 1 > 0 ? mmax - 1 : 1);
  // workspace: one allocation, carved per instance
  std::vector<int64_t> off(K + 1, 0);
  auto words = [&](int64_t n) {
    return 2 * n * (mmax + 1) + 2 * (int64_t)mmax * mmax + mmax + (mmax + 2) + (int64_t)mmax * kBdChunks + 3 * n +
           n * 2 * nkeep;
  };
  for (int i = 0; i < K; ++i) off[i + 1] = off[i] + words(inst[i].n);
  double* ws = nullptr;
  BdSlot* sl = nullptr;
  int* act = nullptr;
  double* gat = nullptr;
  double* gat_h = nullptr;
  auto cleanup = [&]() {
    dev_free(ws, s);
    dev_free(sl, s);
    dev_free(act, s);
    dev_free(gat, s);
    host_pinned_free(gat_h);
  };
  try {
    ws = (double*)dev_alloc(sizeof(double) * off[K], s);
    sl = (BdSlot*)dev_alloc(sizeof(BdSlot) * K, s);
    act = (int*)dev_alloc(sizeof(int) * K, s);
    gat = (double*)dev_alloc(sizeof(double) * 2 * K, s);
    gat_h = (double*)host_pinned_alloc(sizeof(double) * 2 * K);
    std::vector<BdSlot> h(K);
    for (int i = 0; i < K; ++i) {
      const int64_t n = inst[i].n;
      double* p = ws + off[i];
      BdSlot& q = h[i];
      q.V = p; p += n * (mmax + 1);
      q.AV = p; p += n * (mmax + 1);
      q.G = p; p += (int64_t)mmax * mmax;
      q.C = p; p += (int64_t)mmax * mmax;
      q.th = p; p += mmax;
      q.dots = p; p += mmax + 2;
      q.part = p; p += (int64_t)mmax * kBdChunks;
      q.r = p; p += n;
      q.t = p; p += n;
      q.x0 = p; p += n;
      q.tmp = p;
      q.x = inst[i].x;
      q.diag = inst[i].diag;
      q.bx = inst[i].bx;
      q.by = inst[i].by;
      q.n = n;
    }
    dev_zero(ws, sizeof(double) * off[K], s);
    dev_h2d(sl, h.data(), sizeof(BdSlot) * K, s);
    std::vector<int> a(K, 1);
    std::vector<std::vector<double>> rhist(K);
    dev_h2d(act, a.data(), sizeof(int) * K, s);
    auto set_act = [&](const std::vector<int>& v) { dev_h2d(act, v.data(), sizeof(int) * K, s); };
    auto read_gather = [&]() {
      bd_gather(sl, K, gat, s);
      dev_d2h(gat_h, gat, sizeof(double) * 2 * K, s);
      dev_sync(s);
    };
    // H_eff applied to V column `col` of every instance, into AV column `col` (the
    // matvec skips the tiles of the instances that have stopped)
    auto apply = [&](int col) {
      bd_axpby(sl, act, K, nmax, 0, 1.0, BD_V, col, 0.0, BD_BX, 0, s);
      if (tile_active) dev_d2d(tile_active, act, sizeof(int) * K, s);
      matvec();
      bd_axpby(sl, act, K, nmax, 0, 1.0, BD_BY, 0, 0.0, BD_AV, col, s);
    };
    // t -= V (V^T t), twice
    auto orthogonalize = [&](int m) {
      for (int pass = 0; pass < 2; ++pass) {
        bd_dots(sl, act, K, nmax, BD_V, 0, m, BD_T, 0, 0, 0, mmax, s);
        bd_combine(sl, act, K, nmax, BD_V, m, 0, 0, 0.0, BD_TMP, 0, s);
        bd_axpby(sl, act, K, nmax, 0, -1.0, BD_TMP, 0, 1.0, BD_T, 0, s);
      }
      bd_dots(sl, act, K, nmax, BD_T, 0, 1, BD_T, 0, 0, 0, mmax, s);
    };
    // x0 = x, v0 = x / |x|, A v0, G[0][0]
    bd_axpby(sl, act, K, nmax, 0, 1.0, BD_X, 0, 0.0, BD_X0, 0, s);
    bd_axpby(sl, act, K, nmax, 0, 1.0, BD_X, 0, 0.0, BD_V, 0, s);
    bd_dots(sl, act, K, nmax, BD_V, 0, 1, BD_V, 0, 0, 0, mmax, s);
    bd_normalize(sl, act, K, nmax, BD_V, 0, s);
    apply(0);
    bd_dots(sl, act, K, nmax, BD_V, 0, 1, BD_AV, 0, 1, 0, mmax, s);
    int m = 1;
    for (int it = 0; it < maxit; ++it) {
      bd_small_eig(sl, act, K, mmax, m, std::min(m, nkeep), s);
      // x = V c0, r = AV c0 - theta x, |r|^2
      bd_combine(sl, act, K, nmax, BD_V, m, 1, 0, 0.0, BD_X, 0, s);
      bd_combine(sl, act, K, nmax, BD_AV, m, 1, 0, 0.0, BD_R, 0, s);
      bd_axpby(sl, act, K, nmax, 1, 0.0, BD_X, 0, 1.0, BD_R, 0, s);
      bd_dots(sl, act, K, nmax, BD_R, 0, 1, BD_R, 0, 0, 0, mmax, s);
      read_gather();
      int live = 0;
      for (int i = 0; i < K; ++i) {
        if (!a[i]) continue;
        out[i].theta = gat_h[2 * i];
        out[i].iters = it + 1;
        const double rn = std::sqrt(std::max(gat_h[2 * i + 1], 0.0));
        rhist[i].push_back(rn);
        const size_t k = rhist[i].size();
        if (rn <= tol || m >= inst[i].n) {
          out[i].converged = 1;
          a[i] = 0;
        } else if (k > 8 && rn <= 1e-4 * std::fabs(out[i].theta) && rn > 0.8 * rhist[i][k - 9]) {
          // the residual has reached the accuracy of the split-TF32 products (as in
          // Engine::davidson_core): the instance stops, not converged
          a[i] = 0;
        } else {
          ++live;
        }
      }
      if (live == 0 || it + 1 >= maxit) break;  // no use expanding the subspace on the last iteration
      set_act(a);
      bd_precondition(sl, act, K, nmax, s);
      orthogonalize(m);
      read_gather();
      // a preconditioned direction that collapsed falls back to the residual
      std::vector<int> coll(K, 0);
      bool any = false;
      for (int i = 0; i < K; ++i)
        if (a[i] && !(gat_h[2 * i + 1] > 1e-28)) {
          coll[i] = 1;
          any = true;
        }
      if (any) {
        set_act(coll);
        bd_axpby(sl, act, K, nmax, 0, 1.0, BD_R, 0, 0.0, BD_T, 0, s);
        orthogonalize(m);
        read_gather();
        for (int i = 0; i < K; ++i)
          if (coll[i] && !(gat_h[2 * i + 1] > 1e-30)) {
            out[i].converged = 1;
            a[i] = 0;
          }
        set_act(a);
        if (std::none_of(a.begin(), a.end(), [](int v) { return v != 0; })) break;
      }
      bd_normalize(sl, act, K, nmax, BD_T, 0, s);
      if (m == mmax) {
        // restart on the nkeep lowest Ritz vectors
        for (int v = 0; v < nkeep; ++v) {
          bd_combine(sl, act, K, nmax, BD_V, m, 1, v, 0.0, BD_TMP, v, s);
          bd_combine(sl, act, K, nmax, BD_AV, m, 1, v, 0.0, BD_TMP, nkeep + v, s);
        }
        for (int v = 0; v < nkeep; ++v) {
          bd_axpby(sl, act, K, nmax, 0, 1.0, BD_TMP, v, 0.0, BD_V, v, s);
          bd_axpby(sl, act, K, nmax, 0, 1.0, BD_TMP, nkeep + v, 0.0, BD_AV, v, s);
        }
        bd_restart_g(sl, act, K, mmax, nkeep, s);
        m = nkeep;
      }
      bd_axpby(sl, act, K, nmax, 0, 1.0, BD_T, 0, 0.0, BD_V, m, s);
      apply(m);
      // row m of the Rayleigh matrix (lower triangle is what the eigensolver reads)
      bd_dots(sl, act, K, nmax, BD_V, 0, m + 1, BD_AV, m, 1, m, mmax, s);
      ++m;
    }
    // sign of every eigenvector: non-negative overlap with its starting vector
    std::fill(a.begin(), a.end(), 1);
    set_act(a);
    bd_dots(sl, act, K, nmax, BD_X, 0, 1, BD_X0, 0, 0, 0, mmax, s);
    bd_sign(sl, act, K, nmax, s);
    dev_sync(s);
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
}

}  // namespace dmrg

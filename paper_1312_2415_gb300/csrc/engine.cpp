// Engine: symmetry tables, environments, and the micro-iteration pipeline
// (Eq. 25 -> Davidson on H_eff (Eq. 9) -> Eqs. 26-28 -> operator update).
#include "engine.hpp"

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <exception>
#include <functional>
#include <limits>
#include <map>
#include <mutex>
#include <stdexcept>
#include <thread>
#include <tuple>

#include "su2.hpp"

namespace dmrg {

namespace {

inline int64_t bkey(int r, int c) { return ((int64_t)r << 32) | (uint32_t)c; }

// Tasks tagged with an output index, grouped per output in increasing index order
// (stable: a group's tasks keep their order); zs[id] gives the Z offset of a task whose
// B holds a Z id.
struct TaggedTask { int64_t out; GemmTask t; };
void group_by_output(std::vector<TaggedTask>& tagged, int64_t nout, double* Z, const std::vector<int64_t>& zoff,
                     const std::function<void(int64_t, int, int, std::vector<GemmGroup>&)>& make_group,
                     std::vector<GemmTask>& t2, std::vector<GemmGroup>& g2) {
  std::vector<int> cnt(nout + 1, 0);
  for (const auto& q : tagged) ++cnt[q.out + 1];
  for (int64_t o = 0; o < nout; ++o) cnt[o + 1] += cnt[o];
  t2.resize(tagged.size());
  std::vector<int> pos(cnt.begin(), cnt.end() - 1);
  for (const auto& q : tagged) {
    GemmTask t = q.t;
    t.B = Z + zoff[(size_t)(intptr_t)t.B];
    t2[pos[q.out]++] = t;
  }
  for (int64_t o = 0; o < nout; ++o)
    if (cnt[o + 1] > cnt[o]) make_group(o, cnt[o], cnt[o + 1], g2);
}

// f(begin, end) over [0, n) in chunks, on up to 16 threads (the caller's included)
// (an exception in any chunk stops the others and is rethrown on the caller's thread)
template <class F>
void parallel_chunks(size_t n, size_t chunk, F f) {
  std::atomic<size_t> next{0};
  std::mutex mu;
  std::exception_ptr err;
  auto run = [&]() {
    try {
      for (;;) {
        const size_t b = next.fetch_add(chunk);
        if (b >= n) break;
        f(b, std::min(n, b + chunk));
      }
    } catch (...) {
      std::lock_guard<std::mutex> lk(mu);
      if (!err) err = std::current_exception();
      next.store(n);
    }
  };
  const unsigned hc = std::thread::hardware_concurrency();
  const size_t nth = std::min<size_t>(std::max(1u, std::min(16u, hc ? hc : 1u)), (n + chunk - 1) / chunk);
  std::vector<std::thread> th;
  for (size_t t = 1; t < nth; ++t) th.emplace_back(run);
  run();
  for (auto& t : th) t.join();
  if (err) std::rethrow_exception(err);
}

uint64_t splitmix64_next(uint64_t& state) {
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Timer {
  double t0;
  Timer() : t0(now_ms()) {}
  double ms() const { return now_ms() - t0; }
};

}  // namespace

Engine::Engine(int L, int n_irrep, const std::vector<int>& orb_ir, int N, int two_S, int irrep,
               Stream stream)
    : L_(L), N_(N), two_S_(two_S), irrep_(irrep), stream_(stream) {
  sym_.L = L;
  sym_.N = N;
  sym_.two_S = two_S;
  sym_.irrep = irrep;
  sym_.n_irrep = n_irrep;
  sym_.orb_ir = orb_ir;
  opsets_.resize(L + 1);
  for (int k = 0; k <= L; ++k) opsets_[k] = make_op_set(k, L, orb_ir);
  cp_.reset(new Coupling(&pt_));
  lenv_.resize(L + 1);
  renv_.resize(L + 1);
  sites_.resize(L);
  sched_D_ = {64};
  sched_econv_ = {1e-8};
  sched_nmax_ = {4};
  sched_noise_ = {0.0};
}

Engine::~Engine() {
  try {
    flush_events();
    for (auto& e : ev_) event_destroy(e);
    if (cached_) free_plan(cached_);
    cached_ = nullptr;
    for (auto& e : lenv_) free_env(e);
    for (auto& e : renv_) free_env(e);
    for (int k = 0; k < L_; ++k) free_site(k);
    clear_excitations();
    if (reaper_.joinable()) reaper_.join();
    if (side_) {
      dev_sync(side_);
      stream_destroy(side_);
      event_destroy(ev_side_[0]);
      event_destroy(ev_side_[1]);
      dev_free(rq_dev_, stream_);
    }
    dev_sync(stream_);
  } catch (...) {
  }
}

void Engine::check_ready() const {
  if (!have_integrals_) throw std::invalid_argument("integrals not set");
  if (!have_mps_) throw std::invalid_argument("MPS not initialised");
}

// Eq. 11 folding of the one-body integrals into the two-body ones, after checking the
// symmetries the paper requires (Sec. 4.1: eightfold permutation symmetry, real
// orbitals, point-group selection).
void Engine::set_integrals(double econst, const double* h, const double* V) {
  const int L = L_;
  if (N_ < 2) throw std::invalid_argument("the folding of Eq. 11 needs N >= 2");
  double scale = 1e-300;
  for (int i = 0; i < L * L; ++i) scale = std::max(scale, std::fabs(h[i]));
  for (int64_t i = 0; i < (int64_t)L * L * L * L; ++i) scale = std::max(scale, std::fabs(V[i]));
  const double tol = 1e-10 * scale;
  auto Vat = [&](int i, int j, int k, int l) { return V[(((size_t)i * L + j) * L + k) * L + l]; };
  const auto& ir = sym_.orb_ir;
  for (int i = 0; i < L; ++i)
    for (int k = 0; k < L; ++k) {
      if (std::fabs(h[i * L + k] - h[k * L + i]) > tol) throw std::domain_error("h is not symmetric");
      if (ir[i] != ir[k] && std::fabs(h[i * L + k]) > tol)
        throw std::domain_error("h couples orbitals of different irreps");
    }
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j)
      for (int k = 0; k < L; ++k)
        for (int l = 0; l < L; ++l) {
          double v = Vat(i, j, k, l);
          if ((ir[i] ^ ir[j] ^ ir[k] ^ ir[l]) != 0 && std::fabs(v) > tol)
            throw std::domain_error("V breaks the point-group selection rule");
          const double sym[7] = {Vat(j, i, l, k), Vat(k, l, i, j), Vat(l, k, j, i), Vat(k, j, i, l),
                                 Vat(i, l, k, j), Vat(l, i, j, k), Vat(j, k, l, i)};
          for (double s : sym)
            if (std::fabs(v - s) > tol) throw std::domain_error("V lacks eightfold symmetry");
        }
  g_.L = L;
  g_.ir = ir;
  g_.keep_zero = false;
  g_.g.assign((size_t)L * L * L * L, 0.0);
  const double f = 1.0 / (N_ - 1);
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j)
      for (int k = 0; k < L; ++k)
        for (int l = 0; l < L; ++l) {
          double v = Vat(i, j, k, l);
          if (j == l) v += f * h[i * L + k];
          if (i == k) v += f * h[j * L + l];
          g_.g[(((size_t)i * L + j) * L + k) * L + l] = v;
        }
  econst_ = econst;
  Timer t;
  W_.assign(L, {});
  for (int k = 0; k < L; ++k) W_[k] = build_site_recursion(k, opsets_[k], opsets_[k + 1], g_, pt_);
  Wg_.clear();
  st_.t_plan_ms += t.ms();
  have_integrals_ = true;
  for (auto& e : lenv_) free_env(e);
  for (auto& e : renv_) free_env(e);
  if (cached_) { free_plan(cached_); cached_ = nullptr; cached_site_ = -1; }
}

void Engine::set_schedule(const std::vector<int>& D, const std::vector<double>& econv,
                          const std::vector<int>& nmax, const std::vector<double>& noise,
                          double dtol, int dmax) {
  if (D.empty()) throw std::invalid_argument("empty schedule");
  for (int d : D)
    if (d < 1) throw std::invalid_argument("D must be positive");
  sched_D_ = D;
  sched_econv_ = econv;
  sched_nmax_ = nmax;
  sched_noise_ = noise;
  dav_tol_ = dtol;
  dav_max_ = dmax;
}

// ------------------------------------------------------------------ MPS storage

void Engine::free_site(int k) {
  if (sites_[k].data) dev_free(sites_[k].data, stream_);
  sites_[k].data = nullptr;
  sites_[k].size = 0;
  sites_[k].blocks.clear();
}

void Engine::alloc_site(int k) {
  free_site(k);
  Site& S = sites_[k];
  const Bond& bl = bonds_[k];
  const Bond& br = bonds_[k + 1];
  int64_t off = 0;
  for (int l = 0; l < (int)bl.sec.size(); ++l)
    for (int ls = 0; ls < 3; ++ls) {
      const Sector& a = bl.sec[l];
      Sector want{0, a.n + local_n(ls), a.ir ^ local_ir(ls, sym_.orb_ir[k])};
      for (int r = 0; r < (int)br.sec.size(); ++r) {
        const Sector& b = br.sec[r];
        if (b.n != want.n || b.ir != want.ir || !triangle(a.tj, local_ts(ls), b.tj)) continue;
        S.blocks.push_back({ls, l, r, off, bl.dim[l], br.dim[r]});
        off += (int64_t)bl.dim[l] * br.dim[r];
      }
    }
  S.size = off;
  S.data = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(off, 1), stream_);
  dev_zero(S.data, sizeof(double) * std::max<int64_t>(off, 1), stream_);
}

void Engine::invalidate_envs_from_site(int k) {
  for (int b = k + 1; b <= L_; ++b) free_env(lenv_[b]);
  for (int b = 0; b <= k; ++b) free_env(renv_[b]);
  if (cached_) { free_plan(cached_); cached_ = nullptr; cached_site_ = -1; }
}

void Engine::init_mps(uint64_t seed) {
  if (!have_integrals_) throw std::invalid_argument("integrals not set");
  bonds_ = sym_.initial_bonds(sched_D_[0]);
  for (int k = 0; k <= L_; ++k)
    if (bonds_[k].sec.empty()) throw std::domain_error("target symmetry sector is empty");
  uint64_t state = seed;
  for (int k = 0; k < L_; ++k) {
    alloc_site(k);
    std::vector<double> h(sites_[k].size);
    for (auto& v : h) v = (double)(splitmix64_next(state) >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    dev_h2d(sites_[k].data, h.data(), sizeof(double) * h.size(), stream_);
    dev_sync(stream_);
  }
  have_mps_ = true;
  invalidate_envs_from_site(-1);
  for (auto& e : lenv_) free_env(e);
  for (auto& e : renv_) free_env(e);
  reset_noise();
}

// A new state starts without a previous half sweep: no noise until one has ended, and
// the noise streams are numbered from 0 again.
void Engine::reset_noise() {
  w_prev_ = 0.0;
  half_dir_ = 0;
  half_wmax_ = 0.0;
  noise_counter_ = 0;
}

// Serialised MPS: int32 magic, version, L, N, 2S, irrep; per bond: nsec then
// (2j, N, I, dim) per sector; per site: nblk then (ls, left sector, right sector) and
// the dL x dR block row-major in float64 (the reduced tensors of Eq. 22).
std::vector<char> Engine::get_mps() {
  if (!have_mps_) throw std::invalid_argument("MPS not initialised");
  std::vector<char> out;
  auto put = [&](const void* p, size_t n) {
    const char* c = (const char*)p;
    out.insert(out.end(), c, c + n);
  };
  int32_t hdr[6] = {0x444D5247, 1, L_, N_, two_S_, irrep_};
  put(hdr, sizeof(hdr));
  for (int k = 0; k <= L_; ++k) {
    int32_t n = (int32_t)bonds_[k].sec.size();
    put(&n, 4);
    for (int s = 0; s < n; ++s) {
      int32_t v[4] = {bonds_[k].sec[s].tj, bonds_[k].sec[s].n, bonds_[k].sec[s].ir, bonds_[k].dim[s]};
      put(v, 16);
    }
  }
  for (int k = 0; k < L_; ++k) {
    const Site& S = sites_[k];
    std::vector<double> h(S.size);
    dev_d2h(h.data(), S.data, sizeof(double) * S.size, stream_);
    dev_sync(stream_);
    int32_t n = (int32_t)S.blocks.size();
    put(&n, 4);
    for (auto& b : S.blocks) {
      int32_t v[3] = {b.ls, b.l, b.r};
      put(v, 12);
      put(h.data() + b.off, sizeof(double) * (size_t)b.rows * b.cols);
    }
  }
  return out;
}

void Engine::set_mps(const char* buf, size_t len) {
  size_t pos = 0;
  auto get = [&](void* p, size_t n) {
    if (pos + n > len) throw std::invalid_argument("MPS buffer too short");
    std::memcpy(p, buf + pos, n);
    pos += n;
  };
  int32_t hdr[6];
  get(hdr, sizeof(hdr));
  if (hdr[0] != 0x444D5247 || hdr[1] != 1) throw std::invalid_argument("bad MPS header");
  if (hdr[2] != L_ || hdr[3] != N_ || hdr[4] != two_S_ || hdr[5] != irrep_)
    throw std::invalid_argument("MPS belongs to another problem");
  std::vector<Bond> nb(L_ + 1);
  std::vector<std::vector<int>> perm(L_ + 1);
  for (int k = 0; k <= L_; ++k) {
    int32_t n;
    get(&n, 4);
    std::vector<std::pair<Sector, int>> v(n);
    for (int s = 0; s < n; ++s) {
      int32_t x[4];
      get(x, 16);
      if (x[3] <= 0) throw std::invalid_argument("non-positive sector dimension");
      v[s] = {Sector{x[0], x[1], x[2]}, x[3]};
    }
    std::vector<std::pair<Sector, int>> sorted = v;
    std::sort(sorted.begin(), sorted.end(), [](auto& a, auto& b) { return a.first < b.first; });
    for (auto& p : sorted) { nb[k].sec.push_back(p.first); nb[k].dim.push_back(p.second); }
    perm[k].resize(n);
    for (int s = 0; s < n; ++s) perm[k][s] = nb[k].find(v[s].first);
  }
  if (nb[0].sec.size() != 1 || !(nb[0].sec[0] == Sector{0, 0, 0}) || nb[0].dim[0] != 1)
    throw std::invalid_argument("left boundary must be the (0,0,0) singlet");
  if (nb[L_].sec.size() != 1 || !(nb[L_].sec[0] == Sector{two_S_, N_, irrep_}) || nb[L_].dim[0] != 1)
    throw std::invalid_argument("right boundary must be the target sector");
  for (int k = 0; k < L_; ++k) free_site(k);
  bonds_ = nb;
  for (int k = 0; k < L_; ++k) {
    alloc_site(k);
    Site& S = sites_[k];
    std::vector<double> h(S.size, 0.0);
    std::map<std::tuple<int, int, int>, const SiteBlock*> idx;
    for (auto& b : S.blocks) idx[{b.ls, b.l, b.r}] = &b;
    int32_t n;
    get(&n, 4);
    for (int b = 0; b < n; ++b) {
      int32_t x[3];
      get(x, 12);
      if (x[1] < 0 || x[1] >= (int)perm[k].size() || x[2] < 0 || x[2] >= (int)perm[k + 1].size())
        throw std::invalid_argument("block sector index out of range");
      auto it = idx.find({x[0], perm[k][x[1]], perm[k + 1][x[2]]});
      if (it == idx.end()) throw std::invalid_argument("block violates the symmetry of Eq. 22");
      const SiteBlock* sb = it->second;
      get(h.data() + sb->off, sizeof(double) * (size_t)sb->rows * sb->cols);
    }
    dev_h2d(S.data, h.data(), sizeof(double) * h.size(), stream_);
    dev_sync(stream_);
  }
  if (pos != len) throw std::invalid_argument("trailing bytes in MPS buffer");
  have_mps_ = true;
  for (auto& e : lenv_) free_env(e);
  for (auto& e : renv_) free_env(e);
  if (cached_) { free_plan(cached_); cached_ = nullptr; cached_site_ = -1; }
  reset_noise();
}

// ------------------------------------------------------------------ environments

void Engine::free_env(OpStore& e) {
  if (e.data) dev_free(e.data, stream_);
  e = OpStore();
}

void Engine::alloc_env(OpStore& e, int bond, const OpSet& ops) {
  free_env(e);
  const Bond& B = bonds_[bond];
  e.bond = bond;
  e.blocks.resize(ops.ops.size());
  e.at.resize(ops.ops.size());
  int64_t off = 0;
  for (size_t o = 0; o < ops.ops.size(); ++o) {
    const OpInfo& op = ops.ops[o];
    for (int c = 0; c < (int)B.sec.size(); ++c) {
      const Sector& sc = B.sec[c];
      for (int tj = std::abs(sc.tj - op.tk); tj <= sc.tj + op.tk; tj += 2) {
        int r = B.find({tj, sc.n + op.dn, sc.ir ^ op.ir});
        if (r < 0) continue;
        e.at[o][bkey(r, c)] = (int)e.blocks[o].size();
        e.blocks[o].push_back({r, c, off, B.dim[r], B.dim[c]});
        off += (int64_t)B.dim[r] * B.dim[c];
      }
    }
  }
  e.size = off;
  e.data = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(off, 1), stream_);
  dev_zero(e.data, sizeof(double) * std::max<int64_t>(off, 1), stream_);
  e.valid = false;
  e.serial = ++env_serial_;
}

void Engine::identity_fill(OpStore& e, int op) {
  std::vector<ScatterJob> jobs;
  static thread_local std::vector<double> ones;
  int dmax = 1;
  for (auto& b : e.blocks[op]) dmax = std::max(dmax, b.rows);
  std::vector<double> eye((size_t)dmax * dmax, 0.0);
  for (int i = 0; i < dmax; ++i) eye[(size_t)i * dmax + i] = 1.0;
  double* d = (double*)dev_alloc(sizeof(double) * eye.size(), stream_);
  dev_h2d(d, eye.data(), sizeof(double) * eye.size(), stream_);
  for (auto& b : e.blocks[op])
    if (b.r == b.c) jobs.push_back({e.data + b.off, d, nullptr, nullptr, b.cols, dmax, b.rows, b.cols, 0, 0, 0, 1.0});
  scatter_batched(jobs, stream_);
  dev_free(d, stream_);
}

void Engine::ensure_left(int k) {
  if (lenv_[k].valid) return;
  if (k == 0) {
    alloc_env(lenv_[0], 0, opsets_[0]);
    identity_fill(lenv_[0], 0);
    lenv_[0].valid = true;
    return;
  }
  ensure_left(k - 1);
  build_left(k);
}

void Engine::ensure_right(int k) {
  if (renv_[k].valid) return;
  if (k == L_) {
    alloc_env(renv_[L_], L_, opsets_[L_]);
    int h = opsets_[L_].find({OP_H, -1, -1, 0});
    identity_fill(renv_[L_], h);
    renv_[L_].valid = true;
    return;
  }
  ensure_right(k + 1);
  build_right(k);
}

// Blocks ordered by right sector first, so that all blocks with the same right sector
// form one row-major stack (rows = sum dL, cols = dR) that a single GEMM can multiply.
std::vector<XBlock> Engine::x_layout(int i, int64_t* n) const { return x_layout_of(bonds_, i, n); }

std::vector<XBlock> Engine::x_layout_of(const std::vector<Bond>& bonds, int i, int64_t* n) const {
  std::vector<XBlock> X;
  const Bond& bl = bonds[i];
  const Bond& br = bonds[i + 2];
  int64_t off = 0;
  for (int r = 0; r < (int)br.sec.size(); ++r) {
    const Sector& b = br.sec[r];
    int trow = 0;
    for (int l = 0; l < (int)bl.sec.size(); ++l)
      for (int ls1 = 0; ls1 < 3; ++ls1)
        for (int ls2 = 0; ls2 < 3; ++ls2) {
          const Sector& a = bl.sec[l];
          int nn = a.n + local_n(ls1) + local_n(ls2);
          int ir = a.ir ^ local_ir(ls1, sym_.orb_ir[i]) ^ local_ir(ls2, sym_.orb_ir[i + 1]);
          if (b.n != nn || b.ir != ir) continue;
          int t1 = local_ts(ls1), t2 = local_ts(ls2);
          for (int tj = std::abs(t1 - t2); tj <= t1 + t2; tj += 2) {
            if (!triangle(a.tj, tj, b.tj)) continue;
            X.push_back({l, ls1, ls2, tj, r, off, bl.dim[l], br.dim[r], trow});
            off += (int64_t)bl.dim[l] * br.dim[r];
            trow += bl.dim[l];
          }
        }
  }
  *n = off;
  return X;
}

void Engine::layout(int i, std::vector<int64_t>& table, int64_t& n) {
  check_ready();
  if (i < 0 || i > L_ - 2) throw std::out_of_range("site out of range");
  auto X = x_layout(i, &n);
  table.clear();
  for (auto& x : X) {
    const Sector& a = bonds_[i].sec[x.l];
    const Sector& b = bonds_[i + 2].sec[x.r];
    int64_t row[12] = {a.tj, a.n, a.ir, x.ls1, x.ls2, x.tj, b.tj, b.n, b.ir, x.rows, x.cols, x.off};
    table.insert(table.end(), row, row + 12);
  }
}

}  // namespace dmrg

namespace dmrg {

namespace {

// Materialise combined operators with more than one source: dst = sum scalar * src.
double* materialise(std::vector<CombOp>& comb, const OpStore& src, Stream st, int64_t* size) {
  int64_t total = 0;
  for (auto& c : comb)
    if (c.sources.size() > 1)
      for (auto& b : src.blocks[c.sources[0].first]) total += (int64_t)b.rows * b.cols;
  *size = total;
  if (total == 0) return nullptr;
  double* buf = (double*)dev_alloc(sizeof(double) * total, st);
  std::vector<CombSrc> cs;
  std::vector<CombDst> cd;
  int64_t off = 0;
  for (auto& c : comb) {
    if (c.sources.size() <= 1) continue;
    const auto& proto = src.blocks[c.sources[0].first];
    c.own_blocks.clear();
    c.own_at.clear();
    for (size_t bi = 0; bi < proto.size(); ++bi) {
      const BlockRef& pb = proto[bi];
      BlockRef nb = pb;
      nb.off = off;
      c.own_at[bkey(pb.r, pb.c)] = (int)c.own_blocks.size();
      c.own_blocks.push_back(nb);
      CombDst d{buf + off, pb.cols, pb.rows, pb.cols, (int)cs.size(), 0, 0};
      for (auto& s : c.sources) {
        auto it = src.at[s.first].find(bkey(pb.r, pb.c));
        if (it == src.at[s.first].end()) throw std::logic_error("combined sources differ in blocks");
        const BlockRef& sb = src.blocks[s.first][it->second];
        cs.push_back({src.data + sb.off, sb.cols, s.second});
      }
      d.src_end = (int)cs.size();
      cd.push_back(d);
      off += (int64_t)pb.rows * pb.cols;
    }
    c.blocks = &c.own_blocks;
    c.at = &c.own_at;
    c.data = buf;
    c.scalar = 1.0;
  }
  CombPlan* p = comb_plan_upload(cs, cd, st);
  comb_plan_run(p, st);
  comb_plan_free(p, st);
  return buf;
}

}  // namespace

// Left combined operators for the targets at bond i+1: C_{b,P} = sum_a s_a L_a(bond i).
void Engine::group_left(int i, std::vector<CombOp>& out, double** scratch, int64_t* scratch_n) {
  const OpStore& E = lenv_[i];
  std::map<std::pair<int, int>, int> idx;
  out.clear();
  for (const WEntry& w : W_[i]) {
    if (E.blocks[w.a].empty()) continue;
    auto key = std::make_pair(w.b, w.pattern);
    auto it = idx.find(key);
    if (it == idx.end()) {
      CombOp c;
      c.target = w.b;
      c.pattern = w.pattern;
      idx[key] = (int)out.size();
      out.push_back(std::move(c));
      it = idx.find(key);
    }
    out[it->second].sources.push_back({w.a, w.scalar});
    out[it->second].grad.push_back({w.gi, w.gc});
  }
  const int id_op = opsets_[i].find({OP_I, -1, -1, 0});
  for (auto& c : out)
    if (c.sources.size() == 1) {
      c.blocks = &E.blocks[c.sources[0].first];
      c.at = &E.at[c.sources[0].first];
      c.data = E.data;
      c.scalar = c.sources[0].second;
      c.identity = c.sources[0].first == id_op;
    }
  *scratch = materialise(out, E, stream_, scratch_n);
}

// Right combined operators for targets at bond j (site j): D_{a,P} = sum_b s_b R_b(bond j+1).
void Engine::group_right(int j, std::vector<CombOp>& out, double** scratch, int64_t* scratch_n) {
  const OpStore& E = renv_[j + 1];
  std::map<std::pair<int, int>, int> idx;
  out.clear();
  for (const WEntry& w : W_[j]) {
    if (E.blocks[w.b].empty()) continue;
    if (j + 1 == L_ && opsets_[L_].ops[w.b].key.type != OP_H) continue;  // zero partners
    auto key = std::make_pair(w.a, w.pattern);
    auto it = idx.find(key);
    if (it == idx.end()) {
      CombOp c;
      c.target = w.a;
      c.pattern = w.pattern;
      idx[key] = (int)out.size();
      out.push_back(std::move(c));
      it = idx.find(key);
    }
    out[it->second].sources.push_back({w.b, w.scalar});
    out[it->second].grad.push_back({w.gi, w.gc});
  }
  const int h_op = opsets_[j + 1].find({OP_H, -1, -1, 0});
  for (auto& c : out)
    if (c.sources.size() == 1) {
      c.blocks = &E.blocks[c.sources[0].first];
      c.at = &E.at[c.sources[0].first];
      c.data = E.data;
      c.scalar = c.sources[0].second;
      c.identity = c.sources[0].first == h_op;  // partner of H is the identity
    }
  *scratch = materialise(out, E, stream_, scratch_n);
}

// L_b(bond i+1)[jM' <- jM] = sum coef T[i]^T C_{b,P}[jL' <- jL] T[i], T[i] left-normalised.
void Engine::update_left_from(int i, std::vector<CombOp>& comb) {
  Timer tm;
  OpStore& E = lenv_[i + 1];
  alloc_env(E, i + 1, opsets_[i + 1]);
  const Site& T = sites_[i];
  const Bond& bl = bonds_[i];
  const Bond& bm = bonds_[i + 1];
  std::vector<std::vector<int>> by_l(bl.sec.size());
  for (int t = 0; t < (int)T.blocks.size(); ++t) by_l[T.blocks[t].l].push_back(t);
  const int id_op = opsets_[i + 1].find({OP_I, -1, -1, 0});
  std::vector<GemmTask> t1, t2;
  std::vector<GemmGroup> g1;
  std::vector<int64_t> bbase(E.blocks.size() + 1, 0);  // first output index of each operator
  for (size_t o = 0; o < E.blocks.size(); ++o) bbase[o + 1] = bbase[o] + (int64_t)E.blocks[o].size();
  std::vector<TaggedTask> out2;
  int64_t zsize = 0;
  struct ZRef { int64_t off; int rows, cols; };
  std::vector<ZRef> zs;
  t1.reserve(upd_hint_z_ + upd_hint_z_ / 4);
  g1.reserve(upd_hint_z_ + upd_hint_z_ / 4);
  zs.reserve(upd_hint_z_ + upd_hint_z_ / 4);
  out2.reserve(upd_hint_out_ + upd_hint_out_ / 4);
  for (auto& c : comb) {
    if (c.target == id_op) continue;
    for (const BlockRef& cb : *c.blocks) {
      for (int t : by_l[cb.c]) {
        const SiteBlock& tb = T.blocks[t];
        // Z1 = C_blk (rows x cols) . T_t (dL x dM)
        int zid = -1;
        for (int tp : by_l[cb.r]) {
          const SiteBlock& tpb = T.blocks[tp];
          double coef = c.scalar * cp_->left(c.pattern, bl.sec[tb.l].tj, tb.ls, bm.sec[tb.r].tj,
                                              bl.sec[tpb.l].tj, tpb.ls, bm.sec[tpb.r].tj);
          if (coef == 0.0) continue;
          auto it = E.at[c.target].find(bkey(tpb.r, tb.r));
          if (it == E.at[c.target].end()) continue;
          if (zid < 0) {
            zid = (int)zs.size();
            zs.push_back({zsize, cb.rows, tb.cols});
            zsize += (int64_t)cb.rows * tb.cols;
            t1.push_back({c.data + cb.off, T.data + tb.off, cb.cols, tb.cols, cb.cols, 0, 0, 1.0});
            g1.push_back({nullptr, tb.cols, cb.rows, tb.cols, (int)t1.size() - 1, (int)t1.size(), 0});
          }
          out2.push_back({bbase[c.target] + it->second,
                          {T.data + tpb.off, (const double*)(intptr_t)zid, tpb.cols, tb.cols, tpb.rows, 1, 0, coef}});
        }
      }
    }
  }
  upd_hint_z_ = t1.size();
  upd_hint_out_ = out2.size();
  double* Z = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(zsize, 1), stream_);
  for (size_t z = 0; z < g1.size(); ++z) g1[z].C = Z + zs[z].off;
  dev_zero(Z, sizeof(double) * std::max<int64_t>(zsize, 1), stream_);
  std::vector<GemmGroup> g2;
  {
    std::vector<int64_t> zoff(zs.size());
    for (size_t z = 0; z < zs.size(); ++z) zoff[z] = zs[z].off;
    std::vector<std::pair<int, int>> at(bbase.back());  // output index -> (op, block)
    for (size_t o = 0; o + 1 < bbase.size(); ++o)
      for (int64_t b = bbase[o]; b < bbase[o + 1]; ++b) at[b] = {(int)o, (int)(b - bbase[o])};
    group_by_output(out2, bbase.back(), Z, zoff,
                    [&](int64_t id, int b0, int b1, std::vector<GemmGroup>& g) {
                      const BlockRef& ob = E.blocks[at[id].first][at[id].second];
                      g.push_back({E.data + ob.off, ob.cols, ob.rows, ob.cols, b0, b1, 0});
                    }, t2, g2);
  }
  GemmPlan* p1 = gemm_plan_upload(t1, g1, stream_);
  GemmPlan* p2 = gemm_plan_upload(t2, g2, stream_);
  gemm_plan_run(p1, stream_);
  gemm_plan_run(p2, stream_);
  gemm_plan_free(p1, stream_);
  gemm_plan_free(p2, stream_);
  dev_free(Z, stream_);
  identity_fill(E, id_op);
  E.valid = true;
  st_.t_update_ms += tm.ms();
}

// R_a(bond j)[jM' <- jM] = sum coef V D_{a,P}[jR' <- jR] V^T with the mirrored tensor
// V = sqrt((2jR+1)/(2jM+1)) T[j] (Euclidean-orthonormal rows, the bracket of Eq. 27).
void Engine::update_right_from(int j, std::vector<CombOp>& comb) {
  Timer tm;
  OpStore& E = renv_[j];
  alloc_env(E, j, opsets_[j]);
  const Site& T = sites_[j];
  const Bond& bm = bonds_[j];
  const Bond& br = bonds_[j + 1];
  std::vector<std::vector<int>> by_r(br.sec.size());
  for (int t = 0; t < (int)T.blocks.size(); ++t) by_r[T.blocks[t].r].push_back(t);
  const int h_op = opsets_[j].find({OP_H, -1, -1, 0});
  auto f = [&](const SiteBlock& b) {
    return std::sqrt((double)(br.sec[b.r].tj + 1) / (double)(bm.sec[b.l].tj + 1));
  };
  std::vector<GemmTask> t1, t2;
  std::vector<GemmGroup> g1;
  std::vector<int64_t> bbase(E.blocks.size() + 1, 0);  // first output index of each operator
  for (size_t o = 0; o < E.blocks.size(); ++o) bbase[o + 1] = bbase[o] + (int64_t)E.blocks[o].size();
  std::vector<TaggedTask> out2;
  int64_t zsize = 0;
  struct ZRef { int64_t off; int rows, cols; };
  std::vector<ZRef> zs;
  t1.reserve(upd_hint_z_ + upd_hint_z_ / 4);
  g1.reserve(upd_hint_z_ + upd_hint_z_ / 4);
  zs.reserve(upd_hint_z_ + upd_hint_z_ / 4);
  out2.reserve(upd_hint_out_ + upd_hint_out_ / 4);
  for (auto& c : comb) {
    if (c.target == h_op) continue;
    for (const BlockRef& db : *c.blocks) {
      for (int t : by_r[db.c]) {
        const SiteBlock& tb = T.blocks[t];
        int zid = -1;
        for (int tp : by_r[db.r]) {
          const SiteBlock& tpb = T.blocks[tp];
          double coef = c.scalar * f(tb) * f(tpb) *
                        cp_->right(c.pattern, tb.ls, br.sec[tb.r].tj, bm.sec[tb.l].tj, tpb.ls,
                                   br.sec[tpb.r].tj, bm.sec[tpb.l].tj);
          if (coef == 0.0) continue;
          auto it = E.at[c.target].find(bkey(tpb.l, tb.l));
          if (it == E.at[c.target].end()) continue;
          if (zid < 0) {
            // Z1 = D_blk (dR' x dR) . T_t^T (dR x dM)
            zid = (int)zs.size();
            zs.push_back({zsize, db.rows, tb.rows});
            zsize += (int64_t)db.rows * tb.rows;
            t1.push_back({c.data + db.off, T.data + tb.off, db.cols, tb.cols, db.cols, 0, 1, 1.0});
            g1.push_back({nullptr, tb.rows, db.rows, tb.rows, (int)t1.size() - 1, (int)t1.size(), 0});
          }
          out2.push_back({bbase[c.target] + it->second,
                          {T.data + tpb.off, (const double*)(intptr_t)zid, tpb.cols, tb.rows, tpb.cols, 0, 0, coef}});
        }
      }
    }
  }
  upd_hint_z_ = t1.size();
  upd_hint_out_ = out2.size();
  double* Z = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(zsize, 1), stream_);
  for (size_t z = 0; z < g1.size(); ++z) g1[z].C = Z + zs[z].off;
  dev_zero(Z, sizeof(double) * std::max<int64_t>(zsize, 1), stream_);
  std::vector<GemmGroup> g2;
  {
    std::vector<int64_t> zoff(zs.size());
    for (size_t z = 0; z < zs.size(); ++z) zoff[z] = zs[z].off;
    std::vector<std::pair<int, int>> at(bbase.back());  // output index -> (op, block)
    for (size_t o = 0; o + 1 < bbase.size(); ++o)
      for (int64_t b = bbase[o]; b < bbase[o + 1]; ++b) at[b] = {(int)o, (int)(b - bbase[o])};
    group_by_output(out2, bbase.back(), Z, zoff,
                    [&](int64_t id, int b0, int b1, std::vector<GemmGroup>& g) {
                      const BlockRef& ob = E.blocks[at[id].first][at[id].second];
                      g.push_back({E.data + ob.off, ob.cols, ob.rows, ob.cols, b0, b1, 0});
                    }, t2, g2);
  }
  GemmPlan* p1 = gemm_plan_upload(t1, g1, stream_);
  GemmPlan* p2 = gemm_plan_upload(t2, g2, stream_);
  gemm_plan_run(p1, stream_);
  gemm_plan_run(p2, stream_);
  gemm_plan_free(p1, stream_);
  gemm_plan_free(p2, stream_);
  dev_free(Z, stream_);
  identity_fill(E, h_op);
  E.valid = true;
  st_.t_update_ms += tm.ms();
}

void Engine::build_left(int k) {
  std::vector<CombOp> comb;
  double* scr = nullptr;
  int64_t scr_n = 0;
  group_left(k - 1, comb, &scr, &scr_n);
  update_left_from(k - 1, comb);
  if (scr) dev_free(scr, stream_);
}

void Engine::build_right(int k) {
  std::vector<CombOp> comb;
  double* scr = nullptr;
  int64_t scr_n = 0;
  group_right(k, comb, &scr, &scr_n);
  update_right_from(k, comb);
  if (scr) dev_free(scr, stream_);
}

}  // namespace dmrg

namespace dmrg {

struct Engine::MatvecPlan {
  int site = -1;
  int64_t n = 0;
  std::vector<XBlock> X;
  std::vector<CombOp> cl, cr;
  double* scr_l = nullptr;
  double* scr_r = nullptr;
  int64_t scr_l_n = 0, scr_r_n = 0;
  double* Z = nullptr;
  double* W = nullptr;
  CombPlan* pc = nullptr;
  int64_t wsize = 0;
  double* xin = nullptr;
  double* yout = nullptr;
  double* diag = nullptr;
  GemmPlan* p1 = nullptr;
  GemmPlan* p2 = nullptr;
  double flops = 0.0, flops1 = 0.0, flops2 = 0.0;
  // the quadratic form x^T H x with the block pairs of input block >= output block
  // (build_rq; phase 1 restricted to the x rows those pairs read)
  GemmPlan* rq1 = nullptr;
  GemmPlan* rq2 = nullptr;
  CombPlan* rqc = nullptr;
  double rq_flops1 = 0.0, rq_flops2 = 0.0;
  int64_t ntasks = 0;
  int64_t zsize = 0;
  // host tables kept for the mixed-precision plan (built on first use, then released)
  struct ZGroup { const double* D; int n, K; double alpha; int c; int64_t off; };
  // source x block xb; zg < 0: D is the identity; right group gr, coefficient without
  // the group's scalar craw
  struct WSrc { int zg, xb; double coef; int gr; double craw; };
  struct WItem { int gl, cbi, rows, cols, src_begin, src_end; };
  std::vector<ZGroup> zg;
  std::vector<WSrc> wsrc;
  std::vector<WItem> witems;
  std::vector<std::vector<int>> w_by_x;
  std::vector<int64_t> tall_off, tall_rows;
  std::vector<int> sec_dim;
  // mixed-precision matvec: the tiled hi / lo operand pools (operators once per plan, x
  // per matvec), where each block sits in them, the host tables of the current tuning
  // (kept for batched launches) and their device copy
  TcHost tch;
  TcTune tch_tune;
  TcPlan* tc = nullptr;
  float* tc_ops = nullptr;
  float* tc_x = nullptr;
  int64_t tc_ops_lo = 0, tc_x_lo = 0;
  std::vector<int64_t> tc_dmir;                  // Z group -> its right-operator block in the pool
  std::vector<std::vector<int64_t>> tc_cmir;     // (left group, block) -> the block in the pool
  std::unordered_map<int, int64_t> tc_idmir;     // identity of a dimension -> its place in the pool
  std::vector<int64_t> tc_xoff;                  // x block -> its place in the x pool
  double tc_alg_bytes = 0.0;  // operator blocks read once (FP32) + x read and y written (FP64)
  uint64_t serial = 0;      // distinguishes successive plans of an engine
  // excited states: projections v_k of the lower states (nlow x n, row k = v_k) and
  // eta_k v_k, the coefficients c_k = v_k . x and their reduction scratch
  int nlow = 0;
  double* lowv = nullptr;
  double* loww = nullptr;
  double* lowc = nullptr;
};

namespace {
// site transitions allowed by a pattern: ok[ket ls][bra ls]
void allowed(const Pattern& P, bool ok[3][3]) {
  static const int ls_of[4] = {0, 1, 1, 2};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) ok[a][b] = false;
  const int nq = (P.tka + 1) * (P.tkb + 1);
  for (int q = 0; q < nq; ++q)
    for (int br = 0; br < 4; ++br)
      for (int kt = 0; kt < 4; ++kt)
        if (P.w[(size_t)q * 16 + br * 4 + kt] != 0.0) ok[ls_of[kt]][ls_of[br]] = true;
}
}  // namespace

Engine::MatvecPlan* Engine::plan_matvec(int i, bool rdm) {
  Timer tm;
  ensure_left(i);
  ensure_right(i + 2);
  MatvecPlan* P = new MatvecPlan;
  // a plan whose build fails (for instance on the device memory cap) is released whole
  struct Guard {
    Engine* e;
    MatvecPlan* p;
    ~Guard() { if (p) e->free_plan(p); }
  } guard{this, P};
  P->site = i;
  P->X = x_layout(i, &P->n);
  group_left(i, P->cl, &P->scr_l, &P->scr_l_n);
  group_right(i + 1, P->cr, &P->scr_r, &P->scr_r_n);
  const Bond& bl = bonds_[i];
  const Bond& br = bonds_[i + 2];
  const OpSet& mid = opsets_[i + 1];
  const int nl = (int)bl.sec.size(), nr = (int)br.sec.size();
  std::vector<std::vector<int>> byb_l(mid.ops.size()), byb_r(mid.ops.size());
  for (int g = 0; g < (int)P->cl.size(); ++g) byb_l[P->cl[g].target].push_back(g);
  for (int g = 0; g < (int)P->cr.size(); ++g) byb_r[P->cr[g].target].push_back(g);
  // X' lookup: index by (l, ls1, ls2, tj, r) -> dense table
  auto xkey = [&](int l, int ls1, int ls2, int tj, int r) {
    return ((((int64_t)l * 3 + ls1) * 3 + ls2) * 3 + tj) * nr + r;
  };
  std::vector<int> xidx((size_t)nl * 27 * nr, -1);
  std::vector<std::vector<int>> x_by_l(nl);
  std::vector<int64_t> tall_rows(nr, 0), tall_off(nr, -1);
  for (int x = 0; x < (int)P->X.size(); ++x) {
    const XBlock& b = P->X[x];
    xidx[xkey(b.l, b.ls1, b.ls2, b.tj, b.r)] = x;
    x_by_l[b.l].push_back(x);
    tall_rows[b.r] = std::max<int64_t>(tall_rows[b.r], b.trow + b.rows);
    if (tall_off[b.r] < 0) tall_off[b.r] = b.off;
  }
  P->xin = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(P->n, 1), stream_);
  P->yout = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(P->n, 1), stream_);
  // right-group blocks indexed by column sector
  std::vector<std::vector<std::vector<int>>> dby(P->cr.size());
  for (int g = 0; g < (int)P->cr.size(); ++g) {
    dby[g].resize(nr);
    for (int bi = 0; bi < (int)P->cr[g].blocks->size(); ++bi) dby[g][(*P->cr[g].blocks)[bi].c].push_back(bi);
  }
  // phase 1: Z(gr, D block) = stack(r) . D^T ; identity D reads x directly
  struct ZRef { int64_t off; int ld; int zg; };
  std::vector<std::vector<ZRef>> ztab(P->cr.size());  // (gr, dbi) -> Z, zg == INT_MIN: not yet made
  for (size_t g = 0; g < P->cr.size(); ++g)
    ztab[g].assign(P->cr[g].blocks->size(), ZRef{0, 0, std::numeric_limits<int>::min()});
  std::vector<GemmTask> t1;
  std::vector<GemmGroup> g1;
  std::vector<int64_t> g1off;
  int64_t zsize = 0;
  double flops1 = 0.0, flops2 = 0.0;
  auto get_z = [&](int gr, int dbi) -> ZRef {
    const CombOp& D = P->cr[gr];
    const BlockRef& db = (*D.blocks)[dbi];
    ZRef& z = ztab[gr][dbi];
    if (z.zg != std::numeric_limits<int>::min()) return z;
    if (D.identity) {
      z = {-1 - tall_off[db.c], br.dim[db.c], -1 - db.c};  // negative: offset into xin
    } else {
      const int64_t rows = tall_rows[db.c];
      z = {zsize, db.rows, (int)g1.size()};
      P->zg.push_back({D.data + db.off, db.rows, db.cols, D.scalar, db.c, zsize});
      t1.push_back({nullptr, D.data + db.off, db.cols, db.cols, db.cols, 0, 1, D.scalar});
      g1.push_back({nullptr, db.rows, (int)rows, db.rows, (int)t1.size() - 1, (int)t1.size(), 0});
      g1off.push_back(tall_off[db.c]);
      zsize += rows * db.rows;
      flops1 += 2.0 * rows * db.cols * db.rows;
    }
    return z;
  };
  // site transitions allowed by each pattern, and the recoupled coefficient of a
  // (left pattern, right pattern, block labels) combination, memoised
  std::vector<std::array<std::array<bool, 3>, 3>> okp(pt_.pats.size());
  for (size_t q = 0; q < pt_.pats.size(); ++q) {
    bool ok[3][3];
    allowed(pt_.pats[q], ok);
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) okp[q][a][c] = ok[a][c];
  }
  using K2 = CoefKey;
  // W(gl, C block, X') = sum coef * Z rows of X ; phase 2: y_X' += C_blk W
  struct WItem { int gl, cbi, xp; int64_t off; int rows, cols; int src_begin, src_end; };
  std::vector<WItem> ws;
  std::vector<std::vector<DiagTerm>> dout(P->X.size());
  std::vector<std::vector<int>> w_by_x(P->X.size());
  int64_t wsize = 0;
  // Enumeration of the (left block, right block, x block) combinations, in parallel
  // over work items (middle operator b, left group gl, left block cbi) with private
  // coefficient caches, then a serial merge in item order (deterministic tables).
  struct Item { int b, gl, cbi; };
  std::vector<Item> items;
  for (int b = 0; b < (int)mid.ops.size(); ++b) {
    if (byb_l[b].empty() || byb_r[b].empty()) continue;
    for (int gl : byb_l[b])
      for (int cbi = 0; cbi < (int)P->cl[gl].blocks->size(); ++cbi) items.push_back({b, gl, cbi});
  }
  struct Src { int gr, dbi, x; double coef; };
  struct Grp { int xp, begin, end; };      // sources of one W item, first-touch order
  struct DRaw { int x, gr, dbi; double coef; };
  struct Out { std::vector<Grp> g; std::vector<Src> s; std::vector<DRaw> d; int64_t wb = 0; };
  // right-operator blocks some source uses (set by the workers; Z groups are made for these)
  std::vector<int64_t> zbase(P->cr.size() + 1, 0);
  for (size_t g = 0; g < P->cr.size(); ++g) zbase[g + 1] = zbase[g] + (int64_t)P->cr[g].blocks->size();
  std::unique_ptr<std::atomic<uint8_t>[]> zused(new std::atomic<uint8_t>[std::max<int64_t>(zbase.back(), 1)]);
  for (int64_t z = 0; z < zbase.back(); ++z) zused[z].store(0, std::memory_order_relaxed);
  std::vector<Out> outs(items.size());
  std::atomic<size_t> next_item{0};
  const unsigned hcw = std::thread::hardware_concurrency();
  const int nthw = (int)std::max(1u, std::min(16u, hcw ? hcw : 1u));
  std::vector<std::unordered_map<K2, double, CoefKeyHash>> new_coefs(nthw);
  std::atomic<int> next_worker{0};
  const auto& master = coef_master_;  // read-only while the workers run
  std::mutex worker_mu;
  std::exception_ptr worker_err;
  auto worker_body = [&]() {
    Coupling cp = *cp_;  // private memo tables
    auto& coef_cache = new_coefs[next_worker.fetch_add(1)];
    coef_cache.reserve(1 << 12);
    std::vector<int> slot(P->X.size(), -1), touched;
    std::vector<std::vector<Src>> bucket;
    for (;;) {
      const size_t it = next_item.fetch_add(1);
      if (it >= items.size()) break;
      const Item I = items[it];
      const int tkb = mid.ops[I.b].tk, pb = mid.ops[I.b].parity;
      const CombOp& C = P->cl[I.gl];
      const auto& ok1 = okp[C.pattern];
      const BlockRef& cb = (*C.blocks)[I.cbi];
      const int tjL = bl.sec[cb.c].tj, tjLp = bl.sec[cb.r].tj;
      Out& o = outs[it];
      for (int x : x_by_l[cb.c]) {
        const XBlock& X = P->X[x];
        const int tjR = br.sec[X.r].tj;
        const int t1s = local_ts(X.ls1), t2s = local_ts(X.ls2);
        for (int gr : byb_r[I.b]) {
          const CombOp& D = P->cr[gr];
          const auto& ok2 = okp[D.pattern];
          for (int dbi : dby[gr][X.r]) {
            const BlockRef& db = (*D.blocks)[dbi];
            const int tjRp = br.sec[db.r].tj;
            for (int ls1p = 0; ls1p < 3; ++ls1p) {
              if (!ok1[X.ls1][ls1p]) continue;
              const int t1p = local_ts(ls1p);
              for (int ls2p = 0; ls2p < 3; ++ls2p) {
                if (!ok2[X.ls2][ls2p]) continue;
                const int t2p = local_ts(ls2p);
                for (int tjp = std::abs(t1p - t2p); tjp <= t1p + t2p; tjp += 2) {
                  const int xp = xidx[xkey(cb.r, ls1p, ls2p, tjp, db.r)];
                  if (xp < 0) continue;
                  K2 key{(uint64_t)C.pattern | ((uint64_t)D.pattern << 16) | ((uint64_t)tjL << 32) |
                             ((uint64_t)tjR << 40) | ((uint64_t)tjLp << 48) | ((uint64_t)tjRp << 56),
                         (uint64_t)X.ls1 | ((uint64_t)X.ls2 << 2) | ((uint64_t)X.tj << 4) |
                             ((uint64_t)ls1p << 8) | ((uint64_t)ls2p << 10) | ((uint64_t)tjp << 12)};
                  auto ci = coef_cache.find(key);
                  auto mi = ci == coef_cache.end() ? master.find(key) : master.end();
                  double coef = 0.0;
                  if (ci != coef_cache.end()) {
                    coef = ci->second;
                  } else if (mi != master.end()) {
                    coef = mi->second;
                  } else {
                    for (int tjM = std::abs(tjL - t1s); tjM <= tjL + t1s; tjM += 2) {
                      if (!triangle(t2s, tjR, tjM)) continue;
                      double ov = cp.overlap(tjL, X.ls1, X.ls2, X.tj, tjR, tjM);
                      if (ov == 0.0) continue;
                      for (int tjMp = std::abs(tjLp - t1p); tjMp <= tjLp + t1p; tjMp += 2) {
                        if (!triangle(t2p, tjRp, tjMp)) continue;
                        double ovp = cp.overlap(tjLp, ls1p, ls2p, tjp, tjRp, tjMp);
                        if (ovp == 0.0) continue;
                        double sf = cp.singlet(tkb, pb, tjM, tjMp);
                        if (sf == 0.0) continue;
                        double lc = cp.left(C.pattern, tjL, X.ls1, tjM, tjLp, ls1p, tjMp);
                        if (lc == 0.0) continue;
                        double rc = cp.right(D.pattern, X.ls2, tjR, tjM, ls2p, tjRp, tjMp);
                        coef += ov * ovp * sf * lc * rc;
                      }
                    }
                    coef_cache.emplace(key, coef);
                  }
                  if (std::fabs(coef) < 1e-14) continue;
                  int& sl = slot[xp];
                  if (sl < 0) {
                    sl = (int)touched.size();
                    touched.push_back(xp);
                    if (bucket.size() < touched.size()) bucket.emplace_back();
                    bucket[sl].clear();
                  }
                  bucket[sl].push_back({gr, dbi, x, coef});
                  if (!rdm && xp == x && cb.r == cb.c && db.r == db.c) o.d.push_back({x, gr, dbi, coef});
                }
              }
            }
          }
        }
      }
      for (size_t k = 0; k < touched.size(); ++k) {
        o.g.push_back({touched[k], (int)o.s.size(), 0});
        o.s.insert(o.s.end(), bucket[k].begin(), bucket[k].end());
        o.g.back().end = (int)o.s.size();
        o.wb += (int64_t)cb.cols * P->X[touched[k]].cols;
        slot[touched[k]] = -1;
      }
      for (const Src& q : o.s) zused[zbase[q.gr] + q.dbi].store(1, std::memory_order_relaxed);
      touched.clear();
    }
  };
  {
    const unsigned hc = std::thread::hardware_concurrency();
    const int nth = (int)std::max(1u, std::min(16u, hc ? hc : 1u));
    std::vector<std::thread> th;
    auto worker = [&]() {
      try {
        worker_body();
      } catch (...) {
        std::lock_guard<std::mutex> lk(worker_mu);
        if (!worker_err) worker_err = std::current_exception();
        next_item.store(items.size());
      }
    };
    for (int t = 1; t < nth && (size_t)t < items.size(); ++t) th.emplace_back(worker);
    worker();
    for (auto& t : th) t.join();
    if (worker_err) std::rethrow_exception(worker_err);
  }
  for (auto& m : new_coefs)
    for (auto& kv : m) coef_master_.emplace(kv.first, kv.second);
  // Merge in item order (deterministic tables).  Z groups get their ids in (right
  // group, block) order among the blocks some source uses; the W items and sources of
  // every item go to offsets from prefix sums over the items, filled in parallel.
  for (int gr = 0; gr < (int)P->cr.size(); ++gr)
    for (int dbi = 0; dbi < (int)ztab[gr].size(); ++dbi)
      if (zused[zbase[gr] + dbi].load(std::memory_order_relaxed)) get_z(gr, dbi);
  const size_t nit = items.size();
  std::vector<int64_t> it_w(nit + 1, 0), it_s(nit + 1, 0), it_off(nit + 1, 0);
  for (size_t it = 0; it < nit; ++it) {
    const Out& o = outs[it];
    const BlockRef& cb = (*P->cl[items[it].gl].blocks)[items[it].cbi];
    const int64_t wb = o.wb;
    it_w[it + 1] = it_w[it] + (int64_t)o.g.size();
    it_s[it + 1] = it_s[it] + (int64_t)o.s.size();
    it_off[it + 1] = it_off[it] + wb;
    const CombOp& C = P->cl[items[it].gl];
    if (rdm) continue;
    for (const DRaw& dr : o.d) {
      const CombOp& D = P->cr[dr.gr];
      const BlockRef& db = (*D.blocks)[dr.dbi];
      dout[dr.x].push_back({C.data + cb.off, D.data + db.off, cb.cols, db.cols, dr.coef * C.scalar * D.scalar});
    }
  }
  if (it_w[nit] > std::numeric_limits<int>::max() || it_s[nit] > std::numeric_limits<int>::max())
    throw std::runtime_error("matvec tables exceed 2^31 entries");
  wsize = it_off[nit];
  P->zsize = zsize;
  P->Z = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(zsize, 1), stream_);
  P->W = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(wsize, 1), stream_);
  {
    // fix up phase-1 pointers: A = stack of x rows for the column sector
    int64_t zo = 0;
    for (size_t z = 0; z < g1.size(); ++z) {
      t1[z].A = P->xin + g1off[z];
      t1[z].lda = t1[z].ldb;  // stack(r) has ld = d_r = D block columns
      g1[z].C = P->Z + zo;
      zo += (int64_t)g1[z].m * g1[z].n;
    }
  }
  // combine plan for W (one destination per W item, its sources in order)
  std::vector<CombSrc> cs(it_s[nit]);
  std::vector<CombDst> cd(it_w[nit]);
  ws.resize(it_w[nit]);
  // the RDM pass reads the sources' table only at the last pair
  const bool keep_src = !rdm || i == L_ - 2;
  if (keep_src) P->wsrc.resize(it_s[nit]);
  P->witems.resize(it_w[nit]);
  std::vector<double> it_flops(nit, 0.0);
  {
    auto fill = [&](size_t ib, size_t ie) {
        for (size_t it = ib; it < ie; ++it) {
          const Item& I = items[it];
          const CombOp& C = P->cl[I.gl];
          const BlockRef& cb = (*C.blocks)[I.cbi];
          Out& o = outs[it];
          int64_t wi = it_w[it], si = it_s[it], off = it_off[it];
          for (const Grp& g : o.g) {
            const XBlock& Xp = P->X[g.xp];
            WItem w{I.gl, I.cbi, g.xp, off, cb.cols, Xp.cols, (int)si, 0};
            for (int k = g.begin; k < g.end; ++k, ++si) {
              const Src& q = o.s[k];
              const CombOp& D = P->cr[q.gr];
              const XBlock& X = P->X[q.x];
              const ZRef z = ztab[q.gr][q.dbi];
              const int64_t zoff = z.off >= 0 ? z.off + (int64_t)X.trow * z.ld : z.off - (int64_t)X.trow * z.ld;
              // identity right operator: Z is x itself, its alias scalar goes here
              const double coef = D.identity ? q.coef * D.scalar : q.coef;
              cs[si] = {zoff >= 0 ? P->Z + zoff : P->xin + (-1 - zoff), z.ld, coef};
              if (keep_src) P->wsrc[si] = {z.zg, q.x, coef, q.gr, q.coef};
            }
            w.src_end = (int)si;
            P->witems[wi] = {I.gl, I.cbi, w.rows, w.cols, w.src_begin, w.src_end};
            cd[wi] = {P->W + w.off, w.cols, w.rows, w.cols, w.src_begin, w.src_end, 0};
            ws[wi++] = w;
            off += (int64_t)cb.cols * Xp.cols;
            if (!C.identity) it_flops[it] += 2.0 * cb.rows * cb.cols * Xp.cols;
          }
          std::vector<Grp>().swap(o.g);
          std::vector<Src>().swap(o.s);
          std::vector<DRaw>().swap(o.d);
        }
    };
    parallel_chunks(nit, 64, fill);
  }
  for (size_t it = 0; it < nit; ++it) flops2 += it_flops[it];
  {
    std::vector<int> cnt(P->X.size(), 0);
    for (const WItem& w : ws) ++cnt[w.xp];
    for (size_t x = 0; x < P->X.size(); ++x) w_by_x[x].reserve(cnt[x]);
    for (int k = 0; k < (int)ws.size(); ++k) w_by_x[ws[k].xp].push_back(k);
  }
  // phase 2 grouped by output block: the tasks of block x at the prefix of |w_by_x|
  // (none for the RDM pass)
  std::vector<int64_t> xt(P->X.size() + 1, 0), xg(P->X.size() + 1, 0);
  for (size_t x = 0; x < P->X.size() && !rdm; ++x) {
    xt[x + 1] = xt[x] + (int64_t)w_by_x[x].size();
    xg[x + 1] = xg[x] + (w_by_x[x].empty() ? 0 : 1);
  }
  std::vector<GemmTask> t2(xt[P->X.size()]);
  std::vector<GemmGroup> g2(xg[P->X.size()]);
  if (!rdm) parallel_chunks(P->X.size(), 256, [&](size_t xb, size_t xe) {
    for (size_t x = xb; x < xe; ++x) {
      if (w_by_x[x].empty()) continue;
      const XBlock& X = P->X[x];
      int64_t k = xt[x];
      for (int wi : w_by_x[x]) {
        const WItem& w = ws[wi];
        const CombOp& C = P->cl[w.gl];
        const BlockRef& cb = (*C.blocks)[w.cbi];
        if (C.identity) t2[k++] = {nullptr, P->W + w.off, 0, w.cols, w.rows, 0, 0, C.scalar};
        else t2[k++] = {C.data + cb.off, P->W + w.off, cb.cols, w.cols, cb.cols, 0, 0, C.scalar};
      }
      g2[xg[x]] = {P->yout + X.off, X.cols, X.rows, X.cols, (int)xt[x], (int)xt[x + 1], 0};
    }
  });
  // diagonal (not for the RDM pass)
  std::vector<DiagTerm> dt;
  std::vector<DiagOut> dov;
  if (!rdm) {
    P->diag = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(P->n, 1), stream_);
    dev_zero(P->diag, sizeof(double) * std::max<int64_t>(P->n, 1), stream_);
    for (int x = 0; x < (int)P->X.size(); ++x) {
      if (dout[x].empty()) continue;
      const XBlock& X = P->X[x];
      int d0 = (int)dt.size();
      dt.insert(dt.end(), dout[x].begin(), dout[x].end());
      dov.push_back({P->diag + X.off, X.rows, X.cols, d0, (int)dt.size()});
    }
  }
  P->w_by_x = std::move(w_by_x);
  P->tall_off = std::move(tall_off);
  P->tall_rows = std::move(tall_rows);
  P->sec_dim = br.dim;
  P->p1 = gemm_plan_upload(t1, g1, stream_);
  P->pc = comb_plan_upload(cs, cd, stream_);
  if (!rdm) {
    P->p2 = gemm_plan_upload(t2, g2, stream_);
    DiagPlan* pd = diag_plan_upload(dt, dov, stream_);
    diag_plan_run(pd, stream_);
    diag_plan_free(pd, stream_);
  }
  if (!low_.empty() && !rdm) {
    // the lower states' projections onto this pair's basis: + eta |v><v| in every matvec
    const int m = (int)low_.size();
    P->nlow = m;
    P->lowv = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(P->n * m, 1), stream_);
    P->loww = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(P->n * m, 1), stream_);
    P->lowc = (double*)dev_alloc(sizeof(double) * (m + (int64_t)m * 512), stream_);
    for (int k = 0; k < m; ++k) {
      low_projection(low_[k], i, P->X, P->lowv + (int64_t)k * P->n);
      dev_zero(P->loww + (int64_t)k * P->n, sizeof(double) * P->n, stream_);
      vec_axpby(low_[k].eta, P->lowv + (int64_t)k * P->n, 0.0, P->loww + (int64_t)k * P->n, P->n, stream_);
    }
  }
  P->flops1 = flops1;
  P->flops2 = flops2;
  P->flops = flops1 + flops2;
  P->ntasks = (int64_t)t1.size() + (int64_t)t2.size() + (int64_t)cs.size();
  P->wsize = wsize;
  st_.t_plan_ms += tm.ms();
  guard.p = nullptr;
  return P;
}

}  // namespace dmrg

namespace dmrg {

void Engine::release_tc(MatvecPlan* p) {
  tc_plan_free(p->tc, stream_);
  p->tc = nullptr;
  if (p->tc_ops) dev_free(p->tc_ops, stream_);
  if (p->tc_x) dev_free(p->tc_x, stream_);
  p->tc_ops = p->tc_x = nullptr;
  p->tc_dmir.clear();
  p->tc_cmir.clear();
  p->tc_idmir.clear();
  p->tc_xoff.clear();
  p->tch = TcHost();
}

void Engine::free_plan(MatvecPlan* p) {
  if (!p) return;
  release_tc(p);
  gemm_plan_free(p->p1, stream_);
  gemm_plan_free(p->p2, stream_);
  comb_plan_free(p->pc, stream_);
  gemm_plan_free(p->rq1, stream_);
  gemm_plan_free(p->rq2, stream_);
  comb_plan_free(p->rqc, stream_);
  dev_free(p->Z, stream_);
  dev_free(p->W, stream_);
  dev_free(p->xin, stream_);
  dev_free(p->yout, stream_);
  dev_free(p->diag, stream_);
  if (p->scr_l) dev_free(p->scr_l, stream_);
  if (p->scr_r) dev_free(p->scr_r, stream_);
  if (p->lowv) dev_free(p->lowv, stream_);
  if (p->loww) dev_free(p->loww, stream_);
  if (p->lowc) dev_free(p->lowc, stream_);
  // the host tables (millions of entries) are released on a helper thread, one plan at
  // a time, while the caller goes on
  if (reaper_.joinable()) reaper_.join();
  reaper_ = std::thread([p]() { delete p; });
}

Engine::MatvecPlan* Engine::plan_for(int i) {
  if (cached_ && cached_site_ == i) return cached_;
  if (cached_) { free_plan(cached_); cached_ = nullptr; cached_site_ = -1; }
  cached_ = plan_matvec(i);
  cached_->serial = ++plan_serial_;
  cached_site_ = i;
  return cached_;
}

// y = H_eff x on the plan's fixed buffers: Z = x D^T (phase 1), y = sum coef C Z (phase 2).
void Engine::flush_events() {
  if (!ev_pending_) return;
  const double a = event_elapsed_ms(ev_[0], ev_[1]), b = event_elapsed_ms(ev_[1], ev_[2]);
  if (ev_tc_) { st_.tc_phase1_ms += a; st_.tc_phase2_ms += b; }
  else { st_.k_phase1_ms += a; st_.k_phase2_ms += b; }
  ev_pending_ = false;
}

// Operands of the mixed-precision matvec (kernels_tc.cu): every operator block the matvec
// reads, and the identities that identity operators stand for, tiled and split into TF32
// hi / lo in one pool (converted once per plan), and a pool for x (converted per
// matvec); then the tables of the current tuning.
void Engine::build_tc(MatvecPlan* P) {
  Timer tm;
  auto tsize = [](int rows, int cols) -> int64_t { return (int64_t)((cols + 31) / 32) * ((rows + 7) / 8) * 256; };
  std::unordered_map<const double*, int64_t> moff;
  std::vector<TfConv> conv;
  std::vector<int64_t> conv_off;
  int64_t pool = 0;
  double distinct = 0.0;
  auto want = [&](const double* p, int rows, int cols) -> int64_t {
    auto ins = moff.emplace(p, pool);
    if (ins.second) {
      conv.push_back({p, nullptr, rows, cols, (rows + 7) / 8, 0, 0});
      conv_off.push_back(pool);
      pool += tsize(rows, cols);
      distinct += (double)rows * cols;
    }
    return ins.first->second;
  };
  auto want_id = [&](int d) -> int64_t {
    auto it = P->tc_idmir.find(d);
    if (it != P->tc_idmir.end()) return it->second;
    conv.push_back({nullptr, nullptr, d, d, (d + 7) / 8, 1, 0});
    conv_off.push_back(pool);
    P->tc_idmir[d] = pool;
    pool += tsize(d, d);
    return P->tc_idmir[d];
  };
  P->tc_dmir.assign(P->zg.size(), -1);
  for (size_t g = 0; g < P->zg.size(); ++g) P->tc_dmir[g] = want(P->zg[g].D, P->zg[g].n, P->zg[g].K);
  for (const auto& q : P->wsrc)
    if (q.zg < 0) want_id(P->X[q.xb].cols);
  P->tc_cmir.assign(P->cl.size(), {});
  for (const auto& w : P->witems) {
    const CombOp& C = P->cl[w.gl];
    if (C.identity) {
      want_id(w.rows);
      continue;
    }
    auto& cm = P->tc_cmir[w.gl];
    if (cm.empty()) cm.assign(C.blocks->size(), -1);
    if (cm[w.cbi] < 0) {
      const BlockRef& cb = (*C.blocks)[w.cbi];
      cm[w.cbi] = want(C.data + cb.off, cb.rows, cb.cols);
    }
  }
  const int64_t ops = std::max<int64_t>(pool, 256);
  P->tc_ops = (float*)dev_alloc(sizeof(float) * 2 * ops, stream_);
  P->tc_ops_lo = ops;
  dev_zero(P->tc_ops, sizeof(float) * 2 * ops, stream_);
  for (size_t k = 0; k < conv.size(); ++k) {
    conv[k].dst = P->tc_ops + conv_off[k];
    conv[k].lo = ops;
  }
  tc_convert(conv, stream_);
  P->tc_xoff.resize(P->X.size());
  int64_t xp = 0;
  for (size_t x = 0; x < P->X.size(); ++x) {
    P->tc_xoff[x] = xp;
    xp += tsize(P->X[x].rows, P->X[x].cols);
  }
  const int64_t xs = std::max<int64_t>(xp, 256);
  P->tc_x = (float*)dev_alloc(sizeof(float) * 2 * xs, stream_);
  P->tc_x_lo = xs;
  dev_zero(P->tc_x, sizeof(float) * 2 * xs, stream_);  // padding stays zero; x fills the rest
  P->tc_alg_bytes = 4.0 * distinct + 16.0 * (double)P->n;
  tc_tables(P, tune_);
  P->tc = tc_plan_build({&P->tch}, stream_);
  st_.t_plan_ms += tm.ms();
}

// Tiles (one CTA each: up to row_tile rows x 128 columns of one output block), their
// sub-tasks (a term's left-operator block C and its sources, over at most x_chunk x rows)
// and the sources (right-operator block, x block, coefficient with both scalars).
void Engine::tc_tables(MatvecPlan* P, TcTune tune) {
  if (tune.row_tile != 64 && tune.row_tile != 128) throw std::invalid_argument("tc row tile");
  if (tune.x_chunk != 32 && tune.x_chunk != 64) throw std::invalid_argument("tc x chunk");
  const int RT = tune.row_tile, XC = tune.x_chunk;
  TcHost& H = P->tch;
  H = TcHost();
  const size_t nX = P->X.size();
  auto nrg = [](int rows) { return (rows + 7) / 8; };
  H.xb.reserve(nX);
  for (size_t x = 0; x < nX; ++x) {
    const XBlock& X = P->X[x];
    H.xb.push_back({P->xin + X.off, P->tc_x + P->tc_xoff[x], X.rows, X.cols, nrg(X.rows), 0, P->tc_x_lo});
  }
  // sizes per output block, then prefix offsets (the fill runs in parallel)
  std::vector<int64_t> ntile(nX + 1, 0), ntask(nX + 1, 0), nsrc(nX + 1, 0);
  for (size_t x = 0; x < nX; ++x) {
    const XBlock& X = P->X[x];
    const int64_t tiles = (int64_t)((X.rows + RT - 1) / RT) * ((X.cols + 127) / 128);
    int64_t tk = 0, sr = 0;
    for (int wi : P->w_by_x[x]) {
      const auto& w = P->witems[wi];
      const int nch = (w.rows + XC - 1) / XC;
      tk += nch;
      sr += (int64_t)nch * (w.src_end - w.src_begin);
    }
    ntile[x + 1] = ntile[x] + tiles;
    ntask[x + 1] = ntask[x] + tiles * tk;
    nsrc[x + 1] = nsrc[x] + tiles * sr;
  }
  if (nsrc[nX] > std::numeric_limits<int>::max() || ntask[nX] > std::numeric_limits<int>::max())
    throw std::runtime_error("tensor-core tables exceed 2^31 entries");
  H.tiles.resize(ntile[nX]);
  H.t.resize(ntask[nX]);
  H.s.resize(nsrc[nX]);
  parallel_chunks(nX, 64, [&](size_t xb, size_t xe) {
    for (size_t x = xb; x < xe; ++x) {
      const XBlock& X = P->X[x];
      int64_t ti = ntile[x], tk = ntask[x], sr = nsrc[x];
      for (int row0 = 0; row0 < X.rows; row0 += RT)
        for (int col0 = 0; col0 < X.cols; col0 += 128) {
          TfTile T{P->yout + X.off + (int64_t)row0 * X.cols + col0, X.cols, std::min(RT, X.rows - row0),
                   std::min(128, X.cols - col0), (int)tk, 0, P->tc_ops_lo, P->tc_x_lo, 0, 1, 0, X.r, 0, 0};
          int kdl_max = 0, nkc_max = 0;
          for (int wi : P->w_by_x[x]) {
            const auto& w = P->witems[wi];
            const CombOp& C = P->cl[w.gl];
            const int64_t chi = C.identity ? P->tc_idmir.at(w.rows) : P->tc_cmir[w.gl][w.cbi];
            const int cg = nrg(X.rows);  // C has the output block's rows
            for (int kc = 0; kc < w.rows; kc += XC) {
              TfTask q{P->tc_ops + chi + ((int64_t)(kc / 32) * cg + row0 / 8) * 256, cg * 256,
                       std::min(XC, w.rows - kc), (int)sr, 0};
              for (int k = w.src_begin; k < w.src_end; ++k) {
                const auto& src = P->wsrc[k];
                const XBlock& Xs = P->X[src.xb];
                const int drows = src.zg >= 0 ? P->zg[src.zg].n : Xs.cols;
                const int64_t dhi = src.zg >= 0 ? P->tc_dmir[src.zg] : P->tc_idmir.at(Xs.cols);
                const int nkc = (Xs.cols + 31) / 32;
                H.s[sr++] = {P->tc_ops + dhi + (int64_t)(col0 / 8) * 256,
                             P->tc_x + P->tc_xoff[src.xb] + (int64_t)(kc / 8) * 256, nrg(drows) * 256,
                             nrg(Xs.rows) * 256, nkc, Xs.cols - 32 * (nkc - 1),
                             (float)(src.craw * P->cr[src.gr].scalar * C.scalar)};
                T.cost += nkc + (nkc + 1) / 2;
                nkc_max = std::max(nkc_max, nkc);
              }
              q.s_end = (int)sr;
              H.t[tk++] = q;
              T.cost += 2;
              T.kdg = std::max(T.kdg, (q.kdl + 7) / 8);
              kdl_max = std::max(kdl_max, q.kdl);
            }
          }
          T.t_end = (int)tk;
          T.tiny = T.m <= 4 && T.nv <= 4 && kdl_max <= 4 && nkc_max <= 1;
          H.tiles[ti++] = T;
        }
    }
  });
  H.yout = P->yout;
  H.n = P->n;
  P->tch_tune = tune;
}

Engine::TcView Engine::prepare_tc(int i, TcTune tune) {
  check_ready();
  if (!low_.empty()) throw std::invalid_argument("batched matvecs do not carry excited-state projectors");
  if (i < 0 || i > L_ - 2) throw std::out_of_range("site out of range");
  MatvecPlan* p = plan_for(i);
  try {
    if (!p->tc) build_tc(p);
    if (p->tch_tune.row_tile != tune.row_tile || p->tch_tune.x_chunk != tune.x_chunk) tc_tables(p, tune);
  } catch (...) {
    release_tc(p);
    throw;
  }
  return {&p->tch, p->serial, p->xin, p->yout, p->n, p->flops, p->diag};
}

double Engine::rayleigh_fp64(int i, const double* x) {
  check_ready();
  if (i < 0 || i > L_ - 2) throw std::out_of_range("site out of range");
  MatvecPlan* P = plan_for(i);
  if (x != P->xin) dev_d2d(P->xin, x, sizeof(double) * P->n, stream_);
  run_rq(P);
  double* d = (double*)dev_alloc(sizeof(double) * (2 + 1024), stream_);
  double h[2];
  try {
    vec_multidot(P->xin, P->n, 1, P->yout, P->n, d, d + 2, stream_);
    vec_multidot(P->xin, P->n, 1, P->xin, P->n, d + 1, d + 2, stream_);
    dev_d2h(h, d, sizeof(h), stream_);
    dev_sync(stream_);
  } catch (...) {
    dev_free(d, stream_);
    throw;
  }
  dev_free(d, stream_);
  if (!(h[1] > 0.0)) throw std::invalid_argument("zero vector");
  return h[0] / h[1];
}

uint64_t Engine::tc_serial(int i) const {
  return (cached_ && cached_site_ == i && cached_->tc) ? cached_->serial : 0;
}

void Engine::run_matvec(MatvecPlan* p, const double* x, double* y, bool tc) {
  if (tc) {
    flush_events();
    if (!ev_[0]) for (auto& e : ev_) e = event_create();
    if (!p->tc) {
      try {
        build_tc(p);
      } catch (...) {
        release_tc(p);  // a failed build keeps nothing
        throw;
      }
    }
    if (x != p->xin) dev_d2d(p->xin, x, sizeof(double) * p->n, stream_);
    tc_plan_launch(p->tc, ev_, stream_);
    ev_pending_ = true;
    ev_tc_ = true;
    add_projectors(p);
    if (y != p->yout) dev_d2d(y, p->yout, sizeof(double) * p->n, stream_);
    st_.tc_matvecs += 1;
    st_.tc_flops += p->flops;
    st_.tc_phase2_flops += p->flops;
    st_.tc_phase1_bytes += 16.0 * (double)p->n;
    st_.tc_phase2_bytes += p->tc_alg_bytes;
    st_.matvecs += 1;
    st_.matvec_flops += p->flops;
    st_.last_matvec_flops = p->flops;
    st_.last_matvec_tasks = p->ntasks;
    return;
  }
  if (x != p->xin) dev_d2d(p->xin, x, sizeof(double) * p->n, stream_);
  if (p->zsize) dev_zero(p->Z, sizeof(double) * p->zsize, stream_);
  dev_zero(p->yout, sizeof(double) * std::max<int64_t>(p->n, 1), stream_);
  flush_events();
  if (!ev_[0]) for (auto& e : ev_) e = event_create();
  event_record(ev_[0], stream_);
  gemm_plan_run(p->p1, stream_);
  comb_plan_run(p->pc, stream_);
  event_record(ev_[1], stream_);
  gemm_plan_run(p->p2, stream_);
  event_record(ev_[2], stream_);
  ev_pending_ = true;
  ev_tc_ = false;
  add_projectors(p);
  st_.k_launches += 1;
  st_.k_phase1_flops += p->flops1;
  st_.k_phase2_flops += p->flops2;
  if (y != p->yout) dev_d2d(y, p->yout, sizeof(double) * p->n, stream_);
  st_.matvecs += 1;
  st_.matvec_flops += p->flops;
  st_.last_matvec_flops = p->flops;
  st_.last_matvec_tasks = p->ntasks;
}

// The energy x^T H x / x^T x needs only half of the matvec: H_eff is symmetric, so with
// y_X' = sum_X H_X'X x_X blockwise, x^T H x = sum_X' [x_X'^T H_X'X' x_X' +
// 2 sum_{X > X'} x_X'^T H_X'X x_X].  The plan below keeps the sources whose input block
// X is >= the output block X' (those of X > X' with twice the coefficient), drops the W
// items left without sources, and restricts each phase-1 product to the runs of x blocks
// of the stack that a kept source reads; x^T y' then equals x^T H x up to rounding (y'
// itself is not H x).
void Engine::build_rq(MatvecPlan* P) {
  if (P->rqc) return;
  const size_t nw = P->witems.size();
  std::vector<int> wxp(nw, -1);
  for (int x = 0; x < (int)P->w_by_x.size(); ++x)
    for (int k : P->w_by_x[x]) wxp[k] = x;
  std::vector<int64_t> woff(nw + 1, 0);
  for (size_t k = 0; k < nw; ++k) woff[k + 1] = woff[k] + (int64_t)P->witems[k].rows * P->witems[k].cols;
  const size_t nz = P->zg.size();
  // rows of the x stack that each phase-1 product must produce: (first row, rows) of the
  // x blocks its kept sources read
  std::vector<std::vector<std::pair<int64_t, int64_t>>> need(nz);
  std::vector<CombSrc> cs;
  std::vector<CombDst> cd;
  std::vector<char> keep_w(nw, 0);
  for (size_t k = 0; k < nw; ++k) {
    const auto& w = P->witems[k];
    const int xp = wxp[k];
    const int b0 = (int)cs.size();
    for (int q = w.src_begin; q < w.src_end; ++q) {
      const auto& src = P->wsrc[q];
      if (src.xb < xp) continue;
      const XBlock& X = P->X[src.xb];
      const double c = src.xb > xp ? 2.0 * src.coef : src.coef;
      if (src.zg >= 0) {
        const auto& z = P->zg[src.zg];
        cs.push_back({P->Z + z.off + (int64_t)X.trow * z.n, z.n, c});
        need[src.zg].push_back({X.trow, X.rows});
      } else {
        const int sec = -1 - src.zg;  // identity right operator: x rows of the sector
        cs.push_back({P->xin + P->tall_off[sec] + (int64_t)X.trow * P->sec_dim[sec], P->sec_dim[sec], c});
      }
    }
    if ((int)cs.size() == b0) continue;
    keep_w[k] = 1;
    cd.push_back({P->W + woff[k], w.cols, w.rows, w.cols, b0, (int)cs.size(), 0});
  }
  std::vector<GemmTask> t1;
  std::vector<GemmGroup> g1;
  double f1 = 0.0, f2 = 0.0;
  for (size_t z = 0; z < nz; ++z) {
    auto& v = need[z];
    if (v.empty()) continue;
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    const auto& Zg = P->zg[z];
    // one product per run of consecutive needed x blocks
    for (size_t a = 0; a < v.size();) {
      const int64_t r0 = v[a].first;
      int64_t r1 = v[a].first + v[a].second;
      size_t b = a + 1;
      while (b < v.size() && v[b].first <= r1) {
        r1 = std::max(r1, v[b].first + v[b].second);
        ++b;
      }
      const int64_t rows = r1 - r0;
      t1.push_back({P->xin + P->tall_off[Zg.c] + r0 * Zg.K, Zg.D, Zg.K, Zg.K, Zg.K, 0, 1, Zg.alpha});
      g1.push_back({P->Z + Zg.off + r0 * Zg.n, Zg.n, (int)rows, Zg.n, (int)t1.size() - 1, (int)t1.size(), 0});
      f1 += 2.0 * rows * Zg.K * Zg.n;
      a = b;
    }
  }
  std::vector<GemmTask> t2;
  std::vector<GemmGroup> g2;
  for (int x = 0; x < (int)P->w_by_x.size(); ++x) {
    const int b0 = (int)t2.size();
    for (int k : P->w_by_x[x]) {
      if (!keep_w[k]) continue;
      const auto& w = P->witems[k];
      const CombOp& C = P->cl[w.gl];
      const BlockRef& cb = (*C.blocks)[w.cbi];
      if (C.identity) {
        t2.push_back({nullptr, P->W + woff[k], 0, w.cols, w.rows, 0, 0, C.scalar});
      } else {
        t2.push_back({C.data + cb.off, P->W + woff[k], cb.cols, w.cols, cb.cols, 0, 0, C.scalar});
        f2 += 2.0 * cb.rows * cb.cols * w.cols;
      }
    }
    if ((int)t2.size() > b0) {
      const XBlock& X = P->X[x];
      g2.push_back({P->yout + X.off, X.cols, X.rows, X.cols, b0, (int)t2.size(), 0});
    }
  }
  try {
    P->rq1 = gemm_plan_upload(t1, g1, stream_);
    P->rqc = comb_plan_upload(cs, cd, stream_);
    P->rq2 = gemm_plan_upload(t2, g2, stream_);
  } catch (...) {
    gemm_plan_free(P->rq1, stream_);
    comb_plan_free(P->rqc, stream_);
    gemm_plan_free(P->rq2, stream_);
    P->rq1 = P->rq2 = nullptr;
    P->rqc = nullptr;
    throw;
  }
  P->rq_flops1 = f1;
  P->rq_flops2 = f2;
}

// y' of build_rq for the plan's input x (P->xin), into P->yout, on the engine's current
// stream, with the excited-state projectors added as in a matvec
void Engine::run_rq(MatvecPlan* P) {
  build_rq(P);
  if (P->zsize) dev_zero(P->Z, sizeof(double) * P->zsize, stream_);
  dev_zero(P->yout, sizeof(double) * std::max<int64_t>(P->n, 1), stream_);
  flush_events();
  if (!ev_[0]) for (auto& e : ev_) e = event_create();
  event_record(ev_[0], stream_);
  gemm_plan_run(P->rq1, stream_);
  comb_plan_run(P->rqc, stream_);
  event_record(ev_[1], stream_);
  gemm_plan_run(P->rq2, stream_);
  event_record(ev_[2], stream_);
  ev_pending_ = true;
  ev_tc_ = false;
  add_projectors(P);
  st_.k_launches += 1;
  st_.k_phase1_flops += P->rq_flops1;
  st_.k_phase2_flops += P->rq_flops2;
  st_.matvec_flops += P->rq_flops1 + P->rq_flops2;
}

void Engine::matvec(int i, const double* x, double* y) {
  check_ready();
  if (i < 0 || i > L_ - 2) throw std::out_of_range("site out of range");
  MatvecPlan* p = plan_for(i);
  run_matvec(p, x, y, precision_ == 1);
  if (precision_ == 1 && tc_error_flag(stream_)) throw std::runtime_error("cuda: tensor-core wait timed out");
}

// y += sum_k eta_k v_k (v_k . x): the projectors of the excited-state Hamiltonian
void Engine::add_projectors(MatvecPlan* p) {
  if (!p->nlow) return;
  vec_multidot(p->lowv, p->n, p->nlow, p->xin, p->n, p->lowc, p->lowc + p->nlow, stream_);
  vec_combine(p->loww, p->n, p->nlow, p->lowc, 1.0, p->yout, p->n, stream_);
}

void Engine::matvec_noalloc(int i, const double* x, double* y, Stream s) {
  if (!low_.empty())
    throw std::invalid_argument("the allocation-free matvec does not carry excited-state projectors");
  if (!cached_ || cached_site_ != i)
    throw std::invalid_argument(
        "no prepared matvec for this site: call dmrg_heff_matvec (or dmrg_davidson) at this site "
        "first, outside the region where allocation is not allowed");
  MatvecPlan* p = cached_;
  noalloc_matvec_run(p->p1, p->pc, p->p2, p->xin, p->yout, p->n, p->Z, p->zsize, p->W, p->wsize,
                     x, y, s);
}

void Engine::diag(int i, double* d) {
  check_ready();
  if (i < 0 || i > L_ - 2) throw std::out_of_range("site out of range");
  MatvecPlan* p = plan_for(i);
  dev_d2d(d, p->diag, sizeof(double) * p->n, stream_);
}

// Eq. 25 followed by x = sqrt(2jR+1) S.
void Engine::tt_to_x(int i, double* x) {
  check_ready();
  if (i < 0 || i > L_ - 2) throw std::out_of_range("site out of range");
  tt_to_x_of(bonds_, sites_, i, x);
}

void Engine::tt_to_x_of(const std::vector<Bond>& bonds, const std::vector<Site>& sites, int i, double* x) {
  int64_t n;
  auto X = x_layout_of(bonds, i, &n);
  const Bond& bl = bonds[i];
  const Bond& bm = bonds[i + 1];
  const Bond& br = bonds[i + 2];
  const Site& A = sites[i];
  const Site& B = sites[i + 1];
  std::map<std::tuple<int, int, int>, int> ia, ib;  // (ls, l, r) -> block
  for (int t = 0; t < (int)A.blocks.size(); ++t) ia[{A.blocks[t].ls, A.blocks[t].l, A.blocks[t].r}] = t;
  for (int t = 0; t < (int)B.blocks.size(); ++t) ib[{B.blocks[t].ls, B.blocks[t].l, B.blocks[t].r}] = t;
  // the blocks of A by (ls, l), middle sectors m in increasing order: (m, block)
  std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> a_by;
  for (const auto& kv : ia) a_by[{std::get<0>(kv.first), std::get<1>(kv.first)}].push_back({std::get<2>(kv.first), kv.second});
  std::vector<GemmTask> tasks;
  std::vector<GemmGroup> groups;
  for (auto& xb : X) {
    const int tjL = bl.sec[xb.l].tj, tjR = br.sec[xb.r].tj;
    const int t1 = local_ts(xb.ls1), t2 = local_ts(xb.ls2);
    const int ph = (((tjL + tjR + t1 + t2) / 2) & 1) ? -1 : 1;
    int b0 = (int)tasks.size();
    auto la = a_by.find({xb.ls1, xb.l});
    const size_t na = la == a_by.end() ? 0 : la->second.size();
    for (size_t q = 0; q < na; ++q) {
      const int m = la->second[q].first;
      auto b = ib.find({xb.ls2, m, xb.r});
      if (b == ib.end()) continue;
      const int tjM = bm.sec[m].tj;
      double c = std::sqrt((double)(tjR + 1)) * std::sqrt((double)(xb.tj + 1)) * ph *
                 std::sqrt((double)(tjM + 1)) * wigner6j(tjL, tjR, xb.tj, t2, t1, tjM);
      if (c == 0.0) continue;
      const SiteBlock& sa = A.blocks[la->second[q].second];
      const SiteBlock& sb = B.blocks[b->second];
      tasks.push_back({A.data + sa.off, B.data + sb.off, sa.cols, sb.cols, sa.cols, 0, 0, c});
    }
    if ((int)tasks.size() > b0) groups.push_back({x + xb.off, xb.cols, xb.rows, xb.cols, b0, (int)tasks.size(), 0});
  }
  dev_zero(x, sizeof(double) * std::max<int64_t>(n, 1), stream_);
  GemmPlan* p = gemm_plan_upload(tasks, groups, stream_);
  gemm_plan_run(p, stream_);
  gemm_plan_free(p, stream_);
}

// Davidson's algorithm (lowest eigenpair of H_eff, Eq. 9) entirely on the device in
// FP64: subspace up to 32 vectors, restart on the 3 lowest Ritz vectors, diagonal
// preconditioner, two classical Gram-Schmidt passes, convergence on ||r||_2.
double Engine::davidson(int i, double* x, int* iters, bool* converged) {
  return davidson_ex(i, x, iters, converged, false);
}

double Engine::davidson_ex(int i, double* x, int* iters, bool* converged, bool defer) {
  check_ready();
  MatvecPlan* P = plan_for(i);
  if (precision_ != 1) return davidson_core(P, x, dav_tol_, dav_max_, false, iters, converged);
  // mixed precision: Davidson on the tensor-core matvec down to its accuracy, then FP64
  // Davidson iterations from that vector (the residual and Rayleigh quotient in FP64)
  int it1 = 0, it2 = 0;
  bool c1 = false, c2 = false;
  davidson_core(P, x, std::max(dav_tol_, 1e-6), dav_max_, true, &it1, &c1);
  if (tc_error_flag(stream_)) throw std::runtime_error("cuda: tensor-core wait timed out");
  if (defer && refine_iters_ == 1) {
    start_rq(P, x);
    *iters = it1 + 1;
    *converged = false;
    return std::numeric_limits<double>::quiet_NaN();
  }
  double e = davidson_core(P, x, dav_tol_, refine_iters_ > 0 ? refine_iters_ : dav_max_, false, &it2, &c2);
  *iters = it1 + it2;
  *converged = c2;
  return e;
}

// E = x.Hx / x.x with the FP64 matvec on the side stream: x is copied into the plan's
// input on the engine's stream first (so later changes of x do not race), the side
// stream waits for that copy, and the engine's stream waits for the side stream in
// finish_rq before anything the side stream reads can be released.
void Engine::start_rq(MatvecPlan* P, const double* x) {
  if (!side_) {
    side_ = stream_create();
    ev_side_[0] = event_create();
    ev_side_[1] = event_create();
    rq_dev_ = (double*)dev_alloc(sizeof(double) * (2 + 2 * 512), stream_);
  }
  dev_d2d(P->xin, x, sizeof(double) * P->n, stream_);
  event_record(ev_side_[0], stream_);
  rq_plan_ = P;
  rq_pending_ = true;
}

// queue the side stream's FP64 matvec and dot products of the copy start_rq made
void Engine::launch_rq() {
  if (!rq_pending_ || !rq_plan_) return;
  MatvecPlan* P = rq_plan_;
  rq_plan_ = nullptr;
  stream_wait(side_, ev_side_[0]);
  Stream keep = stream_;
  stream_ = side_;
  try {
    run_rq(P);
    vec_multidot(P->xin, P->n, 1, P->yout, P->n, rq_dev_, rq_dev_ + 2, side_);
    vec_multidot(P->xin, P->n, 1, P->xin, P->n, rq_dev_ + 1, rq_dev_ + 2 + 512, side_);
    event_record(ev_side_[1], side_);
  } catch (...) {
    stream_ = keep;
    rq_pending_ = false;
    throw;
  }
  stream_ = keep;
}

double Engine::finish_rq() {
  if (!rq_pending_) return std::numeric_limits<double>::quiet_NaN();
  launch_rq();
  rq_pending_ = false;
  stream_wait(stream_, ev_side_[1]);
  double h[2];
  dev_d2h(h, rq_dev_, sizeof(h), side_);
  dev_sync(side_);
  if (!(h[1] > 0.0)) throw std::runtime_error("Ritz vector has zero norm");
  return h[0] / h[1];
}

double Engine::davidson_core(MatvecPlan* P, double* x, double tol, int maxit, bool tc, int* iters,
                             bool* converged) {
  const int64_t n = P->n;
  const int mmax = std::min<int64_t>(32, std::max<int64_t>(n, 1));
  const int nkeep = std::min(3, mmax - 1 > 0 ? mmax - 1 : 1);
  double *V = nullptr, *AV = nullptr, *G = nullptr, *C = nullptr, *th = nullptr, *sc = nullptr;
  double *dots = nullptr, *r = nullptr, *t = nullptr, *tmp = nullptr, *x0 = nullptr, *hs = nullptr;
  double theta = 0.0;
  bool conv = false;
  int it = 0;
  std::vector<double> rhist;  // residual norms (tensor-core stage)
  auto cleanup = [&]() {
    dev_free(V, stream_); dev_free(AV, stream_); dev_free(G, stream_); dev_free(C, stream_);
    dev_free(th, stream_); dev_free(sc, stream_); dev_free(dots, stream_); dev_free(r, stream_);
    dev_free(t, stream_); dev_free(tmp, stream_); dev_free(x0, stream_);
    host_pinned_free(hs);
  };
  try {
  V = (double*)dev_alloc(sizeof(double) * n * (mmax + 1), stream_);
  AV = (double*)dev_alloc(sizeof(double) * n * (mmax + 1), stream_);
  G = (double*)dev_alloc(sizeof(double) * mmax * mmax, stream_);
  C = (double*)dev_alloc(sizeof(double) * mmax * mmax, stream_);
  th = (double*)dev_alloc(sizeof(double) * mmax, stream_);
  sc = (double*)dev_alloc(sizeof(double) * mmax * 520, stream_);
  dots = (double*)dev_alloc(sizeof(double) * (mmax + 2), stream_);
  r = (double*)dev_alloc(sizeof(double) * n, stream_);
  t = (double*)dev_alloc(sizeof(double) * n, stream_);
  tmp = (double*)dev_alloc(sizeof(double) * n * nkeep * 2, stream_);
  x0 = (double*)dev_alloc(sizeof(double) * n, stream_);  // the starting vector
  dev_zero(G, sizeof(double) * mmax * mmax, stream_);
  hs = (double*)host_pinned_alloc(sizeof(double) * 4);
  dev_d2d(x0, x, sizeof(double) * n, stream_);
  // v0 = x / |x|
  dev_d2d(V, x, sizeof(double) * n, stream_);
  vec_multidot(V, n, 1, V, n, dots, sc, stream_);
  vec_normalize(V, dots, n, stream_);
  run_matvec(P, V, AV, tc);
  vec_multidot(V, n, 1, AV, n, G, sc, stream_);
  int m = 1;
  for (; it < maxit; ++it) {
    small_eig(G, mmax, m, std::min(m, nkeep), th, C, stream_);
    // u = V c0 -> x ; r = AV c0 - theta u
    vec_combine(V, n, m, C, 0.0, x, n, stream_);
    vec_combine(AV, n, m, C, 0.0, r, n, stream_);
    dev_d2h(hs, th, sizeof(double), stream_);
    dev_sync(stream_);
    theta = hs[0];
    vec_axpby(-theta, x, 1.0, r, n, stream_);
    vec_multidot(r, n, 1, r, n, dots, sc, stream_);
    dev_d2h(hs + 1, dots, sizeof(double), stream_);
    dev_sync(stream_);
    st_.davidson_iters += 1;
    const double rn = std::sqrt(std::max(hs[1], 0.0));
    if (rn <= tol) { conv = true; break; }
    if (m >= n) { conv = true; break; }
    if (tc) {
      // The split-TF32 products bound how far the residual can fall (their bias is about
      // 1e-7 of |theta| and grows with the problem): once it is within 1e-4 |theta| and
      // has fallen by less than 20 % over eight iterations, the tensor-core stage stops
      // and the FP64 iterations take over.
      rhist.push_back(rn);
      const size_t k = rhist.size();
      if (k > 8 && rn <= 1e-4 * std::fabs(theta) && rn > 0.8 * rhist[k - 9]) break;
    }
    if (it + 1 >= maxit) break;  // no use expanding the subspace on the last iteration
    vec_precondition(r, P->diag, th, t, n, stream_);
    for (int pass = 0; pass < 2; ++pass) {
      // t -= V (V^T t)
      vec_multidot(V, n, m, t, n, dots, sc, stream_);
      vec_combine(V, n, m, dots, 0.0, tmp, n, stream_);
      vec_axpby(-1.0, tmp, 1.0, t, n, stream_);
    }
    vec_multidot(t, n, 1, t, n, dots, sc, stream_);
    dev_d2h(hs + 2, dots, sizeof(double), stream_);
    dev_sync(stream_);
    if (!(hs[2] > 1e-28)) {
      // preconditioned direction collapsed: fall back to the residual
      dev_d2d(t, r, sizeof(double) * n, stream_);
      for (int pass = 0; pass < 2; ++pass) {
        vec_multidot(V, n, m, t, n, dots, sc, stream_);
        vec_combine(V, n, m, dots, 0.0, tmp, n, stream_);
        vec_axpby(-1.0, tmp, 1.0, t, n, stream_);
      }
      vec_multidot(t, n, 1, t, n, dots, sc, stream_);
      dev_d2h(hs + 2, dots, sizeof(double), stream_);
      dev_sync(stream_);
      if (!(hs[2] > 1e-30)) { conv = true; break; }
    }
    vec_normalize(t, dots, n, stream_);
    if (m == mmax) {
      // restart on the nkeep lowest Ritz vectors
      for (int v = 0; v < nkeep; ++v) {
        vec_combine(V, n, m, C + (size_t)v * m, 0.0, tmp + (size_t)v * n, n, stream_);
        vec_combine(AV, n, m, C + (size_t)v * m, 0.0, tmp + (size_t)(nkeep + v) * n, n, stream_);
      }
      for (int v = 0; v < nkeep; ++v) {
        dev_d2d(V + (size_t)v * n, tmp + (size_t)v * n, sizeof(double) * n, stream_);
        dev_d2d(AV + (size_t)v * n, tmp + (size_t)(nkeep + v) * n, sizeof(double) * n, stream_);
      }
      std::vector<double> hth(nkeep);
      dev_d2h(hth.data(), th, sizeof(double) * nkeep, stream_);
      dev_sync(stream_);
      std::vector<double> Gh((size_t)mmax * mmax, 0.0);
      for (int v = 0; v < nkeep; ++v) Gh[(size_t)v * mmax + v] = hth[v];
      dev_h2d(G, Gh.data(), sizeof(double) * Gh.size(), stream_);
      m = nkeep;
    }
    dev_d2d(V + (size_t)m * n, t, sizeof(double) * n, stream_);
    run_matvec(P, V + (size_t)m * n, AV + (size_t)m * n, tc);
    // row m of the Rayleigh matrix (lower triangle is what small_eig reads)
    vec_multidot(V, n, m + 1, AV + (size_t)m * n, n, G + (size_t)m * mmax, sc, stream_);
    ++m;
  }
  // sign of the eigenvector: non-negative overlap with the starting vector, so that
  // what is added to it afterwards (the noise of Sec. 4.2) does not depend on the
  // arbitrary sign of the small eigensolver
  vec_multidot(x, n, 1, x0, n, dots, sc, stream_);
  dev_d2h(hs + 3, dots, sizeof(double), stream_);
  dev_sync(stream_);
  if (hs[3] < 0.0) vec_axpby(0.0, x0, -1.0, x, n, stream_);
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
  *iters = it + 1;
  *converged = conv;
  return theta;
}

}  // namespace dmrg

namespace dmrg {

// Eqs. 26-28: back-transform x into TT per middle sector (jM, NM, IM), weight the
// columns by sqrt((2jR+1)/(2jM+1)) (which makes the bracket of Eq. 27 right-normalised),
// keep the D largest lambda over all sectors (D counts reduced multiplets), normalise
// with kappa = lambda / sqrt(sum (2jM+1) lambda^2), and write T[i], T[i+1] for the sweep
// direction (dir > 0: A[i] = U, A[i+1] = kappa V; dir < 0: A[i] = U kappa, A[i+1] = V).
// The factor that must be normalised comes from the eigenvectors of the Gram matrix on
// its side (M M^T for U, M^T M for V); the other factor is the projection of M onto
// them (kappa V = U^T M / |M|, U kappa = M V^T / |M|), with no division by lambda.
// Returns the discarded weight sum over dropped (2jM+1) kappa^2 (Eq. 15).
double Engine::truncate(int i, int dir, int D, const double* x, double /*unused*/) {
  check_ready();
  if (i < 0 || i > L_ - 2) throw std::out_of_range("site out of range");
  Timer tm;
  int64_t nx;
  auto X = x_layout(i, &nx);
  const Bond bl = bonds_[i];
  const Bond br = bonds_[i + 2];
  if ((int)fci_.size() != L_ + 1) fci_ = sym_.fci_dims();
  const auto& fci_cache = fci_;
  const int I1 = sym_.orb_ir[i], I2 = sym_.orb_ir[i + 1];
  std::vector<Sector> cands;
  for (int l = 0; l < (int)bl.sec.size(); ++l)
    for (int ls1 = 0; ls1 < 3; ++ls1) {
      const Sector& a = bl.sec[l];
      int t1 = local_ts(ls1);
      for (int tjM = std::abs(a.tj - t1); tjM <= a.tj + t1; tjM += 2) {
        Sector s{tjM, a.n + local_n(ls1), a.ir ^ local_ir(ls1, I1)};
        if (fci_cache[i + 1].count(s)) cands.push_back(s);
      }
    }
  std::sort(cands.begin(), cands.end());
  cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
  struct Grp {
    Sector s;
    std::vector<std::pair<int, int>> rows, cols;  // (l, ls1), (r, ls2)
    std::vector<int> roff, coff;
    int R = 0, C = 0, n = 0;
    int64_t moff = 0, goff = 0, woff = 0, aoff = 0;
  };
  std::vector<Grp> gs;
  for (auto& s : cands) {
    Grp g;
    g.s = s;
    for (int l = 0; l < (int)bl.sec.size(); ++l)
      for (int ls1 = 0; ls1 < 3; ++ls1) {
        const Sector& a = bl.sec[l];
        if (a.n + local_n(ls1) == s.n && (a.ir ^ local_ir(ls1, I1)) == s.ir && triangle(a.tj, local_ts(ls1), s.tj)) {
          g.rows.push_back({l, ls1});
          g.roff.push_back(g.R);
          g.R += bl.dim[l];
        }
      }
    for (int r = 0; r < (int)br.sec.size(); ++r)
      for (int ls2 = 0; ls2 < 3; ++ls2) {
        const Sector& b = br.sec[r];
        if (s.n + local_n(ls2) == b.n && (s.ir ^ local_ir(ls2, I2)) == b.ir && triangle(s.tj, local_ts(ls2), b.tj)) {
          g.cols.push_back({r, ls2});
          g.coff.push_back(g.C);
          g.C += br.dim[r];
        }
      }
    if (g.R == 0 || g.C == 0) continue;
    g.n = dir > 0 ? g.R : g.C;
    gs.push_back(g);
  }
  int64_t msz = 0, gsz = 0, wsz = 0, asz = 0;
  for (auto& g : gs) {
    g.moff = msz; msz += (int64_t)g.R * g.C;
    g.goff = gsz; gsz += (int64_t)g.n * g.n;
    g.woff = wsz; wsz += g.n;
    g.aoff = asz; asz += (int64_t)g.R * g.C;  // room for U (R x r) or V (r x C)
  }
  double* M = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(msz, 1), stream_);
  double* Gm = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(gsz, 1), stream_);
  double* Q = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(gsz, 1), stream_);
  double* W = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(wsz, 1), stream_);
  double* Aux = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(asz, 1), stream_);
  dev_zero(M, sizeof(double) * std::max<int64_t>(msz, 1), stream_);
  dev_zero(Gm, sizeof(double) * std::max<int64_t>(gsz, 1), stream_);
  dev_zero(Aux, sizeof(double) * std::max<int64_t>(asz, 1), stream_);
  // M blocks: sum_j (-1)^(jL+jR+s1+s2) {jL jR j; s2 s1 jM} sqrt(2j+1) x_(l s1 s2 j r)
  std::map<Sector, int> gidx;
  for (int g = 0; g < (int)gs.size(); ++g) gidx[gs[g].s] = g;
  std::map<std::tuple<int, int, int>, std::vector<CombSrc>> dsts;  // (g, row blk, col blk)
  for (auto& xb : X) {
    const Sector& a = bl.sec[xb.l];
    const Sector& b = br.sec[xb.r];
    const int t1 = local_ts(xb.ls1), t2 = local_ts(xb.ls2);
    const int ph = (((a.tj + b.tj + t1 + t2) / 2) & 1) ? -1 : 1;
    for (int tjM = std::abs(a.tj - t1); tjM <= a.tj + t1; tjM += 2) {
      auto it = gidx.find({tjM, a.n + local_n(xb.ls1), a.ir ^ local_ir(xb.ls1, I1)});
      if (it == gidx.end()) continue;
      double c = ph * wigner6j(a.tj, b.tj, xb.tj, t2, t1, tjM) * std::sqrt((double)(xb.tj + 1));
      if (c == 0.0) continue;
      const Grp& g = gs[it->second];
      int rb = -1, cb = -1;
      for (int q = 0; q < (int)g.rows.size(); ++q) if (g.rows[q] == std::make_pair(xb.l, xb.ls1)) rb = q;
      for (int q = 0; q < (int)g.cols.size(); ++q) if (g.cols[q] == std::make_pair(xb.r, xb.ls2)) cb = q;
      if (rb < 0 || cb < 0) continue;
      dsts[{it->second, rb, cb}].push_back({x + xb.off, xb.cols, c});
    }
  }
  {
    std::vector<CombSrc> cs;
    std::vector<CombDst> cd;
    for (auto& kv : dsts) {
      const Grp& g = gs[std::get<0>(kv.first)];
      int rb = std::get<1>(kv.first), cb = std::get<2>(kv.first);
      CombDst d{M + g.moff + (int64_t)g.roff[rb] * g.C + g.coff[cb], g.C,
                bl.dim[g.rows[rb].first], br.dim[g.cols[cb].first], (int)cs.size(), 0, 0};
      cs.insert(cs.end(), kv.second.begin(), kv.second.end());
      d.src_end = (int)cs.size();
      cd.push_back(d);
    }
    CombPlan* p = comb_plan_upload(cs, cd, stream_);
    comb_plan_run(p, stream_);
    comb_plan_free(p, stream_);
  }
  // Gram matrices of the smaller side
  {
    std::vector<GemmTask> t;
    std::vector<GemmGroup> gg;
    for (auto& g : gs) {
      if (dir > 0) t.push_back({M + g.moff, M + g.moff, g.C, g.C, g.C, 0, 1, 1.0});
      else t.push_back({M + g.moff, M + g.moff, g.C, g.C, g.R, 1, 0, 1.0});
      gg.push_back({Gm + g.goff, g.n, g.n, g.n, (int)t.size() - 1, (int)t.size(), 0});
    }
    GemmPlan* p = gemm_plan_upload(t, gg, stream_);
    gemm_plan_run(p, stream_);
    gemm_plan_free(p, stream_);
  }
  std::vector<EigJob> jobs;
  for (auto& g : gs) jobs.push_back({Gm + g.goff, Q + g.goff, W + g.woff, g.n});
  eig_batched(jobs, stream_);
  std::vector<int> goff(1, 0), wgt;
  for (auto& g : gs) { goff.push_back(goff.back() + g.n); wgt.push_back(g.s.tj + 1); }
  std::vector<int> kept;
  double norm2 = 0.0, disc = 0.0;
  // eigenvalues of the Gram matrix are lambda^2 with an error ~ eps lambda_max^2: values
  // with lambda below 3e-8 lambda_max are at that noise level and are treated as zero
  select_largest(W, goff, wgt, D, 3e-8, kept, &norm2, &disc, stream_);
  if (!(norm2 > 0.0)) throw std::runtime_error("two-site vector has zero norm");
  const double w_disc = disc / norm2;
  // the other factor: Q_r^T M (right move) or M Q_r (left move)
  {
    std::vector<GemmTask> t;
    std::vector<GemmGroup> gg;
    for (int q = 0; q < (int)gs.size(); ++q) {
      const Grp& g = gs[q];
      int r = kept[q];
      if (r == 0) continue;
      if (dir > 0) {
        t.push_back({Q + g.goff, M + g.moff, g.n, g.C, g.R, 1, 0, 1.0});
        gg.push_back({Aux + g.aoff, g.C, r, g.C, (int)t.size() - 1, (int)t.size(), 0});
      } else {
        t.push_back({M + g.moff, Q + g.goff, g.C, g.n, g.C, 0, 0, 1.0});
        gg.push_back({Aux + g.aoff, r, g.R, r, (int)t.size() - 1, (int)t.size(), 0});
      }
    }
    GemmPlan* p = gemm_plan_upload(t, gg, stream_);
    gemm_plan_run(p, stream_);
    gemm_plan_free(p, stream_);
  }
  // new middle bond and tensors
  Bond nb;
  std::vector<int> gnew(gs.size(), -1);
  for (int q = 0; q < (int)gs.size(); ++q)
    if (kept[q] > 0) { gnew[q] = (int)nb.sec.size(); nb.sec.push_back(gs[q].s); nb.dim.push_back(kept[q]); }
  if (nb.sec.empty()) throw std::runtime_error("truncation kept no states");
  bonds_[i + 1] = nb;
  for (int b = i + 1; b <= L_; ++b) free_env(lenv_[b]);
  for (int b = 0; b <= i + 1; ++b) free_env(renv_[b]);
  if (cached_) { free_plan(cached_); cached_ = nullptr; cached_site_ = -1; }
  alloc_site(i);
  alloc_site(i + 1);
  const double inv = 1.0 / std::sqrt(norm2);
  std::vector<ScatterJob> sj;
  std::map<std::tuple<int, int, int>, const SiteBlock*> ia, ib;
  for (auto& b : sites_[i].blocks) ia[{b.ls, b.l, b.r}] = &b;
  for (auto& b : sites_[i + 1].blocks) ib[{b.ls, b.l, b.r}] = &b;
  for (int q = 0; q < (int)gs.size(); ++q) {
    const Grp& g = gs[q];
    const int r = kept[q];
    if (r == 0) continue;
    const int m = gnew[q];
    for (int rb = 0; rb < (int)g.rows.size(); ++rb) {
      const SiteBlock* sb = ia.at({g.rows[rb].second, g.rows[rb].first, m});
      double* dst = sites_[i].data + sb->off;
      if (dir > 0) {  // A[i] = U = Q_r (rows of the row block)
        const double* src = Q + g.goff + (int64_t)g.roff[rb] * g.n;
        sj.push_back({dst, src, nullptr, nullptr, r, g.n, sb->rows, r, 0, 0, 0, 1.0});
      } else {        // A[i] = U kappa = M Q_r / |M|
        const double* src = Aux + g.aoff + (int64_t)g.roff[rb] * r;
        sj.push_back({dst, src, nullptr, nullptr, r, r, sb->rows, r, 0, 0, 0, inv});
      }
    }
    for (int cb = 0; cb < (int)g.cols.size(); ++cb) {
      const SiteBlock* sb = ib.at({g.cols[cb].second, m, g.cols[cb].first});
      double* dst = sites_[i + 1].data + sb->off;
      const double f = std::sqrt((double)(g.s.tj + 1) / (double)(br.sec[g.cols[cb].first].tj + 1));
      const int dR = sb->cols;
      if (dir > 0) {  // A[i+1] = kappa V (bracket of Eq. 27) = Q_r^T M / |M|
        const double* src = Aux + g.aoff + g.coff[cb];
        sj.push_back({dst, src, nullptr, nullptr, dR, g.C, r, dR, 0, 0, 0, f * inv});
      } else {        // A[i+1] = V = Q_r^T
        const double* src = Q + g.goff + (int64_t)g.coff[cb] * g.n;
        sj.push_back({dst, src, nullptr, nullptr, dR, g.n, r, dR, 0, 0, 1, f});
      }
    }
  }
  scatter_batched(sj, stream_);
  dev_free(M, stream_);
  dev_free(Gm, stream_);
  dev_free(Q, stream_);
  dev_free(W, stream_);
  dev_free(Aux, stream_);
  st_.last_w_disc = w_disc;
  st_.max_w_disc = std::max(st_.max_w_disc, w_disc);
  st_.t_trunc_ms += tm.ms();
  return w_disc;
}

// Right-normalise site k (reduced Eq. 6) and push the remaining factor into site k-1:
// per left sector, G = sum (2jR+1)/(2jL+1) T T^T = Q lambda Q^T, T <- lambda^-1/2 Q^T T,
// T[k-1] <- T[k-1] Q lambda^1/2.  Directions with lambda below 1e-14 lambda_max of their
// sector (numerically absent from the state) are dropped from the bond.  One pass leaves
// an orthonormality error ~ eps lambda_max / lambda_min; callers run a second pass on
// the then well-conditioned tensor (as in Cholesky-QR2).
void Engine::right_normalize_site(int k) {
  Site& S = sites_[k];
  const Bond bl = bonds_[k];
  const Bond& br = bonds_[k + 1];
  const int nl = (int)bl.sec.size();
  std::vector<int64_t> goff(nl + 1, 0), woff(nl + 1, 0);
  for (int l = 0; l < nl; ++l) {
    goff[l + 1] = goff[l] + (int64_t)bl.dim[l] * bl.dim[l];
    woff[l + 1] = woff[l] + bl.dim[l];
  }
  double* G = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(goff[nl], 1), stream_);
  double* Q = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(goff[nl], 1), stream_);
  double* W = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(woff[nl], 1), stream_);
  dev_zero(G, sizeof(double) * std::max<int64_t>(goff[nl], 1), stream_);
  {
    std::vector<GemmTask> t;
    std::vector<GemmGroup> g;
    for (int l = 0; l < nl; ++l) {
      int b0 = (int)t.size();
      for (auto& b : S.blocks)
        if (b.l == l)
          t.push_back({S.data + b.off, S.data + b.off, b.cols, b.cols, b.cols, 0, 1,
                       (double)(br.sec[b.r].tj + 1) / (double)(bl.sec[l].tj + 1)});
      if ((int)t.size() > b0) g.push_back({G + goff[l], bl.dim[l], bl.dim[l], bl.dim[l], b0, (int)t.size(), 0});
    }
    GemmPlan* p = gemm_plan_upload(t, g, stream_);
    gemm_plan_run(p, stream_);
    gemm_plan_free(p, stream_);
  }
  std::vector<EigJob> jobs;
  for (int l = 0; l < nl; ++l) jobs.push_back({G + goff[l], Q + goff[l], W + woff[l], bl.dim[l]});
  eig_batched(jobs, stream_);
  std::vector<double> w(woff[nl]);
  dev_d2h(w.data(), W, sizeof(double) * w.size(), stream_);
  dev_sync(stream_);
  Bond nb;
  std::vector<int> keep(nl, 0);
  for (int l = 0; l < nl; ++l) {
    const double wmax = bl.dim[l] > 0 ? w[woff[l]] : 0.0;
    for (int a = 0; a < bl.dim[l]; ++a)
      if (w[woff[l] + a] > 1e-14 * wmax && wmax > 0.0) ++keep[l];
    if (keep[l] > 0) { nb.sec.push_back(bl.sec[l]); nb.dim.push_back(keep[l]); }
  }
  // new tensors: site k rows Q_r^T T scaled by lambda^-1/2; site k-1 columns T Q_r lambda^1/2
  Site oldk = S;
  Site oldm = sites_[k - 1];
  sites_[k].data = nullptr;
  sites_[k - 1].data = nullptr;
  bonds_[k] = nb;
  alloc_site(k - 1);
  alloc_site(k);
  std::vector<GemmTask> t;
  std::vector<GemmGroup> g;
  std::vector<double> scl(woff[nl], 0.0);
  for (int l = 0; l < nl; ++l)
    for (int a = 0; a < keep[l]; ++a) scl[woff[l] + a] = w[woff[l] + a];
  for (auto& b : oldk.blocks) {
    const int l = b.l;
    if (keep[l] == 0) continue;
    const int nlid = nb.find(bl.sec[l]);
    for (auto& nbk : sites_[k].blocks)
      if (nbk.ls == b.ls && nbk.l == nlid && nbk.r == b.r) {
        // new block (keep x dR) = Q_r^T (keep x dL) . T (dL x dR); rows scaled afterwards
        t.push_back({Q + goff[l], oldk.data + b.off, bl.dim[l], b.cols, bl.dim[l], 1, 0, 1.0});
        g.push_back({sites_[k].data + nbk.off, nbk.cols, keep[l], nbk.cols, (int)t.size() - 1, (int)t.size(), 0});
      }
  }
  for (auto& b : oldm.blocks) {
    const int l = b.r;  // right sector of site k-1 is the left sector of site k
    if (keep[l] == 0) continue;
    const int nlid = nb.find(bl.sec[l]);
    for (auto& nbk : sites_[k - 1].blocks)
      if (nbk.ls == b.ls && nbk.l == b.l && nbk.r == nlid) {
        t.push_back({oldm.data + b.off, Q + goff[l], b.cols, bl.dim[l], b.cols, 0, 0, 1.0});
        g.push_back({sites_[k - 1].data + nbk.off, nbk.cols, nbk.rows, keep[l], (int)t.size() - 1, (int)t.size(), 0});
      }
  }
  GemmPlan* p = gemm_plan_upload(t, g, stream_);
  gemm_plan_run(p, stream_);
  gemm_plan_free(p, stream_);
  std::vector<ScatterJob> sj;
  for (auto& nbk : sites_[k].blocks) {
    const int l = bl.find(nb.sec[nbk.l]);
    sj.push_back({sites_[k].data + nbk.off, sites_[k].data + nbk.off, W + woff[l], nullptr,
                  nbk.cols, nbk.cols, nbk.rows, nbk.cols, 2, 0, 0, 1.0});
  }
  for (auto& nbk : sites_[k - 1].blocks) {
    const int l = bl.find(nb.sec[nbk.r]);
    sj.push_back({sites_[k - 1].data + nbk.off, sites_[k - 1].data + nbk.off, nullptr, W + woff[l],
                  nbk.cols, nbk.cols, nbk.rows, nbk.cols, 0, 1, 0, 1.0});
  }
  scatter_batched(sj, stream_);
  dev_free(oldk.data, stream_);
  dev_free(oldm.data, stream_);
  dev_free(G, stream_);
  dev_free(Q, stream_);
  dev_free(W, stream_);
}

// Left-normalise site k (reduced Eq. 5, sum T^T T = 1 per right sector) and push the
// remaining factor into site k+1: G = sum T^T T = Q lambda Q^T, T <- T Q lambda^-1/2,
// T[k+1] <- lambda^1/2 Q^T T[k+1]; same threshold and second-pass rule as above.
void Engine::left_normalize_site(int k) {
  Site& S = sites_[k];
  const Bond br = bonds_[k + 1];
  const int nr = (int)br.sec.size();
  std::vector<int64_t> goff(nr + 1, 0), woff(nr + 1, 0);
  for (int r = 0; r < nr; ++r) {
    goff[r + 1] = goff[r] + (int64_t)br.dim[r] * br.dim[r];
    woff[r + 1] = woff[r] + br.dim[r];
  }
  double* G = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(goff[nr], 1), stream_);
  double* Q = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(goff[nr], 1), stream_);
  double* W = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(woff[nr], 1), stream_);
  dev_zero(G, sizeof(double) * std::max<int64_t>(goff[nr], 1), stream_);
  {
    std::vector<GemmTask> t;
    std::vector<GemmGroup> g;
    for (int r = 0; r < nr; ++r) {
      int b0 = (int)t.size();
      for (auto& b : S.blocks)
        if (b.r == r) t.push_back({S.data + b.off, S.data + b.off, b.cols, b.cols, b.rows, 1, 0, 1.0});
      if ((int)t.size() > b0) g.push_back({G + goff[r], br.dim[r], br.dim[r], br.dim[r], b0, (int)t.size(), 0});
    }
    GemmPlan* p = gemm_plan_upload(t, g, stream_);
    gemm_plan_run(p, stream_);
    gemm_plan_free(p, stream_);
  }
  std::vector<EigJob> jobs;
  for (int r = 0; r < nr; ++r) jobs.push_back({G + goff[r], Q + goff[r], W + woff[r], br.dim[r]});
  eig_batched(jobs, stream_);
  std::vector<double> w(woff[nr]);
  dev_d2h(w.data(), W, sizeof(double) * w.size(), stream_);
  dev_sync(stream_);
  Bond nb;
  std::vector<int> keep(nr, 0);
  for (int r = 0; r < nr; ++r) {
    const double wmax = br.dim[r] > 0 ? w[woff[r]] : 0.0;
    for (int a = 0; a < br.dim[r]; ++a)
      if (w[woff[r] + a] > 1e-14 * wmax && wmax > 0.0) ++keep[r];
    if (keep[r] > 0) { nb.sec.push_back(br.sec[r]); nb.dim.push_back(keep[r]); }
  }
  Site oldk = S;
  Site oldn = sites_[k + 1];
  sites_[k].data = nullptr;
  sites_[k + 1].data = nullptr;
  bonds_[k + 1] = nb;
  alloc_site(k);
  alloc_site(k + 1);
  std::vector<GemmTask> t;
  std::vector<GemmGroup> g;
  for (auto& b : oldk.blocks) {  // new block (dL x keep) = T (dL x dR) . Q_r (dR x keep)
    if (keep[b.r] == 0) continue;
    const int nrid = nb.find(br.sec[b.r]);
    for (auto& nbk : sites_[k].blocks)
      if (nbk.ls == b.ls && nbk.l == b.l && nbk.r == nrid) {
        t.push_back({oldk.data + b.off, Q + goff[b.r], b.cols, br.dim[b.r], b.cols, 0, 0, 1.0});
        g.push_back({sites_[k].data + nbk.off, nbk.cols, nbk.rows, keep[b.r], (int)t.size() - 1, (int)t.size(), 0});
      }
  }
  for (auto& b : oldn.blocks) {  // new block (keep x dR') = Q_r^T (keep x dL') . T
    if (keep[b.l] == 0) continue;
    const int nlid = nb.find(br.sec[b.l]);
    for (auto& nbk : sites_[k + 1].blocks)
      if (nbk.ls == b.ls && nbk.l == nlid && nbk.r == b.r) {
        t.push_back({Q + goff[b.l], oldn.data + b.off, br.dim[b.l], b.cols, br.dim[b.l], 1, 0, 1.0});
        g.push_back({sites_[k + 1].data + nbk.off, nbk.cols, keep[b.l], nbk.cols, (int)t.size() - 1, (int)t.size(), 0});
      }
  }
  GemmPlan* p = gemm_plan_upload(t, g, stream_);
  gemm_plan_run(p, stream_);
  gemm_plan_free(p, stream_);
  std::vector<ScatterJob> sj;
  for (auto& nbk : sites_[k].blocks) {
    const int r = br.find(nb.sec[nbk.r]);
    sj.push_back({sites_[k].data + nbk.off, sites_[k].data + nbk.off, nullptr, W + woff[r],
                  nbk.cols, nbk.cols, nbk.rows, nbk.cols, 0, 2, 0, 1.0});
  }
  for (auto& nbk : sites_[k + 1].blocks) {
    const int r = br.find(nb.sec[nbk.l]);
    sj.push_back({sites_[k + 1].data + nbk.off, sites_[k + 1].data + nbk.off, W + woff[r], nullptr,
                  nbk.cols, nbk.cols, nbk.rows, nbk.cols, 1, 0, 0, 1.0});
  }
  scatter_batched(sj, stream_);
  dev_free(oldk.data, stream_);
  dev_free(oldn.data, stream_);
  dev_free(G, stream_);
  dev_free(Q, stream_);
  dev_free(W, stream_);
}

// Mixed canonical form around `center` (Sec. 2.2, Eqs. 5-6): sites L-1..1 are
// right-normalised one by one (the factor moves left into site 0, whose norm is then
// set to 1), then sites 0..center-1 are left-normalised one by one (the factor moves
// right into the centre).  The state is unchanged up to normalisation.
void Engine::canonicalize(int center) {
  check_ready();
  if (center < 0 || center > L_ - 2) throw std::out_of_range("center out of range");
  Timer tm;
  for (int k = L_ - 1; k >= 1; --k) {
    right_normalize_site(k);
    right_normalize_site(k);
  }
  {  // normalise: |Psi|^2 = sum over site-0 blocks of (2jR+1) |T|^2
    const Site& S = sites_[0];
    std::vector<double> h(S.size);
    dev_d2h(h.data(), S.data, sizeof(double) * S.size, stream_);
    dev_sync(stream_);
    double n2 = 0.0;
    for (auto& b : S.blocks)
      for (int e = 0; e < b.rows * b.cols; ++e)
        n2 += (bonds_[1].sec[b.r].tj + 1) * h[b.off + e] * h[b.off + e];
    if (!(n2 > 0.0)) throw std::runtime_error("MPS has zero norm");
    for (auto& v : h) v /= std::sqrt(n2);
    dev_h2d(S.data, h.data(), sizeof(double) * S.size, stream_);
  }
  for (auto& e : lenv_) free_env(e);
  for (auto& e : renv_) free_env(e);
  if (cached_) { free_plan(cached_); cached_ = nullptr; cached_site_ = -1; }
  for (int i = 0; i < center; ++i) {
    left_normalize_site(i);
    left_normalize_site(i);
  }
  (void)tm;
}

// ---------------------------------------------------------------- RDMs
//
// For a fixed state the energy is linear in the folded integrals g of Eq. 11,
// E = E_c + 1/2 sum g_ijkl Gamma_ijkl, so the RDMs are the derivatives dE/dg.  The
// integrals enter the operator recursion only through the scalars s_e of its terms
// (s_e = gc_e g[gi_e]), and with the folded Hamiltonian written as the chain of site
// recursions, dE/ds_e for a term of site k is the expectation value of
// L_a(bond k) (x) [site pattern] (x) R_b(bond k+1): with the two-site object x at sites
// (k, k+1) that is x^T (L_a (x) P_e (x) D_b) x / x^T x, D_b the right combined operator
// of the matvec (Eq. 9).  This is the adjoint of the matvec with respect to its left
// operator blocks: if y = sum C W (phase 2), d(x^T y)/dC = sum x_out W^T =: Gbar, and
// dE/ds_e = <L_a, Gbar_C> summed over the blocks of the combined operator C that holds
// the term.  The sweep therefore visits every site pair once with the centre moving
// right; the terms of the last site (whose right partner is the 1 x 1 end operator) are
// differentiated through the right combined operators at the last pair instead:
// dE/dd = sum coef <C^T x_out, x_src> for a right operator of value d.
void Engine::rdm(double* gamma, double* Gamma) {
  check_ready();
  Timer tm;
  if (Wg_.empty()) {
    Integrals gz = g_;
    gz.keep_zero = true;
    Wg_.assign(L_, {});
    for (int k = 0; k < L_; ++k) Wg_[k] = build_site_recursion(k, opsets_[k], opsets_[k + 1], gz, pt_);
  }
  // the recursion with every allowed term holds the same operator values; it is swapped
  // in for the sweep and back out whatever happens
  struct Swap {
    std::vector<std::vector<WEntry>>& a;
    std::vector<std::vector<WEntry>>& b;
    Swap(std::vector<std::vector<WEntry>>& x, std::vector<std::vector<WEntry>>& y) : a(x), b(y) { std::swap(a, b); }
    ~Swap() { std::swap(a, b); }
  } swap_in(W_, Wg_);
  canonicalize(0);
  const int64_t L4 = (int64_t)L_ * L_ * L_ * L_;
  double* dg = (double*)dev_alloc(sizeof(double) * L4, stream_);
  // |x|^2 of every pair, then the scratch of the dot product
  double* nrm = (double*)dev_alloc(sizeof(double) * (L_ + 1024), stream_);
  dev_zero(dg, sizeof(double) * L4, stream_);
  try {
    for (int i = 0; i <= L_ - 2; ++i) {
      MatvecPlan* P = plan_matvec(i, true);
      try {
        tt_to_x(i, P->xin);
        // x is scaled to unit norm on the device (a zero norm is reported after the
        // pass), so nothing here waits for the device
        vec_multidot(P->xin, P->n, 1, P->xin, P->n, nrm + i, nrm + L_, stream_);
        vec_normalize(P->xin, nrm + i, P->n, stream_);
        // The centre moves on before this pair's products are queued: they read only the
        // copy of x, P's operators and the environment at bond i, none of which the
        // normalisation changes.  Its host synchronisation then waits for the previous
        // pair's products only, and the next pair's tables are built on the host while
        // the device runs this pair's.
        if (i < L_ - 2) {
          left_normalize_site(i);
          left_normalize_site(i);
        }
        rdm_site(P, i, dg, i == L_ - 2);
      } catch (...) {
        free_plan(P);
        throw;
      }
      free_plan(P);
    }
    rdm_finish(dg, L_, N_, gamma, Gamma, stream_);
    std::vector<double> n2(L_ - 1);
    dev_d2h(n2.data(), nrm, sizeof(double) * n2.size(), stream_);
    dev_sync(stream_);
    for (double v : n2)
      if (!(v > 0.0)) throw std::runtime_error("two-site object has zero norm");
  } catch (...) {
    dev_free(dg, stream_);
    dev_free(nrm, stream_);
    for (auto& e : lenv_) free_env(e);
    for (auto& e : renv_) free_env(e);
    throw;
  }
  dev_free(dg, stream_);
  dev_free(nrm, stream_);
  // the environments were built from the full recursion: same values, other tables
  for (auto& e : lenv_) free_env(e);
  for (auto& e : renv_) free_env(e);
  dev_sync(stream_);
  st_.rdm_passes += 1;
  st_.rdm_ms += tm.ms();
}

// x (P->xin) has unit norm.
void Engine::rdm_site(MatvecPlan* P, int i, double* dg, bool last) {
  const double n2 = 1.0;
  // W = sum coef Z (phases 1 and the combine of the FP64 matvec)
  if (P->zsize) dev_zero(P->Z, sizeof(double) * P->zsize, stream_);
  gemm_plan_run(P->p1, stream_);
  comb_plan_run(P->pc, stream_);
  const size_t nw = P->witems.size();
  std::vector<int64_t> woff(nw);
  std::vector<int> wxp(nw, -1);
  {
    int64_t o = 0;
    for (size_t k = 0; k < nw; ++k) {
      woff[k] = o;
      o += (int64_t)P->witems[k].rows * P->witems[k].cols;
    }
    for (int x = 0; x < (int)P->w_by_x.size(); ++x)
      for (int k : P->w_by_x[x]) wxp[k] = x;
  }
  // Gbar(gl, cbi) = sum over its W items of x_out W^T / |x|^2.  The W items of one
  // (left group, block) pair come in runs of consecutive items; the runs, stably sorted
  // by (gl, cbi), give every pair's items in increasing order, pair by pair.
  struct Run { int gl, cbi, b, e; };
  std::vector<Run> runs;
  for (size_t k = 0; k < nw; ++k) {
    const auto& w = P->witems[k];
    if (!runs.empty() && runs.back().gl == w.gl && runs.back().cbi == w.cbi) runs.back().e = (int)k + 1;
    else runs.push_back({w.gl, w.cbi, (int)k, (int)k + 1});
  }
  std::stable_sort(runs.begin(), runs.end(),
                   [](const Run& a, const Run& b) { return a.gl != b.gl ? a.gl < b.gl : a.cbi < b.cbi; });
  std::vector<std::pair<int, int>> by_blk;  // (gl, cbi) of each pair, in order
  std::vector<int> blk_run;                 // the pair's first run (prefix, one past the last pair)
  for (size_t r = 0; r < runs.size(); ++r)
    if (r == 0 || runs[r].gl != runs[r - 1].gl || runs[r].cbi != runs[r - 1].cbi) {
      by_blk.push_back({runs[r].gl, runs[r].cbi});
      blk_run.push_back((int)r);
    }
  blk_run.push_back((int)runs.size());
  std::vector<GemmTask> gt;
  std::vector<GemmGroup> gg;
  std::vector<int64_t> goff;
  int64_t gsize = 0;
  gt.reserve(nw);
  for (size_t q = 0; q < by_blk.size(); ++q) {
    const CombOp& C = P->cl[by_blk[q].first];
    const BlockRef& cb = (*C.blocks)[by_blk[q].second];
    const int b0 = (int)gt.size();
    for (int r = blk_run[q]; r < blk_run[q + 1]; ++r)
      for (int k = runs[r].b; k < runs[r].e; ++k) {
        const XBlock& Xp = P->X[wxp[k]];
        gt.push_back({P->xin + Xp.off, P->W + woff[k], Xp.cols, Xp.cols, Xp.cols, 0, 1, 1.0 / n2});
      }
    goff.push_back(gsize);
    gg.push_back({nullptr, cb.cols, cb.rows, cb.cols, b0, (int)gt.size(), 0});
    gsize += (int64_t)cb.rows * cb.cols;
  }
  double* Gb = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(gsize, 1), stream_);
  dev_zero(Gb, sizeof(double) * std::max<int64_t>(gsize, 1), stream_);
  for (size_t q = 0; q < gg.size(); ++q) gg[q].C = Gb + goff[q];
  {
    GemmPlan* p = gemm_plan_upload(gt, gg, stream_);
    gemm_plan_run(p, stream_);
    gemm_plan_free(p, stream_);
  }
  double flops = P->flops1;
  for (size_t q = 0; q < gg.size(); ++q)
    for (int k = gg[q].task_begin; k < gg[q].task_end; ++k) flops += 2.0 * gg[q].m * gg[q].n * gt[k].k;
  // dE/dg[gi] += gc <L_a, Gbar> over the terms of every left combined operator
  std::map<int64_t, std::vector<DotTask>> dots;
  const OpStore& E = lenv_[i];
  {
    for (size_t q = 0; q < by_blk.size(); ++q) {
      const CombOp& C = P->cl[by_blk[q].first];
      const BlockRef& cb = (*C.blocks)[by_blk[q].second];
      const double* gb = Gb + goff[q];
      for (size_t s = 0; s < C.sources.size(); ++s) {
        const int64_t gi = C.grad[s].first;
        if (gi < 0) continue;
        const int a = C.sources[s].first;
        auto it = E.at[a].find(bkey(cb.r, cb.c));
        if (it == E.at[a].end()) continue;
        const BlockRef& lb = E.blocks[a][it->second];
        dots[gi].push_back({E.data + lb.off, gb, lb.cols, cb.cols, cb.rows, cb.cols, C.grad[s].second});
      }
    }
  }
  double* U = nullptr;
  if (last) {
    // the site's right terms all end in the 1 x 1 operator H(bond L) = 1:
    // dE/ds_e = sum over W items and their sources of this group of craw <C^T x_out, x_src>
    U = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(P->wsize, 1), stream_);
    dev_zero(U, sizeof(double) * std::max<int64_t>(P->wsize, 1), stream_);
    std::vector<GemmTask> ut;
    std::vector<GemmGroup> ug;
    for (size_t k = 0; k < nw; ++k) {
      const auto& w = P->witems[k];
      const CombOp& C = P->cl[w.gl];
      const BlockRef& cb = (*C.blocks)[w.cbi];
      const XBlock& Xp = P->X[wxp[k]];
      const int b0 = (int)ut.size();
      if (C.identity) ut.push_back({nullptr, P->xin + Xp.off, 0, Xp.cols, Xp.cols, 0, 0, C.scalar});
      else ut.push_back({C.data + cb.off, P->xin + Xp.off, cb.cols, Xp.cols, cb.rows, 1, 0, C.scalar});
      ug.push_back({U + woff[k], Xp.cols, cb.cols, Xp.cols, b0, b0 + 1, 0});
      for (int q = w.src_begin; q < w.src_end; ++q) {
        const auto& src = P->wsrc[q];
        const CombOp& D = P->cr[src.gr];
        const XBlock& Xs = P->X[src.xb];
        if (Xs.rows != cb.cols || Xs.cols != Xp.cols)
          throw std::logic_error("rdm: right end operator is not 1 x 1");
        for (size_t s = 0; s < D.sources.size(); ++s) {
          const int64_t gi = D.grad[s].first;
          if (gi < 0) continue;
          dots[gi].push_back({U + woff[k], P->xin + Xs.off, Xp.cols, Xs.cols, cb.cols, Xp.cols,
                              src.craw * D.grad[s].second / n2});
        }
      }
    }
    GemmPlan* p = gemm_plan_upload(ut, ug, stream_);
    gemm_plan_run(p, stream_);
    gemm_plan_free(p, stream_);
    for (size_t q = 0; q < ug.size(); ++q)
      if (ut[q].A) flops += 2.0 * ug[q].m * ug[q].n * ut[q].k;
  }
  std::vector<DotTask> dt;
  std::vector<DotGroup> dgp;
  for (auto& kv : dots)
    for (const DotTask& t : kv.second) flops += 2.0 * t.rows * t.cols;
  st_.rdm_flops += flops;
  for (auto& kv : dots) {
    const int b0 = (int)dt.size();
    dt.insert(dt.end(), kv.second.begin(), kv.second.end());
    dgp.push_back({dg + kv.first, b0, (int)dt.size()});
  }
  dot_grouped(dt, dgp, stream_);
  dev_free(Gb, stream_);
  if (U) dev_free(U, stream_);
}

// ---------------------------------------------------------------- excited states
//
// H_m = H_0 + sum_k eta_{k+1} |Psi_k><Psi_k| (Sec. 4.3).  In the two-site basis of
// sites (i, i+1) the projector is eta v v^T with v = O_L(i) x_k O_R(i+2)^T blockwise:
// x_k the lower state's own two-site object (Eq. 25, x = sqrt(2jR+1) S), O_L / O_R the
// overlaps of the current renormalised basis with the lower state's, per sector:
//   O_L(k+1)[r] = sum_{s, l} T_cur[s, l, r]^T O_L(k)[l] T_low[s, l, r]          (O_L(0) = 1)
//   O_R(k)[l]   = sum_{s, r} (2jR+1)/(2jL+1) T_cur[s, l, r] O_R(k+1)[r] T_low[s, l, r]^T
// (the reduced recursions whose fixed points are the normalisations of Eqs. 5 and 6).
// An overlap is rebuilt whenever the operator environment of the same bond and side has
// been (both depend on the same current tensors).

void Engine::push_excitation(double eta) {
  check_ready();
  canonicalize(0);  // |Psi| = 1
  LowState S;
  S.eta = eta;
  S.bonds = bonds_;
  S.sites.resize(L_);
  for (int k = 0; k < L_; ++k) {
    S.sites[k].blocks = sites_[k].blocks;
    S.sites[k].size = sites_[k].size;
    S.sites[k].data = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(sites_[k].size, 1), stream_);
    dev_d2d(S.sites[k].data, sites_[k].data, sizeof(double) * sites_[k].size, stream_);
  }
  S.left.resize(L_ + 1);
  S.right.resize(L_ + 1);
  low_.push_back(std::move(S));
  if (cached_) { free_plan(cached_); cached_ = nullptr; cached_site_ = -1; }
}

void Engine::clear_excitations() {
  for (auto& S : low_) {
    for (auto& t : S.sites)
      if (t.data) dev_free(t.data, stream_);
    for (auto& o : S.left) free_overlap(o);
    for (auto& o : S.right) free_overlap(o);
  }
  low_.clear();
  if (cached_) { free_plan(cached_); cached_ = nullptr; cached_site_ = -1; }
}

void Engine::free_overlap(Overlap& o) {
  if (o.data) dev_free(o.data, stream_);
  o = Overlap();
}

namespace {
// blocks for the sectors present in both bonds
void overlap_layout(Overlap& O, const Bond& cur, const Bond& low) {
  int64_t off = 0;
  for (int c = 0; c < (int)cur.sec.size(); ++c) {
    const int l = low.find(cur.sec[c]);
    if (l < 0) continue;
    O.by_cur[c] = (int)O.cur.size();
    O.cur.push_back(c);
    O.low.push_back(l);
    O.rows.push_back(cur.dim[c]);
    O.cols.push_back(low.dim[l]);
    O.off.push_back(off);
    off += (int64_t)cur.dim[c] * low.dim[l];
  }
  O.size = off;
}
}  // namespace

void Engine::ensure_ov_left(LowState& S, int k) {
  ensure_left(k);
  Overlap& O = S.left[k];
  if (O.valid && O.env_serial == lenv_[k].serial) return;
  if (k > 0) ensure_ov_left(S, k - 1);
  free_overlap(O);
  overlap_layout(O, bonds_[k], S.bonds[k]);
  O.data = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(O.size, 1), stream_);
  dev_zero(O.data, sizeof(double) * std::max<int64_t>(O.size, 1), stream_);
  if (k == 0) {
    const double one = 1.0;
    for (size_t e = 0; e < O.cur.size(); ++e) dev_h2d(O.data + O.off[e], &one, sizeof(double), stream_);
    dev_sync(stream_);
  } else {
    const Overlap& P = S.left[k - 1];
    const Site& Tc = sites_[k - 1];
    const Site& Tl = S.sites[k - 1];
    const Bond& lowl = S.bonds[k - 1];
    const Bond& lowr = S.bonds[k];
    std::map<std::tuple<int, int, int>, int> lb;  // (ls, low left sector, low right sector)
    for (int t = 0; t < (int)Tl.blocks.size(); ++t) lb[{Tl.blocks[t].ls, Tl.blocks[t].l, Tl.blocks[t].r}] = t;
    std::vector<GemmTask> t1, t2;
    std::vector<GemmGroup> g1;
    std::map<int, std::vector<GemmTask>> out;  // overlap block -> tasks
    std::vector<int64_t> zoff;
    int64_t zsize = 0;
    for (const SiteBlock& c : Tc.blocks) {
      auto pl = P.by_cur.find(c.l);
      auto orr = O.by_cur.find(c.r);
      if (pl == P.by_cur.end() || orr == O.by_cur.end()) continue;
      const int ll = P.low[pl->second], lr = O.low[orr->second];
      auto it = lb.find({c.ls, ll, lr});
      if (it == lb.end()) continue;
      const SiteBlock& b = Tl.blocks[it->second];
      // Z = O_L(k-1)[l] (d_cur(l) x d_low(l)) . T_low (d_low(l) x d_low(r))
      const int dcl = P.rows[pl->second], dll = lowl.dim[ll], dlr = lowr.dim[lr];
      t1.push_back({P.data + P.off[pl->second], Tl.data + b.off, dll, dlr, dll, 0, 0, 1.0});
      g1.push_back({nullptr, dlr, dcl, dlr, (int)t1.size() - 1, (int)t1.size(), 0});
      zoff.push_back(zsize);
      zsize += (int64_t)dcl * dlr;
      // O_L(k)[r] += T_cur^T (d_cur(r) x d_cur(l)) . Z
      out[orr->second].push_back({Tc.data + c.off, (const double*)(intptr_t)(g1.size() - 1), c.cols, dlr,
                                  c.rows, 1, 0, 1.0});
    }
    double* Z = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(zsize, 1), stream_);
    dev_zero(Z, sizeof(double) * std::max<int64_t>(zsize, 1), stream_);
    for (size_t z = 0; z < g1.size(); ++z) g1[z].C = Z + zoff[z];
    std::vector<GemmGroup> g2;
    for (auto& kv : out) {
      const int e = kv.first;
      const int b0 = (int)t2.size();
      for (GemmTask t : kv.second) {
        t.B = Z + zoff[(size_t)(intptr_t)t.B];
        t2.push_back(t);
      }
      g2.push_back({O.data + O.off[e], O.cols[e], O.rows[e], O.cols[e], b0, (int)t2.size(), 0});
    }
    GemmPlan* p1 = gemm_plan_upload(t1, g1, stream_);
    GemmPlan* p2 = gemm_plan_upload(t2, g2, stream_);
    gemm_plan_run(p1, stream_);
    gemm_plan_run(p2, stream_);
    gemm_plan_free(p1, stream_);
    gemm_plan_free(p2, stream_);
    dev_free(Z, stream_);
  }
  O.valid = true;
  O.env_serial = lenv_[k].serial;
}

void Engine::ensure_ov_right(LowState& S, int k) {
  ensure_right(k);
  Overlap& O = S.right[k];
  if (O.valid && O.env_serial == renv_[k].serial) return;
  if (k < L_) ensure_ov_right(S, k + 1);
  free_overlap(O);
  overlap_layout(O, bonds_[k], S.bonds[k]);
  O.data = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(O.size, 1), stream_);
  dev_zero(O.data, sizeof(double) * std::max<int64_t>(O.size, 1), stream_);
  if (k == L_) {
    const double one = 1.0;
    for (size_t e = 0; e < O.cur.size(); ++e) dev_h2d(O.data + O.off[e], &one, sizeof(double), stream_);
    dev_sync(stream_);
  } else {
    const Overlap& P = S.right[k + 1];
    const Site& Tc = sites_[k];
    const Site& Tl = S.sites[k];
    const Bond& lowl = S.bonds[k];
    const Bond& lowr = S.bonds[k + 1];
    std::map<std::tuple<int, int, int>, int> lb;
    for (int t = 0; t < (int)Tl.blocks.size(); ++t) lb[{Tl.blocks[t].ls, Tl.blocks[t].l, Tl.blocks[t].r}] = t;
    std::vector<GemmTask> t1, t2;
    std::vector<GemmGroup> g1;
    std::map<int, std::vector<GemmTask>> out;
    std::vector<int64_t> zoff;
    int64_t zsize = 0;
    for (const SiteBlock& c : Tc.blocks) {
      auto pr = P.by_cur.find(c.r);
      auto ol = O.by_cur.find(c.l);
      if (pr == P.by_cur.end() || ol == O.by_cur.end()) continue;
      const int lr = P.low[pr->second], ll = O.low[ol->second];
      auto it = lb.find({c.ls, ll, lr});
      if (it == lb.end()) continue;
      const SiteBlock& b = Tl.blocks[it->second];
      const double w = (double)(bonds_[k + 1].sec[c.r].tj + 1) / (double)(bonds_[k].sec[c.l].tj + 1);
      // Z = O_R(k+1)[r] (d_cur(r) x d_low(r)) . T_low^T (d_low(r) x d_low(l))
      const int dcr = P.rows[pr->second], dlr = lowr.dim[lr], dll = lowl.dim[ll];
      t1.push_back({P.data + P.off[pr->second], Tl.data + b.off, dlr, dlr, dlr, 0, 1, 1.0});
      g1.push_back({nullptr, dll, dcr, dll, (int)t1.size() - 1, (int)t1.size(), 0});
      zoff.push_back(zsize);
      zsize += (int64_t)dcr * dll;
      // O_R(k)[l] += w T_cur (d_cur(l) x d_cur(r)) . Z
      out[ol->second].push_back({Tc.data + c.off, (const double*)(intptr_t)(g1.size() - 1), c.cols, dll,
                                 c.cols, 0, 0, w});
    }
    double* Z = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(zsize, 1), stream_);
    dev_zero(Z, sizeof(double) * std::max<int64_t>(zsize, 1), stream_);
    for (size_t z = 0; z < g1.size(); ++z) g1[z].C = Z + zoff[z];
    std::vector<GemmGroup> g2;
    for (auto& kv : out) {
      const int e = kv.first;
      const int b0 = (int)t2.size();
      for (GemmTask t : kv.second) {
        t.B = Z + zoff[(size_t)(intptr_t)t.B];
        t2.push_back(t);
      }
      g2.push_back({O.data + O.off[e], O.cols[e], O.rows[e], O.cols[e], b0, (int)t2.size(), 0});
    }
    GemmPlan* p1 = gemm_plan_upload(t1, g1, stream_);
    GemmPlan* p2 = gemm_plan_upload(t2, g2, stream_);
    gemm_plan_run(p1, stream_);
    gemm_plan_run(p2, stream_);
    gemm_plan_free(p1, stream_);
    gemm_plan_free(p2, stream_);
    dev_free(Z, stream_);
  }
  O.valid = true;
  O.env_serial = renv_[k].serial;
}

void Engine::low_projection(LowState& S, int i, const std::vector<XBlock>& X, double* v) {
  ensure_ov_left(S, i);
  ensure_ov_right(S, i + 2);
  const Overlap& OL = S.left[i];
  const Overlap& OR = S.right[i + 2];
  int64_t nl = 0;
  auto XL = x_layout_of(S.bonds, i, &nl);
  double* xl = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(nl, 1), stream_);
  tt_to_x_of(S.bonds, S.sites, i, xl);
  std::map<std::tuple<int, int, int, int, int>, int> at;  // (l, ls1, ls2, tj, r) in low sectors
  for (int q = 0; q < (int)XL.size(); ++q) at[{XL[q].l, XL[q].ls1, XL[q].ls2, XL[q].tj, XL[q].r}] = q;
  std::vector<GemmTask> t1, t2;
  std::vector<GemmGroup> g1, g2;
  std::vector<int64_t> zoff;
  int64_t zsize = 0;
  for (const XBlock& b : X) {
    auto pl = OL.by_cur.find(b.l);
    auto pr = OR.by_cur.find(b.r);
    if (pl == OL.by_cur.end() || pr == OR.by_cur.end()) continue;
    auto it = at.find({OL.low[pl->second], b.ls1, b.ls2, b.tj, OR.low[pr->second]});
    if (it == at.end()) continue;
    const XBlock& c = XL[it->second];
    // Z = x_low (d_low(l) x d_low(r)) . O_R[r]^T (d_low(r) x d_cur(r)); v = O_L[l] . Z
    t1.push_back({xl + c.off, OR.data + OR.off[pr->second], c.cols, c.cols, c.cols, 0, 1, 1.0});
    g1.push_back({nullptr, b.cols, c.rows, b.cols, (int)t1.size() - 1, (int)t1.size(), 0});
    zoff.push_back(zsize);
    zsize += (int64_t)c.rows * b.cols;
    t2.push_back({OL.data + OL.off[pl->second], nullptr, c.rows, b.cols, c.rows, 0, 0, 1.0});
    g2.push_back({v + b.off, b.cols, b.rows, b.cols, (int)t2.size() - 1, (int)t2.size(), 0});
  }
  double* Z = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(zsize, 1), stream_);
  dev_zero(Z, sizeof(double) * std::max<int64_t>(zsize, 1), stream_);
  for (size_t z = 0; z < g1.size(); ++z) {
    g1[z].C = Z + zoff[z];
    t2[z].B = Z + zoff[z];
  }
  int64_t n = 0;
  for (const XBlock& b : X) n = std::max<int64_t>(n, b.off + (int64_t)b.rows * b.cols);
  dev_zero(v, sizeof(double) * std::max<int64_t>(n, 1), stream_);
  GemmPlan* p1 = gemm_plan_upload(t1, g1, stream_);
  GemmPlan* p2 = gemm_plan_upload(t2, g2, stream_);
  gemm_plan_run(p1, stream_);
  gemm_plan_run(p2, stream_);
  gemm_plan_free(p1, stream_);
  gemm_plan_free(p2, stream_);
  dev_free(Z, stream_);
  dev_free(xl, stream_);
}

// True if sites 1..L-1 satisfy the reduced right-normalisation of Eq. 6,
// sum (2jR+1)/(2jL+1) T T^T = 1 per left sector, to 1e-10.
bool Engine::is_right_canonical() {
  for (int k = L_ - 1; k >= 1; --k) {
    const Site& S = sites_[k];
    const Bond& bl = bonds_[k];
    const Bond& br = bonds_[k + 1];
    std::vector<int64_t> goff(bl.sec.size(), 0);
    int64_t tot = 0;
    for (size_t l = 0; l < bl.sec.size(); ++l) { goff[l] = tot; tot += (int64_t)bl.dim[l] * bl.dim[l]; }
    double* G = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(tot, 1), stream_);
    dev_zero(G, sizeof(double) * std::max<int64_t>(tot, 1), stream_);
    std::vector<GemmTask> t;
    std::vector<GemmGroup> g;
    for (size_t l = 0; l < bl.sec.size(); ++l) {
      int b0 = (int)t.size();
      for (auto& b : S.blocks)
        if (b.l == (int)l)
          t.push_back({S.data + b.off, S.data + b.off, b.cols, b.cols, b.cols, 0, 1,
                       (double)(br.sec[b.r].tj + 1) / (double)(bl.sec[l].tj + 1)});
      if ((int)t.size() > b0) g.push_back({G + goff[l], bl.dim[l], bl.dim[l], bl.dim[l], b0, (int)t.size(), 0});
    }
    GemmPlan* p = gemm_plan_upload(t, g, stream_);
    gemm_plan_run(p, stream_);
    gemm_plan_free(p, stream_);
    std::vector<double> h(tot);
    dev_d2h(h.data(), G, sizeof(double) * tot, stream_);
    dev_sync(stream_);
    dev_free(G, stream_);
    for (size_t l = 0; l < bl.sec.size(); ++l)
      for (int a = 0; a < bl.dim[l]; ++a)
        for (int c = 0; c < bl.dim[l]; ++c)
          if (std::fabs(h[goff[l] + (int64_t)a * bl.dim[l] + c] - (a == c ? 1.0 : 0.0)) > 1e-10) return false;
  }
  return true;
}

// ConvergenceScheme of Sec. 4.2: per instruction, macro-iterations (a sweep right then
// a sweep left) until the energy change is below E_conv or N_max is reached; the
// result is the lowest micro-iteration energy (Sec. 4.3).
double Engine::solve(double* e_last_out) {
  check_ready();
  Timer total;
  if (!is_right_canonical()) canonicalize(0);
  double e_min = std::numeric_limits<double>::infinity(), e_last = 0.0;
  double e_prev = std::numeric_limits<double>::infinity();
  bool all_conv = true;
  hist_D_.clear();
  hist_E_.clear();
  hist_w_.clear();
  for (size_t s = 0; s < sched_D_.size(); ++s) {
    const int D = sched_D_[s];
    double e_mac = 0.0, w_mac = 0.0;  // lowest energy / largest discarded weight of the last macro-iteration
    const double econv = s < sched_econv_.size() ? sched_econv_[s] : 1e-8;
    const int nmax = s < sched_nmax_.size() ? sched_nmax_[s] : 1;
    const double gamma = s < sched_noise_.size() ? sched_noise_[s] : 0.0;
    for (int it = 0; it < nmax; ++it) {
      e_mac = std::numeric_limits<double>::infinity();
      w_mac = 0.0;
      for (int dir = 1; dir >= -1; dir -= 2) {
        double wmax = 0.0;
        for (int step = 0; step < L_ - 1; ++step) {
          const int i = dir > 0 ? step : L_ - 2 - step;
          double w = 0.0;
          int iters = 0;
          bool conv = false;
          // the next step is the neighbour in this direction, or the same site where the
          // sweep turns (a half sweep ends where the next one starts)
          next_hint_ = step < L_ - 2 ? i + dir : i;
          double e = sweep_step(i, dir, D, gamma, &w, &iters, &conv);
          all_conv = all_conv && conv;
          e_min = std::min(e_min, e);
          e_last = e;
          wmax = std::max(wmax, w);
          e_mac = std::min(e_mac, e);
          w_mac = std::max(w_mac, w);
        }
      }
      const bool done = std::fabs(e_last - e_prev) < econv;
      e_prev = e_last;
      if (done) break;
    }
    hist_D_.push_back(D);
    hist_E_.push_back(e_mac);
    hist_w_.push_back(w_mac);
  }
  st_.t_total_ms += total.ms();
  if (e_last_out) *e_last_out = e_last;
  (void)all_conv;
  return e_min;
}

// The last part of a sweep step on its own (Sec. 2.5): the operators of the block grown
// by site i (dir > 0, from the left-normalised T[i]) or by site i+1 (dir < 0, from the
// right-normalised T[i+1]), from the combined operators of the environment they extend.
void Engine::update(int i, int dir) {
  check_ready();
  if (i < 0 || i > L_ - 2) throw std::out_of_range("site out of range");
  std::vector<CombOp> comb;
  double* scr = nullptr;
  int64_t scr_n = 0;
  try {
    if (dir > 0) {
      ensure_left(i);
      group_left(i, comb, &scr, &scr_n);
      update_left_from(i, comb);
    } else {
      ensure_right(i + 2);
      group_right(i + 1, comb, &scr, &scr_n);
      update_right_from(i + 1, comb);
    }
  } catch (...) {
    if (scr) dev_free(scr, stream_);
    throw;
  }
  if (scr) dev_free(scr, stream_);
}

double Engine::sweep_step(int i, int dir, int D, double gamma, double* w_disc, int* iters, bool* conv) {
  check_ready();
  if (i < 0 || i > L_ - 2) throw std::out_of_range("site out of range");
  const int next = next_hint_;
  next_hint_ = -1;
  // a change of direction starts a half sweep: the noise of its steps is bounded by the
  // largest discarded weight of the previous one (Sec. 4.2)
  if (dir != half_dir_) {
    w_prev_ = half_dir_ == 0 ? 0.0 : half_wmax_;
    half_wmax_ = 0.0;
    half_dir_ = dir;
  }
  MatvecPlan* P = plan_for(i);
  double* x = (double*)dev_alloc(sizeof(double) * std::max<int64_t>(P->n, 1), stream_);
  tt_to_x(i, x);
  double e = davidson_ex(i, x, iters, conv, true) + econst_;
  if (gamma > 0.0 && w_prev_ > 0.0) {
    // Sec. 4.2: noise bounded by 0.5 gamma w_disc(previous half sweep), then the
    // decomposition renormalises through kappa
    vec_add_noise(x, P->n, 0.5 * gamma * w_prev_, 0x5eed0000ull + (noise_counter_++) * 1000003ull, stream_);
  }
  cached_ = nullptr;  // keep P's combined operators for the update below
  cached_site_ = -1;
  double w;
  bool keep = false;
  try {
    w = truncate(i, dir, D, x, 0.0);
    half_wmax_ = std::max(half_wmax_, w);
    launch_rq();  // after the decomposition, whose kernels would otherwise queue behind it
    if (dir > 0) update_left_from(i, P->cl);
    else update_right_from(i + 1, P->cr);
    // The step changed only the middle bond i+1: the environments at bonds i and i+2 and
    // the x layout of site i, everything P is made of, are unchanged, so a next step at
    // the same site reuses P.  A next step at another site has its tables built here,
    // on the host, while the FP64 Rayleigh quotient runs on the side stream.
    if (next == i) {
      keep = true;
    } else if (next >= 0 && next <= L_ - 2) {
      cached_ = plan_matvec(next);
      cached_->serial = ++plan_serial_;
      cached_site_ = next;
      if (precision_ == 1) {
        try {
          build_tc(cached_);
        } catch (...) {
          release_tc(cached_);
          throw;
        }
        build_rq(cached_);
      }
    }
  } catch (...) {
    if (rq_pending_) { try { finish_rq(); } catch (...) {} }
    free_plan(P);
    dev_free(x, stream_);
    throw;
  }
  if (rq_pending_) e = finish_rq() + econst_;
  if (keep) {
    cached_ = P;
    cached_site_ = i;
  } else {
    free_plan(P);
  }
  dev_free(x, stream_);
  st_.micro_iters += 1;
  *w_disc = w;
  return e;
}

}  // namespace dmrg

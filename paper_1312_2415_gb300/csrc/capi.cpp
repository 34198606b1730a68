// extern "C" boundary: argument checks, host/device pointer handling, error codes.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/dmrg_gb300.h"
#include "batch.hpp"
#include "engine.hpp"

struct dmrg_ctx {
  dmrg::Engine* eng = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
  int L = 0;
  // allocation-free matvecs run on the caller's stream and read the context's tables:
  // `tables` orders them after the context's stream, `noalloc_done` orders the context's
  // next work (which may free or rewrite those tables) after them
  cudaEvent_t tables = nullptr, noalloc_done = nullptr;
  bool noalloc_pending = false;
};

struct dmrg_batch {
  std::vector<dmrg_ctx*> ctx;
  std::vector<int> site;
  std::vector<uint64_t> serial;
  std::vector<double*> x, y;
  std::vector<const double*> diag;
  std::vector<int64_t> n;
  dmrg::TcPlan* plan = nullptr;
  void* graph = nullptr;
  dmrg::TcTune tune;
  double flops = 0.0, best_ms = 0.0, tune_ms = 0.0;
  std::string err;
};

namespace {

const int kGroupOrder[8] = {1, 2, 2, 2, 4, 4, 4, 8};

template <class F>
int guard_err(std::string& err, F&& f) {
  try {
    err.clear();
    return f();
  } catch (const std::bad_alloc& e) {
    err = std::string("allocation failed: ") + e.what();
    return DMRG_ENOMEM;
  } catch (const std::domain_error& e) {
    err = e.what();
    return DMRG_ESYMM;
  } catch (const std::invalid_argument& e) {
    err = e.what();
    return DMRG_EINVAL;
  } catch (const std::out_of_range& e) {
    err = e.what();
    return DMRG_EINVAL;
  } catch (const std::runtime_error& e) {
    err = e.what();
    std::string m = e.what();
    if (m.find("out of memory") != std::string::npos) return DMRG_ENOMEM;
    return m.find("cuda") != std::string::npos || m.find("launch") != std::string::npos ||
                   m.find("Async") != std::string::npos || m.find("sync") != std::string::npos
               ? DMRG_ECUDA
               : DMRG_EINTERNAL;
  } catch (...) {
    err = "unknown failure";
    return DMRG_EINTERNAL;
  }
}

template <class F>
int guard(dmrg_ctx* c, F&& f) {
  if (!c) return DMRG_EINVAL;
  return guard_err(c->err, std::forward<F>(f));
}

// Runs f(dev_in_or_out...) with device buffers: for host pointers, copies in/out.
struct DevBuf {
  double* p = nullptr;
  dmrg::Stream s;
  DevBuf(int64_t n, dmrg::Stream st) : s(st) { p = (double*)dmrg::dev_alloc(sizeof(double) * (n > 0 ? n : 1), st); }
  ~DevBuf() { try { dmrg::dev_free(p, s); } catch (...) {} }
};

// The context's stream is created at the first call that touches the device, so that
// problem setup and its validation work without a GPU.
dmrg::Stream dev_stream(dmrg_ctx* c) {
  if (!c->stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) throw std::runtime_error(std::string("cuda stream: ") + cudaGetErrorString(e));
    c->eng->set_stream((dmrg::Stream)c->stream);
  }
  if (c->noalloc_pending) {
    // work queued from here on (including stream-ordered frees) waits for the
    // allocation-free matvecs still reading the context's tables
    cudaError_t e = cudaStreamWaitEvent(c->stream, c->noalloc_done, 0);
    if (e != cudaSuccess) throw std::runtime_error(std::string("cuda stream wait: ") + cudaGetErrorString(e));
    c->noalloc_pending = false;
  }
  return (dmrg::Stream)c->stream;
}

void wait_user(uintptr_t stream) {
  if (stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) throw std::runtime_error(std::string("cuda user stream: ") + cudaGetErrorString(e));
  }
}

dmrg::Stream dev_stream(dmrg_ctx* c);
int64_t xsize(dmrg_ctx* c, int site) {
  std::vector<int64_t> t;
  int64_t n = 0;
  c->eng->layout(site, t, n);
  return n;
}

}  // namespace

extern "C" {

int dmrg_create(dmrg_ctx** out, int L, int group, const int* orb_irrep, int N, int two_S,
                int target_irrep, int precision) {
  if (!out) return DMRG_EINVAL;
  *out = nullptr;
  if (L < 2 || L > 120 || group < 0 || group > 7 || !orb_irrep) return DMRG_EINVAL;
  const int nir = kGroupOrder[group];
  for (int i = 0; i < L; ++i)
    if (orb_irrep[i] < 0 || orb_irrep[i] >= nir) return DMRG_EINVAL;
  if (N < 2 || N > 2 * L || two_S < 0 || two_S > N || two_S > 2 * L - N || ((N - two_S) & 1))
    return DMRG_EINVAL;
  if (target_irrep < 0 || target_irrep >= nir) return DMRG_EINVAL;
  if (precision != 0 && precision != 1) return DMRG_EINVAL;
  dmrg_ctx* c = new (std::nothrow) dmrg_ctx;
  if (!c) return DMRG_ENOMEM;
  try {
    std::vector<int> ir(orb_irrep, orb_irrep + L);
    c->eng = new dmrg::Engine(L, nir, ir, N, two_S, target_irrep, nullptr);
    c->eng->set_precision(precision, 0);
    c->L = L;
  } catch (...) {
    delete c;
    return DMRG_ENOMEM;
  }
  *out = c;
  return DMRG_OK;
}

int dmrg_set_integrals(dmrg_ctx* c, double econst, const double* h, const double* V) {
  return guard(c, [&] {
    if (!h || !V || !std::isfinite(econst)) return DMRG_EINVAL;
    c->eng->set_integrals(econst, h, V);
    return DMRG_OK;
  });
}

int dmrg_set_schedule(dmrg_ctx* c, int n, const int* D, const double* e_conv, const int* n_max,
                      const double* noise, double davidson_tol, int davidson_max_iter) {
  return guard(c, [&] {
    if (n < 1 || !D || !e_conv || !n_max || !noise || !(davidson_tol > 0) || davidson_max_iter < 1)
      return DMRG_EINVAL;
    for (int i = 0; i < n; ++i)
      if (D[i] < 1 || n_max[i] < 0 || noise[i] < 0 || !(e_conv[i] >= 0)) return DMRG_EINVAL;
    c->eng->set_schedule(std::vector<int>(D, D + n), std::vector<double>(e_conv, e_conv + n),
                         std::vector<int>(n_max, n_max + n), std::vector<double>(noise, noise + n),
                         davidson_tol, davidson_max_iter);
    return DMRG_OK;
  });
}

int dmrg_set_precision(dmrg_ctx* c, int precision, int fp64_iters) {
  return guard(c, [&] {
    if ((precision != 0 && precision != 1) || fp64_iters < 0) return DMRG_EINVAL;
    c->eng->set_precision(precision, fp64_iters);
    return DMRG_OK;
  });
}

int dmrg_init_mps(dmrg_ctx* c, uint64_t seed) {
  return guard(c, [&] {
    dev_stream(c);
    c->eng->init_mps(seed);
    return DMRG_OK;
  });
}

int dmrg_get_mps(dmrg_ctx* c, void* buf, size_t* len) {
  return guard(c, [&] {
    if (!len) return DMRG_EINVAL;
    dev_stream(c);
    auto v = c->eng->get_mps();
    if (!buf) { *len = v.size(); return DMRG_OK; }
    if (*len < v.size()) { *len = v.size(); return DMRG_EINVAL; }
    std::memcpy(buf, v.data(), v.size());
    *len = v.size();
    return DMRG_OK;
  });
}

int dmrg_set_mps(dmrg_ctx* c, const void* buf, size_t len) {
  return guard(c, [&] {
    if (!buf) return DMRG_EINVAL;
    dev_stream(c);
    c->eng->set_mps((const char*)buf, len);
    return DMRG_OK;
  });
}

int dmrg_canonicalize(dmrg_ctx* c, int center) {
  return guard(c, [&] {
    dmrg::Stream s = dev_stream(c);
    c->eng->canonicalize(center);
    dmrg::dev_sync(s);
    return DMRG_OK;
  });
}

int dmrg_solve(dmrg_ctx* c, double* e_min, double* e_last) {
  return guard(c, [&] {
    double el = 0.0;
    dev_stream(c);
    double em = c->eng->solve(&el);
    if (e_min) *e_min = em;
    if (e_last) *e_last = el;
    return DMRG_OK;
  });
}

int dmrg_two_site_layout(dmrg_ctx* c, int site, int64_t* n_elem, int* n_blocks, int64_t* table) {
  return guard(c, [&] {
    std::vector<int64_t> t;
    int64_t n = 0;
    dev_stream(c);
    c->eng->layout(site, t, n);
    if (n_elem) *n_elem = n;
    if (n_blocks) *n_blocks = (int)(t.size() / 12);
    if (table) std::memcpy(table, t.data(), t.size() * sizeof(int64_t));
    return DMRG_OK;
  });
}

int dmrg_tt_to_x(dmrg_ctx* c, int site, double* x, uintptr_t stream) {
  return guard(c, [&] {
    if (!x) return DMRG_EINVAL;
    wait_user(stream);
    const int64_t n = xsize(c, site);
    dmrg::Stream s = dev_stream(c);
    if (stream) {
      c->eng->tt_to_x(site, x);
    } else {
      DevBuf d(n, s);
      c->eng->tt_to_x(site, d.p);
      dmrg::dev_d2h(x, d.p, sizeof(double) * n, s);
    }
    dmrg::dev_sync(s);
    return DMRG_OK;
  });
}

int dmrg_heff_matvec(dmrg_ctx* c, int site, const double* x, double* y, uintptr_t stream) {
  return guard(c, [&] {
    if (!x || !y) return DMRG_EINVAL;
    wait_user(stream);
    const int64_t n = xsize(c, site);
    dmrg::Stream s = dev_stream(c);
    if (stream) {
      c->eng->matvec(site, x, y);
    } else {
      DevBuf dx(n, s), dy(n, s);
      dmrg::dev_h2d(dx.p, x, sizeof(double) * n, s);
      c->eng->matvec(site, dx.p, dy.p);
      dmrg::dev_d2h(y, dy.p, sizeof(double) * n, s);
    }
    dmrg::dev_sync(s);
    return DMRG_OK;
  });
}

int dmrg_energy(dmrg_ctx* c, int site, const double* x, double* energy, uintptr_t stream) {
  return guard(c, [&] {
    if (!x || !energy) return DMRG_EINVAL;
    wait_user(stream);
    const int64_t n = xsize(c, site);
    dmrg::Stream s = dev_stream(c);
    if (stream) {
      *energy = c->eng->rayleigh_fp64(site, x);
    } else {
      DevBuf dx(n, s);
      dmrg::dev_h2d(dx.p, x, sizeof(double) * n, s);
      *energy = c->eng->rayleigh_fp64(site, dx.p);
    }
    return DMRG_OK;
  });
}

int dmrg_heff_matvec_noalloc(dmrg_ctx* c, int site, const double* x, double* y, uintptr_t stream) {
  return guard(c, [&] {
    if (!x || !y || !c->stream) return DMRG_EINVAL;
    auto ck = [](cudaError_t e, const char* what) {
      if (e != cudaSuccess) throw std::runtime_error(std::string("cuda ") + what + ": " + cudaGetErrorString(e));
    };
    if (!c->tables) {
      ck(cudaEventCreateWithFlags(&c->tables, cudaEventDisableTiming), "event");
      ck(cudaEventCreateWithFlags(&c->noalloc_done, cudaEventDisableTiming), "event");
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the prepared tables were written on the context's stream: the caller's stream
    // waits for them on the device (no host synchronisation)
    ck(cudaEventRecord(c->tables, c->stream), "event record");
    ck(cudaStreamWaitEvent(s, c->tables, 0), "stream wait");
    c->eng->matvec_noalloc(site, x, y, (dmrg::Stream)s);
    ck(cudaEventRecord(c->noalloc_done, s), "event record");
    c->noalloc_pending = true;
    return DMRG_OK;
  });
}

int dmrg_rdm(dmrg_ctx* c, double* gamma, double* Gamma, uintptr_t stream) {
  return guard(c, [&] {
    if (!gamma || !Gamma) return DMRG_EINVAL;
    wait_user(stream);
    const int64_t L = c->eng->L();
    dmrg::Stream s = dev_stream(c);
    if (stream) {
      c->eng->rdm(gamma, Gamma);
    } else {
      DevBuf d1(L * L, s), d2(L * L * L * L, s);
      c->eng->rdm(d1.p, d2.p);
      dmrg::dev_d2h(gamma, d1.p, sizeof(double) * L * L, s);
      dmrg::dev_d2h(Gamma, d2.p, sizeof(double) * L * L * L * L, s);
    }
    dmrg::dev_sync(s);
    return DMRG_OK;
  });
}

int dmrg_push_excitation(dmrg_ctx* c, double eta) {
  return guard(c, [&] {
    dev_stream(c);
    c->eng->push_excitation(eta);
    dmrg::dev_sync(c->eng->stream());
    return DMRG_OK;
  });
}

int dmrg_clear_excitations(dmrg_ctx* c) {
  return guard(c, [&] {
    dev_stream(c);
    c->eng->clear_excitations();
    dmrg::dev_sync(c->eng->stream());
    return DMRG_OK;
  });
}

int dmrg_excitation_count(dmrg_ctx* c, int* count) {
  return guard(c, [&] {
    if (!count) return DMRG_EINVAL;
    *count = c->eng->n_excitations();
    return DMRG_OK;
  });
}

int dmrg_heff_diag(dmrg_ctx* c, int site, double* d, uintptr_t stream) {
  return guard(c, [&] {
    if (!d) return DMRG_EINVAL;
    wait_user(stream);
    const int64_t n = xsize(c, site);
    dmrg::Stream s = dev_stream(c);
    if (stream) {
      c->eng->diag(site, d);
    } else {
      DevBuf dd(n, s);
      c->eng->diag(site, dd.p);
      dmrg::dev_d2h(d, dd.p, sizeof(double) * n, s);
    }
    dmrg::dev_sync(s);
    return DMRG_OK;
  });
}

int dmrg_davidson(dmrg_ctx* c, int site, double* x, uintptr_t stream, double* energy, int* iters) {
  return guard(c, [&] {
    if (!x) return DMRG_EINVAL;
    wait_user(stream);
    const int64_t n = xsize(c, site);
    dmrg::Stream s = dev_stream(c);
    int it = 0;
    bool conv = false;
    double e;
    if (stream) {
      e = c->eng->davidson(site, x, &it, &conv);
    } else {
      DevBuf dx(n, s);
      dmrg::dev_h2d(dx.p, x, sizeof(double) * n, s);
      e = c->eng->davidson(site, dx.p, &it, &conv);
      dmrg::dev_d2h(x, dx.p, sizeof(double) * n, s);
    }
    dmrg::dev_sync(s);
    if (energy) *energy = e;
    if (iters) *iters = it;
    if (!conv) { c->err = "Davidson reached its iteration cap"; return DMRG_ENOTCONV; }
    return DMRG_OK;
  });
}

int dmrg_truncate(dmrg_ctx* c, int site, int dir, int D, double noise, const double* x,
                  uintptr_t stream, double* w_disc) {
  return guard(c, [&] {
    if (!x || (dir != 1 && dir != -1) || D < 1 || !(noise >= 0)) return DMRG_EINVAL;
    wait_user(stream);
    const int64_t n = xsize(c, site);
    dmrg::Stream s = dev_stream(c);
    DevBuf dx(n, s);
    if (stream) dmrg::dev_d2d(dx.p, x, sizeof(double) * n, s);
    else dmrg::dev_h2d(dx.p, x, sizeof(double) * n, s);
    if (noise > 0) dmrg::vec_add_noise(dx.p, n, noise, 0x7a11u + (uint64_t)site, s);
    double w = c->eng->truncate(site, dir, D, dx.p, noise);
    dmrg::dev_sync(s);
    if (w_disc) *w_disc = w;
    return DMRG_OK;
  });
}

int dmrg_set_next_site(dmrg_ctx* c, int site) {
  return guard(c, [&] {
    if (site < -1 || site > c->L - 2) return DMRG_EINVAL;
    c->eng->set_next_site(site);
    return DMRG_OK;
  });
}

int dmrg_update_operators(dmrg_ctx* c, int site, int dir) {
  return guard(c, [&] {
    if (dir != 1 && dir != -1) return DMRG_EINVAL;
    dmrg::Stream s = dev_stream(c);
    c->eng->update(site, dir);
    dmrg::dev_sync(s);
    return DMRG_OK;
  });
}

int dmrg_sweep_step(dmrg_ctx* c, int site, int dir, int D, double gamma, double* energy,
                    double* w_disc, int* iters) {
  return guard(c, [&] {
    if ((dir != 1 && dir != -1) || D < 1 || !(gamma >= 0)) return DMRG_EINVAL;
    dmrg::Stream s = dev_stream(c);
    double w = 0.0;
    int it = 0;
    bool conv = false;
    double e = c->eng->sweep_step(site, dir, D, gamma, &w, &it, &conv);
    dmrg::dev_sync(s);
    if (energy) *energy = e;
    if (w_disc) *w_disc = w;
    if (iters) *iters = it;
    if (!conv) { c->err = "Davidson reached its iteration cap"; return DMRG_ENOTCONV; }
    return DMRG_OK;
  });
}

int dmrg_stats(dmrg_ctx* c, dmrg_stats_t* out) {
  return guard(c, [&] {
    if (!out) return DMRG_EINVAL;
    const dmrg::Stats& s = c->eng->stats();
    out->matvecs = s.matvecs;
    out->davidson_iters = s.davidson_iters;
    out->micro_iters = s.micro_iters;
    out->matvec_flops = s.matvec_flops;
    out->last_matvec_flops = s.last_matvec_flops;
    out->last_matvec_tasks = s.last_matvec_tasks;
    out->t_update_ms = s.t_update_ms;
    out->t_trunc_ms = s.t_trunc_ms;
    out->t_plan_ms = s.t_plan_ms;
    out->t_total_ms = s.t_total_ms;
    out->last_w_disc = s.last_w_disc;
    out->max_w_disc = s.max_w_disc;
    out->k_phase1_ms = s.k_phase1_ms;
    out->k_phase2_ms = s.k_phase2_ms;
    out->k_launches = s.k_launches;
    out->k_phase1_flops = s.k_phase1_flops;
    out->k_phase2_flops = s.k_phase2_flops;
    out->kernels_launched = dmrg::kernel_launches();
    out->tc_matvecs = s.tc_matvecs;
    out->tc_flops = s.tc_flops;
    out->tc_phase1_ms = s.tc_phase1_ms;
    out->tc_phase2_ms = s.tc_phase2_ms;
    out->tc_phase1_flops = s.tc_phase1_flops;
    out->tc_phase2_flops = s.tc_phase2_flops;
    out->tc_phase1_bytes = s.tc_phase1_bytes;
    out->tc_phase2_bytes = s.tc_phase2_bytes;
    out->rdm_passes = s.rdm_passes;
    out->rdm_ms = s.rdm_ms;
    out->rdm_flops = s.rdm_flops;
    return DMRG_OK;
  });
}

int dmrg_test_tc_timeout(int on) {
  try {
    dmrg::tc_inject_timeout(on);
  } catch (...) {
    return DMRG_ECUDA;
  }
  return DMRG_OK;
}

int dmrg_set_device_memory_cap(size_t bytes) {
  dmrg::dev_set_cap(bytes);
  return DMRG_OK;
}

int dmrg_device_memory_in_use(size_t* bytes) {
  if (!bytes) return DMRG_EINVAL;
  *bytes = dmrg::dev_bytes_in_use();
  return DMRG_OK;
}

const char* dmrg_last_error(dmrg_ctx* c) { return c ? c->err.c_str() : "null context"; }

void dmrg_destroy(dmrg_ctx* c) {
  if (!c) return;
  if (c->noalloc_pending) cudaStreamWaitEvent(c->stream, c->noalloc_done, 0);
  delete c->eng;
  if (c->stream) cudaStreamDestroy(c->stream);
  if (c->tables) cudaEventDestroy(c->tables);
  if (c->noalloc_done) cudaEventDestroy(c->noalloc_done);
  delete c;
}

int dmrg_solve_history(dmrg_ctx* c, int* n, int* D, double* energy, double* w_disc) {
  return guard(c, [&] {
    if (!n || *n < 0) return DMRG_EINVAL;
    const auto& hd = c->eng->hist_D();
    const int m = std::min<int>(*n, (int)hd.size());
    for (int k = 0; k < m; ++k) {
      if (D) D[k] = hd[k];
      if (energy) energy[k] = c->eng->hist_E()[k];
      if (w_disc) w_disc[k] = c->eng->hist_w()[k];
    }
    *n = (int)hd.size();
    return DMRG_OK;
  });
}

int dmrg_extrapolate(const double* w_disc, const double* energy, int n, double* e_exact, double* c1) {
  if (!w_disc || !energy || n < 2 || !e_exact || !c1) return DMRG_EINVAL;
  // least squares of E = e_exact + c1 w (Eq. 16),
  // centred sums for accuracy
  double mw = 0.0, me = 0.0;
  for (int k = 0; k < n; ++k) {
    mw += w_disc[k];
    me += energy[k];
  }
  mw /= n;
  me /= n;
  double sww = 0.0, swe = 0.0;
  for (int k = 0; k < n; ++k) {
    sww += (w_disc[k] - mw) * (w_disc[k] - mw);
    swe += (w_disc[k] - mw) * (energy[k] - me);
  }
  if (!(sww > 0.0)) return DMRG_EINVAL;  // all discarded weights equal
  *c1 = swe / sww;
  *e_exact = me - *c1 * mw;
  return DMRG_OK;
}

// ---------------------------------------------------------------- batched matvecs

int dmrg_batch_create(dmrg_batch** out, dmrg_ctx* const* ctx, const int* site, int count, int autotune) {
  if (!out || !ctx || !site || count <= 0) return DMRG_EINVAL;
  *out = nullptr;
  for (int i = 0; i < count; ++i)
    if (!ctx[i]) return DMRG_EINVAL;
  dmrg_batch* b = new (std::nothrow) dmrg_batch;
  if (!b) return DMRG_ENOMEM;
  const int rc = guard_err(ctx[0]->err, [&] {
    // the tables of every context at the first candidate tile shape
    std::vector<dmrg::TcTune> cand;
    if (autotune) {
      for (int rt : {128, 64})
        for (int xc : {64, 32}) cand.push_back({rt, xc});
    } else {
      cand.push_back(dmrg::TcTune());
    }
    for (int i = 0; i < count; ++i) {
      dmrg_ctx* c = ctx[i];
      dmrg::Stream s = dev_stream(c);
      dmrg::Engine::TcView v = c->eng->prepare_tc(site[i], cand[0]);
      dmrg::dev_sync(s);
      b->ctx.push_back(c);
      b->site.push_back(site[i]);
      b->serial.push_back(v.serial);
      b->x.push_back(v.x);
      b->y.push_back(v.y);
      b->diag.push_back(v.diag);
      b->n.push_back(v.n);
      b->flops += v.flops;
    }
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) throw std::runtime_error("cuda stream");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const auto t0 = std::chrono::steady_clock::now();
    for (const dmrg::TcTune& t : cand) {
      // every candidate: each context's host tables for this tile shape, merged into one
      // launch; timed as the mean of three launches after a warm-up
      std::vector<const dmrg::TcHost*> hosts;
      for (int i = 0; i < count; ++i) hosts.push_back(ctx[i]->eng->prepare_tc(site[i], t).host);
      dmrg::TcPlan* p = dmrg::tc_plan_build(hosts, (dmrg::Stream)st);
      float ms = 0.0f;
      if (cand.size() > 1) {
        dmrg::tc_plan_launch(p, nullptr, (dmrg::Stream)st);
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r) dmrg::tc_plan_launch(p, nullptr, (dmrg::Stream)st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) throw std::runtime_error("cuda autotune sync");
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.0f;
      }
      if (!b->plan || ms < b->best_ms) {
        if (b->plan) dmrg::tc_plan_free(b->plan, (dmrg::Stream)st);
        b->plan = p;
        b->tune = t;
        b->best_ms = ms;
      } else {
        dmrg::tc_plan_free(p, (dmrg::Stream)st);
      }
    }
    b->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dmrg::dev_sync((dmrg::Stream)st);
    cudaStreamDestroy(st);
    for (int i = 0; i < count; ++i)
      if (ctx[i]->eng->tc_serial(site[i]) != b->serial[i])
        throw std::runtime_error("a context rebuilt its tables while the batch was made");
    if (dmrg::tc_error_flag((dmrg::Stream)cudaStreamLegacy)) throw std::runtime_error("cuda: tensor-core wait timed out");
    b->graph = dmrg::tc_graph_create(b->plan);
    return DMRG_OK;
  });
  if (rc != DMRG_OK) {
    dmrg_batch_destroy(b);
    return rc;
  }
  *out = b;
  return DMRG_OK;
}

int dmrg_batch_io(dmrg_batch* b, int i, double** x, double** y, int64_t* n) {
  if (!b || i < 0 || i >= (int)b->ctx.size()) return DMRG_EINVAL;
  if (x) *x = b->x[i];
  if (y) *y = b->y[i];
  if (n) *n = b->n[i];
  return DMRG_OK;
}

int dmrg_batch_run(dmrg_batch* b, const double* const* x, double* const* y, uintptr_t stream) {
  if (!b || !b->graph) return DMRG_EINVAL;
  return guard_err(b->err, [&] {
    for (size_t i = 0; i < b->ctx.size(); ++i)
      if (b->ctx[i]->eng->tc_serial(b->site[i]) != b->serial[i])
        throw std::invalid_argument("a context of the batch changed its tables since the batch was made");
    cudaStream_t s = stream ? (cudaStream_t)stream : cudaStreamLegacy;
    for (size_t i = 0; x && i < b->ctx.size(); ++i)
      if (x[i] && x[i] != b->x[i])
        if (cudaMemcpyAsync(b->x[i], x[i], sizeof(double) * b->n[i], cudaMemcpyDeviceToDevice, s) != cudaSuccess)
          throw std::runtime_error("cuda batch input copy");
    dmrg::tc_graph_launch(b->graph, (dmrg::Stream)s);
    for (size_t i = 0; y && i < b->ctx.size(); ++i)
      if (y[i] && y[i] != b->y[i])
        if (cudaMemcpyAsync(y[i], b->y[i], sizeof(double) * b->n[i], cudaMemcpyDeviceToDevice, s) != cudaSuccess)
          throw std::runtime_error("cuda batch output copy");
    return DMRG_OK;
  });
}

int dmrg_batch_davidson(dmrg_batch* b, double* const* x, double tol, int max_iter, int fp64_energy,
                        double* energy, int* iters, int* converged, uintptr_t stream) {
  if (!b || !b->graph || !x) return DMRG_EINVAL;
  return guard_err(b->err, [&] {
    const int K = (int)b->ctx.size();
    for (int i = 0; i < K; ++i) {
      if (!x[i]) throw std::invalid_argument("null vector");
      if (b->ctx[i]->eng->tc_serial(b->site[i]) != b->serial[i])
        throw std::invalid_argument("a context of the batch changed its tables since the batch was made");
    }
    cudaStream_t s = stream ? (cudaStream_t)stream : cudaStreamLegacy;
    std::vector<dmrg::BdInst> inst(K);
    for (int i = 0; i < K; ++i) inst[i] = {x[i], b->diag[i], b->x[i], b->y[i], b->n[i]};
    std::vector<dmrg::BdResult> res;
    int* flags = dmrg::tc_plan_active(b->plan);
    const std::vector<int> ones(K, 1);
    try {
      dmrg::batch_davidson(inst, tol, max_iter, [&] { dmrg::tc_graph_launch(b->graph, (dmrg::Stream)s); }, flags,
                           (dmrg::Stream)s, res);
    } catch (...) {
      dmrg::dev_h2d(flags, ones.data(), sizeof(int) * K, (dmrg::Stream)s);
      dmrg::dev_sync((dmrg::Stream)s);
      throw;
    }
    // later batched matvecs compute every instance again
    dmrg::dev_h2d(flags, ones.data(), sizeof(int) * K, (dmrg::Stream)s);
    dmrg::dev_sync((dmrg::Stream)s);
    if (dmrg::tc_error_flag((dmrg::Stream)s)) throw std::runtime_error("cuda: tensor-core wait timed out");
    bool all = true;
    for (int i = 0; i < K; ++i) {
      double e = res[i].theta;
      if (fp64_energy) {
        // the FP64 Rayleigh quotient of the Ritz vector through the context's own tables
        e = b->ctx[i]->eng->rayleigh_fp64(b->site[i], x[i]);
      }
      if (energy) energy[i] = e;
      if (iters) iters[i] = res[i].iters;
      if (converged) converged[i] = res[i].converged;
      all = all && res[i].converged;
    }
    if (!all) {
      b->err = "Davidson reached its iteration cap for some instance";
      return DMRG_ENOTCONV;
    }
    return DMRG_OK;
  });
}

int dmrg_batch_info(dmrg_batch* b, double* flops, int* row_tile, int* x_chunk, double* launch_ms,
                    double* tune_ms) {
  if (!b) return DMRG_EINVAL;
  if (flops) *flops = b->flops;
  if (row_tile) *row_tile = b->tune.row_tile;
  if (x_chunk) *x_chunk = b->tune.x_chunk;
  if (launch_ms) *launch_ms = b->best_ms;
  if (tune_ms) *tune_ms = b->tune_ms;
  return DMRG_OK;
}

const char* dmrg_batch_last_error(dmrg_batch* b) { return b ? b->err.c_str() : "null batch"; }

void dmrg_batch_destroy(dmrg_batch* b) {
  if (!b) return;
  try {
    if (b->graph) dmrg::tc_graph_free(b->graph);
    if (b->plan) {
      dmrg::tc_plan_free(b->plan, (dmrg::Stream)cudaStreamLegacy);
      dmrg::dev_sync((dmrg::Stream)cudaStreamLegacy);
    }
  } catch (...) {
  }
  delete b;
}

}  // extern "C"

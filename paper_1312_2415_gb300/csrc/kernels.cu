// FP64 kernels of the two-site sweep (sm_103a).  Every launch executes a table built
// by the host planner; no kernel waits on another block or on another launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <stdexcept>
#include <string>
#include <unordered_map>

#include "device.hpp"
#include "plans.hpp"

namespace dmrg {

namespace {

thread_local std::string g_err;
int64_t g_launches = 0;  // kernels launched by this library (all contexts)

inline cudaStream_t S(Stream s) { return (cudaStream_t)s; }

inline void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    throw std::runtime_error(g_err);
  }
}

inline int nblk(int64_t n, int t) { return (int)std::min<int64_t>((n + t - 1) / t, 65535 * 8); }

}  // namespace

// ------------------------------------------------------------------ memory

// Device bytes the library holds (all contexts), and an optional cap on them: an
// allocation that would pass the cap fails on the host with std::bad_alloc (reported as
// DMRG_ENOMEM) before any CUDA call is made.
namespace {
std::mutex g_mem_mu;
std::unordered_map<void*, size_t> g_mem_live;
size_t g_mem_in_use = 0, g_mem_cap = 0;
}  // namespace

void* dev_alloc(size_t bytes, Stream s) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    if (g_mem_cap && g_mem_in_use + bytes > g_mem_cap) throw std::bad_alloc();
    g_mem_in_use += bytes;  // reserved before the call, released if it fails
  }
  cudaError_t e = cudaMallocAsync(&p, bytes, S(s));
  std::lock_guard<std::mutex> lk(g_mem_mu);
  if (e != cudaSuccess) {
    g_mem_in_use -= bytes;
    ck(e, "cudaMallocAsync");
  }
  g_mem_live[p] = bytes;
  return p;
}
void dev_free(void* p, Stream s) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    auto it = g_mem_live.find(p);
    if (it != g_mem_live.end()) {
      g_mem_in_use -= it->second;
      g_mem_live.erase(it);
    }
  }
  ck(cudaFreeAsync(p, S(s)), "cudaFreeAsync");
}
size_t dev_bytes_in_use() {
  std::lock_guard<std::mutex> lk(g_mem_mu);
  return g_mem_in_use;
}
void dev_set_cap(size_t bytes) {
  std::lock_guard<std::mutex> lk(g_mem_mu);
  g_mem_cap = bytes;
}
void dev_h2d(void* d, const void* h, size_t b, Stream s) {
  if (b) ck(cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, S(s)), "h2d");
}
void dev_d2h(void* h, const void* d, size_t b, Stream s) {
  if (b) ck(cudaMemcpyAsync(h, d, b, cudaMemcpyDeviceToHost, S(s)), "d2h");
}
void dev_d2d(void* d, const void* x, size_t b, Stream s) {
  if (b) ck(cudaMemcpyAsync(d, x, b, cudaMemcpyDeviceToDevice, S(s)), "d2d");
}
void dev_zero(void* p, size_t b, Stream s) {
  if (b) ck(cudaMemsetAsync(p, 0, b, S(s)), "memset");
}
void dev_sync(Stream s) { ck(cudaStreamSynchronize(S(s)), "stream sync"); }
int64_t kernel_launches() { return g_launches; }
void note_launches(int64_t k) { g_launches += k; }
int dev_check(const char** msg) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return 0;
  g_err = cudaGetErrorString(e);
  if (msg) *msg = g_err.c_str();
  return (int)e;
}
void* host_pinned_alloc(size_t b) {
  void* p = nullptr;
  ck(cudaMallocHost(&p, b ? b : 16), "cudaMallocHost");
  return p;
}
void host_pinned_free(void* p) {
  if (p) cudaFreeHost(p);
}
void* event_create() {
  cudaEvent_t e;
  ck(cudaEventCreate(&e), "cudaEventCreate");
  return (void*)e;
}
void event_destroy(void* e) {
  if (e) cudaEventDestroy((cudaEvent_t)e);
}
void event_record(void* e, Stream s) { ck(cudaEventRecord((cudaEvent_t)e, S(s)), "cudaEventRecord"); }
Stream stream_create() {
  cudaStream_t s;
  ck(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate");
  return (Stream)s;
}
void stream_destroy(Stream s) {
  if (s) cudaStreamDestroy(S(s));
}
void stream_wait(Stream s, void* ev) { ck(cudaStreamWaitEvent(S(s), (cudaEvent_t)ev, 0), "cudaStreamWaitEvent"); }
void event_sync(void* ev) { ck(cudaEventSynchronize((cudaEvent_t)ev), "cudaEventSynchronize"); }
float event_elapsed_ms(void* a, void* b) {
  float ms = 0.f;
  ck(cudaEventSynchronize((cudaEvent_t)b), "cudaEventSynchronize");
  ck(cudaEventElapsedTime(&ms, (cudaEvent_t)a, (cudaEvent_t)b), "cudaEventElapsedTime");
  return ms;
}

// ------------------------------------------------------------------ grouped GEMM

namespace {
constexpr int BM = 32, BN = 32, BK = 16;

__global__ void __launch_bounds__(256) k_grouped_gemm(const GemmTask* __restrict__ tasks,
                                                     const GemmGroup* __restrict__ groups,
                                                     int ngroups) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tile = blockIdx.x;
  int lo = 0, hi = ngroups - 1;
  while (lo < hi) {  // last group with tile_begin <= tile
    int mid = (lo + hi + 1) >> 1;
    if (groups[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
  }
  const GemmGroup g = groups[lo];
  const int local = tile - g.tile_begin;
  const int tn = (g.n + BN - 1) / BN;
  const int row0 = (local / tn) * BM, col0 = (local % tn) * BN;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int t = g.task_begin; t < g.task_end; ++t) {
    const GemmTask T = tasks[t];
    if (T.A == nullptr) {  // op(A) = identity: C += alpha op(B)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
          if (r < g.m && c < g.n)
            acc[i][j] += T.alpha * (T.transB ? T.B[(size_t)c * T.ldb + r] : T.B[(size_t)r * T.ldb + c]);
        }
      continue;
    }
    for (int k0 = 0; k0 < T.k; k0 += BK) {
      for (int e = tid; e < BM * BK; e += 256) {
        int r, kk;
        double v = 0.0;
        if (T.transA) { kk = e / BM; r = e % BM; } else { r = e / BK; kk = e % BK; }
        int gr = row0 + r, gk = k0 + kk;
        if (gr < g.m && gk < T.k)
          v = T.transA ? T.A[(size_t)gk * T.lda + gr] : T.A[(size_t)gr * T.lda + gk];
        As[kk][r] = v * T.alpha;
      }
      for (int e = tid; e < BK * BN; e += 256) {
        int c, kk;
        double v = 0.0;
        if (T.transB) { c = e / BK; kk = e % BK; } else { kk = e / BN; c = e % BN; }
        int gc = col0 + c, gk = k0 + kk;
        if (gc < g.n && gk < T.k)
          v = T.transB ? T.B[(size_t)gc * T.ldb + gk] : T.B[(size_t)gk * T.ldb + gc];
        Bs[kk][c] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double a0 = As[kk][ty], a1 = As[kk][ty + 16];
        double b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
        acc[0][0] = fma(a0, b0, acc[0][0]);
        acc[0][1] = fma(a0, b1, acc[0][1]);
        acc[1][0] = fma(a1, b0, acc[1][0]);
        acc[1][1] = fma(a1, b1, acc[1][1]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
      if (r < g.m && c < g.n) g.C[(size_t)r * g.ldc + c] += acc[i][j];
    }
}
}  // namespace

GemmPlan* gemm_plan_upload(const std::vector<GemmTask>& t, std::vector<GemmGroup>& g, Stream s) {
  GemmPlan* p = new GemmPlan;
  int tiles = 0;
  for (auto& gr : g) {
    gr.tile_begin = tiles;
    if (gr.m > 0 && gr.n > 0) tiles += ((gr.m + BM - 1) / BM) * ((gr.n + BN - 1) / BN);
  }
  p->ngroups = (int)g.size();
  p->ntiles = tiles;
  p->ntasks = (int64_t)t.size();
  if (!t.empty()) {
    p->tasks = (GemmTask*)dev_alloc(t.size() * sizeof(GemmTask), s);
    dev_h2d(p->tasks, t.data(), t.size() * sizeof(GemmTask), s);
  }
  if (!g.empty()) {
    p->groups = (GemmGroup*)dev_alloc(g.size() * sizeof(GemmGroup), s);
    dev_h2d(p->groups, g.data(), g.size() * sizeof(GemmGroup), s);
  }
  return p;
}

void gemm_plan_run(const GemmPlan* p, Stream s) {
  if (!p || p->ntiles == 0) return;
  k_grouped_gemm<<<p->ntiles, 256, 0, S(s)>>>(p->tasks, p->groups, p->ngroups);
  ++g_launches;
  ck(cudaGetLastError(), "grouped_gemm launch");
}

void gemm_plan_free(GemmPlan* p, Stream s) {
  if (!p) return;
  dev_free(p->tasks, s);
  dev_free(p->groups, s);
  delete p;
}

int64_t gemm_plan_tasks(const GemmPlan* p) { return p ? p->ntasks : 0; }

// ------------------------------------------------------------------ combine

namespace {
__global__ void k_combine(const CombSrc* __restrict__ src, const CombDst* __restrict__ dst) {
  const CombDst d = dst[blockIdx.x];
  const int64_t n = (int64_t)d.rows * d.cols;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    int r = (int)(e / d.cols), c = (int)(e % d.cols);
    double v = d.accumulate ? d.dst[(size_t)r * d.ld + c] : 0.0;
    for (int s = d.src_begin; s < d.src_end; ++s) v += src[s].alpha * src[s].src[(size_t)r * src[s].ld + c];
    d.dst[(size_t)r * d.ld + c] = v;
  }
}
}  // namespace

CombPlan* comb_plan_upload(const std::vector<CombSrc>& s, const std::vector<CombDst>& d, Stream st) {
  CombPlan* p = new CombPlan;
  p->ndst = (int)d.size();
  if (!s.empty()) {
    p->src = (CombSrc*)dev_alloc(s.size() * sizeof(CombSrc), st);
    dev_h2d(p->src, s.data(), s.size() * sizeof(CombSrc), st);
  }
  if (!d.empty()) {
    p->dst = (CombDst*)dev_alloc(d.size() * sizeof(CombDst), st);
    dev_h2d(p->dst, d.data(), d.size() * sizeof(CombDst), st);
  }
  return p;
}

void comb_plan_run(const CombPlan* p, Stream s) {
  if (!p || p->ndst == 0) return;
  for (int off = 0; off < p->ndst; off += 65535) {
    int n = std::min(65535, p->ndst - off);
    k_combine<<<n, 128, 0, S(s)>>>(p->src, p->dst + off);
    ++g_launches;
  }
  ck(cudaGetLastError(), "combine launch");
}

void comb_plan_free(CombPlan* p, Stream s) {
  if (!p) return;
  dev_free(p->src, s);
  dev_free(p->dst, s);
  delete p;
}

// ------------------------------------------------------------------ diagonal

namespace {
__global__ void k_diag(const DiagTerm* __restrict__ t, const DiagOut* __restrict__ o) {
  const DiagOut d = o[blockIdx.x];
  const int64_t n = (int64_t)d.dL * d.dR;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    int a = (int)(e / d.dR), b = (int)(e % d.dR);
    double v = d.out[e];
    for (int s = d.term_begin; s < d.term_end; ++s)
      v += t[s].coef * t[s].C[(size_t)a * t[s].ldc + a] * t[s].D[(size_t)b * t[s].ldd + b];
    d.out[e] = v;
  }
}
}  // namespace

DiagPlan* diag_plan_upload(const std::vector<DiagTerm>& t, const std::vector<DiagOut>& o, Stream s) {
  DiagPlan* p = new DiagPlan;
  p->n = (int)o.size();
  if (!t.empty()) {
    p->t = (DiagTerm*)dev_alloc(t.size() * sizeof(DiagTerm), s);
    dev_h2d(p->t, t.data(), t.size() * sizeof(DiagTerm), s);
  }
  if (!o.empty()) {
    p->o = (DiagOut*)dev_alloc(o.size() * sizeof(DiagOut), s);
    dev_h2d(p->o, o.data(), o.size() * sizeof(DiagOut), s);
  }
  return p;
}

void diag_plan_run(const DiagPlan* p, Stream s) {
  if (!p || p->n == 0) return;
  for (int off = 0; off < p->n; off += 65535) {
    int n = std::min(65535, p->n - off);
    k_diag<<<n, 128, 0, S(s)>>>(p->t, p->o + off);
    ++g_launches;
  }
  ck(cudaGetLastError(), "diag launch");
}

void diag_plan_free(DiagPlan* p, Stream s) {
  if (!p) return;
  dev_free(p->t, s);
  dev_free(p->o, s);
  delete p;
}

// ------------------------------------------------------------------ grouped Frobenius products

namespace {
// one CTA per group: the threads stride over every element of every task of the group,
// then a block reduction; the group's output is written by this CTA only
__global__ void __launch_bounds__(256) k_dot_grouped(const DotTask* __restrict__ t,
                                                    const DotGroup* __restrict__ g) {
  const DotGroup G = g[blockIdx.x];
  double s = 0.0;
  for (int k = G.task_begin; k < G.task_end; ++k) {
    const DotTask T = t[k];
    const int64_t ne = (int64_t)T.rows * T.cols;
    double u = 0.0;
    for (int64_t e = threadIdx.x; e < ne; e += blockDim.x) {
      const int r = (int)(e / T.cols), c = (int)(e % T.cols);
      u = fma(T.A[(size_t)r * T.lda + c], T.B[(size_t)r * T.ldb + c], u);
    }
    s = fma(T.alpha, u, s);
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *G.out += sh[0];
}

// Gamma_ijkl = 2 x mean of dg over (ijkl), (jilk), (klij), (lkji), (kjil), (ilkj), (lijk), (jkli)
__global__ void k_rdm2(const double* __restrict__ dg, int L, double* __restrict__ Gamma) {
  const int64_t L4 = (int64_t)L * L * L * L;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < L4; e += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(e % L), k = (int)(e / L % L), j = (int)(e / L / L % L), i = (int)(e / L / L / L);
    auto at = [&](int a, int b, int c, int d) { return dg[(((int64_t)a * L + b) * L + c) * L + d]; };
    const double s = at(i, j, k, l) + at(j, i, l, k) + at(k, l, i, j) + at(l, k, j, i) + at(k, j, i, l) +
                     at(i, l, k, j) + at(l, i, j, k) + at(j, k, l, i);
    Gamma[e] = 0.25 * s;
  }
}

__global__ void k_rdm1(const double* __restrict__ Gamma, int L, int N, double* __restrict__ gamma) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * L) return;
  const int i = e / L, k = e % L;
  double s = 0.0;
  for (int j = 0; j < L; ++j) s += Gamma[(((int64_t)i * L + j) * L + k) * L + j];
  gamma[e] = s / (N - 1);
}
}  // namespace

void dot_grouped(const std::vector<DotTask>& t, const std::vector<DotGroup>& g, Stream s) {
  if (g.empty()) return;
  DotTask* dt = (DotTask*)dev_alloc(std::max<size_t>(t.size(), 1) * sizeof(DotTask), s);
  DotGroup* dgp = (DotGroup*)dev_alloc(g.size() * sizeof(DotGroup), s);
  if (!t.empty()) dev_h2d(dt, t.data(), t.size() * sizeof(DotTask), s);
  dev_h2d(dgp, g.data(), g.size() * sizeof(DotGroup), s);
  for (size_t off = 0; off < g.size(); off += 65535) {
    const int n = (int)std::min<size_t>(65535, g.size() - off);
    k_dot_grouped<<<n, 256, 0, S(s)>>>(dt, dgp + off);
    ++g_launches;
  }
  ck(cudaGetLastError(), "dot launch");
  dev_free(dt, s);
  dev_free(dgp, s);
}

void rdm_finish(const double* dg, int L, int N, double* gamma, double* Gamma, Stream s) {
  const int64_t L4 = (int64_t)L * L * L * L;
  k_rdm2<<<(int)std::min<int64_t>((L4 + 255) / 256, 4096), 256, 0, S(s)>>>(dg, L, Gamma);
  k_rdm1<<<(L * L + 255) / 256, 256, 0, S(s)>>>(Gamma, L, N, gamma);
  g_launches += 2;
  ck(cudaGetLastError(), "rdm launch");
}

// ------------------------------------------------------------------ vector kernels

namespace {
constexpr int kDotChunk = 4096;
constexpr int kMaxChunks = 512;

__global__ void k_multidot_partial(const double* __restrict__ V, int64_t ldv,
                                   const double* __restrict__ w, int64_t n, int nch,
                                   double* __restrict__ part) {
  __shared__ double sh[256];
  const int j = blockIdx.y, c = blockIdx.x;
  const double* v = V + (size_t)j * ldv;
  double s = 0.0;
  for (int64_t i = (int64_t)c * 256 + threadIdx.x; i < n; i += (int64_t)nch * 256) s += v[i] * w[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)j * nch + c] = sh[0];
}

__global__ void k_multidot_final(const double* __restrict__ part, int nch, int m, double* out) {
  const int j = blockIdx.x;
  __shared__ double sh[256];
  double s = 0.0;
  for (int c = threadIdx.x; c < nch; c += 256) s += part[(size_t)j * nch + c];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = sh[0];
}

__global__ void k_vec_combine(const double* __restrict__ V, int64_t ldv, int m,
                              const double* __restrict__ c, double beta, double* __restrict__ y,
                              int64_t n) {
  __shared__ double cs[128];
  for (int j = threadIdx.x; j < m; j += blockDim.x) cs[j] = c[j];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = beta == 0.0 ? 0.0 : beta * y[i];
    for (int j = 0; j < m; ++j) s += cs[j] * V[(size_t)j * ldv + i];
    y[i] = s;
  }
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y,
                        int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

__global__ void k_normalize(double* __restrict__ y, const double* __restrict__ nrm2, int64_t n) {
  double s = *nrm2 > 0.0 ? 1.0 / sqrt(*nrm2) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] *= s;
}

__global__ void k_precondition(const double* __restrict__ r, const double* __restrict__ d,
                               const double* __restrict__ theta, double* __restrict__ t,
                               int64_t n) {
  const double th = *theta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double den = th - d[i];
    if (fabs(den) < 1e-12) den = den < 0 ? -1e-12 : 1e-12;
    t[i] = r[i] / den;
  }
}

__device__ inline void sym_schur2(double app, double aqq, double apq, double& c, double& s) {
  if (apq == 0.0) { c = 1.0; s = 0.0; return; }
  double th = (aqq - app) / (2.0 * apq);
  double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
  c = 1.0 / sqrt(1.0 + t * t);
  s = t * c;
}

// one CTA: Jacobi on an m x m symmetric matrix in shared memory (m <= 48)
__device__ void small_eig_block(const double* __restrict__ G, int gld, int m, int k,
                                double* __restrict__ theta, double* __restrict__ C) {
  __shared__ double A[48][49];
  __shared__ double Q[48][49];
  __shared__ double cs[32], sn[32];
  __shared__ int pp[32], qq[32];
  __shared__ double off_s;
  __shared__ int order[48];
  const int tid = threadIdx.x;
  for (int e = tid; e < m * m; e += blockDim.x) {
    int i = e / m, j = e % m;
    A[i][j] = i >= j ? G[(size_t)i * gld + j] : G[(size_t)j * gld + i];  // lower triangle
    Q[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int np = (m + 1) & ~1;
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) {
      double off = 0.0, tot = 0.0;
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
          tot += A[i][j] * A[i][j];
          if (i != j) off += A[i][j] * A[i][j];
        }
      off_s = (off <= 1e-30 * tot || off == 0.0) ? -1.0 : off;
    }
    __syncthreads();
    if (off_s < 0.0) break;
    for (int step = 0; step < np - 1; ++step) {
      if (tid < np / 2) {
        // round-robin pairing: position 0 fixed, others rotate
        int a = tid, b = np - 1 - tid;
        auto pos = [&](int x) { return x == 0 ? 0 : 1 + (x - 1 + step) % (np - 1); };
        int p = pos(a), q = pos(b);
        if (p > q) { int t = p; p = q; q = t; }
        pp[tid] = p; qq[tid] = q;
        if (q < m) sym_schur2(A[p][p], A[q][q], A[p][q], cs[tid], sn[tid]);
        else { cs[tid] = 1.0; sn[tid] = 0.0; }
      }
      __syncthreads();
      for (int e = tid; e < (np / 2) * m; e += blockDim.x) {
        int r = e / m, j = e % m;
        int p = pp[r], q = qq[r];
        if (q >= m) continue;
        double c = cs[r], s = sn[r];
        double ap = A[p][j], aq = A[q][j];
        A[p][j] = c * ap - s * aq;
        A[q][j] = s * ap + c * aq;
      }
      __syncthreads();
      for (int e = tid; e < (np / 2) * m; e += blockDim.x) {
        int r = e / m, i = e % m;
        int p = pp[r], q = qq[r];
        if (q >= m) continue;
        double c = cs[r], s = sn[r];
        double ap = A[i][p], aq = A[i][q];
        A[i][p] = c * ap - s * aq;
        A[i][q] = s * ap + c * aq;
        double qp = Q[i][p], qv = Q[i][q];
        Q[i][p] = c * qp - s * qv;
        Q[i][q] = s * qp + c * qv;
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    for (int i = 0; i < m; ++i) order[i] = i;
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j)
        if (A[order[j]][order[j]] < A[order[i]][order[i]]) { int t = order[i]; order[i] = order[j]; order[j] = t; }
  }
  __syncthreads();
  for (int e = tid; e < k * m; e += blockDim.x) {
    int v = e / m, i = e % m;
    C[(size_t)v * m + i] = Q[i][order[v]];
  }
  if (tid < k) theta[tid] = A[order[tid]][order[tid]];
}

__global__ void k_small_eig(const double* __restrict__ G, int gld, int m, int k,
                            double* __restrict__ theta, double* __restrict__ C) {
  small_eig_block(G, gld, m, k, theta, C);
}

// ---- grouped Davidson kernels: one launch per operation over all instances of a batch
// (blockIdx.y or blockIdx.x = instance); instances with act[i] == 0 are skipped.

__device__ __forceinline__ double* bd_pick(const BdSlot& s, int which, int col) {
  switch (which) {
    case BD_V: return s.V + (int64_t)col * s.n;
    case BD_AV: return s.AV + (int64_t)col * s.n;
    case BD_R: return s.r;
    case BD_T: return s.t;
    case BD_X: return s.x;
    case BD_X0: return s.x0;
    case BD_TMP: return s.tmp + (int64_t)col * s.n;
    case BD_BX: return s.bx;
    default: return s.by;
  }
}

// part[(j nch + c)] = partial sums of <A col (a_col + j), B>, j < m (grid: nch x m x count)
__global__ void k_bd_dots_partial(const BdSlot* __restrict__ sl, const int* __restrict__ act, int aw, int a_col,
                                  int bw, int b_col, int nch) {
  __shared__ double sh[256];
  const int i = blockIdx.z, j = blockIdx.y, c = blockIdx.x;
  if (!act[i]) return;
  const BdSlot s = sl[i];
  const double* a = bd_pick(s, aw, a_col + j);
  const double* b = bd_pick(s, bw, b_col);
  double v = 0.0;
  for (int64_t e = (int64_t)c * 256 + threadIdx.x; e < s.n; e += (int64_t)nch * 256) v += a[e] * b[e];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) s.part[(size_t)j * nch + c] = sh[0];
}

// out[j] = sum of the partials; out = G + row * mmax (to_g) or dots (grid: m x count)
__global__ void k_bd_dots_final(const BdSlot* __restrict__ sl, const int* __restrict__ act, int nch, int to_g,
                                int row, int mmax) {
  __shared__ double sh[256];
  const int i = blockIdx.y, j = blockIdx.x;
  if (!act[i]) return;
  const BdSlot s = sl[i];
  double v = 0.0;
  for (int c = threadIdx.x; c < nch; c += 256) v += s.part[(size_t)j * nch + c];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) (to_g ? s.G + (size_t)row * mmax : s.dots)[j] = sh[0];
}

// y = beta y + sum_j c[j] V col j, c = C + cv * m (from_c) or dots
__global__ void k_bd_combine(const BdSlot* __restrict__ sl, const int* __restrict__ act, int vw, int m, int from_c,
                             int cv, double beta, int yw, int y_col) {
  __shared__ double cs[64];
  const int i = blockIdx.y;
  if (!act[i]) return;
  const BdSlot s = sl[i];
  const double* c = from_c ? s.C + (size_t)cv * m : s.dots;
  for (int j = threadIdx.x; j < m; j += blockDim.x) cs[j] = c[j];
  __syncthreads();
  const double* V = bd_pick(s, vw, 0);
  double* y = bd_pick(s, yw, y_col);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < s.n; e += (int64_t)gridDim.x * blockDim.x) {
    double v = beta == 0.0 ? 0.0 : beta * y[e];
    for (int j = 0; j < m; ++j) v += cs[j] * V[(size_t)j * s.n + e];
    y[e] = v;
  }
}

// y = a x + b y; a = -theta[0] when a_theta
__global__ void k_bd_axpby(const BdSlot* __restrict__ sl, const int* __restrict__ act, int a_theta, double a, int xw,
                           int x_col, double b, int yw, int y_col) {
  const int i = blockIdx.y;
  if (!act[i]) return;
  const BdSlot s = sl[i];
  const double av = a_theta ? -s.th[0] : a;
  const double* x = bd_pick(s, xw, x_col);
  double* y = bd_pick(s, yw, y_col);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < s.n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = av * x[e] + (b == 0.0 ? 0.0 : b * y[e]);
}

// y /= sqrt(dots[0])
__global__ void k_bd_normalize(const BdSlot* __restrict__ sl, const int* __restrict__ act, int yw, int y_col) {
  const int i = blockIdx.y;
  if (!act[i]) return;
  const BdSlot s = sl[i];
  const double sc = s.dots[0] > 0.0 ? 1.0 / sqrt(s.dots[0]) : 0.0;
  double* y = bd_pick(s, yw, y_col);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < s.n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] *= sc;
}

// t = r / (theta[0] - diag), |denominator| floored as in the single-instance kernel
__global__ void k_bd_precondition(const BdSlot* __restrict__ sl, const int* __restrict__ act) {
  const int i = blockIdx.y;
  if (!act[i]) return;
  const BdSlot s = sl[i];
  const double th = s.th[0];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < s.n; e += (int64_t)gridDim.x * blockDim.x) {
    double den = th - s.diag[e];
    if (fabs(den) < 1e-12) den = den < 0 ? -1e-12 : 1e-12;
    s.t[e] = s.r[e] / den;
  }
}

__global__ void k_bd_small_eig(const BdSlot* __restrict__ sl, const int* __restrict__ act, int mmax, int m, int k) {
  const int i = blockIdx.x;
  if (!act[i]) return;
  const BdSlot s = sl[i];
  small_eig_block(s.G, mmax, m, k, s.th, s.C);
}

// restart: G = diag(theta[0..k)) (zero elsewhere)
__global__ void k_bd_restart_g(const BdSlot* __restrict__ sl, const int* __restrict__ act, int mmax, int k) {
  const int i = blockIdx.x;
  if (!act[i]) return;
  const BdSlot s = sl[i];
  for (int e = threadIdx.x; e < mmax * mmax; e += blockDim.x) {
    const int r = e / mmax, c = e % mmax;
    s.G[e] = (r == c && r < k) ? s.th[r] : 0.0;
  }
}

__global__ void k_bd_gather(const BdSlot* __restrict__ sl, int count, double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    out[2 * i] = sl[i].th[0];
    out[2 * i + 1] = sl[i].dots[0];
  }
}

// x = -x where <x, x0> (dots[0]) < 0
__global__ void k_bd_sign(const BdSlot* __restrict__ sl, const int* __restrict__ act) {
  const int i = blockIdx.y;
  if (!act[i]) return;
  const BdSlot s = sl[i];
  if (!(s.dots[0] < 0.0)) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < s.n; e += (int64_t)gridDim.x * blockDim.x)
    s.x[e] = -s.x[e];
}

__device__ inline uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_noise(double* x, int64_t n, double amp, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t u = splitmix(seed + (uint64_t)i) >> 11;
    double r = (double)u * (2.0 / 9007199254740992.0) - 1.0;
    x[i] += amp * r;
  }
}
}  // namespace

void vec_multidot(const double* V, int64_t ldv, int m, const double* w, int64_t n, double* out,
                  double* scratch, Stream s) {
  if (m <= 0) return;
  int nch = (int)std::min<int64_t>(kMaxChunks, std::max<int64_t>(1, (n + kDotChunk - 1) / kDotChunk));
  dim3 grid(nch, m);
  k_multidot_partial<<<grid, 256, 0, S(s)>>>(V, ldv, w, n, nch, scratch);
  ++g_launches;
  k_multidot_final<<<m, 256, 0, S(s)>>>(scratch, nch, m, out);
  ++g_launches;
  ck(cudaGetLastError(), "multidot");
}

void vec_combine(const double* V, int64_t ldv, int m, const double* c, double beta, double* y,
                 int64_t n, Stream s) {
  k_vec_combine<<<nblk(n, 256), 256, 0, S(s)>>>(V, ldv, m, c, beta, y, n);
  ++g_launches;
  ck(cudaGetLastError(), "vec_combine");
}

void vec_axpby(double a, const double* x, double b, double* y, int64_t n, Stream s) {
  k_axpby<<<nblk(n, 256), 256, 0, S(s)>>>(a, x, b, y, n);
  ++g_launches;
  ck(cudaGetLastError(), "axpby");
}

void vec_normalize(double* y, const double* nrm2, int64_t n, Stream s) {
  k_normalize<<<nblk(n, 256), 256, 0, S(s)>>>(y, nrm2, n);
  ++g_launches;
  ck(cudaGetLastError(), "normalize");
}

void vec_precondition(const double* r, const double* d, const double* th, double* t, int64_t n,
                      Stream s) {
  k_precondition<<<nblk(n, 256), 256, 0, S(s)>>>(r, d, th, t, n);
  ++g_launches;
  ck(cudaGetLastError(), "precondition");
}

namespace {
inline int bd_blocks(int64_t nmax, int count) {
  // enough CTAs per instance to fill the GPU a few times over, no more than the data needs
  const int per = (int)std::max<int64_t>(1, std::min<int64_t>((nmax + 255) / 256, std::max(1, 2048 / std::max(count, 1))));
  return per;
}
}  // namespace

void bd_dots(const BdSlot* sl, const int* act, int count, int64_t nmax, int aw, int a_col, int m, int bw, int b_col,
             int to_g, int row, int mmax, Stream s) {
  if (m <= 0 || count <= 0) return;
  const int nch = (int)std::min<int64_t>(kBdChunks, std::max<int64_t>(1, (nmax + 256 * 8 - 1) / (256 * 8)));
  k_bd_dots_partial<<<dim3(nch, m, count), 256, 0, S(s)>>>(sl, act, aw, a_col, bw, b_col, nch);
  ++g_launches;
  k_bd_dots_final<<<dim3(m, count), 256, 0, S(s)>>>(sl, act, nch, to_g, row, mmax);
  ++g_launches;
  ck(cudaGetLastError(), "grouped dots");
}

void bd_combine(const BdSlot* sl, const int* act, int count, int64_t nmax, int vw, int m, int from_c, int cv,
                double beta, int yw, int y_col, Stream s) {
  if (count <= 0) return;
  k_bd_combine<<<dim3(bd_blocks(nmax, count), count), 256, 0, S(s)>>>(sl, act, vw, m, from_c, cv, beta, yw, y_col);
  ++g_launches;
  ck(cudaGetLastError(), "grouped combine");
}

void bd_axpby(const BdSlot* sl, const int* act, int count, int64_t nmax, int a_theta, double a, int xw, int x_col,
              double b, int yw, int y_col, Stream s) {
  if (count <= 0) return;
  k_bd_axpby<<<dim3(bd_blocks(nmax, count), count), 256, 0, S(s)>>>(sl, act, a_theta, a, xw, x_col, b, yw, y_col);
  ++g_launches;
  ck(cudaGetLastError(), "grouped axpby");
}

void bd_normalize(const BdSlot* sl, const int* act, int count, int64_t nmax, int yw, int y_col, Stream s) {
  if (count <= 0) return;
  k_bd_normalize<<<dim3(bd_blocks(nmax, count), count), 256, 0, S(s)>>>(sl, act, yw, y_col);
  ++g_launches;
  ck(cudaGetLastError(), "grouped normalize");
}

void bd_precondition(const BdSlot* sl, const int* act, int count, int64_t nmax, Stream s) {
  if (count <= 0) return;
  k_bd_precondition<<<dim3(bd_blocks(nmax, count), count), 256, 0, S(s)>>>(sl, act);
  ++g_launches;
  ck(cudaGetLastError(), "grouped precondition");
}

void bd_small_eig(const BdSlot* sl, const int* act, int count, int mmax, int m, int k, Stream s) {
  if (count <= 0) return;
  k_bd_small_eig<<<count, 256, 0, S(s)>>>(sl, act, mmax, m, k);
  ++g_launches;
  ck(cudaGetLastError(), "grouped small eig");
}

void bd_restart_g(const BdSlot* sl, const int* act, int count, int mmax, int k, Stream s) {
  if (count <= 0) return;
  k_bd_restart_g<<<count, 256, 0, S(s)>>>(sl, act, mmax, k);
  ++g_launches;
  ck(cudaGetLastError(), "grouped restart");
}

void bd_gather(const BdSlot* sl, int count, double* out, Stream s) {
  if (count <= 0) return;
  k_bd_gather<<<(count + 127) / 128, 128, 0, S(s)>>>(sl, count, out);
  ++g_launches;
  ck(cudaGetLastError(), "grouped gather");
}

void bd_sign(const BdSlot* sl, const int* act, int count, int64_t nmax, Stream s) {
  if (count <= 0) return;
  k_bd_sign<<<dim3(bd_blocks(nmax, count), count), 256, 0, S(s)>>>(sl, act);
  ++g_launches;
  ck(cudaGetLastError(), "grouped sign");
}

void small_eig(const double* G, int gld, int m, int k, double* theta, double* C, Stream s) {
  k_small_eig<<<1, 256, 0, S(s)>>>(G, gld, m, k, theta, C);
  ++g_launches;
  ck(cudaGetLastError(), "small_eig");
}

void vec_add_noise(double* x, int64_t n, double amp, uint64_t seed, Stream s) {
  k_noise<<<nblk(n, 256), 256, 0, S(s)>>>(x, n, amp, seed);
  ++g_launches;
  ck(cudaGetLastError(), "noise");
}

// ------------------------------------------------------------------ batched Jacobi

namespace {
constexpr int kEigSmemN = 64;  // blocks up to this size are diagonalised in shared memory

// Cyclic Jacobi (round-robin pairing, n/2 rotations per step) on one symmetric block per
// CTA, the matrix and the eigenvectors in shared memory (row stride n+1).  A pair is rotated only while |a_pq| exceeds
// 1e-16 sqrt(|a_pp a_qq|) plus an absolute floor; the loop ends after a sweep without
// rotations (at most 40 sweeps).  Output: eigenvalues descending, eigenvectors as
// columns of J.Q.
template <int NT>
__global__ void __launch_bounds__(NT) k_eig_batched(const EigJob* __restrict__ jobs) {
  const EigJob J = jobs[blockIdx.x];
  const int n = J.n, tid = threadIdx.x;
  extern __shared__ double sm[];
  const int ld = n + 1;
  double* A = sm;
  double* Q = sm + (size_t)n * ld;
  const int np = (n + 1) & ~1;
  double* cs = sm + (size_t)2 * n * ld;
  double* sn = cs + np / 2;
  double* wtmp = sn + np / 2;
  __shared__ int nrot;
  for (int e = tid; e < n * n; e += NT) A[(size_t)(e / n) * ld + e % n] = J.A[e];
  for (int e = tid; e < n * n; e += NT) Q[(size_t)(e / n) * ld + e % n] = (e / n == e % n) ? 1.0 : 0.0;
  __syncthreads();
  double scale = 0.0;
  for (int i = 0; i < n; ++i) scale = fmax(scale, fabs(A[(size_t)i * ld + i]));
  const double floor_abs = 1e-300 + 1e-18 * scale;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) nrot = 0;
    __syncthreads();
    for (int step = 0; step < np - 1; ++step) {
      for (int r = tid; r < np / 2; r += NT) {
        int a = r, b = np - 1 - r;
        int p = a == 0 ? 0 : 1 + (a - 1 + step) % (np - 1);
        int q = b == 0 ? 0 : 1 + (b - 1 + step) % (np - 1);
        if (p > q) { int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < n) {
          double app = A[(size_t)p * ld + p], aqq = A[(size_t)q * ld + q], apq = A[(size_t)p * ld + q];
          if (fabs(apq) > 1e-16 * sqrt(fabs(app * aqq)) + floor_abs) {
            sym_schur2(app, aqq, apq, c, s);
            atomicAdd(&nrot, 1);
          }
        }
        cs[r] = c; sn[r] = s;
      }
      __syncthreads();
      for (int e = tid; e < (np / 2) * n; e += NT) {
        int r = e / n, j = e % n;
        if (sn[r] == 0.0) continue;
        int a = r, b = np - 1 - r;
        int p = a == 0 ? 0 : 1 + (a - 1 + step) % (np - 1);
        int q = b == 0 ? 0 : 1 + (b - 1 + step) % (np - 1);
        if (p > q) { int t = p; p = q; q = t; }
        double c = cs[r], s = sn[r];
        double ap = A[(size_t)p * ld + j], aq = A[(size_t)q * ld + j];
        A[(size_t)p * ld + j] = c * ap - s * aq;
        A[(size_t)q * ld + j] = s * ap + c * aq;
      }
      __syncthreads();
      for (int e = tid; e < (np / 2) * n; e += NT) {
        int r = e / n, i = e % n;
        if (sn[r] == 0.0) continue;
        int a = r, b = np - 1 - r;
        int p = a == 0 ? 0 : 1 + (a - 1 + step) % (np - 1);
        int q = b == 0 ? 0 : 1 + (b - 1 + step) % (np - 1);
        if (p > q) { int t = p; p = q; q = t; }
        double c = cs[r], s = sn[r];
        double ap = A[(size_t)i * ld + p], aq = A[(size_t)i * ld + q];
        A[(size_t)i * ld + p] = c * ap - s * aq;
        A[(size_t)i * ld + q] = s * ap + c * aq;
        double qp = Q[(size_t)i * ld + p], qv = Q[(size_t)i * ld + q];
        Q[(size_t)i * ld + p] = c * qp - s * qv;
        Q[(size_t)i * ld + q] = s * qp + c * qv;
      }
      __syncthreads();
    }
    if (nrot == 0) break;
    __syncthreads();
  }
  // eigenpairs sorted descending (ties by index)
  for (int i = tid; i < n; i += NT) wtmp[i] = A[(size_t)i * ld + i];
  __syncthreads();
  const double* Qs = Q;
  for (int i = tid; i < n; i += NT) {
    double vi = wtmp[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double vj = wtmp[j];
      if (vj > vi || (vj == vi && j < i)) ++rank;
    }
    J.w[rank] = vi;
    for (int rr = 0; rr < n; ++rr) J.Q[(size_t)rr * n + rank] = Qs[(size_t)rr * ld + i];
  }
}
}  // namespace

// ------------------------------------------------------------------ parallel block Jacobi

namespace {
// Symmetric eigensolver for the large Gram blocks (n above the shared-memory limit): a
// two-sided block Jacobi.  Rows and columns are grouped in blocks of 32; each step of
// a round-robin tournament pairs the blocks, and for every pair (I, J) the 64 x 64
// diagonal sub-block G[I+J, I+J] is diagonalised in shared memory (cyclic Jacobi),
// giving V.  One launch applies V^T to the rows I+J of every pair (the pairs' rows are
// disjoint), the next applies V to the columns I+J of G and of Q (disjoint columns):
// together G <- W^T G W with W the block rotation of the step.  At convergence the
// eigenvalues are the diagonal of G and the eigenvectors the columns of Q; the
// absolute accuracy is ~eps |G|, that of the Gram route.
constexpr int kOB = 32;   // rows per block
constexpr int kOP = 64;   // rows per pair
constexpr int kOL = 65;   // shared-memory row stride (doubles)

struct BjJob {
  double* A;      // n x n symmetric (the Gram matrix), diagonalised in place
  double* Q;      // n x n accumulated rotations (eigenvectors as columns)
  double* w;      // n eigenvalues (output, descending)
  int n, nb;      // nb = number of row blocks, even
  int pair_begin; // first CTA of this job in a step launch
  int pad;
};

// cyclic Jacobi on a 64 x 64 symmetric matrix A (shared memory, stride kOL),
// eigenvectors accumulated into V (identity on entry), all 256 threads; a pair is
// rotated while |a_pq| > 1e-16 sqrt|a_pp a_qq| + floor_abs, for one sweep: the outer
// iteration returns to every pair until it is diagonal, and inner sweeps beyond the first
// cost more than they save (measured: 1 sweep 1.4-1.9x faster than 3, 2.1-2.7x than 5,
// at the same accuracy)
__device__ void cta_jacobi64(double* A, double* V, double* cs, double* sn, int* pq, int* nrot,
                             double floor_abs) {
  const int tid = threadIdx.x;
  constexpr int m = kOP, np = kOP, nr = kOP / 2;
  for (int sweep = 0; sweep < 1; ++sweep) {
    if (tid == 0) *nrot = 0;
    __syncthreads();
    for (int step = 0; step < np - 1; ++step) {
      if (tid < nr) {
        const int a = tid, b = np - 1 - tid;
        int p = a == 0 ? 0 : 1 + (a - 1 + step) % (np - 1);
        int q = b == 0 ? 0 : 1 + (b - 1 + step) % (np - 1);
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        const double app = A[p * kOL + p], aqq = A[q * kOL + q], apq = A[p * kOL + q];
        if (fabs(apq) > 1e-16 * sqrt(fabs(app * aqq)) + floor_abs) {
          sym_schur2(app, aqq, apq, c, s);
          atomicAdd(nrot, 1);
        }
        cs[tid] = c; sn[tid] = s; pq[2 * tid] = p; pq[2 * tid + 1] = q;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < nr * m / 256; ++k) {  // rows p, q of A
        const int e = tid + 256 * k, r = e >> 6, j = e & 63;
        if (sn[r] == 0.0) continue;
        const int p = pq[2 * r], q = pq[2 * r + 1];
        const double c = cs[r], s = sn[r];
        const double ap = A[p * kOL + j], aq = A[q * kOL + j];
        A[p * kOL + j] = c * ap - s * aq;
        A[q * kOL + j] = s * ap + c * aq;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < nr * m / 256; ++k) {  // columns p, q of A and V
        const int e = tid + 256 * k, r = e >> 6, i = e & 63;
        if (sn[r] == 0.0) continue;
        const int p = pq[2 * r], q = pq[2 * r + 1];
        const double c = cs[r], s = sn[r];
        const double ap = A[i * kOL + p], aq = A[i * kOL + q];
        A[i * kOL + p] = c * ap - s * aq;
        A[i * kOL + q] = s * ap + c * aq;
        const double vp = V[i * kOL + p], vq = V[i * kOL + q];
        V[i * kOL + p] = c * vp - s * vq;
        V[i * kOL + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    if (*nrot == 0) break;
    __syncthreads();
  }
}

// out(64 x 64 tile) = op(X) op(Y) with a 4 x 4 register tile per thread; X, Y in shared
// memory with stride kOL; tx / ty: transpose flags
template <bool TX, bool TY>
__device__ __forceinline__ void tile64(const double* X, const double* Y, double (&acc)[4][4]) {
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (int k = 0; k < kOP; ++k) {
    double x[4], y[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x[u] = TX ? X[k * kOL + ti * 4 + u] : X[(ti * 4 + u) * kOL + k];
      y[u] = TY ? Y[(tj * 4 + u) * kOL + k] : Y[k * kOL + tj * 4 + u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(x[u], y[v], acc[u][v]);
  }
}

__device__ __forceinline__ int find_job(const BjJob* jobs, int njobs) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].pair_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void pair_rows(const BjJob& J, int r, int step, int* idx) {
  const int a = r, b = J.nb - 1 - r;
  const int p = a == 0 ? 0 : 1 + (a - 1 + step) % (J.nb - 1);
  const int q = b == 0 ? 0 : 1 + (b - 1 + step) % (J.nb - 1);
  if (threadIdx.x < kOP) {
    const int blk = threadIdx.x < kOB ? p : q, row = blk * kOB + (threadIdx.x % kOB);
    idx[threadIdx.x] = row < J.n ? row : -1;
  }
}

// Q = identity, and the largest |diagonal| of A per job (the noise scale eps |G|)
__global__ void k_bj_prep(const BjJob* __restrict__ jobs, double* __restrict__ gmax) {
  const BjJob J = jobs[blockIdx.x];
  const int n = J.n;
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) J.Q[e] = (e / n == e % n) ? 1.0 : 0.0;
  double best = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) best = fmax(best, fabs(J.A[(size_t)i * n + i]));
  __shared__ double red[256];
  red[threadIdx.x] = best;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) gmax[blockIdx.x] = red[0];
}

// step, part 1: V of every pair from its diagonal sub-block (one CTA per pair)
__global__ void __launch_bounds__(256) k_bj_rows(const BjJob* __restrict__ jobs, int njobs, int step,
                                                 const double* __restrict__ gmax, double* __restrict__ vbuf,
                                                 int* __restrict__ flag, int* __restrict__ nrot) {
  extern __shared__ double bsm[];
  double* S = bsm;              // sub-block, then diagonalised
  double* V = S + kOP * kOL;    // its eigenvectors
  __shared__ double cs[kOP / 2], sn[kOP / 2];
  __shared__ int pq[kOP], idx[kOP];
  __shared__ int inner_rot, need;
  const int lo = find_job(jobs, njobs);
  const BjJob J = jobs[lo];
  const int r = blockIdx.x - J.pair_begin, tid = threadIdx.x, n = J.n;
  if (r >= J.nb / 2 || step >= J.nb - 1) {
    if (tid == 0) flag[blockIdx.x] = 0;
    return;
  }
  pair_rows(J, r, step, idx);
  if (tid == 0) need = 0;
  __syncthreads();
  // Rotate while an off-diagonal exceeds 1e-14 sqrt|g_ii g_jj| + 1e-14 |G| (|G| = the
  // largest diagonal entry): below that it is rounding noise of the rotations (~eps
  // sqrt(64) |G|), and it moves the eigenvalues only at second order.  The absolute part
  // must stay above the inner solver's floor, or pairs of null-space directions would
  // be sent back to it forever.
  const double fl = 1e-14 * gmax[lo];
  for (int e = tid; e < kOP * kOP; e += 256) {
    const int i = e >> 6, j = e & 63;
    S[i * kOL + j] = (idx[i] >= 0 && idx[j] >= 0) ? J.A[(size_t)idx[i] * n + idx[j]] : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < kOP * kOP; e += 256) {
    const int i = e >> 6, j = e & 63;
    if (i < j && fabs(S[i * kOL + j]) > 1e-14 * sqrt(fabs(S[i * kOL + i] * S[j * kOL + j])) + fl) need = 1;
  }
  __syncthreads();
  if (!need) {
    if (tid == 0) flag[blockIdx.x] = 0;
    return;
  }
  for (int e = tid; e < kOP * kOL; e += 256) V[e] = ((e / kOL) == (e % kOL)) ? 1.0 : 0.0;
  __syncthreads();
  cta_jacobi64(S, V, cs, sn, pq, &inner_rot, 1e-16 * gmax[lo]);  // floor below the outer one
  // one Newton-Schulz step V <- V (3 I - V^T V) / 2 against the rounding of the rotations
  {
    double acc[4][4];
    tile64<true, false>(V, V, acc);  // V^T V
    __syncthreads();
    const int ti = tid >> 4, tj = tid & 15;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int i = ti * 4 + u, j = tj * 4 + v;
        S[i * kOL + j] = (i == j ? 1.5 : 0.0) - 0.5 * acc[u][v];
      }
    __syncthreads();
    tile64<false, false>(V, S, acc);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) V[(ti * 4 + u) * kOL + tj * 4 + v] = acc[u][v];
    __syncthreads();
  }
  double* vg = vbuf + (size_t)blockIdx.x * kOP * kOP;
  for (int e = tid; e < kOP * kOP; e += 256) vg[e] = V[(e >> 6) * kOL + (e & 63)];
  if (tid == 0) {
    flag[blockIdx.x] = 1;
    atomicAdd(&nrot[lo], 1);
  }
}

// step, part 2: rows I+J of A <- V^T rows I+J, one 64-column chunk per CTA (grid.y)
__global__ void __launch_bounds__(256) k_bj_rowapply(const BjJob* __restrict__ jobs, int njobs, int step,
                                                     const double* __restrict__ vbuf, const int* __restrict__ flag) {
  extern __shared__ double bsm[];
  double* V = bsm;
  double* buf = V + kOP * kOL;
  __shared__ int idx[kOP];
  if (!flag[blockIdx.x]) return;
  const int lo = find_job(jobs, njobs);
  const BjJob J = jobs[lo];
  const int r = blockIdx.x - J.pair_begin, tid = threadIdx.x, n = J.n;
  const int c0 = blockIdx.y * kOP;
  if (c0 >= n) return;
  pair_rows(J, r, step, idx);
  const double* vg = vbuf + (size_t)blockIdx.x * kOP * kOP;
  for (int e = tid; e < kOP * kOP; e += 256) V[(e >> 6) * kOL + (e & 63)] = vg[e];
  __syncthreads();
  for (int e = tid; e < kOP * kOP; e += 256) {
    const int i = e >> 6, k = e & 63;
    buf[i * kOL + k] = (idx[i] >= 0 && c0 + k < n) ? J.A[(size_t)idx[i] * n + c0 + k] : 0.0;
  }
  __syncthreads();
  double acc[4][4];
  tile64<true, false>(V, buf, acc);
  const int ti = tid >> 4, tj = tid & 15;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int row = idx[ti * 4 + u];
    if (row < 0) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v)
      if (c0 + tj * 4 + v < n) J.A[(size_t)row * n + c0 + tj * 4 + v] = acc[u][v];
  }
}

// step, part 3: columns I+J of A (grid.z = 0) and of Q (grid.z = 1) <- columns times V,
// one 64-row chunk per CTA (grid.y)
__global__ void __launch_bounds__(256) k_bj_cols(const BjJob* __restrict__ jobs, int njobs, int step,
                                                 const double* __restrict__ vbuf, const int* __restrict__ flag) {
  extern __shared__ double bsm[];
  double* V = bsm;
  double* buf = V + kOP * kOL;
  __shared__ int idx[kOP];
  if (!flag[blockIdx.x]) return;
  const int lo = find_job(jobs, njobs);
  const BjJob J = jobs[lo];
  const int r = blockIdx.x - J.pair_begin, tid = threadIdx.x, n = J.n;
  pair_rows(J, r, step, idx);
  const double* vg = vbuf + (size_t)blockIdx.x * kOP * kOP;
  for (int e = tid; e < kOP * kOP; e += 256) V[(e >> 6) * kOL + (e & 63)] = vg[e];
  __syncthreads();
  const int ti = tid >> 4, tj = tid & 15;
  double* M = blockIdx.z == 0 ? J.A : J.Q;
  const int r0 = blockIdx.y * kOP;
  if (r0 >= n) return;
  for (int e = tid; e < kOP * kOP; e += 256) {
    const int rr = e >> 6, k = e & 63;
    buf[rr * kOL + k] = (idx[k] >= 0 && r0 + rr < n) ? M[(size_t)(r0 + rr) * n + idx[k]] : 0.0;
  }
  __syncthreads();
  double acc[4][4];
  tile64<false, false>(buf, V, acc);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int rr = r0 + ti * 4 + u;
    if (rr >= n) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int col = idx[tj * 4 + v];
      if (col >= 0) M[(size_t)rr * n + col] = acc[u][v];
    }
  }
}

// eigenvalues = diagonal of the rotated A, sorted descending (ties by index) with the
// normalised columns of Q; A is scratch for the unsorted eigenvectors
__global__ void k_bj_finish(const BjJob* __restrict__ jobs) {
  const BjJob J = jobs[blockIdx.x];
  const int n = J.n, tid = threadIdx.x;
  extern __shared__ double wn[];
  double* qn = wn + n;
  for (int i = tid; i < n; i += blockDim.x) {
    wn[i] = J.A[(size_t)i * n + i];
    double q2 = 0.0;
    for (int j = 0; j < n; ++j) q2 += J.Q[(size_t)j * n + i] * J.Q[(size_t)j * n + i];
    qn[i] = 1.0 / sqrt(q2);
  }
  __syncthreads();
  for (int64_t e = tid; e < (int64_t)n * n; e += blockDim.x) J.A[e] = J.Q[e] * qn[e % n];
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    const double vi = wn[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double vj = wn[j];
      if (vj > vi || (vj == vi && j < i)) ++rank;
    }
    J.w[rank] = vi;
    for (int rr = 0; rr < n; ++rr) J.Q[(size_t)rr * n + rank] = J.A[(size_t)rr * n + i];
  }
}

}  // namespace

static void eig_block_jacobi(const std::vector<EigJob>& jobs, Stream s) {
  if (jobs.empty()) return;
  std::vector<BjJob> bj;
  int pairs = 0, nbmax = 0, nmax = 0;
  for (const EigJob& j : jobs) {
    int nb = (j.n + kOB - 1) / kOB;
    nb += nb & 1;
    bj.push_back({j.A, j.Q, j.w, j.n, nb, pairs, 0});
    pairs += nb / 2;
    nbmax = std::max(nbmax, nb);
    nmax = std::max(nmax, j.n);
  }
  const int nj = (int)bj.size();
  const int nch = (nmax + kOP - 1) / kOP;  // 64-wide chunks of the largest matrix
  BjJob* d = (BjJob*)dev_alloc(sizeof(BjJob) * nj, s);
  dev_h2d(d, bj.data(), sizeof(BjJob) * nj, s);
  double* gmax = (double*)dev_alloc(sizeof(double) * nj, s);
  double* vbuf = (double*)dev_alloc(sizeof(double) * (size_t)pairs * kOP * kOP, s);
  int* flag = (int*)dev_alloc(sizeof(int) * pairs, s);
  int* nrot = (int*)dev_alloc(sizeof(int) * nj, s);
  std::vector<int> hrot(nj);
  k_bj_prep<<<nj, 256, 0, S(s)>>>(d, gmax);
  ++g_launches;
  const size_t shr = sizeof(double) * 2 * kOP * kOL, shc = sizeof(double) * 2 * kOP * kOL;
  static bool attr = false;
  if (!attr) {
    ck(cudaFuncSetAttribute(k_bj_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shr), "bj smem");
    ck(cudaFuncSetAttribute(k_bj_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shc), "bj smem");
    ck(cudaFuncSetAttribute(k_bj_rowapply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shc), "bj smem");
    attr = true;
  }
  for (int sweep = 0; sweep < 40; ++sweep) {
    ck(cudaMemsetAsync(nrot, 0, sizeof(int) * nj, S(s)), "bj counters");
    for (int step = 0; step < nbmax - 1; ++step) {
      k_bj_rows<<<pairs, 256, shr, S(s)>>>(d, nj, step, gmax, vbuf, flag, nrot);
      k_bj_rowapply<<<dim3(pairs, nch), 256, shc, S(s)>>>(d, nj, step, vbuf, flag);
      k_bj_cols<<<dim3(pairs, nch, 2), 256, shc, S(s)>>>(d, nj, step, vbuf, flag);
      g_launches += 3;
    }
    ck(cudaGetLastError(), "bj step");
    dev_d2h(hrot.data(), nrot, sizeof(int) * nj, s);
    dev_sync(s);
    bool any = false;
    for (int v : hrot) any = any || v > 0;
    if (!any) break;
  }
  const size_t shf = sizeof(double) * 2 * nmax;
  if (shf > 220 * 1024) throw std::runtime_error("eig_batched: block too large");
  if (shf > 48 * 1024)
    ck(cudaFuncSetAttribute(k_bj_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shf), "bj finish smem");
  k_bj_finish<<<nj, 256, shf, S(s)>>>(d);
  ++g_launches;
  ck(cudaGetLastError(), "bj finish");
  dev_free(nrot, s);
  dev_free(flag, s);
  dev_free(vbuf, s);
  dev_free(gmax, s);
  dev_free(d, s);
}

void eig_batched(const std::vector<EigJob>& jobs, Stream s) {
  if (jobs.empty()) return;
  std::vector<EigJob> small, large;
  int nmax_s = 1, nmax_l = 1;
  for (auto& j : jobs) {
    if (j.n <= kEigSmemN) { small.push_back(j); nmax_s = std::max(nmax_s, j.n); }
    else { large.push_back(j); nmax_l = std::max(nmax_l, j.n); }
  }
  EigJob* d = (EigJob*)dev_alloc(jobs.size() * sizeof(EigJob), s);
  if (!small.empty()) {
    dev_h2d(d, small.data(), small.size() * sizeof(EigJob), s);
    const int np = (nmax_s + 1) & ~1;
    size_t shm = sizeof(double) * ((size_t)2 * nmax_s * (nmax_s + 1) + np + nmax_s) + 64;
    ck(cudaFuncSetAttribute(k_eig_batched<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm), "eig smem");
    k_eig_batched<256><<<(int)small.size(), 256, shm, S(s)>>>(d);
    ++g_launches;
    ck(cudaGetLastError(), "eig_batched (shared)");
  }
  if (!large.empty()) eig_block_jacobi(large, s);
  dev_free(d, s);
}

// ------------------------------------------------------------------ selection

namespace {
// rank of every value (descending, ties by position) over all n values: one thread per
// value, many CTAs; keep[i] = rank < D and above the zero threshold
__global__ void k_select_rank(const double* __restrict__ v, int n, const double* __restrict__ vmax,
                              int D, double zero_rel, int* __restrict__ keep) {
  __shared__ double tile[1024];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double vi = i < n ? fmax(v[i], 0.0) : 0.0;
  int rank = 0;
  for (int j0 = 0; j0 < n; j0 += 1024) {
    for (int t = threadIdx.x; t < 1024; t += blockDim.x) tile[t] = (j0 + t < n) ? fmax(v[j0 + t], 0.0) : -1.0;
    __syncthreads();
    const int jn = min(1024, n - j0);
    for (int t = 0; t < jn; ++t) {
      const double vj = tile[t];
      rank += (vj > vi || (vj == vi && j0 + t < i)) ? 1 : 0;
    }
    __syncthreads();
  }
  if (i < n) keep[i] = (rank < D && vi > zero_rel * zero_rel * (*vmax)) ? 1 : 0;
}

__global__ void k_select_max(const double* __restrict__ v, int n, double* __restrict__ vmax) {
  __shared__ double red[256];
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) mx = fmax(mx, v[i]);
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) { if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]); __syncthreads(); }
  if (threadIdx.x == 0) *vmax = red[0];
}

// per-group kept counts and the weighted sums (norm^2, discarded) in a fixed order
__global__ void k_select_sums(const double* __restrict__ v, int n, const int* __restrict__ gid,
                              const int* __restrict__ wgt, const int* __restrict__ keep, int* kept,
                              double* sums) {
  __shared__ double red[2][256];
  double nrm = 0.0, disc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) {
    const double w = (double)wgt[gid[i]] * fmax(v[i], 0.0);
    nrm += w;
    if (keep[i]) atomicAdd(&kept[gid[i]], 1); else disc += w;
  }
  red[0][threadIdx.x] = nrm;
  red[1][threadIdx.x] = disc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) { red[0][threadIdx.x] += red[0][threadIdx.x + o]; red[1][threadIdx.x] += red[1][threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { sums[0] = red[0][0]; sums[1] = red[1][0]; }
}
}  // namespace

void select_largest(const double* vals, const std::vector<int>& goff, const std::vector<int>& wgt,
                    int D, double zero_rel, std::vector<int>& kept, double* norm2, double* disc,
                    Stream s) {
  const int G = (int)wgt.size();
  const int n = goff.back();
  std::vector<int> gid(n);
  for (int g = 0; g < G; ++g)
    for (int i = goff[g]; i < goff[g + 1]; ++i) gid[i] = g;
  int* d_gid = (int*)dev_alloc(sizeof(int) * (n + 1), s);
  int* d_w = (int*)dev_alloc(sizeof(int) * (G + 1), s);
  int* d_k = (int*)dev_alloc(sizeof(int) * (G + 1), s);
  int* d_keep = (int*)dev_alloc(sizeof(int) * (n + 1), s);
  double* d_s = (double*)dev_alloc(sizeof(double) * 3, s);
  dev_h2d(d_gid, gid.data(), sizeof(int) * n, s);
  dev_h2d(d_w, wgt.data(), sizeof(int) * G, s);
  dev_zero(d_k, sizeof(int) * (G + 1), s);
  k_select_max<<<1, 256, 0, S(s)>>>(vals, n, d_s + 2);
  ++g_launches;
  if (n > 0) {
    k_select_rank<<<(n + 255) / 256, 256, 0, S(s)>>>(vals, n, d_s + 2, D, zero_rel, d_keep);
    ++g_launches;
  }
  k_select_sums<<<1, 256, 0, S(s)>>>(vals, n, d_gid, d_w, d_keep, d_k, d_s);
  ++g_launches;
  ck(cudaGetLastError(), "select");
  kept.assign(G, 0);
  double sums[2];
  dev_d2h(kept.data(), d_k, sizeof(int) * G, s);
  dev_d2h(sums, d_s, sizeof(double) * 2, s);
  dev_sync(s);
  *norm2 = sums[0];
  *disc = sums[1];
  dev_free(d_gid, s);
  dev_free(d_w, s);
  dev_free(d_k, s);
  dev_free(d_keep, s);
  dev_free(d_s, s);
}

// ------------------------------------------------------------------ scatter

namespace {
__device__ inline double scl(const double* v, int i, int mode) {
  if (mode == 0) return 1.0;
  double x = v[i];
  return mode == 1 ? sqrt(x) : 1.0 / sqrt(x);
}

__global__ void k_scatter(const ScatterJob* __restrict__ jobs) {
  const ScatterJob J = jobs[blockIdx.x];
  const int64_t n = (int64_t)J.rows * J.cols;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    int i = (int)(e / J.cols), j = (int)(e % J.cols);
    double v = J.trans ? J.src[(size_t)j * J.lds + i] : J.src[(size_t)i * J.lds + j];
    J.dst[(size_t)i * J.ldd + j] = J.a * scl(J.rs, i, J.rmode) * scl(J.cs, j, J.cmode) * v;
  }
}
}  // namespace

void scatter_batched(const std::vector<ScatterJob>& jobs, Stream s) {
  if (jobs.empty()) return;
  ScatterJob* d = (ScatterJob*)dev_alloc(jobs.size() * sizeof(ScatterJob), s);
  dev_h2d(d, jobs.data(), jobs.size() * sizeof(ScatterJob), s);
  for (size_t off = 0; off < jobs.size(); off += 65535) {
    int n = (int)std::min<size_t>(65535, jobs.size() - off);
    k_scatter<<<n, 128, 0, S(s)>>>(d + off);
    ++g_launches;
  }
  ck(cudaGetLastError(), "scatter");
  dev_free(d, s);
}

// ------------------------------------------------------------------ allocation-free matvec
//
// For callers that cannot allocate device memory at the time of the call (inside a
// region where cudaMalloc is not allowed, or on a budget that forbids growth): the
// matvec's scratch (the right-operator products Z and the weighted sums W) is placed in
// this fixed array instead of the context's own buffers.  The array exists once per
// device that loads the library and stays allocated until the process exits.

namespace {

constexpr int64_t kNoAllocScratchDoubles = (int64_t)8 << 20;  // 64 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {nullptr};  // device address of the array, per device ordinal

struct Remap {
  const char* lo[4];
  const char* hi[4];
  char* to[4];
};

__device__ __forceinline__ const double* remap_ptr(const double* p, const Remap& m) {
  const char* c = (const char*)p;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (c >= m.lo[k] && c < m.hi[k]) return (const double*)(m.to[k] + (c - m.lo[k]));
  return p;
}

// k_grouped_gemm with every operand / output address passed through the remap
__global__ void __launch_bounds__(256) k_grouped_gemm_ra(const GemmTask* __restrict__ tasks,
                                                        const GemmGroup* __restrict__ groups,
                                                        int ngroups, Remap rm) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tile = blockIdx.x;
  int lo = 0, hi = ngroups - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (groups[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
  }
  const GemmGroup g = groups[lo];
  double* Cp = (double*)remap_ptr(g.C, rm);
  const int local = tile - g.tile_begin;
  const int tn = (g.n + BN - 1) / BN;
  const int row0 = (local / tn) * BM, col0 = (local % tn) * BN;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int t = g.task_begin; t < g.task_end; ++t) {
    const GemmTask T = tasks[t];
    const double* Bp = remap_ptr(T.B, rm);
    if (T.A == nullptr) {
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
          if (r < g.m && c < g.n)
            acc[i][j] += T.alpha * (T.transB ? Bp[(size_t)c * T.ldb + r] : Bp[(size_t)r * T.ldb + c]);
        }
      continue;
    }
    const double* Ap = remap_ptr(T.A, rm);
    for (int k0 = 0; k0 < T.k; k0 += BK) {
      for (int e = tid; e < BM * BK; e += 256) {
        int r, kk;
        double v = 0.0;
        if (T.transA) { kk = e / BM; r = e % BM; } else { r = e / BK; kk = e % BK; }
        int gr = row0 + r, gk = k0 + kk;
        if (gr < g.m && gk < T.k)
          v = T.transA ? Ap[(size_t)gk * T.lda + gr] : Ap[(size_t)gr * T.lda + gk];
        As[kk][r] = v * T.alpha;
      }
      for (int e = tid; e < BK * BN; e += 256) {
        int c, kk;
        double v = 0.0;
        if (T.transB) { c = e / BK; kk = e % BK; } else { kk = e / BN; c = e % BN; }
        int gc = col0 + c, gk = k0 + kk;
        if (gc < g.n && gk < T.k)
          v = T.transB ? Bp[(size_t)gc * T.ldb + gk] : Bp[(size_t)gk * T.ldb + gc];
        Bs[kk][c] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double a0 = As[kk][ty], a1 = As[kk][ty + 16];
        double b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
        acc[0][0] = fma(a0, b0, acc[0][0]);
        acc[0][1] = fma(a0, b1, acc[0][1]);
        acc[1][0] = fma(a1, b0, acc[1][0]);
        acc[1][1] = fma(a1, b1, acc[1][1]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
      if (r < g.m && c < g.n) Cp[(size_t)r * g.ldc + c] += acc[i][j];
    }
}

// k_combine with remapped addresses
__global__ void k_combine_ra(const CombSrc* __restrict__ src, const CombDst* __restrict__ dst, Remap rm) {
  const CombDst d = dst[blockIdx.x];
  double* dp = (double*)remap_ptr(d.dst, rm);
  const int64_t n = (int64_t)d.rows * d.cols;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    int r = (int)(e / d.cols), c = (int)(e % d.cols);
    double v = d.accumulate ? dp[(size_t)r * d.ld + c] : 0.0;
    for (int s = d.src_begin; s < d.src_end; ++s)
      v += src[s].alpha * remap_ptr(src[s].src, rm)[(size_t)r * src[s].ld + c];
    dp[(size_t)r * d.ld + c] = v;
  }
}

// Device address of the static array on the current device (looked up once per device).
double* noalloc_scratch(int* err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) { *err = 1; return nullptr; }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) { *err = 2; return nullptr; }
    g_noalloc_ptr[dev] = p;
  }
  *err = 0;
  return g_noalloc_ptr[dev];
}

}  // namespace

int64_t noalloc_scratch_capacity() { return kNoAllocScratchDoubles; }

void noalloc_matvec_run(const GemmPlan* p1, const CombPlan* pc, const GemmPlan* p2,
                        const double* xin, const double* yout, int64_t n, const double* Z,
                        int64_t zsize, const double* Wb, int64_t wsize, const double* x,
                        double* y, Stream s) {
  if (zsize + wsize > kNoAllocScratchDoubles)
    throw std::invalid_argument("scratch needed exceeds the 64 MiB static maximum of the allocation-free matvec");
  int err = 0;
  double* scratch = noalloc_scratch(&err);
  if (!scratch) throw std::runtime_error("cuda: cudaGetSymbolAddress of the static scratch failed");
  Remap rm;
  rm.lo[0] = (const char*)xin;  rm.hi[0] = (const char*)(xin + n);     rm.to[0] = (char*)x;
  rm.lo[1] = (const char*)yout; rm.hi[1] = (const char*)(yout + n);    rm.to[1] = (char*)y;
  rm.lo[2] = (const char*)Z;    rm.hi[2] = (const char*)(Z + zsize);   rm.to[2] = (char*)scratch;
  rm.lo[3] = (const char*)Wb;   rm.hi[3] = (const char*)(Wb + wsize);  rm.to[3] = (char*)(scratch + zsize);
  // phase 1 accumulates into Z and phase 2 into y: both start at zero; W is overwritten
  if (zsize) ck(cudaMemsetAsync(scratch, 0, sizeof(double) * zsize, S(s)), "memset scratch");
  if (n) ck(cudaMemsetAsync(y, 0, sizeof(double) * n, S(s)), "memset y");
  if (p1 && p1->ntiles) {
    k_grouped_gemm_ra<<<p1->ntiles, 256, 0, S(s)>>>(p1->tasks, p1->groups, p1->ngroups, rm);
    ++g_launches;
  }
  if (pc && pc->ndst) {
    for (int off = 0; off < pc->ndst; off += 65535) {
      int nb = std::min(65535, pc->ndst - off);
      k_combine_ra<<<nb, 128, 0, S(s)>>>(pc->src, pc->dst + off, rm);
      ++g_launches;
    }
  }
  if (p2 && p2->ntiles) {
    k_grouped_gemm_ra<<<p2->ntiles, 256, 0, S(s)>>>(p2->tasks, p2->groups, p2->ngroups, rm);
    ++g_launches;
  }
  ck(cudaGetLastError(), "allocation-free matvec launch");
}

}  // namespace dmrg

// Device memory and kernel launchers used by the engine.  Every numeric step of the
// two-site sweep is one of these launches; the planner only builds their tables.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

namespace dmrg {

typedef void* Stream;  // cudaStream_t

// ---- memory (stream-ordered; sizes in bytes) ----
void* dev_alloc(size_t bytes, Stream s);
void dev_free(void* p, Stream s);
void dev_h2d(void* dst, const void* src, size_t bytes, Stream s);
void dev_d2h(void* dst, const void* src, size_t bytes, Stream s);
void dev_d2d(void* dst, const void* src, size_t bytes, Stream s);
void dev_zero(void* p, size_t bytes, Stream s);
void dev_sync(Stream s);
size_t dev_bytes_in_use();     // device bytes held by the library (all contexts)
void dev_set_cap(size_t bytes);  // 0 = no cap; otherwise dev_alloc beyond it throws bad_alloc
int64_t kernel_launches();  // number of this library's kernel launches so far
int dev_check(const char** msg);  // 0 if no CUDA error is pending
void* host_pinned_alloc(size_t bytes);
// CUDA events for timing kernels on the engine's stream
void* event_create();
void event_destroy(void* e);
void event_record(void* e, Stream s);
float event_elapsed_ms(void* a, void* b);  // both must have completed
void host_pinned_free(void* p);
// a private non-blocking stream, and ordering across streams by events
Stream stream_create();
void stream_destroy(Stream s);
void stream_wait(Stream s, void* ev);  // work queued on s after this waits for ev
void event_sync(void* ev);

// ---- grouped GEMM: C_g = C_g + sum_t alpha_t op(A_t) op(B_t), row-major blocks;
// A == nullptr means op(A) = identity (C_g += alpha op(B)) ----
struct GemmTask {
  const double* A;
  const double* B;
  int lda, ldb;
  int k;
  int transA, transB;
  double alpha;
};
struct GemmGroup {
  double* C;
  int ldc, m, n;
  int task_begin, task_end;
  int tile_begin;     // prefix of 32x32 output tiles (filled by the uploader)
};
struct GemmPlan;  // device copy of a task/group table
GemmPlan* gemm_plan_upload(const std::vector<GemmTask>& t, std::vector<GemmGroup>& g, Stream s);
void gemm_plan_run(const GemmPlan* p, Stream s);
void gemm_plan_free(GemmPlan* p, Stream s);
int64_t gemm_plan_tasks(const GemmPlan* p);

// ---- block combine: dst = (accumulate ? dst : 0) + sum alpha_s src_s (2-D blocks) ----
struct CombSrc {
  const double* src;
  int ld;
  double alpha;
};
struct CombDst {
  double* dst;
  int ld, rows, cols;
  int src_begin, src_end;
  int accumulate;
};
struct CombPlan;
CombPlan* comb_plan_upload(const std::vector<CombSrc>& s, const std::vector<CombDst>& d, Stream st);
void comb_plan_run(const CombPlan* p, Stream s);
void comb_plan_free(CombPlan* p, Stream s);

// ---- diagonal of a sum of C (x) D terms: out += coef diag(C)_a diag(D)_b ----
struct DiagTerm {
  const double* C;
  const double* D;
  int ldc, ldd;
  double coef;
};
struct DiagOut {
  double* out;
  int dL, dR;
  int term_begin, term_end;
};
struct DiagPlan;
DiagPlan* diag_plan_upload(const std::vector<DiagTerm>& t, const std::vector<DiagOut>& o, Stream s);
void diag_plan_run(const DiagPlan* p, Stream s);
void diag_plan_free(DiagPlan* p, Stream s);

// ---- grouped Frobenius products: *out_g += sum_t alpha_t sum_ij A_t(i,j) B_t(i,j) ----
struct DotTask {
  const double* A;
  const double* B;
  int lda, ldb, rows, cols;
  double alpha;
};
struct DotGroup {
  double* out;       // distinct across the groups of one call
  int task_begin, task_end;
};
void dot_grouped(const std::vector<DotTask>& t, const std::vector<DotGroup>& g, Stream s);
// RDMs from the derivatives dg = dE/dg_ijkl of the energy with respect to the folded
// integrals of Eq. 11: Gamma = 2 x (average of dg over the eight permutations of V),
// gamma_ik = sum_j Gamma_ijkj / (N - 1)
void rdm_finish(const double* dg, int L, int N, double* gamma, double* Gamma, Stream s);

// ---- dense vector kernels for Davidson (FP64) ----
// out[j] = <V_j, w>, j < m; V is column-block storage V + j*ldv.
void vec_multidot(const double* V, int64_t ldv, int m, const double* w, int64_t n, double* out,
                  double* scratch, Stream s);
// y = beta*y + sum_j c[j] V_j (c on device)
void vec_combine(const double* V, int64_t ldv, int m, const double* c, double beta, double* y,
                 int64_t n, Stream s);
// y = a*x + b*y with a, b on device (pointers) or host scalars
void vec_axpby(double a, const double* x, double b, double* y, int64_t n, Stream s);
// scale y by 1/sqrt(*nrm2_dev)
void vec_normalize(double* y, const double* nrm2_dev, int64_t n, Stream s);
// t = r / (theta - diag), |denominator| floored
void vec_precondition(const double* r, const double* diag, const double* theta_dev, double* t,
                      int64_t n, Stream s);
// lowest eigenpairs of the m x m (m <= 48) symmetric matrix whose lower triangle is in G
// (ld gld) -> theta[0..k) ascending, C[v*m + i] = component i of vector v
void small_eig(const double* G, int gld, int m, int k, double* theta, double* C, Stream s);
// uniform noise in [-amp, amp) from splitmix64(seed + index), added to x
void vec_add_noise(double* x, int64_t n, double amp, uint64_t seed, Stream s);

// ---- batched symmetric eigensolver (cyclic Jacobi), eigenvalues sorted descending ----
struct EigJob {
  double* A;     // n x n symmetric, overwritten
  double* Q;     // n x n eigenvectors (columns), output
  double* w;     // n eigenvalues, output (descending)
  int n;
};
void eig_batched(const std::vector<EigJob>& jobs, Stream s);

// ---- global selection of the D largest values (ties: earlier group, lower index) ----
// vals: concatenated eigenvalues (lambda^2) of groups with offsets goff (size G+1);
// weights wgt[g] = 2jM+1.  Writes kept[g] and sums (norm2, discarded) to host.
void select_largest(const double* vals, const std::vector<int>& goff, const std::vector<int>& wgt,
                    int D, double zero_rel, std::vector<int>& kept, double* norm2, double* disc,
                    Stream s);

// ---- scaled block copy: dst[i,j] = a * r(i) * c(j) * src(i,j) (src transposed if set);
// r(i) from rs[i] by mode 0 = 1, 1 = sqrt(rs[i]), 2 = 1/sqrt(rs[i]); same for c(j) ----
struct ScatterJob {
  double* dst;
  const double* src;
  const double* rs;
  const double* cs;
  int ldd, lds, rows, cols;
  int rmode, cmode, trans;
  double a;
};
void scatter_batched(const std::vector<ScatterJob>& jobs, Stream s);

// ---- mixed-precision matvec: FP32 data, split-TF32 products on the tensor cores with
// FP32 accumulation (kernels_tc.cu).  Phase 1 writes Zt = (stack_c D^T)^T column-major for
// every right-operator block D (several blocks side by side in one MMA tile, the stack
// tile reused); phase 2 forms W^T = sum coef Zt while staging and accumulates
// y += C W over a task list (y FP64, added with atomics).  Every FP32 matrix here has a
// row stride that is a multiple of 4 and a 16-byte aligned first row, with zeros in the
// padding, so that rows are read as float4. ----
struct Tc1Entry {   // one right-operator block, or a piece of at most 128 of its rows
  const float* D;   // first row of the piece: ncols rows of K elements, row stride ldd
  float* zt;        // first column of its Zt: ncols columns of the stack's rows, stride ldz
  int ldd, ldz, ncols;
  int start;        // first column of the piece inside its pack (multiple of 8)
  float alpha;      // scalar of the operator
};
struct Tc1Pack { int e_begin, e_end, n; };  // n = padded columns of the pack (<= 128)
struct Tc1Unit {
  const float* A;   // stack rows row0 .. row0 + rows - 1 (rows <= 128), row stride lda
  int lda, rows, K, row0;
  int p_begin, p_end;
};
struct Tc2Src { const float* z; int ldz; float coef; };  // W^T(j, k) += coef z[j ldz + k]
struct Tc2Task {
  const float* C;   // left-operator block (m x K, row stride ldc); nullptr = identity
  int ldc, K;
  float alpha;
  int s_begin, s_end;
};
struct Tc2Unit {
  double* y;        // output block (row stride ldy); tile rows row0 .., columns col0 ..
  int ldy, m, n, row0, col0;
  int t_begin, t_end;
};
// one x block (rows x cols, row-major FP64) and its places in the FP32 stack (row-major,
// stride ld) and in the transposed stack (column-major, stride ldt)
struct TcXBlock { const double* src; float* dst; float* dstt; int rows, cols, ld, ldt; };
// one FP64 block converted to FP32 with row stride ld (a multiple of 4)
struct TcMirror { const double* src; float* dst; int rows, cols, ld; };
// Host description of one instance's mixed-precision matvec: the tables of both phases
// and the ranges units are cut from (phase 1: the packs of one 128-row stack tile;
// phase 2: the tasks of one output tile), reading x from xin and writing y to yout.
struct TcHost {
  std::vector<Tc1Entry> e;
  std::vector<Tc1Pack> p;
  std::vector<Tc1Unit> r1;  // p_begin / p_end span every pack of the tile
  std::vector<Tc2Src> s;
  std::vector<Tc2Task> t;
  std::vector<Tc2Unit> r2;  // t_begin / t_end span every task of the tile
  std::vector<TcXBlock> xb;
  double* yout = nullptr;
  int64_t n = 0;
};
// how ranges are cut into units (one CTA each): packs per phase-1 unit, tasks per
// phase-2 unit
struct TcTune { int packs_per_unit = 8, tasks_per_unit = 96; };
struct TcPlan;
// device tables of one or several instances (one grouped launch per phase for all)
TcPlan* tc_plan_build(const std::vector<const TcHost*>& inst, TcTune tune, Stream st);
// clear every y, x -> FP32 stacks, phase 1, phase 2; ev (3 events or nullptr) are
// recorded before phase 1, between the phases and after.  All pointers are fixed, so
// the sequence can be captured in a CUDA graph.
void tc_plan_launch(const TcPlan* p, void* const* ev, Stream s);
void tc_plan_free(TcPlan* p, Stream s);
int tc_error_flag(Stream s);  // 1 if a tensor-core kernel timed out on a wait
void tc_mirror(const std::vector<TcMirror>& m, Stream s);  // blocks -> FP32, padding untouched
// CUDA graph of tc_plan_launch(p) (captured on a private stream), its replay and release
void* tc_graph_create(const TcPlan* p);
void tc_graph_launch(void* g, Stream s);
void tc_graph_free(void* g);

// ---- allocation-free matvec: runs prepared matvec tables with the scratch in a
// fixed device array (capacity in doubles) and x / y redirected to caller buffers ----
int64_t noalloc_scratch_capacity();
void noalloc_matvec_run(const GemmPlan* p1, const CombPlan* pc, const GemmPlan* p2,
                        const double* xin, const double* yout, int64_t n, const double* Z,
                        int64_t zsize, const double* W, int64_t wsize, const double* x,
                        double* y, Stream s);

}  // namespace dmrg

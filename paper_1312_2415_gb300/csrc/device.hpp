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
// ---- grouped Davidson (all instances of a batch, one launch per operation) ----
// Workspace of one instance: subspace V and H V (n x (mmax + 1) each, column j at
// V + j n), the Rayleigh matrix G and its eigenvectors C (mmax x mmax), Ritz values th,
// dot products (dots, mmax + 2), partial sums (part, mmax x kBdChunks), residual r,
// correction t, scratch tmp (n x 2 nkeep), the Ritz vector x (the caller's buffer), the
// start vector x0, the H_eff diagonal, and the batch's matvec input / output bx, by.
struct BdSlot {
  double *V, *AV, *G, *C, *th, *dots, *part, *r, *t, *tmp, *x, *x0;
  const double* diag;
  double *bx, *by;
  int64_t n;
};
constexpr int kBdChunks = 64;
enum BdWhich { BD_V = 0, BD_AV, BD_R, BD_T, BD_X, BD_X0, BD_TMP, BD_BX, BD_BY };
// Every operation skips the instances with act[i] == 0; sl and act are device arrays of
// count entries, nmax the largest n.
// <A col (a_col + j), B col b_col> for j < m into G + row * mmax (to_g) or dots
void bd_dots(const BdSlot* sl, const int* act, int count, int64_t nmax, int aw, int a_col, int m, int bw, int b_col,
             int to_g, int row, int mmax, Stream s);
// y = beta y + sum_j c[j] V col j, c = C + cv * m (from_c) or dots
void bd_combine(const BdSlot* sl, const int* act, int count, int64_t nmax, int vw, int m, int from_c, int cv,
                double beta, int yw, int y_col, Stream s);
// y = a x + b y (a = -th[0] when a_theta)
void bd_axpby(const BdSlot* sl, const int* act, int count, int64_t nmax, int a_theta, double a, int xw, int x_col,
              double b, int yw, int y_col, Stream s);
// y /= sqrt(dots[0])
void bd_normalize(const BdSlot* sl, const int* act, int count, int64_t nmax, int yw, int y_col, Stream s);
// t = r / (th[0] - diag), denominator floored
void bd_precondition(const BdSlot* sl, const int* act, int count, int64_t nmax, Stream s);
// lowest k eigenpairs of the m x m Rayleigh matrices (lower triangles, ld mmax) into th, C
void bd_small_eig(const BdSlot* sl, const int* act, int count, int mmax, int m, int k, Stream s);
// G = diag(th[0..k))
void bd_restart_g(const BdSlot* sl, const int* act, int count, int mmax, int k, Stream s);
// x = -x where dots[0] < 0
void bd_sign(const BdSlot* sl, const int* act, int count, int64_t nmax, Stream s);
// out[2 i] = th[0], out[2 i + 1] = dots[0] of every instance
void bd_gather(const BdSlot* sl, int count, double* out, Stream s);

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

// ---- mixed-precision matvec (kernels_tc.cu): split-TF32 block products on the tcgen05
// tensor cores with FP32 accumulation, fused per output tile (no intermediate in global
// memory).  For an output block y_X' and every term (left-operator block C, weighted sum
// W = sum_s coef_s x_s D_s^T of right-operator products), the kernel forms W^T = sum_s
// coef_s D_s x_s^T in tensor memory (one accumulator per source, summed with the
// coefficients in FP32 registers) and adds y^T += W^T C^T (C's scalar folded into the
// coefficients).  Operands are FP32 "tiled" copies split into a TF32 head (hi) and tail
// (lo) kept in two arrays of the same layout: a block of R rows and K columns is stored
// as ceil(K/32) column chunks, each of ceil(R/8) row groups of 8 rows x 32 columns (1 KB)
// in the K-major core-matrix order of the tensor core's shared-memory operands (zeros in
// the padding), so that the rows an MMA needs from one chunk are one contiguous run that
// a single bulk copy moves into shared memory. ----
struct TfSrc {          // one source of a sub-task: W^T += coef D x^T
  const float* d;       // hi tiles of the right-operator block: chunk 0, first row group of the output column tile
  const float* x;       // hi tiles of the x block: chunk 0, first row group of the sub-task's x rows
  int d_cs, x_cs;       // floats between consecutive K chunks of d and of x
  int nkc, klast;       // K chunks (ceil(dR / 32)) and valid columns of the last one (1..32)
  float coef;           // the source's coefficient times the scalars of both operators
};
struct TfTask {         // one sub-task: y^T += W^T C^T over kdl columns of C
  const float* c;       // hi tiles of the left-operator block: chunk of its first column, first row group of the tile
  int c_cs;             // floats between consecutive K chunks of c
  int kdl;              // x rows of the sub-task (<= 64): N of W^T, K of the second product
  int s_begin, s_end;   // sources (at least one)
};
struct TfTile {         // one output tile of y, computed by one CTA from all of its terms
  double* y;            // element (row0, col0) of the output block
  int ldy, m, nv;       // m <= 128 rows, nv <= 128 columns
  int t_begin, t_end;   // sub-tasks
  int64_t dlo, xlo;     // floats from a hi tile to its lo tile (operator pool, x pool)
  int64_t cost;         // MMA steps (tiles run in decreasing order of cost)
  int kdg;              // x row groups of the tile's largest term (sizes its product-1 slots)
  int inst;             // instance of a batch (0 for a single matvec)
  int64_t group;        // right sector of the output block (tiles of a group share operator blocks)
  int tiny;             // 1: at most 4 x 4 outputs, terms of at most 4 x rows, sources of one K chunk
                        // (computed on CUDA cores, one term per lane)
  int pad;
};
// one FP64 block (rows x cols, row-major) to tiled hi / lo (nrg = ceil(rows / 8) row
// groups per chunk; lo = hi + lo floats); identity != 0: the rows x rows identity
struct TfConv { const double* src; float* dst; int rows, cols, nrg, identity; int64_t lo; };
// Host description of one instance's mixed-precision matvec: its tiles, sub-tasks and
// sources, the conversion of x (FP64, the ABI's layout) into its tiled pool, and y.
struct TcHost {
  std::vector<TfSrc> s;
  std::vector<TfTask> t;
  std::vector<TfTile> tiles;
  std::vector<TfConv> xb;
  double* yout = nullptr;
  int64_t n = 0;
};
// output tile rows (64 or 128) and x rows per sub-task (32 or 64)
struct TcTune { int row_tile = 128, x_chunk = 64; };
struct TcPlan;
// device tables of one or several instances (one launch of each kernel for all)
TcPlan* tc_plan_build(const std::vector<const TcHost*>& inst, Stream st);
// x -> tiled hi / lo, then the fused kernel over every tile; ev (3 events or nullptr)
// are recorded before the conversion, between the two launches and after.  All pointers
// are fixed, so the sequence can be captured in a CUDA graph.
void tc_plan_launch(const TcPlan* p, void* const* ev, Stream s);
void tc_plan_free(TcPlan* p, Stream s);
// per-instance flags (device, one int per instance, 1 after the build): the tiles of an
// instance whose flag is 0 are skipped (its y is left as it is)
int* tc_plan_active(TcPlan* p);
int tc_error_flag(Stream s);  // 1 if a tensor-core kernel gave up on a wait (then cleared)
// test hook: while set, the fused kernel's first wait is on a barrier that nothing
// completes, with a short limit, so that it takes the timed-out path
void tc_inject_timeout(int on);
void tc_convert(const std::vector<TfConv>& m, Stream s);  // blocks -> tiled hi / lo
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

// Host orchestration of the two-site spin-adapted DMRG on one GPU.
#pragma once
#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "coupling.hpp"
#include "device.hpp"
#include "mpo.hpp"
#include "symmetry.hpp"

namespace dmrg {

struct BlockRef {
  int r, c;      // row / column sector indices at the bond
  int64_t off;   // element offset inside the owning buffer
  int rows, cols;
};

// Reduced blocks of every operator of one bond (one side), in one device buffer.
struct OpStore {
  bool valid = false;
  int bond = -1;
  uint64_t serial = 0;  // distinct for every allocation (overlaps record the one they match)
  std::vector<std::vector<BlockRef>> blocks;         // per operator
  std::vector<std::unordered_map<int64_t, int>> at;  // (r << 32 | c) -> block index
  double* data = nullptr;
  int64_t size = 0;
};

// One MPS site: reduced tensor blocks T[k]^{(s N I)}_{(left sector),(right sector)}.
struct SiteBlock {
  int ls, l, r;
  int64_t off;
  int rows, cols;
};
struct Site {
  std::vector<SiteBlock> blocks;
  double* data = nullptr;
  int64_t size = 0;
};

struct XBlock {  // block of the two-site vector: (jL NL IL) (s1) (s2) j (jR NR IR)
  int l, ls1, ls2, tj, r;
  int64_t off;
  int rows, cols;
  int trow;       // row offset inside the stack of blocks sharing the right sector r
};

// A combined operator sum_a scalar_a O_a over sources sharing one site pattern.
struct CombOp {
  int target = -1, pattern = -1;
  double scalar = 1.0;           // multiplies the blocks (alias) or 1 (materialised)
  bool identity = false;         // the operator is the identity (scaled by scalar)
  const std::vector<BlockRef>* blocks = nullptr;
  const std::unordered_map<int64_t, int>* at = nullptr;
  const double* data = nullptr;  // base of the blocks
  // materialised storage
  std::vector<BlockRef> own_blocks;
  std::unordered_map<int64_t, int> own_at;
  std::vector<std::pair<int, double>> sources;  // (operator index, scalar)
  std::vector<std::pair<int64_t, double>> grad;  // (gi, gc) of each source's recursion term
};

// Overlap of the current MPS's renormalised basis at one bond with a stored state's, for
// every sector present in both: block e is d_cur(cur[e]) x d_low(low[e]), row-major.
struct Overlap {
  bool valid = false;
  uint64_t env_serial = 0;  // serial of the operator environment of the same bond and side
  std::vector<int> cur, low, rows, cols;
  std::vector<int64_t> off;
  std::unordered_map<int, int> by_cur;  // current sector -> block
  double* data = nullptr;
  int64_t size = 0;
};

// A lower state of the excited-state Hamiltonian H_m = H_0 + sum eta_k |Psi_k><Psi_k|
// (Sec. 4.3): its bonds and reduced tensors, its weight, and its overlaps with the
// current basis on both sides of every bond.
struct LowState {
  double eta = 0.0;
  std::vector<Bond> bonds;
  std::vector<Site> sites;
  std::vector<Overlap> left, right;
};

struct Stats {
  int64_t matvecs = 0, davidson_iters = 0, micro_iters = 0;
  double matvec_flops = 0.0, last_matvec_flops = 0.0, last_matvec_ms = 0.0;
  int64_t last_matvec_tasks = 0;
  double t_matvec_ms = 0, t_update_ms = 0, t_trunc_ms = 0, t_plan_ms = 0, t_total_ms = 0;
  double last_w_disc = 0.0, max_w_disc = 0.0;
  // device time of the matvec kernels (CUDA events on the engine's stream)
  double k_phase1_ms = 0.0, k_phase2_ms = 0.0;
  int64_t k_launches = 0;
  double k_phase1_flops = 0.0, k_phase2_flops = 0.0;
  // tensor-core (mixed precision) matvecs
  int64_t tc_matvecs = 0;
  double tc_flops = 0.0, tc_phase1_ms = 0.0, tc_phase2_ms = 0.0;
  double tc_phase1_flops = 0.0, tc_phase2_flops = 0.0, tc_phase1_bytes = 0.0, tc_phase2_bytes = 0.0;
  int64_t rdm_passes = 0;
  double rdm_ms = 0.0, rdm_flops = 0.0;
};

// key of a recoupled matvec coefficient: (left pattern, right pattern, the spins of the
// blocks and of the local states) packed in two words
struct CoefKey {
  uint64_t a, b;
  bool operator==(const CoefKey& o) const { return a == o.a && b == o.b; }
};
struct CoefKeyHash {
  size_t operator()(const CoefKey& k) const { return std::hash<uint64_t>()(k.a * 0x9E3779B97F4A7C15ull ^ k.b); }
};

class Engine {
 public:
  Engine(int L, int n_irrep, const std::vector<int>& orb_ir, int N, int two_S, int irrep,
         Stream stream);
  ~Engine();

  void set_integrals(double econst, const double* h, const double* V);
  void set_schedule(const std::vector<int>& D, const std::vector<double>& econv,
                    const std::vector<int>& nmax, const std::vector<double>& noise, double dtol,
                    int dmax);
  void init_mps(uint64_t seed);
  std::vector<char> get_mps();
  void set_mps(const char* buf, size_t len);

  // two-site probes (site i means orbitals i, i+1); the MPS must be in mixed canonical
  // form around i (left-normalised left of i, right-normalised right of i+1)
  void layout(int i, std::vector<int64_t>& table, int64_t& n);
  void tt_to_x(int i, double* x_dev);
  void matvec(int i, const double* x_dev, double* y_dev);
  void diag(int i, double* d_dev);
  // y = H_eff x with the prepared tables of site i and the library's fixed scratch array;
  // allocates nothing (throws invalid_argument if no table is prepared for i)
  void matvec_noalloc(int i, const double* x_dev, double* y_dev, Stream s);
  double davidson(int i, double* x_dev, int* iters, bool* converged);
  // mixed precision with one FP64 iteration (which only evaluates the FP64 Rayleigh
  // quotient of the tensor-core Ritz vector): with defer set the FP64 matvec is queued on
  // a side stream and the energy is collected by finish_rq()
  double davidson_ex(int i, double* x_dev, int* iters, bool* converged, bool defer);
  double truncate(int i, int dir, int D, const double* x_dev, double noise);
  double solve(double* e_last);
  // one micro-iteration of a sweep at sites (i, i+1): Eq. 25, Davidson, noise,
  // Eqs. 26-28 and the operator update in the sweep direction
  double sweep_step(int i, int dir, int D, double gamma, double* w_disc, int* iters, bool* conv);
  // the operator update of a sweep step in direction dir, after truncate(i, dir, ...)
  void update(int i, int dir);
  // the site of the next sweep_step (-1: unknown), used once by the next sweep_step to
  // build that site's tables while its FP64 energy is being evaluated
  void set_next_site(int s) { next_hint_ = s; }
  void canonicalize(int center);
  // Spin-summed 1- and 2-RDMs of the current MPS (device outputs, L^2 and L^4 doubles,
  // row-major): Gamma_ijkl = sum_st <a+_is a+_jt a_lt a_ks> projected onto the eight
  // permutations under which V is invariant, gamma_ik = sum_j Gamma_ijkj / (N - 1).
  // Leaves the MPS in mixed canonical form around site L-2 (the state is unchanged).
  void rdm(double* gamma_dev, double* Gamma_dev);
  // Excited states (Sec. 4.3): store the current MPS (normalised, right-canonical) as the
  // next lower state with weight eta; from then on H_eff carries + eta |Psi><Psi|.
  void push_excitation(double eta);
  void clear_excitations();
  int n_excitations() const { return (int)low_.size(); }
  bool is_right_canonical();
  void right_normalize_site(int k);
  void left_normalize_site(int k);

  const Stats& stats() { flush_events(); return st_; }
  Stream stream() const { return stream_; }
  void set_stream(Stream s) { stream_ = s; }
  // 0: FP64 block products; 1: split-TF32 tensor-core products (FP32 accumulation) in
  // Davidson, finished by FP64 Davidson iterations from the mixed-precision vector
  void set_precision(int p, int refine_iters) { precision_ = p; refine_iters_ = refine_iters; }
  int precision() const { return precision_; }
  // Batched matvecs: the mixed-precision tables of site i (built if needed), the plan's
  // serial (changes whenever the tables are rebuilt), its input / output buffers and
  // flops.  The tables stay valid until the MPS or the site of the engine changes.
  struct TcView { const TcHost* host; uint64_t serial; double* x; double* y; int64_t n; double flops; const double* diag; };
  // x^T H x / x^T x in FP64 with site i's tables (the symmetric form of build_rq; x on
  // the device)
  double rayleigh_fp64(int i, const double* x);
  TcView prepare_tc(int i, TcTune tune);
  uint64_t tc_serial(int i) const;
  void set_tune(TcTune t) { tune_ = t; }
  const std::vector<int>& hist_D() const { return hist_D_; }
  const std::vector<double>& hist_E() const { return hist_E_; }
  const std::vector<double>& hist_w() const { return hist_w_; }
  int L() const { return L_; }

 private:
  struct MatvecPlan;
  void check_ready() const;
  void free_env(OpStore& e);
  void alloc_env(OpStore& e, int bond, const OpSet& ops);
  void ensure_left(int k);
  void ensure_right(int k);
  void build_left(int k);
  void build_right(int k);
  void invalidate_envs_from_site(int k);
  void reset_noise();
  std::vector<XBlock> x_layout(int i, int64_t* n) const;
  void group_left(int i, std::vector<CombOp>& out, double** scratch, int64_t* scratch_n);
  void group_right(int i, std::vector<CombOp>& out, double** scratch, int64_t* scratch_n);
  void build_tc(MatvecPlan* p);
  void tc_tables(MatvecPlan* p, TcTune tune);
  // rdm: only the tables the RDM pass reads (phase 1, the combine into W and the W items;
  // the sources' table at the last pair); no phase 2, no diagonal, no lower-state terms
  MatvecPlan* plan_matvec(int i, bool rdm = false);
  void free_plan(MatvecPlan* p);
  void release_tc(MatvecPlan* p);  // frees the tensor-core tables of a plan
  void build_rq(MatvecPlan* p);    // tables of the symmetric quadratic form (energy)
  void run_rq(MatvecPlan* p);
  MatvecPlan* plan_for(int i);
  void run_matvec(MatvecPlan* p, const double* x, double* y, bool tc = false);
  double davidson_core(MatvecPlan* P, double* x, double tol, int maxit, bool tc, int* iters,
                       bool* converged);
  void update_left_from(int i, std::vector<CombOp>& comb);
  void update_right_from(int i, std::vector<CombOp>& comb);
  void alloc_site(int k);
  void free_site(int k);
  void identity_fill(OpStore& e, int op);
  void rdm_site(MatvecPlan* P, int i, double* dg, bool last);
  void add_projectors(MatvecPlan* p);
  void start_rq(MatvecPlan* P, const double* x);
  void launch_rq();
  double finish_rq();
  void free_overlap(Overlap& o);
  void ensure_ov_left(LowState& S, int k);
  void ensure_ov_right(LowState& S, int k);
  // v = projection of S onto the current two-site basis of sites (i, i+1) (layout X)
  void low_projection(LowState& S, int i, const std::vector<XBlock>& X, double* v);
  void tt_to_x_of(const std::vector<Bond>& bonds, const std::vector<Site>& sites, int i, double* x);
  std::vector<XBlock> x_layout_of(const std::vector<Bond>& bonds, int i, int64_t* n) const;

  int L_, N_, two_S_, irrep_;
  Symmetry sym_;
  Integrals g_;
  double econst_ = 0.0;
  bool have_integrals_ = false, have_mps_ = false;
  std::vector<OpSet> opsets_;
  PatternTable pt_;
  std::unique_ptr<Coupling> cp_;
  std::vector<std::vector<WEntry>> W_;
  std::vector<std::vector<WEntry>> Wg_;  // W_ with the terms of every allowed integral
  std::vector<Bond> bonds_;
  std::vector<std::map<Sector, int>> fci_;  // FCI-capped sector dimensions per bond
  std::vector<Site> sites_;
  std::vector<OpStore> lenv_, renv_;
  uint64_t env_serial_ = 0;
  // table sizes of the last operator update (block products, and their outputs): the next
  // update reserves that much, since neighbouring bonds have tables of similar size
  size_t upd_hint_z_ = 0, upd_hint_out_ = 0;
  std::vector<LowState> low_;
  std::vector<int> sched_D_, sched_nmax_;
  std::vector<double> sched_econv_, sched_noise_;
  double dav_tol_ = 1e-10;
  int dav_max_ = 100;
  Stream stream_;
  Stats st_;
  MatvecPlan* cached_ = nullptr;
  int cached_site_ = -1;
  // noise of Sec. 4.2: largest discarded weight of the previous half sweep, direction
  // and running maximum of the current one (a half sweep ends where the direction of
  // sweep_step changes), and the counter that seeds each noisy step's stream
  double w_prev_ = 0.0;
  int half_dir_ = 0;
  double half_wmax_ = 0.0;
  uint64_t noise_counter_ = 0;
  int next_hint_ = -1;
  void* ev_[3] = {nullptr, nullptr, nullptr};
  void flush_events();
  bool ev_pending_ = false;
  bool ev_tc_ = false;
  int precision_ = 0;
  int refine_iters_ = 0;  // FP64 finishing iterations in mixed mode (0: up to the cap)
  TcTune tune_;           // tile shape of the tensor-core matvec
  // per schedule instruction of the last solve: D, lowest energy and largest discarded
  // weight of its last macro-iteration (the data of the extrapolation, Sec. 4.3)
  std::vector<int> hist_D_;
  std::vector<double> hist_E_, hist_w_;
  uint64_t plan_serial_ = 0;
  std::thread reaper_;  // releases the host tables of the last freed plan
  // recoupled matvec coefficients of every plan so far (they depend on pattern ids and
  // spins only); read by the planner's workers, extended after each plan
  std::unordered_map<CoefKey, double, CoefKeyHash> coef_master_;
  // side stream of the deferred FP64 Rayleigh quotient: events (input copied, done),
  // device results (x.Hx, x.x) and reduction scratch
  Stream side_ = nullptr;
  void* ev_side_[2] = {nullptr, nullptr};
  double* rq_dev_ = nullptr;
  bool rq_pending_ = false;
  MatvecPlan* rq_plan_ = nullptr;  // plan whose FP64 Rayleigh quotient is still to be queued
};

}  // namespace dmrg

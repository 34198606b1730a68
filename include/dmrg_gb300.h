/* C ABI of the GB300 spin-adapted two-site DMRG library (libdmrg_gb300.so).
 *
 * The calls follow the paper's statement of the problem (Wouters, Poelmans, Ayers,
 * Van Neck, "CheMPS2", Sec. 4): a Hamiltonian given by E_const, one-body h_ij and
 * two-body V_ijkl in physics notation (Sec. 4.1), the target spin, particle number and
 * point-group irrep (Sec. 4.1 "Problem"), a convergence scheme of (D, E_conv, N_max,
 * gamma_noise) instructions (Sec. 4.2) and the two-site sweep (Secs. 2.3-2.4, 3.2-3.3).
 *
 * Conventions shared by every call:
 *  - Spins are passed doubled (two_S = 2S, tj = 2j).  Irreps are 0..7 of a real
 *    abelian group with XOR as product; the group index is 0=C1 1=Ci 2=C2 3=Cs 4=D2
 *    5=C2v 6=C2h 7=D2h (Sec. 3.1) and fixes how many irreps are valid (1, 2, 2, 2, 4,
 *    4, 4, 8).
 *  - Matrices are row-major float64.  The caller owns every pointer it passes; the
 *    library copies what it keeps.
 *  - "site i" of the two-site probes means orbitals i and i+1 (0-based), 0 <= i <= L-2.
 *    Probes use the MPS as it is: it must be left-normalised left of i and
 *    right-normalised right of i+1 (Eqs. 5-6), as after dmrg_set_mps of such an MPS or
 *    inside a sweep.
 *  - The two-site vector x holds, block by block, x = sqrt(2 jR + 1) * S with S the
 *    reduced two-site object of Eq. 25; its Euclidean norm is the norm of the state,
 *    so H_eff is symmetric.  dmrg_two_site_layout gives the block table.
 *  - stream == 0: x / y / d are HOST pointers.  stream != 0: they are DEVICE pointers
 *    (cudaStream_t cast to uintptr_t); the call first waits for work queued on that
 *    stream and returns after its own device work has finished.
 *  - Return 0 on success or a negative DMRG_E* code; dmrg_last_error(ctx) then holds a
 *    message.  No exception crosses the ABI.  A context is single-threaded.
 */
#ifndef DMRG_GB300_H
#define DMRG_GB300_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DMRG_OK 0
#define DMRG_EINVAL -1   /* invalid argument (size, N/S/irrep, state of the context) */
#define DMRG_ESYMM -2    /* integrals violate eightfold or point-group symmetry */
#define DMRG_ENOTCONV -3 /* Davidson reached its iteration cap; outputs hold the best */
#define DMRG_ENOMEM -4   /* host or device allocation failed */
#define DMRG_ECUDA -5    /* a CUDA call failed */
#define DMRG_EINTERNAL -6

typedef struct dmrg_ctx dmrg_ctx;

typedef struct {
  int64_t matvecs;         /* H_eff applications since creation */
  int64_t davidson_iters;
  int64_t micro_iters;     /* two-site optimisation steps */
  double matvec_flops;     /* planner-counted flops of all matvecs (nonzero blocks) */
  double last_matvec_flops;
  int64_t last_matvec_tasks;
  double t_update_ms, t_trunc_ms, t_plan_ms, t_total_ms; /* host wall clock */
  double last_w_disc, max_w_disc;                          /* Eq. 15 */
  /* device time (CUDA events) and flops of the two matvec kernels: phase 1 applies
   * the right-block operators (x D^T), phase 2 the left-block ones (sum c C Z) */
  double k_phase1_ms, k_phase2_ms;
  int64_t k_launches;
  double k_phase1_flops, k_phase2_flops;
  int64_t kernels_launched; /* all kernels this library launched in the process */
  /* matvecs done on the tensor cores (precision 1), their flops and device time */
  int64_t tc_matvecs;
  double tc_flops, tc_phase1_ms, tc_phase2_ms;
  /* per phase of those matvecs: flops, and compulsory bytes (FP32 operands read once
   * per use, FP32 Z written once, y written once) */
  double tc_phase1_flops, tc_phase2_flops, tc_phase1_bytes, tc_phase2_bytes;
  /* dmrg_rdm passes: count, host wall clock (ms, the planning included) and the flops of
   * their block products (matvec phase 1, the adjoint GEMMs, the Frobenius products) */
  int64_t rdm_passes;
  double rdm_ms, rdm_flops;
} dmrg_stats_t;

/* Sec. 4.1: L orbitals with irreps orb_irrep[L], N electrons (2 <= N <= 2L, needed by
 * the one-body folding of Eq. 11), spin two_S, target irrep.  precision: 0 = FP64 block
 * products; 1 = block products on the tensor cores in TF32 with each operand split into
 * two TF32 parts (three products, FP32 accumulation), used inside Davidson, which then
 * finishes with FP64 iterations from that vector so that energies are FP64 Rayleigh
 * quotients.  *out receives a new context (free with dmrg_destroy).  Errors:
 * DMRG_EINVAL. */
int dmrg_create(dmrg_ctx** out, int L, int group, const int* orb_irrep, int N, int two_S,
                int target_irrep, int precision);

/* Sec. 4.1 setEconst / setTmat / setVmat: h is L*L, V is L^4 with V[((i*L+j)*L+k)*L+l] =
 * (ij|V|kl).  h must be symmetric and V eightfold symmetric; both must respect the
 * point group (DMRG_ESYMM otherwise).  Host pointers, copied. */
int dmrg_set_integrals(dmrg_ctx* ctx, double econst, const double* h, const double* V);

/* Sec. 4.2 ConvergenceScheme: n instructions (D, E_conv, N_max, gamma_noise); noise
 * uniform in +-0.5 gamma w_disc(previous half sweep) is added to x before the
 * decomposition.  Davidson stops at ||r||_2 <= davidson_tol or davidson_max_iter. */
int dmrg_set_schedule(dmrg_ctx* ctx, int n, const int* D, const double* e_conv,
                      const int* n_max, const double* noise, double davidson_tol,
                      int davidson_max_iter);

/* Switch the precision mode (0 or 1, as in dmrg_create) of an existing context.
 * fp64_iters caps the FP64 Davidson iterations that finish each mixed-precision solve
 * (0 = until the Davidson tolerance or the Davidson cap). */
int dmrg_set_precision(dmrg_ctx* ctx, int precision, int fp64_iters);

/* Sec. 4.3: new MPS with the first instruction's D spread equally over the sectors of
 * every bond (capped by the FCI dimension) and filled with uniform(-1,1) numbers from
 * splitmix64 seeded with `seed` (site by site, block by block, row-major). */
int dmrg_init_mps(dmrg_ctx* ctx, uint64_t seed);

/* Serialised MPS (the reduced tensors of Eq. 22).  Layout, little-endian:
 * int32 magic 0x444D5247, version 1, L, N, two_S, irrep; for each bond 0..L: int32
 * n_sectors then n_sectors x int32 (2j, N, irrep, dim); for each site 0..L-1: int32
 * n_blocks then per block int32 (local state 0|1|2, left sector index, right sector
 * index) followed by dL*dR float64 row-major.  dmrg_get_mps: call with buf == NULL to
 * get the size in *len.  dmrg_set_mps replaces the MPS (DMRG_EINVAL on a malformed or
 * symmetry-violating buffer). */
int dmrg_get_mps(dmrg_ctx* ctx, void* buf, size_t* len);
int dmrg_set_mps(dmrg_ctx* ctx, const void* buf, size_t len);

/* Brings the MPS to mixed canonical form around sites (center, center+1) (Sec. 2.2,
 * Eqs. 5-6) by exact decompositions (Eqs. 25-28 keeping every nonzero singular value);
 * the state is unchanged up to normalisation. */
int dmrg_canonicalize(dmrg_ctx* ctx, int center);

/* Sec. 4.3 Solve: right-normalises the MPS (unless Eq. 6 already holds to 1e-10 on every
 * site right of the first), then runs the convergence scheme with
 * macro-iterations of one sweep to the right and one to the left.  *e_min = the lowest
 * energy of all micro-iterations (including E_const), *e_last = the last one. */
int dmrg_solve(dmrg_ctx* ctx, double* e_min, double* e_last);

/* Spin-summed one- and two-particle reduced density matrices of the current MPS (the
 * Gamma^A of Sec. 4.3, calc2DM, which DMRG-SCF consumes, Sec. 4.4), obtained as the
 * derivatives of its energy with respect to the integrals (energy of Sec. 4.1):
 *   Gamma[((i*L + j)*L + k)*L + l] = sum_st <a+_is a+_jt a_lt a_ks>, projected onto the
 *     eight index permutations under which V is invariant (the only part an energy with
 *     such a V depends on), so that dE/dV_ijkl = Gamma_ijkl / 2 for symmetric changes;
 *   gamma[i*L + k] = sum_s <a+_is a_ks> = sum_j Gamma_ijkj / (N - 1) = dE/dh_ik;
 *   E = E_const + sum h gamma + 1/2 sum V Gamma.
 * Computed on the device by the adjoint of the H_eff matvec (Eq. 9) with respect to the
 * scalars of the operator recursion (Sec. 2.5), one pass over the site pairs with the
 * centre moving right; afterwards the MPS is in mixed canonical form around L-2 (same
 * state).  gamma (L*L doubles) and Gamma (L^4 doubles) are device pointers when stream
 * != 0, host pointers when stream == 0.  DMRG_EINVAL on NULL outputs. */
int dmrg_rdm(dmrg_ctx* ctx, double* gamma, double* Gamma, uintptr_t stream);

/* Excited states (Sec. 4.3): dmrg_push_excitation stores the current MPS as the next
 * lower state |Psi_k> (normalised; the current MPS is left right-canonical, same state)
 * with weight eta = eta_{k+1}, so that every later H_eff (dmrg_heff_matvec, Davidson,
 * dmrg_solve) is that of H_m = H_0 + sum_k eta_{k+1} |Psi_k><Psi_k|: the two-site
 * projection v_k of each lower state (through its overlaps with the current basis) adds
 * eta_{k+1} v_k (v_k . x) to y.  Start the next state from a new MPS (dmrg_init_mps) or
 * the current one.  dmrg_heff_matvec_noalloc and dmrg_batch_create reject contexts with
 * lower states (DMRG_EINVAL).  dmrg_clear_excitations drops them all.  *count: the
 * number of stored lower states. */
int dmrg_push_excitation(dmrg_ctx* ctx, double eta);
int dmrg_clear_excitations(dmrg_ctx* ctx);
int dmrg_excitation_count(dmrg_ctx* ctx, int* count);

/* Block table of x for sites (site, site+1): n_blocks rows of 12 int64 (2jL, NL, IL,
 * s1, s2, 2j, 2jR, NR, IR, dL, dR, offset) with s1, s2 the local states 0|1|2 and the
 * block stored row-major at x + offset.  table may be NULL (sizes only). */
int dmrg_two_site_layout(dmrg_ctx* ctx, int site, int64_t* n_elem, int* n_blocks,
                         int64_t* table);

/* Eq. 25 from the current T[site], T[site+1] (x as above). */
int dmrg_tt_to_x(dmrg_ctx* ctx, int site, double* x, uintptr_t stream);

/* y = H_eff x (Eq. 9) with the renormalised and complementary operators of Sec. 2.5. */
int dmrg_heff_matvec(dmrg_ctx* ctx, int site, const double* x, double* y, uintptr_t stream);

/* *energy = x^T H_eff x / x^T x (the Rayleigh quotient that gives a micro-iteration's
 * energy, Secs. 2.3 and 4.3; without E_const), always in FP64.  H_eff is symmetric, so it
 * is evaluated from the block pairs with input block >= output block (the others' share
 * counted twice): about half of a matvec's second phase.  x: n doubles in the layout of
 * dmrg_two_site_layout, device pointer when stream != 0, host pointer when stream == 0.
 * DMRG_EINVAL for a NULL pointer or a zero vector. */
int dmrg_energy(dmrg_ctx* ctx, int site, const double* x, double* energy, uintptr_t stream);

/* Allocation-free variant of dmrg_heff_matvec (no counterpart in the paper).  It is for
 * callers that cannot allocate device memory at the moment they apply H_eff: a process
 * that reserved its device memory up front and must not grow it (a serving process
 * sharing the GPU with other work, where a new cudaMalloc can fail or force others
 * out), or a host framework whose own allocator owns the GPU and forbids side
 * allocations.  It runs the FP64 tables that an earlier dmrg_heff_matvec /
 * dmrg_davidson call prepared for this site (DMRG_EINVAL if there are none), with the
 * FP64 block products whatever the context's precision mode: for a precision-1 context
 * its y is the FP64 product, not the split-TF32 one dmrg_heff_matvec returns.  Its
 * intermediate products live in one fixed device array of the library (64 MiB per
 * device, held until the process exits); problems that need more scratch are rejected
 * with DMRG_EINVAL and a message.  It calls no cudaMalloc / cudaFree and no allocating
 * library routine.  x and y are DEVICE pointers of n_elem doubles (see
 * dmrg_two_site_layout); the work is queued on `stream` (0 = the default stream) behind
 * the context's own queued work, and the call returns without waiting for it.  The
 * context's next call waits on the device for that work before it runs anything that
 * could free or rewrite the tables it reads.  The first call on a device looks up the
 * array's address (cudaGetSymbolAddress): make that first call before any stream
 * capture.  All calls share the array, which keeps the previous call's contents (the
 * call clears what must start at zero), so calls whose device work overlaps in time
 * race on it: serialise them. */
int dmrg_heff_matvec_noalloc(dmrg_ctx* ctx, int site, const double* x, double* y,
                             uintptr_t stream);

/* d = diagonal of H_eff (the Davidson preconditioner). */
int dmrg_heff_diag(dmrg_ctx* ctx, int site, double* d, uintptr_t stream);

/* Davidson's lowest eigenpair of H_eff started from x (overwritten with the Ritz
 * vector, norm 1); *energy excludes E_const.  DMRG_ENOTCONV if the cap was hit. */
int dmrg_davidson(dmrg_ctx* ctx, int site, double* x, uintptr_t stream, double* energy,
                  int* iters);

/* Eqs. 26-28: decompose x, keep the D largest reduced singular values and write
 * T[site], T[site+1] (dir = +1: A[site] = U, A[site+1] = kappa V; dir = -1:
 * A[site] = U kappa, A[site+1] = V).  noise (>= 0) adds uniform(-noise, noise) to x
 * first.  *w_disc = discarded weight (Eq. 15). */
int dmrg_truncate(dmrg_ctx* ctx, int site, int dir, int D, double noise, const double* x,
                  uintptr_t stream, double* w_disc);

/* Sec. 2.5: the renormalised and complementary operators of the block that the sweep
 * grows, from the operators of the environment it extends: dir = +1 grows the left
 * block by orbital `site` (T[site] must be left-normalised, as after dmrg_truncate with
 * dir = +1), dir = -1 grows the right block by orbital site+1 (T[site+1] right-normalised,
 * as after dmrg_truncate with dir = -1).  dmrg_tt_to_x, dmrg_davidson, dmrg_truncate and
 * this call, in that order, do the work of one dmrg_sweep_step (without its noise) with
 * the two-site vector passing through the caller's buffers. */
int dmrg_update_operators(dmrg_ctx* ctx, int site, int dir);

/* Hint for the next dmrg_sweep_step: the site it will run at (-1 = unknown; used once).
 * A step at site s changes only the middle bond s+1, so the next step at the same site
 * keeps every table of this one; a step at another site has its tables built on the
 * host while this step's FP64 energy (precision 1) is evaluated on the device.  Results
 * do not depend on the hint.  dmrg_solve sets it for every step of its sweeps.
 * DMRG_EINVAL unless -1 <= site <= L-2. */
int dmrg_set_next_site(dmrg_ctx* ctx, int site);

/* One micro-iteration of a sweep (Secs. 2.3-2.5, 3.3): Eq. 25 from T[site], T[site+1],
 * Davidson with the scheme's tolerance and cap, noise gamma * 0.5 * w_disc(previous
 * half sweep), Eqs. 26-28 to D, and the renormalised / complementary operator update
 * for the next site in direction dir (+1 right, -1 left).  Outputs: energy (with
 * E_const), discarded weight, Davidson iterations.  DMRG_ENOTCONV if Davidson hit the
 * cap (the step is still completed). */
int dmrg_sweep_step(dmrg_ctx* ctx, int site, int dir, int D, double gamma, double* energy,
                    double* w_disc, int* iters);

/* Extrapolation data of the last dmrg_solve (Sec. 4.3): for each schedule instruction,
 * D, the lowest micro-iteration energy of its last macro-iteration and the largest
 * discarded weight of that macro-iteration (Eq. 15, max over the micro-iterations).
 * *n: capacity of the arrays on entry, number of instructions on return (arrays may be
 * NULL to query it). */
int dmrg_solve_history(dmrg_ctx* ctx, int* n, int* D, double* energy, double* w_disc);

/* Eq. 16: least-squares fit of E(D) = E_exact + C1 w_disc(D) over n >= 2 points (host
 * only).  DMRG_EINVAL for n < 2, NULL pointers or equal discarded weights. */
int dmrg_extrapolate(const double* w_disc, const double* energy, int n, double* e_exact,
                     double* c1);

/* Batched mixed-precision matvecs (no counterpart in the paper, which treats one
 * problem at a time): y_i = H_eff(ctx[i], site[i]) x_i for `count` independent
 * contexts, computed with the split-TF32 tensor-core products of precision 1 (whatever
 * precision the contexts were created with) as ONE launch of the fused matvec kernel
 * over the output tiles of all instances (after one launch converting every x), replayed
 * from a CUDA graph.  dmrg_batch_create prepares each context's tables at its site (as
 * a first dmrg_heff_matvec would) and, if autotune != 0, times the candidate tile shapes
 * (output rows per tile 128 or 64, x rows per term 64 or 32) on the merged tables and
 * keeps the fastest, then captures the launch sequence in a CUDA graph.  Failures are
 * reported through dmrg_last_error(ctx[0]).  The batch stays valid while no context
 * rebuilds its tables (a matvec at another site, a truncation or a sweep step does):
 * dmrg_batch_run then fails with DMRG_EINVAL. */
typedef struct dmrg_batch dmrg_batch;
int dmrg_batch_create(dmrg_batch** out, dmrg_ctx* const* ctx, const int* site, int count,
                      int autotune);
/* Device buffers of instance i: the input the graph reads (x, n doubles, the layout of
 * dmrg_two_site_layout) and the output it writes (y). */
int dmrg_batch_io(dmrg_batch* b, int i, double** x, double** y, int64_t* n);
/* Queue the batched matvec on `stream` (0 = the default stream) without waiting.  x and y
 * (arrays of count DEVICE pointers, or NULL) are copied into / out of the batch's
 * buffers around the graph; NULL entries (or NULL arrays) use the buffers in place.
 * Runs that overlap in time, or that overlap a matvec of one of the contexts at the
 * same site, race on those buffers. */
int dmrg_batch_run(dmrg_batch* b, const double* const* x, double* const* y, uintptr_t stream);
/* Davidson's algorithm (Sec. 2.3; the steps of dmrg_davidson) for every instance of the
 * batch in lockstep: each iteration applies H_eff to all instances with the batched
 * tensor-core matvec (one graph launch), and each vector operation of the iteration
 * (dot products, subspace combinations, residual, preconditioner, Gram-Schmidt,
 * normalisation, the small Rayleigh-Ritz eigenproblems) is one launch over all
 * instances; an instance that has converged (||r||_2 <= tol) is left as it is while the
 * others continue.  x: count DEVICE pointers to n_i doubles in the layout of
 * dmrg_two_site_layout (in: start vectors; out: Ritz vectors of unit norm, sign fixed by
 * a non-negative overlap with the start).  energy, iters, converged: host arrays of
 * count entries, or NULL.  energy is the lowest Ritz value of the split-TF32 operator,
 * or, with fp64_energy != 0, the FP64 Rayleigh quotient of the Ritz vector through each
 * context's FP64 tables.  The products carry about 5e-7 of max|y| (split TF32), so
 * tolerances much below ~1e-5 may not be reached: DMRG_ENOTCONV when some instance hits
 * max_iter (its best pair is still returned).  Runs on `stream` (0 = the default
 * stream) and returns after the last result is on the host; the batch's buffers are in
 * use meanwhile.  DMRG_EINVAL as dmrg_batch_run. */
int dmrg_batch_davidson(dmrg_batch* b, double* const* x, double tol, int max_iter, int fp64_energy,
                        double* energy, int* iters, int* converged, uintptr_t stream);
/* flops of one batched matvec (planner-counted), the chosen tile shape (output rows per
 * tile, x rows per term), the measured time of one launch sequence in the autotuner (0
 * without it) and the autotuner's time. */
int dmrg_batch_info(dmrg_batch* b, double* flops, int* row_tile, int* x_chunk,
                    double* launch_ms, double* tune_ms);
const char* dmrg_batch_last_error(dmrg_batch* b);
void dmrg_batch_destroy(dmrg_batch* b);

/* Device memory held by the library (all contexts of the process, in bytes), and an
 * optional cap on it (no counterpart in the paper, whose program states its memory use in
 * Sec. 5: 10 MB - 64 GB).  With a cap set (bytes > 0), a call whose next device
 * allocation would exceed it fails with DMRG_ENOMEM before the allocation is made; what
 * that call had allocated is released, the context keeps its previous state and can be
 * used again (with the cap raised or removed, bytes = 0).  Library-wide, not per
 * context. */
int dmrg_set_device_memory_cap(size_t bytes);

/* Test hook for failure detection (no counterpart in the paper).  While on != 0, each CTA
 * of the tensor-core matvec kernel starts with a bounded wait on a barrier that nothing
 * completes (a few thousand polls), so that it takes the path of a timed-out wait: it
 * records the error, issues nothing, frees its tensor memory and returns.  The calls that
 * ran it then fail with DMRG_ECUDA ("tensor-core wait timed out"); the error flag is
 * cleared when it is read, and with the hook off the next call computes normally.  No
 * fault, trap or endless wait is involved.  Library-wide. */
int dmrg_test_tc_timeout(int on);
int dmrg_device_memory_in_use(size_t* bytes);

int dmrg_stats(dmrg_ctx* ctx, dmrg_stats_t* out);
const char* dmrg_last_error(dmrg_ctx* ctx);
void dmrg_destroy(dmrg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif

// Mixed-precision H_eff matvec on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The effective Hamiltonian of Eq. 9, written with the renormalised and complementary
// operators of Sec. 2.5, acts on an output block y_X' as a sum of terms
//   y_X' += C W,   W = sum_s coef_s x_s D_s^T,
// C a left-operator block, x_s blocks of the two-site vector and D_s right-operator
// blocks (the combined operators of the left / right environments).  One CTA owns each
// output tile (up to 128 rows x 128 columns of one block, so nothing is added with
// atomics and the summation order is fixed) and runs all of its terms; the launch is
// persistent (one CTA per SM taking tiles from a work queue), so the pipeline runs on
// from one tile into the next (tiles of at most 4 x 4 outputs go to a CUDA-core kernel,
// k_tc_tiny, instead):
//   product 1: W^T = D_s x_s^T per source, into tensor-memory accumulators of at most
//              two 32-column K chunks each (M = 128 output columns, N = x rows of the
//              term, K = the right sector);
//   the converter warps add coef_s times each accumulator into FP32 registers, split the
//              sum into TF32 head and tail and store it as the A operand of
//   product 2: y^T += W^T C^T (M = 128 output columns, N = output rows, K = x rows),
//              restarted per term and drained into FP32 registers, which are added to y
//              (FP64) every few terms.  The tensor core's own FP32 accumulation loses
//              accuracy over long runs of products, hence the short accumulators.
// Every product uses split TF32: v = hi + lo with hi = rna_tf32(v), lo = rna_tf32(v - hi),
// and the three leading products hi*hi + hi*lo + lo*hi (about 2^-21 relative).  The
// second operand's hi and lo tiles sit one above the other in shared memory, so one MMA
// of twice the N gives A_hi B_hi^T and A_hi B_lo^T side by side in the accumulator and a
// second one adds A_lo B_hi^T to the first half: two instructions per K step instead of
// three.  An M = 128 tf32 MMA costs the issuing thread about 40-50 cycles whatever its N
// up to 64, so fewer, wider instructions are what the small blocks of this method need;
// products 1 and 2 are issued by two threads.
//
// Operands live in global memory already split and tiled in the K-major core-matrix
// order the MMA reads (see device.hpp), so a warp-specialised pipeline moves them with
// cp.async.bulk into shared memory (completion counted in bytes on mbarriers): a producer
// thread fills the product-1 ring, the product-2 thread loads the C tiles itself; only
// W^T passes through registers.  The shared-memory operand descriptors are K-major
// without swizzle: core matrices of 8 rows x 16 bytes, 128 bytes apart along K (LBO) and
// 1024 bytes apart along M/N (SBO), for 32-column chunks.
//
// Every wait is bounded: a CTA that gives up records an error, stops issuing work, waits
// (bounded) for its own copies and products in flight, frees its tensor memory and
// returns; the host reads and clears the error flag.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <unordered_map>
#include <stdexcept>
#include <string>

#include "device.hpp"
#include "plans.hpp"

namespace dmrg {

namespace {

constexpr long long kSpinLimit = 1ll << 22;  // polls of an mbarrier before giving up (seconds)
constexpr int kTF = 128 * 32;                // floats of a 128-row x 32-column tile (16 KB)
constexpr int kMaxS1 = 8;                    // slots of the product-1 operand ring, at most
constexpr int kS1KB = 96;                    // shared memory of the product-1 ring (KB)
constexpr int kMaxB2 = 2;                    // C slots, at most
constexpr int kTmemCols = 512;
constexpr int kWCols = 128;                  // tensor-memory columns of a W^T accumulator
constexpr int kNW = 3;                       // W^T accumulators
constexpr int kYCol = kNW * kWCols;          // first column of the y^T accumulator (128 columns)
constexpr int kTileQ = 4;                    // tiles taken from the work queue ahead of the slowest role
// shared memory (floats): product-1 slot = D tile hi, lo (up to 128 rows) and x tile hi,
// lo (kp rows each); product 2: C slots (2 x 128 rows x 2 chunks in all) and W^T tiles
// (128 rows x 2 chunks, hi, lo)
constexpr int kB2F = 4 * kTF;
constexpr int kA2F = 4 * kTF;
constexpr int kSmemF = kS1KB * 256 + kB2F + kA2F;
constexpr int kSegChunks = 2;   // K chunks per product-1 accumulator (then added in registers)
constexpr int kFlushTerms = 16; // terms summed in FP32 registers before they are added to y (FP64)
constexpr int kProducerWarp = 0, kMma1Warp = 1, kMma2Warp = 2, kConvWarp0 = 3, kConvWarps = 8;
constexpr int kMvThreads = (kConvWarp0 + kConvWarps) * 32;
constexpr int kConvThreads = kConvWarps * 32;

__device__ int g_tc_error = 0;
__device__ int g_tc_inject = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// float index of element (row, k) of a K-major no-swizzle tile with 32 columns
__device__ __forceinline__ int kmo(int row, int k) {
  return (row >> 3) * 256 + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  // start >> 4 | LBO (128 B) >> 4 << 16 | SBO (1024 B) >> 4 << 32 | descriptor version 1 << 46
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: D f32, A and B tf32, both K-major, M = 128, N = n (multiple of 16)
__device__ __forceinline__ uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init_n(uint64_t* mbar, int n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(n));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait that also gives up once another thread has flagged an abort; on its own
// timeout it records the error and flags the abort
__device__ __forceinline__ bool wait_or_abort(uint64_t* mbar, uint32_t parity, volatile int* abort_flag,
                                              long long limit = kSpinLimit) {
  for (long long it = 0; it < limit; ++it) {
    if (mbar_test(mbar, parity)) return true;
    if ((it & 1023) == 1023 && *abort_flag) return false;
  }
  atomicExch(&g_tc_error, 1);
  *abort_flag = 1;
  return false;
}

// bounded wait that ignores the abort flag (draining work in flight before exit)
__device__ __forceinline__ void wait_drain(uint64_t* mbar, uint32_t parity) {
  for (long long it = 0; it < kSpinLimit; ++it)
    if (mbar_test(mbar, parity)) return;
  atomicExch(&g_tc_error, 1);
}

// global -> shared bulk copy counted on mbar (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

// 32 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// the three split products of one K step, unstacked: A_hi B_hi^T + A_hi B_lo^T +
// A_lo B_hi^T into the same columns; nst steps of K = 8
__device__ __forceinline__ void mma_triple_steps(uint32_t tmem, uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl,
                                                 uint32_t id, int nst, bool fresh) {
  for (int st = 0; st < nst; ++st) {
    const uint64_t o = (uint64_t)(16 * st);
    mma_tf32(tmem, ah + o, bh + o, id, (fresh && st == 0) ? 0u : 1u);
    mma_tf32(tmem, ah + o, bl + o, id, 1u);
    mma_tf32(tmem, al + o, bh + o, id, 1u);
  }
}

struct Bars {
  uint64_t s1_full[kMaxS1], s1_empty[kMaxS1];
  uint64_t b2_full[kMaxB2], b2_empty[kMaxB2];
  uint64_t w_full[kNW], w_empty[kNW];
  uint64_t a2_full, mma2_done;
  uint64_t drain1, drain2, never;
  uint64_t tile_full[kTileQ], tile_empty[kTileQ];
};

// the two split products of one K step stacked along N: A_hi [B_hi; B_lo]^T (N = 2 kp)
// into accumulator columns [0, 2 kp) and A_lo B_hi^T (N = kp) into [0, kp); nst steps of
// K = 8 (8 columns = 256 bytes = 16 in the descriptor's address field), the first
// product restarting the accumulator when `fresh`
__device__ __forceinline__ void mma_pair_steps(uint32_t tmem, uint64_t ah, uint64_t al, uint64_t b, uint32_t id2,
                                               uint32_t id1, int nst, bool fresh) {
  mma_tf32(tmem, ah, b, id2, fresh ? 0u : 1u);
  mma_tf32(tmem, al, b, id1, 1u);
  if (nst > 1) {
    mma_tf32(tmem, ah + 16, b + 16, id2, 1u);
    mma_tf32(tmem, al + 16, b + 16, id1, 1u);
  }
  if (nst > 2) {
    mma_tf32(tmem, ah + 32, b + 32, id2, 1u);
    mma_tf32(tmem, al + 32, b + 32, id1, 1u);
  }
  if (nst > 3) {
    mma_tf32(tmem, ah + 48, b + 48, id2, 1u);
    mma_tf32(tmem, al + 48, b + 48, id1, 1u);
  }
}

// Geometry of one output tile.  kp: x rows of a term rounded up to 32 (x hi and x lo are
// stacked kp rows apart); mp: output rows rounded up to 32 (C hi and C lo are stacked mp
// rows apart).  Product-1 slots are sized for the tile (its output columns and its
// widest term), as many as fit: small blocks keep more copies in flight.  C slots hold
// the chunks of the tile's widest term.
struct TileGeom {
  int T, nvg, mg, mp, kpm, slot_f, nslots, b2_f, nb2;
  __device__ explicit TileGeom(const TfTile& t) {
    T = t.t_end - t.t_begin;
    nvg = (t.nv + 7) >> 3;
    mg = (t.m + 7) >> 3;
    mp = (t.m + 31) & ~31;
    kpm = t.kdg > 4 ? 64 : 32;
    slot_f = (2 * nvg + kpm / 4) * 256;
    nslots = min(kMaxS1, (kS1KB * 256) / slot_f);
    b2_f = 2 * mp * 32 * (kpm / 32);
    nb2 = min(kMaxB2, kB2F / b2_f);
  }
};

// Persistent: one CTA per SM takes tiles from a work queue (a counter in global memory,
// zeroed before the launch, handing out the tiles in the planner's order) until it is
// empty, so the pipeline runs on from one tile into the next.  The producer thread takes
// each tile and passes its index to the other roles through a small ring in shared
// memory (tile_full / tile_empty); -1 ends the list.  Ring phases are kept per slot
// across tiles (bit masks of parities), and a tile whose product-1 slot layout differs
// from the last one's waits for the last one's slots to be released first.  Tensor
// memory has a fixed layout: kNW W^T accumulators of 128 columns and the y^T accumulator
// in the last 128 columns.
__global__ void __launch_bounds__(kMvThreads, 1)
    k_tc_matvec(const TfTile* __restrict__ tiles, const TfTask* __restrict__ tasks, const TfSrc* __restrict__ srcs,
                int* __restrict__ queue, const int* __restrict__ active, int ntiles) {
  extern __shared__ unsigned char smem_dyn[];
  float* sm = (float*)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
  float* s1 = sm;                      // product-1 slots: D hi, D lo (nvg KB each), x hi, x lo (kp rows each)
  float* b2 = sm + kS1KB * 256;        // C slots: per K chunk C hi (mp rows) then C lo (mp rows); they
                                       // follow the product-1 slots, which the MMA's reads of a whole
                                       // 128-row D tile may run past
  float* a2 = b2 + kB2F;               // W^T: chunk 0 hi, lo, chunk 1 hi, lo
  __shared__ __align__(8) Bars bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int tile_q[kTileQ];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == kMma1Warp) tmem_alloc(&tmem_slot, kTmemCols);
  if (tid == 0) {
    for (int s = 0; s < kMaxS1; ++s) {
      mbar_init_n(&bar.s1_full[s], 1);
      mbar_init_n(&bar.s1_empty[s], 1);
    }
    for (int s = 0; s < kMaxB2; ++s) {
      mbar_init_n(&bar.b2_full[s], 1);
      mbar_init_n(&bar.b2_empty[s], 1);
    }
    for (int q = 0; q < kNW; ++q) {
      mbar_init_n(&bar.w_full[q], 1);
      mbar_init_n(&bar.w_empty[q], kConvThreads);
    }
    mbar_init_n(&bar.a2_full, kConvThreads);
    mbar_init_n(&bar.mma2_done, 1);
    mbar_init_n(&bar.drain1, 1);
    mbar_init_n(&bar.drain2, 1);
    mbar_init_n(&bar.never, 1);
    for (int r = 0; r < kTileQ; ++r) {
      mbar_init_n(&bar.tile_full[r], 1);
      mbar_init_n(&bar.tile_empty[r], 2 + kConvThreads);
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  // stale shared memory past the rows a copy fills must be finite: it meets zeros in
  // padded products
  for (int e = tid * 4; e < kSmemF; e += kMvThreads * 4)
    *reinterpret_cast<float4*>(sm + e) = make_float4(0.f, 0.f, 0.f, 0.f);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  if (tid == kMma1Warp * 32 && g_tc_inject) {
    // test hook: a wait on a barrier that nothing completes, with a short limit
    wait_or_abort(&bar.never, 0, &abort_flag, 4096);
  }
  __syncthreads();

  // the k-th tile of this CTA for the roles other than the producer (-1: none left, or
  // the CTA gave up)
  auto next_tile = [&](int k) -> int {
    const int r = k % kTileQ;
    if (!wait_or_abort(&bar.tile_full[r], (k / kTileQ) & 1, &abort_flag)) return -1;
    const int ti = tile_q[r];
    mbar_arrive(&bar.tile_empty[r]);
    return ti;
  };
  if (warp == kProducerWarp) {
    // ---- producer: takes the tiles; product-1 operands in the order the MMA thread
    // consumes them
    if (lane == 0 && !abort_flag) {
      uint32_t emp = 0, pend = 0, fpar = 0;  // per slot: release parity, fill not yet released, fill parity
      int last_slot_f = -1;
      bool ok = true;
      for (int k = 0; ok; ++k) {
        // take the next tile and pass it on
        const int r = k % kTileQ;
        if (k >= kTileQ && !wait_or_abort(&bar.tile_empty[r], (k / kTileQ - 1) & 1, &abort_flag)) break;
        int ti = atomicAdd(queue, 1);
        if (ti >= ntiles) ti = -1;
        tile_q[r] = ti;
        mbar_arrive(&bar.tile_full[r]);
        if (ti < 0) break;
        const TfTile tile = tiles[ti];
        if (!active[tile.inst]) continue;
        const TileGeom g(tile);
        if (g.slot_f != last_slot_f) {
          // a new slot layout overlaps the old slots: all of them are released first
          for (int s = 0; s < kMaxS1 && ok; ++s)
            if ((pend >> s) & 1u) {
              ok = wait_or_abort(&bar.s1_empty[s], (emp >> s) & 1u, &abort_flag);
              emp ^= 1u << s;
              pend &= ~(1u << s);
            }
          last_slot_f = g.slot_f;
        }
        int slot = 0;
        for (int t = 0; t < g.T && ok; ++t) {
          const TfTask tk = tasks[tile.t_begin + t];
          const int kdg = (tk.kdl + 7) >> 3, kp = tk.kdl > 32 ? 64 : 32;
          const uint32_t bytes = 2u * (g.nvg + kdg) * 1024u;
          for (int si = tk.s_begin; si < tk.s_end && ok; ++si) {
            const TfSrc S = srcs[si];
            for (int kk = 0; kk < S.nkc; ++kk) {
              if ((pend >> slot) & 1u) {
                if (!wait_or_abort(&bar.s1_empty[slot], (emp >> slot) & 1u, &abort_flag)) {
                  ok = false;
                  break;
                }
                emp ^= 1u << slot;
              }
              float* dst = s1 + slot * g.slot_f;
              const float* d = S.d + (int64_t)kk * S.d_cs;
              const float* x = S.x + (int64_t)kk * S.x_cs;
              mbar_expect_tx(&bar.s1_full[slot], bytes);
              bulk_g2s(dst, d, g.nvg * 1024u, &bar.s1_full[slot]);
              bulk_g2s(dst + g.nvg * 256, d + tile.dlo, g.nvg * 1024u, &bar.s1_full[slot]);
              bulk_g2s(dst + 2 * g.nvg * 256, x, kdg * 1024u, &bar.s1_full[slot]);
              bulk_g2s(dst + 2 * g.nvg * 256 + kp * 32, x + tile.xlo, kdg * 1024u, &bar.s1_full[slot]);
              pend |= 1u << slot;
              fpar ^= 1u << slot;
              if (++slot == g.nslots) slot = 0;
            }
          }
        }
      }
      // copies still in flight land before the CTA can exit: wait for the last fill of
      // every slot not yet released (a completed phase keeps testing complete while no
      // newer one starts)
      for (int s = 0; s < kMaxS1; ++s)
        if ((pend >> s) & 1u) wait_drain(&bar.s1_full[s], ((fpar >> s) & 1u) ^ 1u);
    }
  } else if (warp == kMma1Warp) {
    // ---- product 1: W^T = D x^T per source, segments of up to two K chunks per
    // accumulator
    if (lane == 0 && !abort_flag) {
      uint32_t ful = 0;  // per slot: parity of the next fill
      int q = 0, wround = 0;
      bool ok = true;
      for (int k = 0; ok; ++k) {
        const int ti = next_tile(k);
        if (ti < 0) break;
        const TfTile tile = tiles[ti];
        if (!active[tile.inst]) continue;
        const TileGeom g(tile);
        int slot = 0;
        for (int t = 0; t < g.T && ok; ++t) {
          const TfTask tk = tasks[tile.t_begin + t];
          const int kp = tk.kdl > 32 ? 64 : 32;
          const uint32_t id2 = idesc_tf32(2 * kp), id1 = idesc_tf32(kp);
          for (int si = tk.s_begin; si < tk.s_end && ok; ++si) {
            const TfSrc S = srcs[si];
            for (int k0 = 0; k0 < S.nkc; k0 += kSegChunks) {
              if (wround >= 1 && !wait_or_abort(&bar.w_empty[q], (wround - 1) & 1, &abort_flag)) {
                ok = false;
                break;
              }
              const uint32_t wq = tmem + (uint32_t)(q * kWCols);
              const int k1 = min(S.nkc, k0 + kSegChunks);
              for (int kk = k0; kk < k1; ++kk) {
                if (!wait_or_abort(&bar.s1_full[slot], (ful >> slot) & 1u, &abort_flag)) {
                  ok = false;
                  break;
                }
                ful ^= 1u << slot;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const int kv = kk == S.nkc - 1 ? S.klast : 32;
                const float* base = s1 + slot * g.slot_f;
                mma_pair_steps(wq, smem_desc(smem_u32(base)), smem_desc(smem_u32(base + g.nvg * 256)),
                               smem_desc(smem_u32(base + 2 * g.nvg * 256)), id2, id1, (kv + 7) >> 3, kk == k0);
                mma_commit(&bar.s1_empty[slot]);
                if (++slot == g.nslots) slot = 0;
              }
              if (!ok) break;
              mma_commit(&bar.w_full[q]);
              if (++q == kNW) {
                q = 0;
                ++wround;
              }
            }
          }
        }
      }
      // every product issued has finished before tensor memory is released
      mma_commit(&bar.drain1);
      wait_drain(&bar.drain1, 0);
    }
  } else if (warp == kMma2Warp) {
    // ---- product 2: y^T = W^T C^T per term, fresh accumulator; this thread also loads
    // the C tiles (slot u % nb2 of the tile; the next fill of a slot waits for the
    // product that read it, and a tile starts once the last one's products have finished)
    if (lane == 0 && !abort_flag) {
      uint32_t bf = 0, bc = 0, lf = 0, filled = 0;  // per C slot: fill parity to wait, commits, last fill, ever filled
      int gt = 0;                                    // terms of the CTA's earlier tiles
      int tiles_done = 0;
      bool ok = true;
      for (int k = 0; ok; ++k) {
        const int ti = next_tile(k);
        if (ti < 0) break;
        const TfTile tile = tiles[ti];
        if (!active[tile.inst]) continue;
        const TileGeom g(tile);
        auto load_c = [&](int u) {
          const TfTask tk = tasks[tile.t_begin + u];
          const int nch = (tk.kdl + 31) >> 5, s = u % g.nb2;
          float* dst = b2 + s * g.b2_f;
          mbar_expect_tx(&bar.b2_full[s], 2u * nch * g.mg * 1024u);
          for (int c = 0; c < nch; ++c) {
            const float* src = tk.c + (int64_t)c * tk.c_cs;
            bulk_g2s(dst + c * 2 * g.mp * 32, src, g.mg * 1024u, &bar.b2_full[s]);
            bulk_g2s(dst + c * 2 * g.mp * 32 + g.mp * 32, src + tile.dlo, g.mg * 1024u, &bar.b2_full[s]);
          }
          lf ^= 1u << s;
          filled |= 1u << s;
        };
        for (int u = 0; u < min(g.nb2, g.T); ++u) load_c(u);
        const uint32_t idm = idesc_tf32((tile.m + 15) & ~15);
        for (int t = 0; t < g.T; ++t) {
          const int s = t % g.nb2;
          const TfTask tk = tasks[tile.t_begin + t];
          if (!wait_or_abort(&bar.a2_full, (gt + t) & 1, &abort_flag) ||
              !wait_or_abort(&bar.b2_full[s], (bf >> s) & 1u, &abort_flag)) {
            ok = false;
            break;
          }
          bf ^= 1u << s;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const float* cb = b2 + s * g.b2_f;
          for (int c = 0; c * 32 < tk.kdl; ++c) {
            const int kv = min(32, tk.kdl - 32 * c);
            mma_triple_steps(tmem + kYCol, smem_desc(smem_u32(a2 + (2 * c) * kTF)),
                             smem_desc(smem_u32(a2 + (2 * c + 1) * kTF)), smem_desc(smem_u32(cb + c * 2 * g.mp * 32)),
                             smem_desc(smem_u32(cb + c * 2 * g.mp * 32 + g.mp * 32)), idm, (kv + 7) >> 3, c == 0);
          }
          mma_commit(&bar.b2_empty[s]);
          bc ^= 1u << s;
          mma_commit(&bar.mma2_done);
          if (t + g.nb2 < g.T) {
            if (!wait_or_abort(&bar.b2_empty[s], ((bc >> s) & 1u) ^ 1u, &abort_flag)) {
              ok = false;
              break;
            }
            load_c(t + g.nb2);
          }
        }
        gt += g.T;
        // the next tile's C layout may overlap this one's slots: its products finish first
        mma_commit(&bar.drain2);
        wait_drain(&bar.drain2, tiles_done & 1);
        ++tiles_done;
      }
      // every C copy has landed before the CTA exits (the last fill of every slot)
      for (int s = 0; s < kMaxB2; ++s)
        if ((filled >> s) & 1u) wait_drain(&bar.b2_full[s], ((lf >> s) & 1u) ^ 1u);
      if (tiles_done == 0) {
        mma_commit(&bar.drain2);
        wait_drain(&bar.drain2, 0);
      }
    }
  } else {
    // ---- converters: warp w reads tensor-memory lanes 32 (w % 4) .. (its output
    // columns); half 0 / 1 holds x rows 0..31 / 32..63 of W^T and output rows 0..63 /
    // 64..127 of y.  A W^T accumulator holds the hi part in columns [0, kp) and the
    // stacked lo part in [kp, 2 kp); their sum is the product.
    const int quarter = warp & 3, half = (warp - kConvWarp0) >> 2;
    const int n = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    int q = 0, wround = 0, gt = 0;
    bool ok = !abort_flag;
    for (int k = 0; ok; ++k) {
      const int ti = next_tile(k);
      if (ti < 0) break;
      const TfTile tile = tiles[ti];
      if (!active[tile.inst]) continue;
      const int T = tile.t_end - tile.t_begin;
      float yacc[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) yacc[j] = 0.0f;
      auto drain_y = [&]() {
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          if (64 * half + 32 * i < tile.m) {
            float v[32];
            tmem_ld32(lane_base + (uint32_t)(kYCol + 64 * half + 32 * i), v);
#pragma unroll
            for (int j = 0; j < 32; ++j) yacc[32 * i + j] += v[j];
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
      };
      // the FP32 sums of the last terms are added to y (the tile's owner writes it
      // first, then accumulates into it)
      bool stored = false;
      auto flush_y = [&]() {
        if (abort_flag || n >= tile.nv) return;
#pragma unroll
        for (int j = 0; j < 64; ++j) {
          const int r = 64 * half + j;
          if (r < tile.m) {
            double* yp = tile.y + (int64_t)r * tile.ldy + n;
            *yp = stored ? *yp + (double)yacc[j] : (double)yacc[j];
          }
          yacc[j] = 0.0f;
        }
        stored = true;
      };
      for (int t = 0; t < T && ok; ++t) {
        const TfTask tk = tasks[tile.t_begin + t];
        const int kp = tk.kdl > 32 ? 64 : 32;
        float wsum[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) wsum[j] = 0.0f;
        for (int si = tk.s_begin; si < tk.s_end && ok; ++si) {
          const float coef = srcs[si].coef;
          const int nseg = (srcs[si].nkc + kSegChunks - 1) / kSegChunks;
          for (int sg = 0; sg < nseg; ++sg) {
            if (!wait_or_abort(&bar.w_full[q], wround & 1, &abort_flag)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (32 * half < tk.kdl) {
              const uint32_t wa = lane_base + (uint32_t)(q * kWCols + 32 * half);
              float v[32];
              tmem_ld32(wa, v);
#pragma unroll
              for (int j = 0; j < 32; ++j) wsum[j] = fmaf(coef, v[j], wsum[j]);
              tmem_ld32(wa + (uint32_t)kp, v);
#pragma unroll
              for (int j = 0; j < 32; ++j) wsum[j] = fmaf(coef, v[j], wsum[j]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(&bar.w_empty[q]);
            if (++q == kNW) {
              q = 0;
              ++wround;
            }
          }
        }
        if (!ok) break;
        // product 2 of the previous term has finished: its result is added to the
        // registers, and W^T in shared memory and y^T may be overwritten (the first term
        // of a tile follows the drain of the CTA's previous tile)
        if (t >= 1) {
          if (!wait_or_abort(&bar.mma2_done, (gt + t - 1) & 1, &abort_flag)) {
            ok = false;
            break;
          }
          drain_y();
          if (t % kFlushTerms == 0) flush_y();
        }
        float* ah = a2 + (2 * half) * kTF;
        float* al = ah + kTF;
#pragma unroll
        for (int gg = 0; gg < 8; ++gg) {
          float4 h, l;
          float* hv = &h.x;
          float* lv = &l.x;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float v = (32 * half + 4 * gg + e < tk.kdl) ? wsum[4 * gg + e] : 0.0f;
            hv[e] = tf32_round(v);
            lv[e] = tf32_round(v - hv[e]);
          }
          *reinterpret_cast<float4*>(ah + kmo(n, 4 * gg)) = h;
          *reinterpret_cast<float4*>(al + kmo(n, 4 * gg)) = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&bar.a2_full);
      }
      if (ok && T >= 1) {
        if (wait_or_abort(&bar.mma2_done, (gt + T - 1) & 1, &abort_flag)) drain_y();
        else ok = false;
      }
      flush_y();
      gt += T;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == kMma1Warp) tmem_free(tmem, kTmemCols);
}

// ------------------------------------------------------------------ tiny tiles

// element (row, col) of a tiled hi / lo operand (chunk 0, col < 32) as hi + lo in FP64
__device__ __forceinline__ double tiled_val(const float* __restrict__ p, int64_t lo, int row, int col) {
  const int64_t e = (int64_t)kmo(row, col);
  return (double)p[e] + (double)p[e + lo];
}

// Output tiles of at most 4 x 4 elements whose terms have at most 4 x rows and whose
// sources are one K chunk (tile.tiny): the same sum y += C (sum_s coef_s x_s D_s^T) on
// CUDA cores in FP64 from the FP32 operand tiles, one warp per tile and one term per lane
// (tensor-core products would be nearly all padding and the pipeline's per-term handoffs
// would dominate).  The lanes' partial sums are reduced in a fixed order and written
// once: deterministic, no atomics.
__global__ void __launch_bounds__(256) k_tc_tiny(const TfTile* __restrict__ tiles, const TfTask* __restrict__ tasks,
                                                 const TfSrc* __restrict__ srcs, const int* __restrict__ active,
                                                 int n) {
  const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (w >= n) return;
  const TfTile tile = tiles[w];
  if (!active[tile.inst]) return;
  double y[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) y[i][j] = 0.0;
  for (int t = tile.t_begin + lane; t < tile.t_end; t += 32) {
    const TfTask tk = tasks[t];
    double W[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int j = 0; j < 4; ++j) W[k][j] = 0.0;
    for (int si = tk.s_begin; si < tk.s_end; ++si) {
      const TfSrc S = srcs[si];
      const double coef = (double)S.coef;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k >= tk.kdl) break;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (j >= tile.nv) break;
          double acc = 0.0;
          for (int r = 0; r < S.klast; ++r) acc += tiled_val(S.x, tile.xlo, k, r) * tiled_val(S.d, tile.dlo, j, r);
          W[k][j] += coef * acc;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i >= tile.m) break;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k >= tk.kdl) break;
        const double c = tiled_val(tk.c, tile.dlo, i, k);
#pragma unroll
        for (int j = 0; j < 4; ++j) y[i][j] += c * W[k][j];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double v = y[i][j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && i < tile.m && j < tile.nv) tile.y[(int64_t)i * tile.ldy + j] = v;
    }
}

// ------------------------------------------------------------------ conversions

// FP64 blocks -> tiled hi / lo (one CTA per block); identity blocks write their diagonal
__global__ void k_tiled_convert(const TfConv* __restrict__ m) {
  const TfConv M = m[blockIdx.x];
  const int n = M.identity ? M.rows : M.rows * M.cols;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    int r, c;
    double v;
    if (M.identity) {
      r = c = e;
      v = 1.0;
    } else {
      r = e / M.cols;
      c = e - r * M.cols;
      v = M.src[e];
    }
    const int64_t off = ((int64_t)(c >> 5) * M.nrg + (r >> 3)) * 256 + ((c & 31) >> 2) * 32 + (r & 7) * 4 + (c & 3);
    const float f = (float)v;
    const float hi = tf32_round(f);
    M.dst[off] = hi;
    M.dst[off + M.lo] = tf32_round(f - hi);
  }
}

inline void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw std::runtime_error(std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
T* upload(const std::vector<T>& v, Stream s) {
  if (v.empty()) return nullptr;
  T* p = (T*)dev_alloc(v.size() * sizeof(T), s);
  dev_h2d(p, v.data(), v.size() * sizeof(T), s);
  return p;
}

size_t smem_bytes() { return sizeof(float) * (size_t)kSmemF + 1024; }

}  // namespace

struct TcPlan {
  TfTile* tiles = nullptr;
  TfTask* tasks = nullptr;
  TfSrc* srcs = nullptr;
  TfConv* xb = nullptr;
  TfTile* tiny = nullptr;      // tiles for k_tc_tiny
  int ntiny = 0;
  int* queue = nullptr;        // the persistent kernel's tile counter
  int* active = nullptr;       // per instance: 0 = skip its tiles
  int ninst = 0;
  int ntiles = 0, nxb = 0, grid = 0;
  int launches = 0;  // kernels of one launch sequence
};

namespace {

int sm_count() {
  int dev = 0, n = 0;
  ck(cudaGetDevice(&dev), "device");
  ck(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev), "SM count");
  return std::max(n, 1);
}

}  // namespace

TcPlan* tc_plan_build(const std::vector<const TcHost*>& inst, Stream st) {
  TcPlan* P = new TcPlan;
  try {
    std::vector<TfSrc> s;
    std::vector<TfTask> t;
    std::vector<TfTile> tl;
    std::vector<TfConv> xb;
    const bool single = inst.size() == 1;
    int64_t inst_id = 0;
    for (const TcHost* H : inst) {
      if (single) break;  // one instance: its tables are uploaded as they are
      const int s0 = (int)s.size(), t0 = (int)t.size();
      s.insert(s.end(), H->s.begin(), H->s.end());
      for (TfTask q : H->t) {
        q.s_begin += s0;
        q.s_end += s0;
        t.push_back(q);
      }
      for (TfTile q : H->tiles) {
        q.t_begin += t0;
        q.t_end += t0;
        q.group += inst_id << 32;  // groups never span instances
        q.inst = (int)inst_id;
        tl.push_back(q);
      }
      ++inst_id;
      xb.insert(xb.end(), H->xb.begin(), H->xb.end());
    }
    const std::vector<TfTile>& tiles0 = single ? inst[0]->tiles : tl;
    // Tiles of output blocks with the same right sector read the same right-operator
    // blocks: they run together (so that those blocks stay in L2), groups in decreasing
    // order of their largest tile and tiles in decreasing order of work within a group
    // (the hardware starts CTAs in launch order, so the longest work does not finish last)
    std::unordered_map<int64_t, int64_t> gmax;
    for (const TfTile& q : tiles0) {
      int64_t& g = gmax[q.group];
      g = std::max(g, q.cost);
    }
    std::vector<int> order(tiles0.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      const TfTile &A = tiles0[a], &B = tiles0[b];
      const int64_t ga = gmax[A.group], gb = gmax[B.group];
      if (ga != gb) return ga > gb;
      if (A.group != B.group) return A.group < B.group;
      return A.cost > B.cost;
    });
    std::vector<TfTile> sorted, tiny;
    sorted.reserve(tiles0.size());
    for (size_t i = 0; i < order.size(); ++i) (tiles0[order[i]].tiny ? tiny : sorted).push_back(tiles0[order[i]]);
    P->tiny = upload(tiny, st);
    P->ntiny = (int)tiny.size();
    P->grid = (int)std::min<size_t>(sorted.size(), (size_t)sm_count());
    P->queue = (int*)dev_alloc(sizeof(int), st);
    P->ninst = (int)inst.size();
    P->active = upload(std::vector<int>(inst.size(), 1), st);
    P->tiles = upload(sorted, st);
    P->tasks = upload(single ? inst[0]->t : t, st);
    P->srcs = upload(single ? inst[0]->s : s, st);
    P->xb = upload(single ? inst[0]->xb : xb, st);
    P->ntiles = (int)sorted.size();
    P->nxb = (int)(single ? inst[0]->xb.size() : xb.size());
    P->launches = (P->nxb > 0) + (P->ntiles > 0) + (P->ntiny > 0);
  } catch (...) {
    tc_plan_free(P, st);
    throw;
  }
  return P;
}

int* tc_plan_active(TcPlan* p) { return p ? p->active : nullptr; }

void tc_plan_free(TcPlan* p, Stream s) {
  if (!p) return;
  dev_free(p->tiles, s);
  dev_free(p->tasks, s);
  dev_free(p->srcs, s);
  dev_free(p->xb, s);
  dev_free(p->queue, s);
  dev_free(p->tiny, s);
  dev_free(p->active, s);
  delete p;
}

namespace {

void tc_set_attributes() {
  static bool attr = false;
  if (attr) return;
  ck(cudaFuncSetAttribute(k_tc_matvec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes()),
     "tc matvec smem");
  attr = true;
}

void tc_enqueue(const TcPlan* p, void* const* ev, cudaStream_t cs) {
  if (ev) event_record(ev[0], cs);
  if (p->nxb > 0) k_tiled_convert<<<p->nxb, 256, 0, cs>>>(p->xb);
  if (ev) event_record(ev[1], cs);
  if (p->ntiny > 0)
    k_tc_tiny<<<(p->ntiny + 7) / 8, 256, 0, cs>>>(p->tiny, p->tasks, p->srcs, p->active, p->ntiny);
  if (p->ntiles > 0) {
    ck(cudaMemsetAsync(p->queue, 0, sizeof(int), cs), "tile queue reset");
    k_tc_matvec<<<p->grid, kMvThreads, smem_bytes(), cs>>>(p->tiles, p->tasks, p->srcs, p->queue, p->active,
                                                           p->ntiles);
  }
  if (ev) event_record(ev[2], cs);
  ck(cudaGetLastError(), "tc matvec launch");
}

struct TcGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  int launches = 0;
};

}  // namespace

void tc_plan_launch(const TcPlan* p, void* const* ev, Stream s) {
  tc_set_attributes();
  tc_enqueue(p, ev, (cudaStream_t)s);
  note_launches(p->launches);
}

void* tc_graph_create(const TcPlan* p) {
  tc_set_attributes();
  cudaStream_t cs;
  ck(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "graph stream");
  TcGraph* G = new TcGraph;
  G->launches = p->launches;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    tc_enqueue(p, nullptr, cs);
    e = cudaStreamEndCapture(cs, &G->g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&G->ex, G->g, 0);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    if (G->g) cudaGraphDestroy(G->g);
    delete G;
    throw std::runtime_error(std::string("cuda graph of the batched matvec: ") + cudaGetErrorString(e));
  }
  return G;
}

void tc_graph_launch(void* g, Stream s) {
  TcGraph* G = (TcGraph*)g;
  ck(cudaGraphLaunch(G->ex, (cudaStream_t)s), "graph launch");
  note_launches(G->launches);
}

void tc_graph_free(void* g) {
  TcGraph* G = (TcGraph*)g;
  if (!G) return;
  if (G->ex) cudaGraphExecDestroy(G->ex);
  if (G->g) cudaGraphDestroy(G->g);
  delete G;
}

void tc_convert(const std::vector<TfConv>& m, Stream s) {
  if (m.empty()) return;
  TfConv* d = upload(m, s);
  k_tiled_convert<<<(int)m.size(), 256, 0, (cudaStream_t)s>>>(d);
  note_launches(1);
  ck(cudaGetLastError(), "tc convert launch");
  dev_free(d, s);
}

int tc_error_flag(Stream s) {
  int h = 0;
  ck(cudaMemcpyFromSymbolAsync(&h, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, (cudaStream_t)s),
     "tc error flag");
  ck(cudaStreamSynchronize((cudaStream_t)s), "tc error flag");
  if (h) {
    const int zero = 0;
    ck(cudaMemcpyToSymbolAsync(g_tc_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, (cudaStream_t)s),
       "tc error flag");
    ck(cudaStreamSynchronize((cudaStream_t)s), "tc error flag");
  }
  return h;
}

void tc_inject_timeout(int on) {
  const int v = on ? 1 : 0;
  ck(cudaMemcpyToSymbol(g_tc_inject, &v, sizeof(int)), "tc inject");
}

}  // namespace dmrg

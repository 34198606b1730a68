// Mixed-precision H_eff matvec on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Data are FP32 (operators mirrored once per two-site problem, x converted per matvec);
// every block product runs on the tensor cores in TF32 with each operand split into a
// TF32 head and tail (v = hi + lo) and the three leading products hi*hi + hi*lo + lo*hi
// accumulated in FP32 in tensor memory (about 2^-21 relative per product, the accuracy
// of FP32 data).  Operands are staged by the threads into shared memory in the canonical
// K-major layout without swizzle: core matrices of 8 rows x 16 bytes, 128 bytes apart
// along K (LBO) and 1024 bytes apart along M/N (SBO) for a 32-column K chunk.  A thread
// moves one core-matrix row at a time: a float4 from global memory (every FP32 matrix
// has 16-byte aligned rows padded with zeros), split into two float4 stores.  The
// blocks are small and irregular (reduced symmetry blocks of a few to a few hundred
// rows) and are gathered and split while staging, so tensor maps do not apply.
//
// Phase 1 (k_tc_phase1): for a right sector c the x blocks with that sector form a stack
// (rows = sum of their left dimensions, columns = d_c).  Every right-operator block D
// with column sector c gives Z = stack D^T, written transposed (Zt, column-major) so
// that phase 2 reads it K-contiguously.  A CTA keeps a 128-row tile of the stack in
// shared memory and runs through packs of operator blocks placed side by side in the
// MMA's N dimension (up to 128 columns); two accumulators in tensor memory alternate so
// that the epilogue of one pack overlaps the products of the next.
//
// Phase 2 (k_tc_phase2): for an output block of y and a run of its tasks, each task
// stages a left-operator block C (or the identity) as A and W^T = sum coef Zt (the
// complementary-operator sums) as B, and accumulates C W in tensor memory; the tile is
// added to y (FP64) with atomics, since a block's tasks may be split over several CTAs.
//
// Every wait on an MMA-completion barrier is bounded; on timeout the CTA records an
// error, stops issuing work, frees its tensor memory and returns.
#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>

#include "device.hpp"
#include "plans.hpp"

namespace dmrg {

namespace {

constexpr int kThreads = 256;               // 8 warps: all stage, warps w and w+4 share TMEM lanes
constexpr long long kSpinLimit = 1ll << 22; // polls of an mbarrier before giving up (seconds)
constexpr int kTileF = 128 * 32;            // floats of a 128-row x 32-column operand tile

__device__ int g_tc_error = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// float index of element (row, k) in a K-major no-swizzle tile with 32 columns
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

// the three split products of one 32-column K chunk (kpad / 8 steps of K = 8)
__device__ __forceinline__ void mma_chunk(uint32_t tmem, const float* Ah, const float* Al,
                                          const float* Bh, const float* Bl, int kpad, uint32_t idesc,
                                          bool first) {
  const uint32_t ah = smem_u32(Ah), al = smem_u32(Al), bh = smem_u32(Bh), bl = smem_u32(Bl);
  for (int st = 0; st < kpad / 8; ++st) {
    const uint32_t ko = st * 256;  // 8 columns = two core matrices along K
    mma_tf32(tmem, smem_desc(ah + ko), smem_desc(bh + ko), idesc, (first && st == 0) ? 0u : 1u);
    mma_tf32(tmem, smem_desc(ah + ko), smem_desc(bl + ko), idesc, 1u);
    mma_tf32(tmem, smem_desc(al + ko), smem_desc(bh + ko), idesc, 1u);
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  const uint32_t a = smem_u32(mbar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

// 16 consecutive accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

__device__ __forceinline__ void put_split4(float* hi, float* lo, int off, float4 v) {
  float4 h, l;
  h.x = tf32_round(v.x);
  h.y = tf32_round(v.y);
  h.z = tf32_round(v.z);
  h.w = tf32_round(v.w);
  l.x = tf32_round(v.x - h.x);
  l.y = tf32_round(v.y - h.y);
  l.z = tf32_round(v.z - h.z);
  l.w = tf32_round(v.w - h.w);
  *reinterpret_cast<float4*>(hi + off) = h;
  *reinterpret_cast<float4*>(lo + off) = l;
}

__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

// Work item e of a tile with nrows rows: 64 items per 8-row group, item = (row group,
// 4-column group kb, row r7); 32 consecutive items fill 512 consecutive bytes of the tile.
struct Item { int r, kb; };
__device__ __forceinline__ Item item(int e) { return {(e >> 6) * 8 + (e & 7), (e >> 3) & 7}; }

// Stage rows [0, nrows) of a 32-column chunk into hi / lo tiles from row-major FP32 data:
// tile(row_base + r, k) = a X[r ld + k0 + k] for the first kval4 groups of 4 columns,
// zero for the following groups up to nkg (kpad / 4).  Columns past K inside the last
// group read the zero padding of X.  Threads t0, t0 + nthr, ... of the caller; each
// thread issues the loads of up to four items before it uses any of them.
__device__ __forceinline__ void stage4(float* hi, float* lo, int row_base, int nrows, int nkg, int kval4,
                                       const float* __restrict__ X, int ld, int k0, float a, int t0,
                                       int nthr) {
  const int ne = ((nrows + 7) >> 3) * 64;
  if (ne <= nthr) {  // one item per thread at most
    if (t0 >= ne) return;
    const Item it = item(t0);
    if (it.r >= nrows || it.kb >= nkg) return;
    float4 v = it.kb < kval4 ? ldg4(X + (size_t)it.r * ld + k0 + it.kb * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
    v.x *= a;
    v.y *= a;
    v.z *= a;
    v.w *= a;
    put_split4(hi, lo, kmo(row_base + it.r, it.kb * 4), v);
    return;
  }
  for (int e0 = 0; e0 < ne; e0 += 4 * nthr) {
    float4 v[4];
    Item it[4];
    bool st[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = e0 + t0 + i * nthr;
      it[i] = item(e);
      st[i] = e < ne && it[i].r < nrows && it[i].kb < nkg;
      v[i] = (st[i] && it[i].kb < kval4) ? ldg4(X + (size_t)it[i].r * ld + k0 + it[i].kb * 4)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (st[i]) {
        v[i].x *= a;
        v[i].y *= a;
        v[i].z *= a;
        v[i].w *= a;
        put_split4(hi, lo, kmo(row_base + it[i].r, it[i].kb * 4), v[i]);
      }
  }
}

// A = alpha * identity rows row0 .. row0 + nrows - 1 of a K x K identity, columns k0 ..
__device__ __forceinline__ void stage4_identity(float* hi, float* lo, int nrows, int nkg, int kvalid, int row0,
                                                int k0, float alpha, int t0, int nthr) {
  const int ne = ((nrows + 7) >> 3) * 64;
  for (int e = t0; e < ne; e += nthr) {
    const Item it = item(e);
    if (it.r >= nrows || it.kb >= nkg) continue;
    const int d = row0 + it.r - k0 - it.kb * 4;  // column of the diagonal inside the group
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (d >= 0 && d < 4 && k0 + it.kb * 4 + d < k0 + kvalid) (&v.x)[d] = alpha;
    put_split4(hi, lo, kmo(it.r, it.kb * 4), v);
  }
}

// B = W^T rows col0 .. col0 + nrows - 1: sum over sources of coef * z[(col0 + j) ldz + k0 + k].
// Up to four items per thread; the loads of two sources are issued before their sums.
__device__ __forceinline__ void stage4_wsum(float* hi, float* lo, int nrows, int nkg, int kval4,
                                            const Tc2Src* __restrict__ srcs, int s_begin, int s_end, int col0,
                                            int k0, int t0, int nthr) {
  const int ne = ((nrows + 7) >> 3) * 64;
  for (int e0 = 0; e0 < ne; e0 += 4 * nthr) {
    float4 acc[4];
    Item it[4];
    bool ld[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = e0 + t0 + i * nthr;
      it[i] = item(e);
      if (e >= ne) it[i].r = 1 << 20;
      ld[i] = it[i].r < nrows && it[i].kb < kval4;
      acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int si = s_begin; si < s_end; si += 2) {
      const bool two = si + 1 < s_end;
      const Tc2Src S0 = srcs[si];
      const Tc2Src S1 = two ? srcs[si + 1] : S0;
      const float* z0 = S0.z + (size_t)col0 * S0.ldz + k0;
      const float* z1 = S1.z + (size_t)col0 * S1.ldz + k0;
      float4 v0[4], v1[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        v0[i] = ld[i] ? ldg4(z0 + (size_t)it[i].r * S0.ldz + it[i].kb * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
        v1[i] = (ld[i] && two) ? ldg4(z1 + (size_t)it[i].r * S1.ldz + it[i].kb * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = fma4(S1.coef, v1[i], fma4(S0.coef, v0[i], acc[i]));
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (it[i].r < nrows && it[i].kb < nkg) put_split4(hi, lo, kmo(it[i].r, it[i].kb * 4), acc[i]);
  }
}

// ------------------------------------------------------------------ phase 1

constexpr int kMaxPackEntries = 16;  // pack columns are padded per entry to multiples of 8

// shared-memory floats: one-chunk units keep the stack tile (hi, lo) and two B buffers;
// multi-chunk units double-buffer A and B together
template <bool kOne>
constexpr int p1_smem_floats() { return kOne ? 6 * kTileF : 8 * kTileF; }

template <bool kOne>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_phase1(const Tc1Unit* __restrict__ units, const Tc1Pack* __restrict__ packs,
                const Tc1Entry* __restrict__ ents) {
  extern __shared__ unsigned char smem_dyn[];
  float* sm = (float*)(((uintptr_t)smem_dyn + 127) & ~(uintptr_t)127);
  __shared__ __align__(8) uint64_t mbar_buf[2];
  __shared__ __align__(8) uint64_t mbar_acc[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ Tc1Entry pent[2][kMaxPackEntries];
  __shared__ signed char pgrp[2][16];  // entry of each 8-column group, -1 = none
  __shared__ int pn[2];

  const Tc1Unit u = units[blockIdx.x];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&tmem_slot, 256);
  if (tid == 0) {
    mbar_init(&mbar_buf[0]);
    mbar_init(&mbar_buf[1]);
    mbar_init(&mbar_acc[0]);
    mbar_init(&mbar_acc[1]);
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  const int nch = (u.K + 31) >> 5;
  if (kOne) {
    const int kpad = (u.K + 7) & ~7;
    stage4(sm, sm + kTileF, 0, u.rows, kpad >> 2, (u.K + 3) >> 2, u.A, u.lda, 0, 1.0f, tid, kThreads);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  uint32_t ph_buf[2] = {0, 0}, ph_acc[2] = {0, 0};

  // epilogue of pack slot a: accumulator columns -> Zt (column-major, coalesced along rows)
  auto epilogue = [&](int a) {
    if (tid == 0 && !mbar_wait(&mbar_acc[a], ph_acc[a])) {
      atomicExch(&g_tc_error, 1);
      abort_flag = 1;
    }
    ph_acc[a] ^= 1;
    __syncthreads();
    if (abort_flag) return;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int q = warp & 3, h = warp >> 2;
    const int r = q * 32 + lane;
    const int n16 = (pn[a] + 15) & ~15;
    for (int c0 = h * 16; c0 < n16; c0 += 32) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * 128 + c0), v);
#pragma unroll
      for (int g8 = 0; g8 < 2; ++g8) {
        const int e = pgrp[a][(c0 >> 3) + g8];
        if (e < 0 || r >= u.rows) continue;
        const Tc1Entry& E = pent[a][e];
        const int j0 = c0 + 8 * g8 - E.start, nc = E.ncols, ldz = E.ldz;
        float* zp = E.zt + (size_t)j0 * ldz + u.row0 + r;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (j0 + j < nc) zp[(size_t)j * ldz] = v[8 * g8 + j];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  };

  int s = 0;
  const int npk = u.p_end - u.p_begin;
  for (int pi = 0; pi < npk && !abort_flag; ++pi) {
    const Tc1Pack P = packs[u.p_begin + pi];
    const int slot = pi & 1;
    const int nent = P.e_end - P.e_begin;
    if (tid < nent) pent[slot][tid] = ents[P.e_begin + tid];
    if (tid == 0) pn[slot] = P.n;
    for (int ch = 0; ch < nch; ++ch, ++s) {
      const int b = s & 1;
      if (s >= 2) {
        if (tid == 0 && !mbar_wait(&mbar_buf[b], ph_buf[b])) {
          atomicExch(&g_tc_error, 1);
          abort_flag = 1;
        }
        ph_buf[b] ^= 1;
      }
      __syncthreads();
      if (abort_flag) break;
      if (ch == 0 && tid < 16) {
        int g = -1;
        for (int e = 0; e < nent; ++e) {
          const int st = pent[slot][e].start, en = st + ((pent[slot][e].ncols + 7) & ~7);
          if (tid * 8 >= st && tid * 8 < en) g = e;
        }
        pgrp[slot][tid] = (signed char)g;
      }
      const int k0 = ch * 32, kvalid = min(32, u.K - k0), kpad = (kvalid + 7) & ~7;
      const int nkg = kpad >> 2, kval4 = (kvalid + 3) >> 2;
      float* Ah = kOne ? sm : sm + b * 4 * kTileF;
      float* Al = Ah + kTileF;
      float* Bh = kOne ? sm + (2 + 2 * b) * kTileF : Ah + 2 * kTileF;
      float* Bl = Bh + kTileF;
      if (!kOne) stage4(Ah, Al, 0, u.rows, nkg, kval4, u.A, u.lda, k0, 1.0f, tid, kThreads);
      for (int e = 0; e < nent; ++e) {
        const Tc1Entry& E = pent[slot][e];
        stage4(Bh, Bl, E.start, E.ncols, nkg, kval4, E.D, E.ldd, k0, E.alpha, tid, kThreads);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        mma_chunk(tmem + (uint32_t)(slot * 128), Ah, Al, Bh, Bl, kpad, idesc_tf32((P.n + 15) & ~15), ch == 0);
        mma_commit(&mbar_buf[b]);
        if (ch == nch - 1) mma_commit(&mbar_acc[slot]);
      }
    }
    if (abort_flag) break;
    if (pi >= 1) epilogue((pi - 1) & 1);
  }
  if (!abort_flag && npk > 0) epilogue((npk - 1) & 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 256);
}

// ------------------------------------------------------------------ phase 2

// The tensor core's FP32 accumulation loses accuracy over long runs of products (the
// error of a 48-task run measured ~10x that of a 2-task run), so phase 2 adds its
// accumulator into FP32 registers every kSegSteps steps and restarts it.
constexpr int kSegSteps = 2;

// Output tiles of more than 32 rows: all 8 warps stage each step, double-buffered, and
// drain the accumulator at segment ends.
constexpr int kP2BufF = 3 * kTileF;  // A hi, A lo (128 rows), B hi, B lo (64 rows)

__global__ void __launch_bounds__(kThreads, 1)
    k_tc_phase2(const Tc2Unit* __restrict__ units, const Tc2Task* __restrict__ tasks,
                const Tc2Src* __restrict__ srcs) {
  extern __shared__ unsigned char smem_dyn[];
  float* sm = (float*)(((uintptr_t)smem_dyn + 127) & ~(uintptr_t)127);
  __shared__ __align__(8) uint64_t mbar_buf[2];
  __shared__ __align__(8) uint64_t mbar_seg;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const Tc2Unit u = units[blockIdx.x];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mv = min(128, u.m - u.row0), nv = min(64, u.n - u.col0);
  const int n16 = (nv + 15) & ~15;
  const int q = warp & 3, h = warp >> 2;
  if (warp == 0) tmem_alloc(&tmem_slot, 64);
  if (tid == 0) {
    mbar_init(&mbar_buf[0]);
    mbar_init(&mbar_buf[1]);
    mbar_init(&mbar_seg);
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_tf32(n16);
  uint32_t ph_buf[2] = {0, 0}, ph_seg = 0;
  float acc[2][16];  // this thread's row, columns h*16 + 32*i + j, summed over segments
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[i][j] = 0.0f;
  int nsteps = 0;
  for (int t = u.t_begin; t < u.t_end; ++t) nsteps += (tasks[t].K + 31) >> 5;
  int s = 0, seg_first = 0;
  for (int t = u.t_begin; t < u.t_end && !abort_flag; ++t) {
    const Tc2Task T = tasks[t];
    const int nch = (T.K + 31) >> 5;
    for (int ch = 0; ch < nch; ++ch, ++s) {
      const int b = s & 1;
      if (s >= 2) {  // the MMA of step s - 2 must be done with this buffer
        if (tid == 0 && !mbar_wait(&mbar_buf[b], ph_buf[b])) {
          atomicExch(&g_tc_error, 1);
          abort_flag = 1;
        }
        ph_buf[b] ^= 1;
      }
      __syncthreads();
      if (abort_flag) break;
      const int k0 = ch * 32, kvalid = min(32, T.K - k0), kpad = (kvalid + 7) & ~7;
      const int nkg = kpad >> 2, kval4 = (kvalid + 3) >> 2;
      float* Ah = sm + b * kP2BufF;
      float* Al = Ah + kTileF;
      float* Bh = Al + kTileF;
      float* Bl = Bh + kTileF / 2;
      if (T.C) stage4(Ah, Al, 0, mv, nkg, kval4, T.C + (size_t)u.row0 * T.ldc, T.ldc, k0, T.alpha, tid, kThreads);
      else stage4_identity(Ah, Al, mv, nkg, kvalid, u.row0, k0, T.alpha, tid, kThreads);
      stage4_wsum(Bh, Bl, nv, nkg, kval4, srcs, T.s_begin, T.s_end, u.col0, k0, tid, kThreads);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      const bool seg_end = (s + 1 - seg_first == kSegSteps) || (s + 1 == nsteps);
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        mma_chunk(tmem, Ah, Al, Bh, Bl, kpad, idesc, s == seg_first);
        mma_commit(&mbar_buf[b]);
        if (seg_end) mma_commit(&mbar_seg);
      }
      if (seg_end) {
        // promote the segment's FP32 accumulator to the register sums, then restart it
        if (tid == 0 && !mbar_wait(&mbar_seg, ph_seg)) {
          atomicExch(&g_tc_error, 1);
          abort_flag = 1;
        }
        ph_seg ^= 1;
        __syncthreads();
        if (abort_flag) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int c0 = h * 16 + 32 * i;
          if (c0 < n16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[i][j] += v[j];
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        seg_first = s + 1;
      }
    }
  }
  __syncthreads();
  const int r = q * 32 + lane;
  if (s > 0 && !abort_flag && r < mv) {
    double* yr = u.y + (size_t)(u.row0 + r) * u.ldy + u.col0;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = h * 16 + 32 * i + j;
        if (c < nv) atomicAdd(yr + c, (double)acc[i][j]);
      }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) tmem_free(tmem, 64);
}

// Phase 2 for output tiles of at most 32 rows (the common case of small symmetry
// blocks), as a warp-specialised pipeline: four producer groups of two warps each own
// one shared-memory stage and fill it for every fourth step (a step is one 32-column K
// chunk of one task); one thread issues the MMAs of the steps in order and releases
// each stage with tcgen05.commit.  A stage holds A = 32 rows of C (hi, lo) and B = 64
// rows of W^T (hi, lo); the MMA still reads 128 rows of A, and rows 32..127 fall on the
// rest of the same stage: they only produce accumulator rows that are never read.
constexpr int kGroups = 4, kGroupThreads = 64;
constexpr int kAcc = 4;  // TMEM accumulators (64 columns each) of the MMA warp's segments
constexpr int kUnitTasks = 128, kUnitSrcs = 384;  // descriptors held in shared memory
constexpr int kP2sThreads = kGroups * kGroupThreads + 32;
constexpr int kSA = 32 * 32, kSB = 64 * 32;   // floats of an A (32-row) / B (64-row) tile
constexpr int kP2sStageF = 2 * kSA + 2 * kSB;  // 24 KB: the 16 KB A footprint stays inside

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_init_n(uint64_t* mbar, int n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(n));
}

// bounded wait that also gives up once another thread has flagged an abort
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* mbar, uint32_t parity, volatile int* abort_flag) {
  const uint32_t a = smem_u32(mbar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 1023) == 1023 && *abort_flag) return false;
  }
  atomicExch(&g_tc_error, 1);
  *abort_flag = 1;
  return false;
}

__global__ void __launch_bounds__(kP2sThreads, 2)
    k_tc_phase2s(const Tc2Unit* __restrict__ units, const Tc2Task* __restrict__ tasks,
                 const Tc2Src* __restrict__ srcs) {
  extern __shared__ unsigned char smem_dyn[];
  float* sm = (float*)(((uintptr_t)smem_dyn + 127) & ~(uintptr_t)127);
  __shared__ __align__(8) uint64_t full[kGroups];
  __shared__ __align__(8) uint64_t empty[kGroups];
  __shared__ __align__(8) uint64_t accf[kAcc];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  // the unit's task and source descriptors, loaded once (the loops would otherwise put
  // a dependent global load in front of every step)
  __shared__ Tc2Task stask[kUnitTasks];
  __shared__ Tc2Src ssrc[kUnitSrcs];

  const Tc2Unit u = units[blockIdx.x];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mv = u.m - u.row0, nv = min(64, u.n - u.col0);  // mv <= 32 by construction
  const int n16 = (nv + 15) & ~15;
  const int ntask = u.t_end - u.t_begin;  // <= kUnitTasks by construction
  const int s0 = tasks[u.t_begin].s_begin, nsrc = tasks[u.t_end - 1].s_end - s0;
  const Tc2Src* S = nsrc <= kUnitSrcs ? ssrc : srcs + s0;  // sources relative to s0
  for (int k = tid; k < ntask; k += kP2sThreads) stask[k] = tasks[u.t_begin + k];
  if (nsrc <= kUnitSrcs)
    for (int k = tid; k < nsrc; k += kP2sThreads) ssrc[k] = srcs[s0 + k];
  if (warp == kGroups * 2) tmem_alloc(&tmem_slot, 64 * kAcc);
  if (tid == 0) {
    for (int g = 0; g < kGroups; ++g) {
      mbar_init_n(&full[g], kGroupThreads);
      mbar_init_n(&empty[g], 1);
    }
    for (int a = 0; a < kAcc; ++a) mbar_init_n(&accf[a], 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  if (warp < kGroups * 2) {
    // ---- producers: group g fills stage g for steps s = g, g + 4, ...
    const int g = warp >> 1, gt = tid & (kGroupThreads - 1);
    float* Ah = sm + g * kP2sStageF;
    float* Al = Ah + kSA;
    float* Bh = Al + kSA;
    float* Bl = Bh + kSB;
    int s = 0;
    for (int t = 0; t < ntask && !abort_flag; ++t) {
      const Tc2Task& T = stask[t];
      const int nch = (T.K + 31) >> 5;
      for (int ch = 0; ch < nch; ++ch, ++s) {
        if ((s & (kGroups - 1)) != g) continue;
        const int k = s / kGroups;  // fill number of this stage
        if (k > 0 && !mbar_wait_or_abort(&empty[g], (k - 1) & 1, &abort_flag)) break;
        const int k0 = ch * 32, kvalid = min(32, T.K - k0), kpad = (kvalid + 7) & ~7;
        const int nkg = kpad >> 2, kval4 = (kvalid + 3) >> 2;
        if (T.C) stage4(Ah, Al, 0, mv, nkg, kval4, T.C + (size_t)u.row0 * T.ldc, T.ldc, k0, T.alpha, gt, kGroupThreads);
        else stage4_identity(Ah, Al, mv, nkg, kvalid, u.row0, k0, T.alpha, gt, kGroupThreads);
        stage4_wsum(Bh, Bl, nv, nkg, kval4, S, T.s_begin - s0, T.s_end - s0, u.col0, k0, gt, kGroupThreads);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&full[g]);
      }
    }
  } else {
    // ---- warp 8: lane 0 issues the MMAs of segment j into accumulator j % kAcc; the
    // warp adds finished segments (accumulator rows 0..31 = TMEM lanes 0..31) to its
    // registers kAcc - 1 segments behind, so the tensor core always has work queued
    const uint32_t idesc = idesc_tf32(n16);
    float acc[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) acc[i] = 0.0f;
    uint32_t ph_acc[kAcc];
#pragma unroll
    for (int a = 0; a < kAcc; ++a) ph_acc[a] = 0;
    auto drain = [&](int a) {
      int ok = 1;
      if (lane == 0) ok = mbar_wait_or_abort(&accf[a], ph_acc[a], &abort_flag);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) return;
      ph_acc[a] ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (16 * i < n16) {
          float v[16];
          tmem_ld16(tmem + (uint32_t)(a * 64 + 16 * i), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[16 * i + j] += v[j];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
    };
    int s = 0, seg = 0, in_seg = 0, drained = 0;
    bool stop = false;
    for (int t = 0; t < ntask && !stop; ++t) {
      const int K = stask[t].K;
      const int nch = (K + 31) >> 5;
      for (int ch = 0; ch < nch; ++ch, ++s) {
        const int g = s & (kGroups - 1);
        if (lane == 0) {
          if (mbar_wait_or_abort(&full[g], (s / kGroups) & 1, &abort_flag)) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int kvalid = min(32, K - ch * 32), kpad = (kvalid + 7) & ~7;
            float* Ah = sm + g * kP2sStageF;
            mma_chunk(tmem + (uint32_t)((seg % kAcc) * 64), Ah, Ah + kSA, Ah + 2 * kSA, Ah + 2 * kSA + kSB, kpad,
                      idesc, in_seg == 0);
            mma_commit(&empty[g]);
          }
        }
        if (__shfl_sync(0xffffffffu, (int)abort_flag, 0)) { stop = true; break; }
        if (++in_seg == kSegSteps) {
          if (lane == 0) mma_commit(&accf[seg % kAcc]);
          __syncwarp();
          ++seg;
          in_seg = 0;
          // the accumulator of segment `seg` is reused next: keep at most kAcc - 1 pending
          while (seg - drained > kAcc - 1) drain(drained++ % kAcc);
        }
      }
    }
    if (!stop && !__shfl_sync(0xffffffffu, (int)abort_flag, 0)) {
      if (in_seg > 0) {
        if (lane == 0) mma_commit(&accf[seg % kAcc]);
        __syncwarp();
        ++seg;
      }
      while (drained < seg) drain(drained++ % kAcc);
      if (!__shfl_sync(0xffffffffu, (int)abort_flag, 0) && lane < mv) {
        double* yr = u.y + (size_t)(u.row0 + lane) * u.ldy + u.col0;
#pragma unroll
        for (int j = 0; j < 64; ++j)
          if (j < nv) atomicAdd(yr + j, (double)acc[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == kGroups * 2) tmem_free(tmem, 64 * kAcc);
}

// ------------------------------------------------------------------ conversions

// x (FP64) -> the FP32 stacks (row-major) and their transposes, one CTA per x block
__global__ void k_x_prep(const TcXBlock* __restrict__ xb) {
  const TcXBlock B = xb[blockIdx.x];
  const int n = B.rows * B.cols;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int r = e / B.cols, c = e - r * B.cols;
    const float v = (float)B.src[e];
    B.dst[(int64_t)r * B.ld + c] = v;
    B.dstt[(int64_t)c * B.ldt + r] = v;
  }
}

// FP64 blocks (row-major, stride cols) -> FP32 with row stride ld, one CTA per block
__global__ void k_mirror(const TcMirror* __restrict__ m) {
  const TcMirror M = m[blockIdx.x];
  const int n = M.rows * M.cols;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int r = e / M.cols, c = e - r * M.cols;
    M.dst[(int64_t)r * M.ld + c] = (float)M.src[e];
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

size_t smem_bytes(int floats) { return sizeof(float) * (size_t)floats + 128; }

}  // namespace

struct TcPlan {
  Tc1Entry* ents = nullptr;
  Tc1Pack* packs = nullptr;
  Tc1Unit* u1 = nullptr;      // one-chunk units first, then multi-chunk units
  int n1_one = 0, n1_multi = 0;
  Tc2Src* srcs = nullptr;
  Tc2Task* tasks = nullptr;
  Tc2Unit* u2 = nullptr;      // tiles of at most 32 rows first, then the others
  int n2_small = 0, n2 = 0;
  TcXBlock* xb = nullptr;
  int nxb = 0;
  std::vector<std::pair<double*, int64_t>> clear;  // outputs zeroed before the products
  int launches = 0;           // kernels of one launch sequence
};

TcPlan* tc_plan_build(const std::vector<const TcHost*>& inst, TcTune tune, Stream st) {
  if (tune.packs_per_unit < 1 || tune.tasks_per_unit < 1 || tune.tasks_per_unit > kUnitTasks)
    throw std::invalid_argument("tc tuning");
  std::vector<Tc1Entry> e;
  std::vector<Tc1Pack> p;
  std::vector<Tc1Unit> u1, u1m;
  std::vector<Tc2Src> sr;
  std::vector<Tc2Task> t;
  std::vector<Tc2Unit> u2, u2g;
  std::vector<TcXBlock> xb;
  TcPlan* P = new TcPlan;
  // one instance: its tables are uploaded as they are (indices need no offsets)
  const bool single = inst.size() == 1;
  for (const TcHost* H : inst) {
    const int e0 = (int)e.size(), p0 = (int)p.size(), s0 = (int)sr.size(), t0 = (int)t.size();
    for (const Tc1Pack& q : H->p)
      if (q.e_end - q.e_begin > kMaxPackEntries || q.n > 128) throw std::logic_error("tc pack too large");
    if (!single) {
      e.insert(e.end(), H->e.begin(), H->e.end());
      for (Tc1Pack q : H->p) {
        q.e_begin += e0;
        q.e_end += e0;
        p.push_back(q);
      }
    }
    for (const Tc1Unit& r : H->r1)
      for (int pb = r.p_begin; pb < r.p_end; pb += tune.packs_per_unit) {
        Tc1Unit u = r;
        u.p_begin = p0 + pb;
        u.p_end = p0 + std::min(r.p_end, pb + tune.packs_per_unit);
        (r.K <= 32 ? u1 : u1m).push_back(u);
      }
    if (!single) {
      sr.insert(sr.end(), H->s.begin(), H->s.end());
      for (Tc2Task q : H->t) {
        q.s_begin += s0;
        q.s_end += s0;
        t.push_back(q);
      }
    }
    for (const Tc2Unit& r : H->r2)
      for (int tb = r.t_begin; tb < r.t_end; tb += tune.tasks_per_unit) {
        Tc2Unit u = r;
        u.t_begin = t0 + tb;
        u.t_end = t0 + std::min(r.t_end, tb + tune.tasks_per_unit);
        (r.m - r.row0 <= 32 ? u2 : u2g).push_back(u);
      }
    if (!single) xb.insert(xb.end(), H->xb.begin(), H->xb.end());
    if (H->yout && H->n > 0) P->clear.push_back({H->yout, H->n});
  }
  P->n1_one = (int)u1.size();
  P->n1_multi = (int)u1m.size();
  u1.insert(u1.end(), u1m.begin(), u1m.end());
  P->n2_small = (int)u2.size();
  u2.insert(u2.end(), u2g.begin(), u2g.end());
  P->n2 = (int)u2.size();
  const TcHost* H0 = single ? inst[0] : nullptr;
  P->ents = upload(single ? H0->e : e, st);
  P->packs = upload(single ? H0->p : p, st);
  P->u1 = upload(u1, st);
  P->srcs = upload(single ? H0->s : sr, st);
  P->tasks = upload(single ? H0->t : t, st);
  P->u2 = upload(u2, st);
  P->xb = upload(single ? H0->xb : xb, st);
  P->nxb = (int)(single ? H0->xb.size() : xb.size());
  P->launches = (P->nxb > 0) + (P->n1_one > 0) + (P->n1_multi > 0) + (P->n2_small > 0) + (P->n2 > P->n2_small);
  return P;
}

void tc_plan_free(TcPlan* p, Stream s) {
  if (!p) return;
  dev_free(p->ents, s);
  dev_free(p->packs, s);
  dev_free(p->u1, s);
  dev_free(p->srcs, s);
  dev_free(p->tasks, s);
  dev_free(p->u2, s);
  dev_free(p->xb, s);
  delete p;
}

namespace {

void tc_set_attributes() {
  static bool attr = false;
  if (attr) return;
  ck(cudaFuncSetAttribute(k_tc_phase1<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem_bytes(p1_smem_floats<true>())), "tc phase 1 smem");
  ck(cudaFuncSetAttribute(k_tc_phase1<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem_bytes(p1_smem_floats<false>())), "tc phase 1 smem");
  ck(cudaFuncSetAttribute(k_tc_phase2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem_bytes(2 * kP2BufF)), "tc phase 2 smem");
  ck(cudaFuncSetAttribute(k_tc_phase2s, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)smem_bytes(kGroups * kP2sStageF)), "tc phase 2 smem");
  attr = true;
}

void tc_enqueue(const TcPlan* p, void* const* ev, cudaStream_t cs) {
  if (ev) event_record(ev[0], cs);
  for (const auto& c : p->clear) ck(cudaMemsetAsync(c.first, 0, sizeof(double) * (size_t)c.second, cs), "tc zero y");
  if (p->nxb > 0) k_x_prep<<<p->nxb, 256, 0, cs>>>(p->xb);
  if (p->n1_one > 0)
    k_tc_phase1<true><<<p->n1_one, kThreads, smem_bytes(p1_smem_floats<true>()), cs>>>(p->u1, p->packs, p->ents);
  if (p->n1_multi > 0)
    k_tc_phase1<false><<<p->n1_multi, kThreads, smem_bytes(p1_smem_floats<false>()), cs>>>(
        p->u1 + p->n1_one, p->packs, p->ents);
  if (ev) event_record(ev[1], cs);
  if (p->n2_small > 0)
    k_tc_phase2s<<<p->n2_small, kP2sThreads, smem_bytes(kGroups * kP2sStageF), cs>>>(p->u2, p->tasks, p->srcs);
  if (p->n2 > p->n2_small)
    k_tc_phase2<<<p->n2 - p->n2_small, kThreads, smem_bytes(2 * kP2BufF), cs>>>(p->u2 + p->n2_small, p->tasks,
                                                                                 p->srcs);
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

void tc_mirror(const std::vector<TcMirror>& m, Stream s) {
  if (m.empty()) return;
  TcMirror* d = upload(m, s);
  k_mirror<<<(int)m.size(), 256, 0, (cudaStream_t)s>>>(d);
  note_launches(1);
  ck(cudaGetLastError(), "tc mirror launch");
  dev_free(d, s);
}

int tc_error_flag(Stream s) {
  int h = 0;
  ck(cudaMemcpyFromSymbolAsync(&h, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, (cudaStream_t)s),
     "tc error flag");
  ck(cudaStreamSynchronize((cudaStream_t)s), "tc error flag");
  return h;
}

}  // namespace dmrg

// Tensor-core (tcgen05, sm_103a) grouped block GEMM for the mixed-precision matvec.
//
// C_g += sum_t alpha_t op(A_t) op(B_t) as in k_grouped_gemm, with every product done on
// the 5th-generation tensor cores in TF32 with FP32 accumulation, each operand split
// into a TF32 head and a TF32 tail (a = a_hi + a_lo) and the three leading products
// a_hi b_hi + a_hi b_lo + a_lo b_hi accumulated (about 2^-21 relative per product).
// One CTA (4 warps) owns a 128 x 64 tile of one output block (the MMA N is the block's
// width rounded up to 16, at most 64); its FP32 accumulator lives in tensor memory for
// the whole task list of the block and is added to the FP64 output once.  Two staging
// buffers alternate, so the next K chunk is staged while the tensor core consumes the
// previous one.  Operands are read from FP64 global memory (the coefficient alpha
// is applied while staging), rounded / split, and written to shared memory in the
// canonical K-major layout without swizzle: 8-row x 16-byte core matrices, core
// matrices adjacent in K 128 bytes apart (LBO), adjacent in M/N 1024 bytes apart (SBO)
// for a 32-wide K chunk.  The operand blocks are small and irregular (reduced symmetry
// blocks of tens to a few hundred rows), so they are staged by the threads rather than
// by TMA tensor maps.  Every wait on the MMA-completion barrier is bounded; on timeout
// the CTA records an error, frees its tensor memory and returns.
#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>

#include "device.hpp"
#include "plans.hpp"

namespace dmrg {

namespace {

constexpr int TM = 128, TN = 64, TK = 32;
constexpr int kThreads = 128;
constexpr uint32_t kTmemCols = 64;
constexpr long long kSpinLimit = 1ll << 22;  // a few seconds at most

__device__ int g_tc_error = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of element (row, k) inside a K-major no-swizzle tile with TK columns
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  // start address >> 4 | LBO (128 B) >> 4 << 16 | SBO (1024 B) >> 4 << 32 | version 1 << 46
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: D f32, A/B tf32, both K-major, N = TN, M = TM
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Stage alpha * op(X)[r0 + r][k0 + k] for r < vrows, k < kpad into hi / lo tiles (the
// other rows of the tile stay zero from the initial clear; columns in [kvalid, kpad) are
// written as zeros).  op = identity if trans == 0, transpose otherwise; X == nullptr
// stands for the identity matrix.  Threads walk core matrices (8 rows x 4 columns =
// 128 contiguous bytes) so that consecutive threads write consecutive words.
__device__ __forceinline__ void stage(float* hi, float* lo, int vrows, int kvalid, int kpad,
                                      const double* X, int ld, int trans, int r0, int k0,
                                      double alpha) {
  const int nkb = kpad >> 2;                 // 4-column groups
  const int ncm = ((vrows + 7) >> 3) * nkb;  // core matrices touched
  for (int e = threadIdx.x; e < ncm * 32; e += kThreads) {
    const int q = e & 31, cm = e >> 5;
    const int r = (cm / nkb) * 8 + (q >> 2), k = (cm % nkb) * 4 + (q & 3);
    if (r >= vrows) continue;
    double v = 0.0;
    if (k < kvalid) {
      const int gr = r0 + r, gk = k0 + k;
      if (X == nullptr) v = (gr == gk) ? alpha : 0.0;
      else v = alpha * (trans ? X[(size_t)gk * ld + gr] : X[(size_t)gr * ld + gk]);
    }
    const float h = tf32_round((float)v);
    const float l = tf32_round((float)(v - (double)h));
    const uint32_t off = kmajor_off(r, k) >> 2;
    hi[off] = h;
    lo[off] = l;
  }
}

constexpr int kStageFloats = 2 * TM * TK + 2 * TN * TK;  // A hi, A lo, B hi, B lo

__global__ void __launch_bounds__(kThreads, 1) k_grouped_gemm_tc(const GemmTask* __restrict__ tasks,
                                                                const GemmGroup* __restrict__ groups,
                                                                int ngroups) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float* buf[2] = {(float*)smem_raw, (float*)smem_raw + kStageFloats};
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int tile = blockIdx.x;
  int lo_g = 0, hi_g = ngroups - 1;
  while (lo_g < hi_g) {
    int mid = (lo_g + hi_g + 1) >> 1;
    if (groups[mid].tile_begin_tc <= tile) lo_g = mid; else hi_g = mid - 1;
  }
  const GemmGroup g = groups[lo_g];
  const int local = tile - g.tile_begin_tc;
  const int tn = (g.n + TN - 1) / TN;
  const int row0 = (local / tn) * TM, col0 = (local % tn) * TN;
  const int vrows_a = min(TM, g.m - row0), vrows_b = min(TN, g.n - col0);
  const int nmma = min(TN, (vrows_b + 15) & ~15);  // MMA N: multiple of 16, at most 64
  const uint32_t idesc = (kIdesc & ~(0x3Fu << 17)) | ((uint32_t)(nmma >> 3) << 17);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  for (int e = threadIdx.x; e < 2 * kStageFloats; e += kThreads) ((float*)smem_raw)[e] = 0.0f;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  uint32_t phase[2] = {0, 0};
  bool pending[2] = {false, false};
  uint32_t accumulate = 0;
  int chunk = 0;

  for (int t = g.task_begin; t < g.task_end && !abort_flag; ++t) {
    const GemmTask T = tasks[t];
    // op(A) is m x k, op(B) is k x n; the tensor core reads B as n x k (K-major), i.e.
    // op(B)^T: rows n, columns k  ->  stage B with the opposite transpose flag
    const int K = T.A ? T.k : g.m;
    for (int k0 = 0; k0 < K && !abort_flag; k0 += TK, ++chunk) {
      const int b = chunk & 1;
      if (pending[b]) {  // the tensor core must be done with this buffer
        if (!mbar_wait(smem_u32(&mbar[b]), phase[b])) { atomicExch(&g_tc_error, 1); abort_flag = 1; }
        phase[b] ^= 1;
        pending[b] = false;
        __syncthreads();
        if (abort_flag) break;
      }
      const int kvalid = min(TK, K - k0);
      const int kpad = (kvalid + 7) & ~7;
      float* Ahi = buf[b];
      float* Alo = Ahi + TM * TK;
      float* Bhi = Alo + TM * TK;
      float* Blo = Bhi + TN * TK;
      stage(Ahi, Alo, vrows_a, kvalid, kpad, T.A, T.lda, T.transA, row0, k0, T.alpha);
      stage(Bhi, Blo, vrows_b, kvalid, kpad, T.B, T.ldb, !T.transB, col0, k0, 1.0);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a_hi = smem_u32(Ahi), a_lo = smem_u32(Alo);
        const uint32_t b_hi = smem_u32(Bhi), b_lo = smem_u32(Blo);
        for (int st = 0; st < kpad / 8; ++st) {  // K = 8 per instruction
          const uint32_t ko = st * 256;
          mma_tf32(tmem, smem_desc(a_hi + ko), smem_desc(b_hi + ko), idesc, accumulate);
          accumulate = 1;
          mma_tf32(tmem, smem_desc(a_hi + ko), smem_desc(b_lo + ko), idesc, 1);
          mma_tf32(tmem, smem_desc(a_lo + ko), smem_desc(b_hi + ko), idesc, 1);
        }
        mma_commit(smem_u32(&mbar[b]));
      }
      pending[b] = true;
      accumulate = 1;
    }
  }
  for (int b = 0; b < 2; ++b)
    if (pending[b] && !abort_flag) {
      if (!mbar_wait(smem_u32(&mbar[b]), phase[b])) { atomicExch(&g_tc_error, 1); abort_flag = 1; }
    }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!abort_flag && accumulate) {
    // epilogue: warp w reads TMEM lanes 32w..32w+31 (= rows), 16 columns at a time
    const int r = row0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < nmma; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (r < g.m) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = col0 + c0 + j;
          if (c < g.n) g.C[(size_t)r * g.ldc + c] += (double)__uint_as_float(v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

}  // namespace

void gemm_plan_run_tc(const GemmPlan* p, Stream s) {
  if (!p || p->ntiles_tc == 0) return;
  const size_t shm = sizeof(float) * (size_t)(2 * kStageFloats) + 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_grouped_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) throw std::runtime_error(std::string("cuda tc smem attr: ") + cudaGetErrorString(e));
    attr = true;
  }
  k_grouped_gemm_tc<<<p->ntiles_tc, kThreads, shm, (cudaStream_t)s>>>(p->tasks, p->groups, p->ngroups);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw std::runtime_error(std::string("cuda tc gemm launch: ") + cudaGetErrorString(e));
}

int tc_error_flag(Stream s) {
  int h = 0;
  cudaMemcpyFromSymbolAsync(&h, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, (cudaStream_t)s);
  cudaStreamSynchronize((cudaStream_t)s);
  return h;
}

}  // namespace dmrg

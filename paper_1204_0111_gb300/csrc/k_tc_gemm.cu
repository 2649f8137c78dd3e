// Tensor-core (tcgen05 / TMEM) complex64 front GEMM of the complex64 path:
//   C (128 x 128 tile) (+)= +-A B^T
// for the Schur update F_BR -= (Z D^{-1}) Z^T and the two triangular multiplies of selective
// inversion (§2.2), whose contraction depth is the full supernode size.
//
// Complex products use three real products (Gauss): T1 = Ar Br, T2 = Ai Bi,
// T3 = (Ar + Ai)(Br + Bi), Re = T1 - T2, Im = T3 - T1 - T2.  Each real operand x is split into
// TF32 parts x = hi + lo (hi = tf32(x), lo = tf32(x - hi)) and each real product is formed as
// hi*hi + hi*lo + lo*hi (about 22 significant bits): nine kind::tf32 MMAs per k-step of 8,
// accumulated in FP32 in tensor memory (3 x 128 columns).
//
// Two kernels.  k_tc_pack splits an operand once per front into the six TF32 planes (hi/lo of
// re, im, re+im), already laid out as the MMA reads them from shared memory (K-major, no swizzle,
// 8-row x 16-byte core matrices): one 48 KB block per 128 rows x 16 k.  k_tc_gemm then streams the
// A and B blocks of each k-block with bulk asynchronous copies into one of two shared-memory
// stages (96 KB each): thread 0 produces (waits for a free stage, posts the expected bytes, issues
// the copies), thread 32 issues the MMAs once a stage is full and commits them to the stage's
// "empty" barrier, and all eight warps read the accumulators back for the epilogue.  Every
// mbarrier wait is bounded; a wait that gives up records an error in status[1], and the CTA skips
// its epilogue, frees its tensor memory and returns.
#include <cstdint>

#include "cplx.cuh"
#include "psp_internal.h"

namespace psp {

namespace {

constexpr int TM = 128, TN = 128, KB = 16;     // tile and k-block (two tf32 MMAs of K = 8)
constexpr int PLANE_BYTES = TM * KB * 4;       // 8 KB: 128 rows x 16 tf32
constexpr int NPLANE = 6;                      // hi/lo of re, im, re+im
constexpr int BLOCK_BYTES = NPLANE * PLANE_BYTES;      // one packed operand block: 48 KB
constexpr int STAGE_BYTES = 2 * BLOCK_BYTES;           // A and B blocks: 96 KB
constexpr int NSTAGE = 2;
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024;  // + barriers and the TMEM slot
constexpr uint32_t LBO = 128;                  // next core matrix along K
constexpr uint32_t SBO = 512;                  // next 8-row group (4 core matrices of K per group)
constexpr uint32_t TMEM_COLS = 512;
constexpr long long WAIT_LIMIT = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row r, k) inside one plane
__host__ __device__ __forceinline__ uint32_t plane_off(int r, int k) {
  return (uint32_t)((r >> 3) * SBO + (k >> 2) * LBO + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((LBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((SBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; layout type 0 = no swizzle
  return d;
}

// kind::tf32 instruction descriptor: D f32, A and B tf32, both K-major, M = 128, N = 128
__host__ __device__ constexpr uint32_t make_idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ uint32_t tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_round(x);
  lo = tf32_round(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try(mbar, parity)) return true;
  return false;
}

__device__ __forceinline__ void expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

}  // namespace

// ---------------------------------------------------------------------------
// k_tc_pack: one 48 KB block (rows r0..r0+127, k k0..k0+15) of a packed operand per CTA.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tc_pack(const TcPackTask* __restrict__ tasks) {
  const TcPackTask tk = tasks[blockIdx.x];
  for (int u = threadIdx.x; u < TM * (KB / 4); u += 256) {
    const int r = u % TM, c = u / TM;
    const int rg = tk.r0 + r;
    uint32_t hr[4], lr[4], hi_[4], li[4], hs[4], ls[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = tk.k0 + 4 * c + q;
      float2 v = make_float2(0.f, 0.f);
      if (rg < tk.R && k < tk.K) {
        if (tk.mode == TC_PACK_PLAIN) {
          v = tk.src[(int64_t)k * tk.ld + rg];
          if (tk.d) v = cdiv(v, tk.d[(int64_t)k * tk.ldd]);
        } else if (tk.mode == TC_PACK_UNIT_LOWER) {          // T[rg, k], unit lower
          v = (k == rg) ? make_float2(1.f, 0.f) : (k < rg ? tk.src[(int64_t)k * tk.ld + rg] : make_float2(0.f, 0.f));
        } else {                                             // T[k, rg], unit lower (transposed read)
          v = (k == rg) ? make_float2(1.f, 0.f) : (k > rg ? tk.src[(int64_t)rg * tk.ld + k] : make_float2(0.f, 0.f));
        }
      }
      split(v.x, hr[q], lr[q]);
      split(v.y, hi_[q], li[q]);
      split(v.x + v.y, hs[q], ls[q]);
    }
    unsigned char* dst = reinterpret_cast<unsigned char*>(tk.dst) + plane_off(r, 4 * c);
    *reinterpret_cast<uint4*>(dst + 0 * PLANE_BYTES) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
    *reinterpret_cast<uint4*>(dst + 1 * PLANE_BYTES) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
    *reinterpret_cast<uint4*>(dst + 2 * PLANE_BYTES) = make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
    *reinterpret_cast<uint4*>(dst + 3 * PLANE_BYTES) = make_uint4(li[0], li[1], li[2], li[3]);
    *reinterpret_cast<uint4*>(dst + 4 * PLANE_BYTES) = make_uint4(hs[0], hs[1], hs[2], hs[3]);
    *reinterpret_cast<uint4*>(dst + 5 * PLANE_BYTES) = make_uint4(ls[0], ls[1], ls[2], ls[3]);
  }
}

// ---------------------------------------------------------------------------
// k_tc_gemm: one 128 x 128 output tile per CTA from packed operand blocks.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 1) k_tc_gemm(const TcGemmTask* __restrict__ tasks, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const TcGemmTask tk = tasks[blockIdx.x];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NSTAGE * STAGE_BYTES);
  uint64_t* empty = full + NSTAGE;
  uint64_t* done = empty + NSTAGE;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int nkb = tk.nkb;

  if (tid == 0) {
    // producer: stage i & 1 holds k-block i; refill a stage once its MMAs have completed
    for (int i = 0; i < nkb; ++i) {
      const int s = i & 1;
      if (i >= 2 && !mbar_wait(smem_u32(&empty[s]), (uint32_t)(((i >> 1) - 1) & 1))) {
        *abort_flag = 1;
        atomicCAS(status + 1, 0, 1);
        break;
      }
      const uint32_t fb = smem_u32(&full[s]);
      const uint32_t dst = smem_u32(smem + s * STAGE_BYTES);
      expect_tx(fb, STAGE_BYTES);
      bulk_copy(dst, tk.A + (int64_t)(tk.kb0 + i) * BLOCK_BYTES, BLOCK_BYTES, fb);
      bulk_copy(dst + BLOCK_BYTES, tk.B + (int64_t)(tk.kb0 + i) * BLOCK_BYTES, BLOCK_BYTES, fb);
    }
  } else if (tid == 32) {
    // MMA issuer
    const uint32_t idesc = make_idesc();
    for (int i = 0; i < nkb; ++i) {
      const int s = i & 1;
      if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((i >> 1) & 1))) {
        *abort_flag = 1;
        atomicCAS(status + 1, 0, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(smem + s * STAGE_BYTES), b0 = a0 + BLOCK_BYTES;
#pragma unroll
      for (int t = 0; t < KB / 8; ++t) {
        const uint32_t ko = (uint32_t)t * 2 * LBO;  // two core matrices of K per MMA
#pragma unroll
        for (int p = 0; p < 3; ++p) {               // T1: re*re, T2: im*im, T3: sum*sum
          const uint32_t dt = tmem + (uint32_t)(p * TN);
          const uint32_t ahi = a0 + (2 * p) * PLANE_BYTES + ko, alo = a0 + (2 * p + 1) * PLANE_BYTES + ko;
          const uint32_t bhi = b0 + (2 * p) * PLANE_BYTES + ko, blo = b0 + (2 * p + 1) * PLANE_BYTES + ko;
          const uint32_t first = (i == 0 && t == 0) ? 0u : 1u;
          mma_tf32(dt, make_desc(ahi), make_desc(bhi), idesc, first);
          mma_tf32(dt, make_desc(ahi), make_desc(blo), idesc, 1u);
          mma_tf32(dt, make_desc(alo), make_desc(bhi), idesc, 1u);
        }
      }
      mma_commit(smem_u32(&empty[s]));
    }
    mma_commit(smem_u32(done));   // completes when every MMA above has completed
  }
  __syncthreads();
  // every thread waits for the accumulators (bounded); skipped when the main loop gave up
  if (!*abort_flag && nkb > 0 && !mbar_wait(smem_u32(done), 0u)) {
    *abort_flag = 1;
    atomicCAS(status + 1, 0, 1);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (!*abort_flag) {
    const int q = warp & 3, half = warp >> 2;
    const int row = 32 * q + lane;
    const bool neg = tk.flags & GF_NEG, beta0 = tk.flags & GF_BETA0, lower = tk.flags & GF_C_LOWER;
    for (int cc = 0; cc < TN / 2; cc += 16) {
      const int col0 = half * (TN / 2) + cc;
      uint32_t t1[16], t2[16], t3[16];
      if (nkb > 0) {
        const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col0;
        tmem_ld16(base, t1);
        tmem_ld16(base + TN, t2);
        tmem_ld16(base + 2 * TN, t3);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) t1[i] = t2[i] = t3[i] = 0u;
      }
      if (row < tk.m) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int col = col0 + i;
          if (col >= tk.n || (lower && row < col)) continue;
          const float a = __uint_as_float(t1[i]), b = __uint_as_float(t2[i]), c = __uint_as_float(t3[i]);
          float2 v = make_float2(a - b, c - a - b);
          if (neg) v = make_float2(-v.x, -v.y);
          float2* dst = tk.C + (int64_t)col * tk.ldc + row;
          *dst = beta0 ? v : cadd(*dst, v);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

void launch_tc_pack(const TcPackTask* tasks, int ntasks, cudaStream_t st) {
  if (ntasks > 0) k_tc_pack<<<ntasks, 256, 0, st>>>(tasks);
}

void launch_tc_gemm(const TcGemmTask* tasks, int ntasks, int* status, cudaStream_t st) {
  if (ntasks <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    attr = true;
  }
  k_tc_gemm<<<ntasks, 256, SMEM_BYTES, st>>>(tasks, status);
}

int tc_gemm_tile() { return TM; }
int tc_block_k() { return KB; }
int64_t tc_block_bytes() { return BLOCK_BYTES; }

}  // namespace psp

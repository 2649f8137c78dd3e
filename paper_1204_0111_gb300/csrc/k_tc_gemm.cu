// Tensor-core (tcgen05 / TMEM) complex64 front GEMM of the complex64 path:
//   C (128 x 128 tile) (+)= +-A diag(d)^{+-1} B^T,
// the Schur update F_BR -= Z D^{-1} Z^T and the two triangular multiplies of selective inversion
// (§2.2), whose contraction depth is the full supernode size.
//
// Complex products use three real products (Gauss): T1 = Ar Br, T2 = Ai Bi,
// T3 = (Ar + Ai)(Br + Bi), Re = T1 - T2, Im = T3 - T1 - T2.  Each real operand x is split into
// TF32 parts x = hi + lo (hi = tf32(x), lo = tf32(x - hi)) and each real product is formed as
// hi*hi + hi*lo + lo*hi, which keeps about 22 significant bits: nine kind::tf32 MMAs per k-step,
// accumulated in FP32 in tensor memory (3 x 128 columns).
//
// One CTA of 256 threads per output tile.  All threads load the operands from global memory,
// apply the diagonal scaling and the unit-triangular masks, split them and store the twelve
// planes in the canonical K-major no-swizzle layout (8-row x 16-byte core matrices); thread 0
// issues the MMAs and commits them to an mbarrier per stage, so loading k-block kb+1 overlaps
// the MMAs of k-block kb (two stages).  Every mbarrier wait is bounded; a wait that gives up
// records an error in `status` and the CTA skips its epilogue, frees its tensor memory and exits.
#include <cstdint>

#include "cplx.cuh"
#include "psp_internal.h"

namespace psp {

namespace {

constexpr int TM = 128, TN = 128, KB = 16;     // tile and k-block (two tf32 MMAs of K = 8)
constexpr int PLANE_BYTES = TM * KB * 4;       // 8 KB: 128 rows x 16 tf32
constexpr int NPLANE = 6;                      // hi/lo of re, im, re+im
constexpr int STAGE_BYTES = 2 * NPLANE * PLANE_BYTES;   // A and B planes: 96 KB
constexpr int NSTAGE = 2;
constexpr int SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024;  // + barriers, scaling, TMEM slot
constexpr uint32_t LBO = 128;                  // next core matrix along K
constexpr uint32_t SBO = 512;                  // next 8-row group (4 core matrices of K per group)
constexpr uint32_t TMEM_COLS = 512;
constexpr long long WAIT_LIMIT = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row r, k) inside one plane
__device__ __forceinline__ uint32_t plane_off(int r, int k) {
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

}  // namespace

__global__ void __launch_bounds__(256, 1) k_tc_gemm(const GemmTask<float2>* __restrict__ tasks, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const GemmTask<float2> tk = tasks[blockIdx.x];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* stage_base = smem;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + NSTAGE * STAGE_BYTES);        // 2 barriers
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + NSTAGE * STAGE_BYTES + 64);
  int* abort_flag = reinterpret_cast<int*>(smem + NSTAGE * STAGE_BYTES + 68);

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])) : "memory");
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

  const bool bnn = tk.flags & GF_B_NN;
  const bool dmul = tk.flags & GF_D_MUL, ddiv = tk.flags & GF_D_DIV;
  const bool bmask = tk.flags & (GF_B_UNIT_LOWER_NT | GF_B_UNIT_LOWER_NN);
  const bool mask_nt = tk.flags & GF_B_UNIT_LOWER_NT;
  const int nkb = (tk.k + KB - 1) / KB;
  const uint32_t idesc = make_idesc();

  // Register-staged operands of one k-block: each thread owns two A units and two B units
  // (a unit = one row x 4 consecutive k).  All loads of a block are issued together, and the next
  // block's loads are issued before the current block's MMAs, so global latency overlaps compute.
  float2 ra[2][4], rd[2][4], rb[2][4];
  auto load_block = [&](int kb) {
    const int k0 = kb * KB;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int uA = tid + 256 * i;
      const int r = uA % TM, c = uA / TM;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + 4 * c + q;
        const bool in = r < tk.m && k < tk.k;
        ra[i][q] = in ? tk.A[(int64_t)k * tk.lda + r] : make_float2(0.f, 0.f);
        if (dmul || ddiv) rd[i][q] = (k < tk.k) ? tk.d[(int64_t)k * tk.ldd] : make_float2(1.f, 0.f);
      }
      int j, cb;
      if (bnn) { cb = uA % (KB / 4); j = uA / (KB / 4); } else { j = uA % TN; cb = uA / TN; }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + 4 * cb + q;
        const bool in = j < tk.n && k < tk.k;
        rb[i][q] = in ? (bnn ? tk.B[(int64_t)j * tk.ldb + k] : tk.B[(int64_t)k * tk.ldb + j]) : make_float2(0.f, 0.f);
      }
    }
  };
  // value-dependent work happens at store time so that the loads above stay in flight
  auto finish_block = [&](int kb) {
    const int k0 = kb * KB;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int uA = tid + 256 * i;
      if (dmul || ddiv) {
#pragma unroll
        for (int q = 0; q < 4; ++q) ra[i][q] = dmul ? cmul(ra[i][q], rd[i][q]) : cdiv(ra[i][q], rd[i][q]);
      }
      if (bmask) {
        int j, cb;
        if (bnn) { cb = uA % (KB / 4); j = uA / (KB / 4); } else { j = uA % TN; cb = uA / TN; }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int kg = tk.kg0 + k0 + 4 * cb + q, ng = tk.ng0 + j;
          if (j < tk.n && k0 + 4 * cb + q < tk.k) {
            if (kg == ng) rb[i][q] = make_float2(1.f, 0.f);
            else if (mask_nt ? (kg > ng) : (kg < ng)) rb[i][q] = make_float2(0.f, 0.f);
          }
        }
      }
    }
  };
  auto store_unit = [&](unsigned char* planes, uint32_t o, const float2 (&v)[4]) {
    uint32_t hr[4], lr[4], hi_[4], li[4], hs[4], ls[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      split(v[q].x, hr[q], lr[q]);
      split(v[q].y, hi_[q], li[q]);
      split(v[q].x + v[q].y, hs[q], ls[q]);
    }
    *reinterpret_cast<uint4*>(planes + 0 * PLANE_BYTES + o) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
    *reinterpret_cast<uint4*>(planes + 1 * PLANE_BYTES + o) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
    *reinterpret_cast<uint4*>(planes + 2 * PLANE_BYTES + o) = make_uint4(hi_[0], hi_[1], hi_[2], hi_[3]);
    *reinterpret_cast<uint4*>(planes + 3 * PLANE_BYTES + o) = make_uint4(li[0], li[1], li[2], li[3]);
    *reinterpret_cast<uint4*>(planes + 4 * PLANE_BYTES + o) = make_uint4(hs[0], hs[1], hs[2], hs[3]);
    *reinterpret_cast<uint4*>(planes + 5 * PLANE_BYTES + o) = make_uint4(ls[0], ls[1], ls[2], ls[3]);
  };

  if (nkb > 0) load_block(0);
  for (int kb = 0; kb < nkb; ++kb) {
    const int s = kb & 1;
    unsigned char* st = stage_base + s * STAGE_BYTES;
    unsigned char* sb = st + NPLANE * PLANE_BYTES;
    if (kb >= 2) {
      if (tid == 0 && !mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((kb >> 1) - 1) & 1))) {
        *abort_flag = 1;
        atomicCAS(status + 1, 0, 1);
      }
      __syncthreads();
      if (*abort_flag) break;
    }
    finish_block(kb);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int uA = tid + 256 * i;
      store_unit(st, plane_off(uA % TM, 4 * (uA / TM)), ra[i]);
      int j, cb;
      if (bnn) { cb = uA % (KB / 4); j = uA / (KB / 4); } else { j = uA % TN; cb = uA / TN; }
      store_unit(sb, plane_off(j, 4 * cb), rb[i]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(st), b0 = smem_u32(sb);
#pragma unroll
      for (int t = 0; t < KB / 8; ++t) {
        const uint32_t ko = (uint32_t)t * 2 * LBO;  // two core matrices of K per MMA
        // product p: accumulator, A plane pair, B plane pair  (T1: re*re, T2: im*im, T3: sum*sum)
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const uint32_t dt = tmem + (uint32_t)(p * TN);
          const uint32_t ahi = a0 + (2 * p) * PLANE_BYTES + ko, alo = a0 + (2 * p + 1) * PLANE_BYTES + ko;
          const uint32_t bhi = b0 + (2 * p) * PLANE_BYTES + ko, blo = b0 + (2 * p + 1) * PLANE_BYTES + ko;
          const uint32_t first = (kb == 0 && t == 0) ? 0u : 1u;
          mma_tf32(dt, make_desc(ahi), make_desc(bhi), idesc, first);
          mma_tf32(dt, make_desc(ahi), make_desc(blo), idesc, 1u);
          mma_tf32(dt, make_desc(alo), make_desc(bhi), idesc, 1u);
        }
      }
      mma_commit(smem_u32(&mbar[s]));
    }
    if (kb + 1 < nkb) load_block(kb + 1);   // next block's loads overlap this block's MMAs
  }

  // wait for the last commit (it covers every earlier MMA of this thread)
  if (nkb > 0 && !*abort_flag) {
    if (tid == 0) {
      const int kl = nkb - 1;
      if (!mbar_wait(smem_u32(&mbar[kl & 1]), (uint32_t)((kl >> 1) & 1))) {
        *abort_flag = 1;
        atomicCAS(status + 1, 0, 1);
      }
    }
    __syncthreads();
  }
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

void launch_tc_gemm(const GemmTask<float2>* tasks, int ntasks, int* status, cudaStream_t st) {
  if (ntasks <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    attr = true;
  }
  k_tc_gemm<<<ntasks, 256, SMEM_BYTES, st>>>(tasks, status);
}

int tc_gemm_tile() { return TM; }

}  // namespace psp

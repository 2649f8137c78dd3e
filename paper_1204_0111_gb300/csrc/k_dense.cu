// Dense front kernels of the partial factorisation (§2.2), CUDA-core path for complex128
// and complex64:  blocked unpivoted LDL^T of F_TL, the blocked inverse of L_TL for selective
// inversion, and a batched complex GEMM C (+)= alpha A diag(d)^{+-1} B^T with triangle masks
// that carries the trailing updates, the Schur update F_BR -= Z F_BL^T and the two
// triangular multiplies.
#include "cplx.cuh"
#include "psp_internal.h"

namespace psp {

constexpr int kNB = 32;  // diagonal block size of the blocked LDL^T and inverse

// ---------------------------------------------------------------------------
// LDL^T of the kb-th diagonal block of F_TL (unblocked, right-looking, in shared memory).
// The block is overwritten by its unit lower factor (strict part) and D (diagonal).
// A pivot with |d| < tiny records 1 + (front's global id) in status[0]; the smallest |d| of all
// pivots is kept in status[4..5] as the bitwise complement of its double (atomicMax of the
// complement = minimum of the non-negative value; 0 = no pivot yet).
// ---------------------------------------------------------------------------
template <typename T, typename C>
__global__ void __launch_bounds__(128) k_diag_ldlt(const FrontTask<T>* __restrict__ fronts, const int* __restrict__ list,
                                                   int kb, double tiny, int* status) {
  __shared__ C S[kNB][kNB + 1];  // S[col][row], in the compute precision C
  __shared__ C colv[kNB];
  const FrontTask<T> ft = fronts[list[blockIdx.x]];
  const int ld = ft.s + ft.u;
  const int o = kb * kNB;
  const int bs = min(kNB, ft.s - o);
  T* B = ft.G + (int64_t)o * ld + o;
  for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
    const int r = e % bs, c = e / bs;
    if (r >= c) S[c][r] = CplxTraits<C>::from(to_c128(B[(int64_t)c * ld + r]));
  }
  __syncthreads();
  double dmin = INFINITY;
  for (int j = 0; j < bs; ++j) {
    const C d = S[j][j];
    if (threadIdx.x == 0) {
      if (fmax(fabs((double)d.x), fabs((double)d.y)) < tiny) atomicCAS(status, 0, (int)(1 + ft.gfid));
      dmin = fmin(dmin, hypot((double)d.x, (double)d.y));
    }
    const C dinv = cdiv(CplxTraits<C>::one(), d);
    for (int i = j + 1 + threadIdx.x; i < bs; i += blockDim.x) {
      const C a = S[j][i];
      colv[i] = a;
      S[j][i] = cmul(a, dinv);
    }
    __syncthreads();
    // S(i,k) -= a_i * l_k for j < k <= i
    const int m = bs - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e % m, k = j + 1 + e / m;
      if (i >= k) cfms(S[k][i], colv[i], S[j][k]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
    const int r = e % bs, c = e / bs;
    if (r >= c) B[(int64_t)c * ld + r] = CplxTraits<T>::from(to_c128(S[c][r]));
  }
  if (threadIdx.x == 0 && dmin == dmin)   // a NaN pivot leaves the minimum alone (status[0] reports it if tiny)
    atomicMax(reinterpret_cast<unsigned long long*>(status + 4), ~(unsigned long long)__double_as_longlong(dmin));
}

// ---------------------------------------------------------------------------
// Rows of F_TL below diagonal block kb:  X L_kk^T = F(r, block)  ->  F(r, block) := X D^{-1}.
// One thread per row; L_kk and D in shared memory.
// ---------------------------------------------------------------------------
template <typename T, typename C>
__global__ void __launch_bounds__(64) k_panel_right(const FrontTask<T>* __restrict__ fronts,
                                                    const ColTask* __restrict__ tasks, int kb) {
  __shared__ C L[kNB][kNB + 1];  // L[col][row]
  __shared__ C dinv[kNB];
  const ColTask tk = tasks[blockIdx.x];
  const FrontTask<T> ft = fronts[tk.front];
  const int ld = ft.s + ft.u;
  const int o = kb * kNB;
  const int bs = min(kNB, ft.s - o);
  const T* Bd = ft.G + (int64_t)o * ld + o;
  for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
    const int r = e % bs, c = e / bs;
    L[c][r] = (r > c) ? CplxTraits<C>::from(to_c128(Bd[(int64_t)c * ld + r])) : CplxTraits<C>::zero();
  }
  for (int c = threadIdx.x; c < bs; c += blockDim.x) dinv[c] = cdiv(CplxTraits<C>::one(), CplxTraits<C>::from(to_c128(Bd[(int64_t)c * ld + c])));
  __syncthreads();
  const int r = tk.c0 + threadIdx.x;
  if (r >= tk.c1) return;
  T* row = ft.G + (int64_t)o * ld + r;
  C x[kNB];
#pragma unroll
  for (int c = 0; c < kNB; ++c) {
    if (c < bs) {
      C v = CplxTraits<C>::from(to_c128(row[(int64_t)c * ld]));
      for (int k = 0; k < c; ++k) cfms(v, x[k], L[k][c]);
      x[c] = v;
    }
  }
#pragma unroll
  for (int c = 0; c < kNB; ++c)
    if (c < bs) row[(int64_t)c * ld] = CplxTraits<T>::from(to_c128(cmul(x[c], dinv[c])));
}

// ---------------------------------------------------------------------------
// Block row kb of W (the inverse of L_TL under construction): W(kb, cols) := L_kk^{-1} W(kb, cols).
// A 32 x 64 tile is staged through shared memory; one thread per column.
// ---------------------------------------------------------------------------
template <typename T, typename C>
__global__ void __launch_bounds__(64) k_panel_left(const FrontTask<T>* __restrict__ fronts,
                                                   const ColTask* __restrict__ tasks, int kb) {
  __shared__ C L[kNB][kNB + 1];   // L[col][row]
  __shared__ C Wt[64][kNB + 1];   // Wt[col][row]
  const ColTask tk = tasks[blockIdx.x];
  const FrontTask<T> ft = fronts[tk.front];
  const int ld = ft.s + ft.u;
  const int o = kb * kNB;
  const int bs = min(kNB, ft.s - o);
  const int ncol = tk.c1 - tk.c0;
  const T* Bd = ft.G + (int64_t)o * ld + o;
  for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
    const int r = e % bs, c = e / bs;
    L[c][r] = (r > c) ? CplxTraits<C>::from(to_c128(Bd[(int64_t)c * ld + r])) : CplxTraits<C>::zero();
  }
  T* W0 = ft.W + (int64_t)tk.c0 * ft.s + o;
  for (int e = threadIdx.x; e < bs * ncol; e += blockDim.x) {
    const int r = e % bs, c = e / bs;
    Wt[c][r] = CplxTraits<C>::from(to_c128(W0[(int64_t)c * ft.s + r]));
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c < ncol) {
    for (int r = 1; r < bs; ++r) {
      C v = Wt[c][r];
      for (int k = 0; k < r; ++k) cfms(v, L[k][r], Wt[c][k]);
      Wt[c][r] = v;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < bs * ncol; e += blockDim.x) {
    const int r = e % bs, cc = e / bs;
    W0[(int64_t)cc * ft.s + r] = CplxTraits<T>::from(to_c128(Wt[cc][r]));
  }
}

// ---------------------------------------------------------------------------
// Block column kb of the second inverse X of L_TL (two-inverse form, X L_TL = I row by row):
// X(r, block) := X(r, block) L_kk^{-1} for rows r of the task, i.e. x L_kk = b by backward
// substitution along each row.  One thread per row; L_kk in shared memory.
// ---------------------------------------------------------------------------
template <typename T, typename C>
__global__ void __launch_bounds__(64) k_panel_rsolve(const FrontTask<T>* __restrict__ fronts,
                                                     const ColTask* __restrict__ tasks, int kb) {
  __shared__ C L[kNB][kNB + 1];  // L[col][row], strictly lower part of L_kk
  const ColTask tk = tasks[blockIdx.x];
  const FrontTask<T> ft = fronts[tk.front];
  const int ld = ft.s + ft.u;
  const int o = kb * kNB;
  const int bs = min(kNB, ft.s - o);
  const T* Bd = ft.G + (int64_t)o * ld + o;
  for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
    const int r = e % bs, c = e / bs;
    L[c][r] = (r > c) ? CplxTraits<C>::from(to_c128(Bd[(int64_t)c * ld + r])) : CplxTraits<C>::zero();
  }
  __syncthreads();
  const int r = tk.c0 + threadIdx.x;
  if (r >= tk.c1) return;
  T* row = ft.W2 + (int64_t)o * ft.s + r;   // X(r, o + c) at row[c * s]
  C x[kNB];
#pragma unroll
  for (int c = 0; c < kNB; ++c) x[c] = c < bs ? CplxTraits<C>::from(to_c128(row[(int64_t)c * ft.s])) : CplxTraits<C>::zero();
  // x_c = b_c - sum_{k > c} x_k L(k, c), from the last column
#pragma unroll
  for (int c = kNB - 1; c >= 0; --c) {
    if (c < bs) {
      C v = x[c];
#pragma unroll
      for (int k = c + 1; k < kNB; ++k)
        if (k < bs) cfms(v, x[k], L[c][k]);
      x[c] = v;
    }
  }
#pragma unroll
  for (int c = 0; c < kNB; ++c)
    if (c < bs) row[(int64_t)c * ft.s] = CplxTraits<T>::from(to_c128(x[c]));
}

// ---------------------------------------------------------------------------
// Batched complex GEMM, one 64 x 64 output tile per CTA (16 x 16 threads, 4 x 4 each; thread
// (tx, ty) owns rows ty + 16 a and columns tx + 16 b, so each 16 x 16 block (a, b) is spread over
// the whole CTA and can be skipped as a unit).
// Complex products use three real multiplications (Gauss): with the pre-sums ar + ai and
// br + bi staged in shared memory, t1 += ar br, t2 += ai bi, t3 += (ar + ai)(br + bi), and at the
// end re = t1 - t2, im = t3 - t1 - t2.  Three FMAs per complex MAC instead of four.
// ---------------------------------------------------------------------------
constexpr int GT = 64, GK = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_gemm(const GemmTask<T>* __restrict__ tasks) {
  using R = typename CplxTraits<T>::real;
  // single precision: rows of 68 floats (16-byte aligned, so a thread reads its 4 consecutive rows
  // or columns with one 128-bit load); double precision: 65 (no bank conflicts in the staging)
  constexpr bool kSingle = sizeof(R) == 4;
  constexpr int GP = kSingle ? GT + 4 : GT + 1;
  __shared__ __align__(16) R Ar[GK][GP], Ai[GK][GP], As[GK][GP];
  __shared__ __align__(16) R Br[GK][GP], Bi[GK][GP], Bs[GK][GP];
  const GemmTask<T> tk = tasks[blockIdx.x];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const T zero = CplxTraits<T>::zero();
  R t1[4][4], t2[4][4], t3[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) t1[a][b] = t2[a][b] = t3[a][b] = R(0);

  const bool bnn = tk.flags & GF_B_NN, lower = tk.flags & GF_C_LOWER;
  for (int k0 = 0; k0 < tk.k; k0 += GK) {
    // A chunk: 64 rows x GK k
    for (int e = threadIdx.x; e < GT * GK; e += 256) {
      const int i = e % GT, kk = e / GT;
      T v = zero;
      if (i < tk.m && k0 + kk < tk.k) {
        v = tk.A[(int64_t)(k0 + kk) * tk.lda + i];
        if (tk.flags & (GF_D_MUL | GF_D_DIV)) {
          const T dd = tk.d[(int64_t)(k0 + kk) * tk.ldd];
          v = (tk.flags & GF_D_MUL) ? cmul(v, dd) : cdiv(v, dd);
        }
      }
      Ar[kk][i] = v.x;
      Ai[kk][i] = v.y;
      As[kk][i] = v.x + v.y;
    }
    // B chunk: 64 n x GK k
    for (int e = threadIdx.x; e < GT * GK; e += 256) {
      int j, kk;
      if (bnn) { kk = e % GK; j = e / GK; } else { j = e % GT; kk = e / GT; }
      T v = zero;
      if (j < tk.n && k0 + kk < tk.k) {
        v = bnn ? tk.B[(int64_t)j * tk.ldb + (k0 + kk)] : tk.B[(int64_t)(k0 + kk) * tk.ldb + j];
        if (tk.flags & (GF_B_UNIT_LOWER_NT | GF_B_UNIT_LOWER_NN)) {
          const int kg = tk.kg0 + k0 + kk, ng = tk.ng0 + j;
          if (kg == ng) v = CplxTraits<T>::one();
          else if ((tk.flags & GF_B_UNIT_LOWER_NT) ? (kg > ng) : (kg < ng)) v = zero;
        }
      }
      Br[kk][j] = v.x;
      Bi[kk][j] = v.y;
      Bs[kk][j] = v.x + v.y;
    }
    __syncthreads();
    if constexpr (kSingle) {
      // single precision: the FP32 pipe is fast enough that issue slots, not FMAs, bound the
      // loop, so all 16 blocks run; thread (tx, ty) owns rows 4 ty .. 4 ty + 3 and columns
      // 4 tx .. 4 tx + 3, each operand quadruple one 128-bit shared load (six loads per 48 FMAs)
#pragma unroll
      for (int kk = 0; kk < GK; ++kk) {
        R ar[4], ai[4], as[4], br[4], bi[4], bs[4];
        *reinterpret_cast<float4*>(ar) = *reinterpret_cast<const float4*>(&Ar[kk][4 * ty]);
        *reinterpret_cast<float4*>(ai) = *reinterpret_cast<const float4*>(&Ai[kk][4 * ty]);
        *reinterpret_cast<float4*>(as) = *reinterpret_cast<const float4*>(&As[kk][4 * ty]);
        *reinterpret_cast<float4*>(br) = *reinterpret_cast<const float4*>(&Br[kk][4 * tx]);
        *reinterpret_cast<float4*>(bi) = *reinterpret_cast<const float4*>(&Bi[kk][4 * tx]);
        *reinterpret_cast<float4*>(bs) = *reinterpret_cast<const float4*>(&Bs[kk][4 * tx]);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            t1[a][b] = fma(ar[a], br[b], t1[a][b]);
            t2[a][b] = fma(ai[a], bi[b], t2[a][b]);
            t3[a][b] = fma(as[a], bs[b], t3[a][b]);
          }
      }
      __syncthreads();
      continue;
    }
    // double precision (2 DFMA per clock per SM): only the 16 x 16 blocks (a, b) of the tile that
    // carry work in this k-chunk run: rows and columns inside the task, the lower triangle of a
    // diagonal tile, the non-zero part of a triangular B.  The tests are uniform over the CTA, so
    // skipped blocks cost no FP64 issue slots.
    bool bact[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      bool on = 16 * b < tk.n;
      if (tk.flags & GF_B_UNIT_LOWER_NT) on = on && (k0 + tk.kg0 <= 16 * b + 15 + tk.ng0);
      if (tk.flags & GF_B_UNIT_LOWER_NN) on = on && (k0 + GK - 1 + tk.kg0 >= 16 * b + tk.ng0);
      bact[b] = on;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (16 * a >= tk.m) continue;
#pragma unroll
      for (int kk = 0; kk < GK; ++kk) {
        const R ar = Ar[kk][ty + 16 * a], ai = Ai[kk][ty + 16 * a], as = As[kk][ty + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (!bact[b] || (lower && b > a)) continue;
          const R br = Br[kk][tx + 16 * b], bi = Bi[kk][tx + 16 * b], bs = Bs[kk][tx + 16 * b];
          t1[a][b] = fma(ar, br, t1[a][b]);
          t2[a][b] = fma(ai, bi, t2[a][b]);
          t3[a][b] = fma(as, bs, t3[a][b]);
        }
      }
    }
    __syncthreads();
  }
  const bool neg = tk.flags & GF_NEG, beta0 = tk.flags & GF_BETA0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = kSingle ? 4 * ty + a : ty + 16 * a;
    if (i >= tk.m) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = kSingle ? 4 * tx + b : tx + 16 * b;
      if (j >= tk.n || (lower && i < j)) continue;
      T v;
      v.x = t1[a][b] - t2[a][b];
      v.y = t3[a][b] - t1[a][b] - t2[a][b];
      if (neg) v = cneg(v);
      T* c = tk.C + (int64_t)j * tk.ldc + i;
      *c = beta0 ? v : cadd(*c, v);
    }
  }
}

// strict lower part of W -> strict lower part of F_TL (D stays on the diagonal)
template <typename T>
__global__ void __launch_bounds__(256) k_copy_linv(const FrontTask<T>* __restrict__ fronts,
                                                   const ColTask* __restrict__ tasks) {
  const ColTask tk = tasks[blockIdx.x];
  const FrontTask<T> ft = fronts[tk.front];
  const int ld = ft.s + ft.u;
  for (int c = tk.c0; c < tk.c1; ++c)
    for (int r = c + 1 + threadIdx.x; r < ft.s; r += blockDim.x)
      ft.G[(int64_t)c * ld + r] = ft.W[(int64_t)c * ft.s + r];
  if (ft.W2) {   // the second inverse, whole (unit lower, zero above), after G
    T* G2 = ft.G + second_inverse_offset(ft.s, ft.u);
    for (int c = tk.c0; c < tk.c1; ++c)
      for (int r = threadIdx.x; r < ft.s; r += blockDim.x) G2[(int64_t)c * ft.s + r] = ft.W2[(int64_t)c * ft.s + r];
  }
}

// ZD = Z D^{-1}, column by column, once per front: the Schur update and the M_BL product then
// read plain operands in every tile instead of dividing each element by its pivot again.  When the
// factor keeps L_BL = F_BL L^{-T} D^{-1} itself, ZD is G's bottom block (ldzd = s + u)
template <typename T>
__global__ void __launch_bounds__(256) k_scale_zd(const FrontTask<T>* __restrict__ fronts,
                                                  const ColTask* __restrict__ tasks) {
  __shared__ T dinv[64];   // the task's pivots' reciprocals, one division each (at most 64 columns)
  const ColTask tk = tasks[blockIdx.x];
  const FrontTask<T> ft = fronts[tk.front];
  const int ld = ft.s + ft.u;
  const int nc = tk.c1 - tk.c0;
  for (int c = threadIdx.x; c < nc; c += blockDim.x)
    dinv[c] = cdiv(CplxTraits<T>::one(), ft.G[(int64_t)(tk.c0 + c) * (ld + 1)]);
  __syncthreads();
  // every (column, row) of the task over all threads
  for (int64_t e = threadIdx.x; e < (int64_t)nc * ft.u; e += blockDim.x) {
    const int c = (int)(e / ft.u), r = (int)(e % ft.u);
    ft.ZD[(int64_t)(tk.c0 + c) * ft.ldzd + r] = cmul(ft.Z[(int64_t)(tk.c0 + c) * ft.u + r], dinv[c]);
  }
}

// wide: the diagonal blocks' LDL^T and the solves against them in complex128 whatever the storage
// precision (the complex64 factors' FP64 refinement of the diagonal blocks)
template <typename T>
void launch_diag_ldlt(const FrontTask<T>* fronts, const int* list, int nlist, int kb, double tiny, int* status,
                      bool wide, cudaStream_t st) {
  if (nlist <= 0) return;
  // 128 threads: a 32 x 32 block keeps few busy, and smaller CTAs let more fronts' blocks share an SM
  if (wide) k_diag_ldlt<T, double2><<<nlist, 128, 0, st>>>(fronts, list, kb, tiny, status);
  else k_diag_ldlt<T, T><<<nlist, 128, 0, st>>>(fronts, list, kb, tiny, status);
}
template <typename T>
void launch_panel_right(const FrontTask<T>* fronts, const ColTask* tasks, int ntasks, int kb, bool wide,
                        cudaStream_t st) {
  if (ntasks <= 0) return;
  if (wide) k_panel_right<T, double2><<<ntasks, 64, 0, st>>>(fronts, tasks, kb);
  else k_panel_right<T, T><<<ntasks, 64, 0, st>>>(fronts, tasks, kb);
}
template <typename T>
void launch_panel_left(const FrontTask<T>* fronts, const ColTask* tasks, int ntasks, int kb, bool wide,
                       cudaStream_t st) {
  if (ntasks <= 0) return;
  if (wide) k_panel_left<T, double2><<<ntasks, 64, 0, st>>>(fronts, tasks, kb);
  else k_panel_left<T, T><<<ntasks, 64, 0, st>>>(fronts, tasks, kb);
}
template <typename T>
void launch_panel_rsolve(const FrontTask<T>* fronts, const ColTask* tasks, int ntasks, int kb, bool wide,
                         cudaStream_t st) {
  if (ntasks <= 0) return;
  if (wide) k_panel_rsolve<T, double2><<<ntasks, 64, 0, st>>>(fronts, tasks, kb);
  else k_panel_rsolve<T, T><<<ntasks, 64, 0, st>>>(fronts, tasks, kb);
}
template <typename T>
void launch_gemm(const GemmTask<T>* tasks, int ntasks, cudaStream_t st) {
  if (ntasks > 0) k_gemm<T><<<ntasks, 256, 0, st>>>(tasks);
}
template <typename T>
void launch_copy_linv(const FrontTask<T>* fronts, const ColTask* tasks, int ntasks, cudaStream_t st) {
  if (ntasks > 0) k_copy_linv<T><<<ntasks, 256, 0, st>>>(fronts, tasks);
}
template <typename T>
void launch_scale_zd(const FrontTask<T>* fronts, const ColTask* tasks, int ntasks, cudaStream_t st) {
  if (ntasks > 0) k_scale_zd<T><<<ntasks, 256, 0, st>>>(fronts, tasks);
}

#define PSP_INST(T)                                                                                           \
  template void launch_diag_ldlt<T>(const FrontTask<T>*, const int*, int, int, double, int*, bool, cudaStream_t);    \
  template void launch_panel_right<T>(const FrontTask<T>*, const ColTask*, int, int, bool, cudaStream_t);            \
  template void launch_panel_left<T>(const FrontTask<T>*, const ColTask*, int, int, bool, cudaStream_t);             \
  template void launch_panel_rsolve<T>(const FrontTask<T>*, const ColTask*, int, int, bool, cudaStream_t);     \
  template void launch_gemm<T>(const GemmTask<T>*, int, cudaStream_t);                                         \
  template void launch_copy_linv<T>(const FrontTask<T>*, const ColTask*, int, cudaStream_t);                 \
  template void launch_scale_zd<T>(const FrontTask<T>*, const ColTask*, int, cudaStream_t);
PSP_INST(double2)
PSP_INST(float2)
#undef PSP_INST

}  // namespace psp

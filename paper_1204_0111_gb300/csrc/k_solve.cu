// Multifrontal solve with selectively inverted fronts (§2.2), one tree level per launch, as the
// T_i of Alg. 1.3 inside the sweep of Alg. 1.5.
//
// Each front stores G = [inv(L_TL) (unit lower, D on the diagonal); M_BL = L_BL inv(L_TL)], so
//   up the tree:   v_S = inv(L_TL) w_S,  x_S = D^{-1} v_S,  update_U = w_U - M_BL w_S
//   down the tree: x_S = inv(L_TL)^T x_S - M_BL^T x_U
// which are matrix-vector products (the point of selective inversion): every task reads its
// block of G once, column segments contiguous, and no task depends on another task of the same
// level.  Children's update vectors are pulled (at most two per row), never scattered, so the
// summation order is fixed.  Extension by zero over the pad, the plane coupling J_{i+1,i} of
// the previous / next panel and the extraction of the panel's planes are fused into the
// gathers and the final write.
#include "cplx.cuh"
#include "psp_internal.h"

namespace psp {

template <typename T>
__device__ __forceinline__ T input_value(const SolveCtx<T>& cx, int node, int q) {
  const int nx = cx.sh.nx;
  const int plane = nx * cx.sh.ny;
  const int own = node - cx.lead * plane;                 // index within the panel's planes
  if (own < 0) return CplxTraits<T>::zero();              // extension by zero over the pad (Alg. 1.3)
  const int64_t g = (int64_t)own + (int64_t)plane * cx.z0;
  const double2* uq = cx.u + (int64_t)q * cx.N;
  double2 v;
  if (cx.mode == 0) {
    // u_i - J_{i,i-1} u_{i-1}: J's coupling entry is -s1 s2 / s3(z0 - 1/2) / h^2
    v = __ldcg(uq + g);
    if (cx.has_prev && own < plane) {
      const int x = own % nx, y = own / nx;
      const double2 a = cscale(cmul(cmul(cx.s1n[x], cx.s2n[y]), cx.s3h[cx.z0]), cx.inv_h2);
      cfma(v, a, __ldcg(uq + g - plane));
    }
  } else {
    // J_{i+1,i}^T u_{i+1}: supported on the panel's last plane
    v = make_double2(0.0, 0.0);
    const int last = own - (cx.z1 - cx.z0 - 1) * plane;
    if (cx.has_next && last >= 0) {
      const int x = last % nx, y = last / nx;
      const double2 a = cscale(cmul(cmul(cx.s1n[x], cx.s2n[y]), cx.s3h[cx.z1]), -cx.inv_h2);
      v = cmul(a, __ldcg(uq + g + plane));
    }
  }
  return CplxTraits<T>::from(v);
}

template <typename T, int RG>
__device__ __forceinline__ void pull_add(const SolveCtx<T>& cx, const int32_t* pl, int rhs0, T* out) {
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int32_t o = pl[t];
    if (o < 0) break;
#pragma unroll
    for (int q = 0; q < RG; ++q)
      if (rhs0 + q < cx.nrhs) out[q] = cadd(out[q], __ldcg(cx.upd + (int64_t)(rhs0 + q) * cx.upd_ld + o));
  }
}

// w_S entries [j0, j1) of front sn (zero-extended input + children's updates) for right-hand sides
// [rhs0, rhs0 + RG) into w (right-hand side major, ld chunk).  Each thread first loads the node ids
// and pull offsets of GU entries, then all of their values, so that a thread has GU independent
// gathers in flight rather than one chain of dependent loads after another.
template <typename T, int RG>
__device__ __forceinline__ void gather_w(const SolveCtx<T>& cx, const int first, const int32_t* pull, const int j0,
                                         const int j1, const int rhs0, T* w, const int chunk) {
  constexpr int GU = RG >= 4 ? 1 : (RG == 2 ? 2 : 4);
  for (int p0 = j0 + threadIdx.x; p0 < j1; p0 += GU * blockDim.x) {
    int node[GU];
    int32_t pa[GU], pb[GU];
#pragma unroll
    for (int t = 0; t < GU; ++t) {
      const int p = p0 + t * blockDim.x;
      const bool in = p < j1;
      node[t] = in ? cx.sh.order[first + p] : 0;
      pa[t] = in ? pull[2 * p] : -1;
      pb[t] = in ? pull[2 * p + 1] : -1;
    }
    T v[GU][RG];
#pragma unroll
    for (int t = 0; t < GU; ++t)
#pragma unroll
      for (int q = 0; q < RG; ++q) {
        T x = CplxTraits<T>::zero();
        if (p0 + t * blockDim.x < j1 && rhs0 + q < cx.nrhs) {
          x = input_value(cx, node[t], rhs0 + q);
          const T* uq = cx.upd + (int64_t)(rhs0 + q) * cx.upd_ld;
          if (pa[t] >= 0) x = cadd(x, __ldcg(uq + pa[t]));
          if (pb[t] >= 0) x = cadd(x, __ldcg(uq + pb[t]));
        }
        v[t][q] = x;
      }
#pragma unroll
    for (int t = 0; t < GU; ++t) {
      const int p = p0 + t * blockDim.x;
      if (p < j1)
#pragma unroll
        for (int q = 0; q < RG; ++q) w[q * chunk + (p - j0)] = v[t][q];
    }
  }
}

// up-the-tree task: rows [r0, r1) of front sn, right-hand sides [rhs0, rhs0 + RG).
// phase 0 gathers w_S (zero-extended input + children's updates) and, for rows r < s, writes
// x_r = D^{-1} y_r with y_S = inv(L_TL) w_S (and y_r itself into xb when the second phase needs it);
// for rows r >= s it writes the update w_U - M_BL w_S (extended selective inversion).
// phase 1 (factors keeping L_BL) takes y_S from xb and writes the update w_U - L_BL y_S of rows r >= s.
template <typename T, int RG>
__device__ __forceinline__ void fwd_task(const SolveTask tk, const int rhs0, const SolveCtx<T>& cx, const int R,
                                         unsigned char* smem_raw, const int phase, const int chunk) {
  const int sn = tk.sn;
  const int s = cx.sh.s[sn], u = cx.sh.u[sn], ld = s + u;
  const int first = cx.sh.first[sn];
  const T* G = cx.G + cx.sh.g_off[sn];
  const int32_t* pull = cx.sh.pull + 2 * cx.sh.pull_ptr[sn];
  // the vector w_S (or y_S) passes through shared memory in chunks of `chunk` entries (a multiple of
  // 256), so a CTA carries RG right-hand sides over a factor block of any width and reads it once
  T* w = reinterpret_cast<T*>(smem_raw);        // RG x chunk (right-hand side major: no bank conflicts
                                                 // when a warp spans several columns, R < 32)
  T* red = w + (int64_t)chunk * RG;              // blockDim x RG

  const int i = threadIdx.x % R, grp = threadIdx.x / R, ngrp = blockDim.x / R;
  const int r = tk.r0 + i;
  const int jmax = r < tk.r1 ? (r < s ? r : s) : 0;   // strictly lower part of inv(L_TL), all of the bottom block
  const int jend = min(tk.r1, s);                      // entries of w_S this task needs (w_r of its rows r < s too)
  T acc[RG], wr[RG];
#pragma unroll
  for (int q = 0; q < RG; ++q) acc[q] = wr[q] = CplxTraits<T>::zero();
  const T* Gr = G + r;
  const int64_t step = (int64_t)ngrp * ld;
  for (int j0 = 0; j0 < jend; j0 += chunk) {
    const int j1 = min(j0 + chunk, jend);
    if (j0 > 0) __syncthreads();   // the previous chunk is consumed
    if (phase == 0) {
      gather_w<T, RG>(cx, first, pull, j0, j1, rhs0, w, chunk);   // w_S = zero-extended input + children's updates
    } else {
      for (int p = j0 + threadIdx.x; p < j1; p += blockDim.x)
#pragma unroll
        for (int q = 0; q < RG; ++q)
          w[q * chunk + (p - j0)] = (rhs0 + q < cx.nrhs) ? __ldcg(cx.xb + (int64_t)(rhs0 + q) * cx.n_loc + first + p)
                                                      : CplxTraits<T>::zero();
    }
    __syncthreads();
    if (r < tk.r1) {
      if (r < s && r >= j0 && r < j1)
#pragma unroll
        for (int q = 0; q < RG; ++q) wr[q] = w[q * chunk + (r - j0)];
      // the same j sequence j = grp, grp + ngrp, ... in every chunking (j0 is a multiple of ngrp)
      const int jm = min(jmax, j1);
      int j = j0 + grp;
      // eight independent factor loads in flight per thread
      for (; j + 7 * ngrp < jm; j += 8 * ngrp) {
        T gv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) gv[t] = __ldg(Gr + (int64_t)j * ld + t * step);
#pragma unroll
        for (int t = 0; t < 8; ++t)
#pragma unroll
          for (int q = 0; q < RG; ++q) cfma(acc[q], gv[t], w[q * chunk + (j - j0 + t * ngrp)]);
      }
      for (; j < jm; j += ngrp) {
        const T gv = __ldg(Gr + (int64_t)j * ld);
#pragma unroll
        for (int q = 0; q < RG; ++q) cfma(acc[q], gv, w[q * chunk + (j - j0)]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < RG; ++q) red[threadIdx.x * RG + q] = acc[q];
  __syncthreads();
  if (grp == 0 && r < tk.r1) {
    for (int g2 = 1; g2 < ngrp; ++g2)
#pragma unroll
      for (int q = 0; q < RG; ++q) acc[q] = cadd(acc[q], red[(g2 * R + i) * RG + q]);
    if (r < s) {
      const T dinv = cdiv(CplxTraits<T>::one(), G[(int64_t)r * ld + r]);
#pragma unroll
      for (int q = 0; q < RG; ++q)
        if (rhs0 + q < cx.nrhs) {
          const T y = cadd(acc[q], wr[q]);
          const int64_t o = (int64_t)(rhs0 + q) * cx.n_loc + first + r;
          cx.xf[o] = cmul(y, dinv);
          if (cx.si != PSP_SI_EXTENDED) cx.xb[o] = y;
        }
    } else {
      T wu[RG];
#pragma unroll
      for (int q = 0; q < RG; ++q) wu[q] = CplxTraits<T>::zero();
      pull_add<T, RG>(cx, pull + 2 * r, rhs0, wu);
      const int64_t o = cx.sh.upd_off[sn] + (r - s);
#pragma unroll
      for (int q = 0; q < RG; ++q)
        if (rhs0 + q < cx.nrhs) cx.upd[(int64_t)(rhs0 + q) * cx.upd_ld + o] = csub(wu[q], acc[q]);
    }
  }
}

// Without inversion (G keeps L_TL): the first phase up the tree of front sn by one CTA: w_S gathered
// as above, then forward substitution y_S = L_TL^{-1} w_S in blocks of 32 columns (one warp solves
// the diagonal block, all threads update the rows below it), x_S = D^{-1} y_S into xf, y_S into xb.
template <typename T, int RG>
__device__ __forceinline__ void fwd_tri_task(const SolveTask tk, const int rhs0, const SolveCtx<T>& cx,
                                             unsigned char* smem_raw) {
  const int sn = tk.sn;
  const int s = cx.sh.s[sn], ld = s + cx.sh.u[sn];
  const int first = cx.sh.first[sn];
  const T* G = cx.G + cx.sh.g_off[sn];
  const int32_t* pull = cx.sh.pull + 2 * cx.sh.pull_ptr[sn];
  T* w = reinterpret_cast<T*>(smem_raw);        // RG x s (right-hand side major)
  for (int p = threadIdx.x; p < s; p += blockDim.x) {
    const int node = cx.sh.order[first + p];
    T v[RG];
#pragma unroll
    for (int q = 0; q < RG; ++q) v[q] = (rhs0 + q < cx.nrhs) ? input_value(cx, node, rhs0 + q) : CplxTraits<T>::zero();
    pull_add<T, RG>(cx, pull + 2 * p, rhs0, v);
#pragma unroll
    for (int q = 0; q < RG; ++q) w[q * s + p] = v[q];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int b = 0; b < s; b += 32) {
    const int be = min(b + 32, s);
    if (warp == 0) {
      // diagonal block: y_j final, then w_k -= L[k, j] y_j for b <= j < k < be
      for (int j = b; j < be; ++j) {
        const int k = b + lane;
        const T l = (k > j && k < be) ? __ldg(G + (int64_t)j * ld + k) : CplxTraits<T>::zero();
        __syncwarp();
        if (k > j && k < be)
#pragma unroll
          for (int q = 0; q < RG; ++q) cfms(w[q * s + k], l, w[q * s + j]);
        __syncwarp();
      }
    }
    __syncthreads();
    // rows below the block: w_i -= sum_{j in block} L[i, j] y_j
    for (int i = be + threadIdx.x; i < s; i += blockDim.x) {
      T acc[RG];
#pragma unroll
      for (int q = 0; q < RG; ++q) acc[q] = CplxTraits<T>::zero();
      for (int j = b; j < be; ++j) {
        const T l = __ldg(G + (int64_t)j * ld + i);
#pragma unroll
        for (int q = 0; q < RG; ++q) cfma(acc[q], l, w[q * s + j]);
      }
#pragma unroll
      for (int q = 0; q < RG; ++q) w[q * s + i] = csub(w[q * s + i], acc[q]);
    }
    __syncthreads();
  }
  for (int r = threadIdx.x; r < s; r += blockDim.x) {
    const T dinv = cdiv(CplxTraits<T>::one(), G[(int64_t)r * ld + r]);
#pragma unroll
    for (int q = 0; q < RG; ++q)
      if (rhs0 + q < cx.nrhs) {
        const int64_t o = (int64_t)(rhs0 + q) * cx.n_loc + first + r;
        cx.xb[o] = w[q * s + r];
        cx.xf[o] = cmul(w[q * s + r], dinv);
      }
  }
}

template <typename T, int RG>
__global__ void __launch_bounds__(256) k_solve_fwd(const SolveTask* __restrict__ tasks, SolveCtx<T> cx, int R,
                                                   int phase, int chunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (phase == 0 && cx.si == PSP_SI_NONE) fwd_tri_task<T, RG>(tasks[blockIdx.x], blockIdx.y * RG, cx, smem_raw);
  else fwd_task<T, RG>(tasks[blockIdx.x], blockIdx.y * RG, cx, R, smem_raw, phase, chunk);
}

// the final write of x_S column c of a front: xb (elimination order) and, for the panel's own
// planes, the global vector (Alg. 1.3 extraction; assigned in the forward sweep, subtracted in the
// backward sweep)
template <typename T>
__device__ __forceinline__ void write_solution(const SolveCtx<T>& cx, const int first, const int c, const int q,
                                               const T out) {
  cx.xb[(int64_t)q * cx.n_loc + first + c] = out;
  const int node = cx.sh.order[first + c];
  const int nx = cx.sh.nx, ny = cx.sh.ny;
  const int k = node / (nx * ny);
  if (k >= cx.lead) {
    const int64_t g = (node % (nx * ny)) + (int64_t)nx * ny * (cx.z0 + k - cx.lead);
    double2* uq = cx.u + (int64_t)q * cx.N + g;
    const double2 o = to_c128(out);
    *uq = (cx.mode == 0) ? o : csub(__ldcg(uq), o);
  }
}

// down-the-tree task: columns [r0, r1) of S of front sn.
//   extended factors (phase 0): x_c = xf_c + sum_{r > c} G[r, c] y_r over all s + u rows, with
//     y = xf on S and -x_U on the struct rows; writes the solution.
//   factors keeping L_BL, phase 0: t_c = xf_c - sum_{r >= s} L_BL[r, c] x_U[r] into xf.
//   paper's factors, phase 1: x_c = t_c + sum_{c < r < s} inv(L_TL)[r, c] t_r; writes the solution.
template <typename T, int RG>
__device__ __forceinline__ void bwd_task(const SolveTask tk, const int rhs0, const SolveCtx<T>& cx,
                                         unsigned char* smem_raw, const int phase, const int chunk) {
  const int sn = tk.sn;
  const int s = cx.sh.s[sn], u = cx.sh.u[sn], ld = s + u;
  const int first = cx.sh.first[sn];
  const T* G = cx.G + cx.sh.g_off[sn];
  const int32_t* sel = cx.sh.struct_elim + cx.sh.struct_ptr[sn];
  const int c0 = tk.r0;
  const bool ext = cx.si == PSP_SI_EXTENDED;
  // rows of the inner sums: [lo, hi), passed through shared memory in chunks of `chunk` rows
  const int lo = (ext || phase == 1) ? c0 : s;
  const int hi = (ext || phase == 0) ? ld : s;
  // the columns the inner sums read: G's, or in the two-inverse form's second phase the second
  // inverse of L_TL (s x s after G), which was built row by row for this direction
  const bool second = phase == 1 && cx.si == PSP_SI_TWO;
  const T* Gs = second ? G + second_inverse_offset(s, u) : G;
  const int lds = second ? s : ld;
  // right-hand side major (y[q * chunk + row]): the lanes of a warp read consecutive rows, so the
  // loads are free of bank conflicts whatever RG is
  T* y = reinterpret_cast<T*>(smem_raw);        // RG x chunk
  T* sums = y + (int64_t)chunk * RG;            // (r1 - c0) x RG column sums (<= 256 columns)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int e = threadIdx.x; e < (tk.r1 - c0) * RG; e += blockDim.x) sums[e] = CplxTraits<T>::zero();
  for (int rb = lo; rb < hi; rb += chunk) {
    const int re = min(rb + chunk, hi);
    __syncthreads();   // sums initialised / the previous chunk consumed
    for (int r = rb + threadIdx.x; r < re; r += blockDim.x) {
#pragma unroll
      for (int q = 0; q < RG; ++q) {
        T v = CplxTraits<T>::zero();
        if (rhs0 + q < cx.nrhs) {
          const int64_t base = (int64_t)(rhs0 + q) * cx.n_loc;
          v = (r < s) ? __ldcg(cx.xf + base + first + r) : cneg(__ldcg(cx.xb + base + sel[r - s]));
        }
        y[q * chunk + (r - rb)] = v;
      }
    }
    __syncthreads();
    for (int c = c0 + warp; c < tk.r1; c += nw) {
      T acc[RG];
#pragma unroll
      for (int q = 0; q < RG; ++q) acc[q] = CplxTraits<T>::zero();
      const T* Gc = Gs + (int64_t)c * lds;
      int r = (rb > c + 1 ? rb : c + 1) + lane;
      for (; r + 7 * 32 < re; r += 8 * 32) {   // eight independent factor loads in flight per lane
        T gv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) gv[t] = __ldg(Gc + r + 32 * t);
#pragma unroll
        for (int t = 0; t < 8; ++t)
#pragma unroll
          for (int q = 0; q < RG; ++q) cfma(acc[q], gv[t], y[q * chunk + (r + 32 * t - rb)]);
      }
      for (; r < re; r += 32) {
        const T gv = __ldg(Gc + r);
#pragma unroll
        for (int q = 0; q < RG; ++q) cfma(acc[q], gv, y[q * chunk + (r - rb)]);
      }
#pragma unroll
      for (int q = 0; q < RG; ++q) {
        for (int off = 16; off > 0; off >>= 1) {
          acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, off);
          acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, off);
        }
        if (lane == 0) sums[(c - c0) * RG + q] = cadd(sums[(c - c0) * RG + q], acc[q]);
      }
    }
  }
  __syncthreads();
  for (int c = c0 + threadIdx.x; c < tk.r1; c += blockDim.x) {
#pragma unroll
    for (int q = 0; q < RG; ++q) {
      if (rhs0 + q >= cx.nrhs) continue;
      const int64_t o = (int64_t)(rhs0 + q) * cx.n_loc + first + c;
      const T v = cadd(sums[(c - c0) * RG + q], __ldcg(cx.xf + o));   // + xf_c (z_c, or t_c in phase 1)
      if (!ext && phase == 0) cx.xf[o] = v;                           // t_c: this thread's column only
      else write_solution(cx, first, c, rhs0 + q, v);
    }
  }
}

// Without inversion: the second phase down the tree of front sn by one CTA: back substitution
// L_TL^T x_S = t (t in xf) in blocks of 32 columns from the last, each block first takes the
// products with the solved rows below it (one warp per column), then one warp solves the block.
template <typename T, int RG>
__device__ __forceinline__ void bwd_tri_task(const SolveTask tk, const int rhs0, const SolveCtx<T>& cx,
                                             unsigned char* smem_raw) {
  const int sn = tk.sn;
  const int s = cx.sh.s[sn], ld = s + cx.sh.u[sn];
  const int first = cx.sh.first[sn];
  const T* G = cx.G + cx.sh.g_off[sn];
  T* x = reinterpret_cast<T*>(smem_raw);   // RG x s (right-hand side major): t, overwritten by x block by block
  for (int r = threadIdx.x; r < s; r += blockDim.x)
#pragma unroll
    for (int q = 0; q < RG; ++q)
      x[q * s + r] = (rhs0 + q < cx.nrhs) ? __ldcg(cx.xf + (int64_t)(rhs0 + q) * cx.n_loc + first + r)
                                           : CplxTraits<T>::zero();
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nblk = (s + 31) / 32;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int b = bi * 32, be = min(b + 32, s);
    // x_c -= sum_{r >= be} L[r, c] x_r for the block's columns
    for (int c = b + warp; c < be; c += nw) {
      T acc[RG];
#pragma unroll
      for (int q = 0; q < RG; ++q) acc[q] = CplxTraits<T>::zero();
      for (int r = be + lane; r < s; r += 32) {
        const T l = __ldg(G + (int64_t)c * ld + r);
#pragma unroll
        for (int q = 0; q < RG; ++q) cfma(acc[q], l, x[q * s + r]);
      }
#pragma unroll
      for (int q = 0; q < RG; ++q) {
        for (int off = 16; off > 0; off >>= 1) {
          acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, off);
          acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, off);
        }
        if (lane == 0) x[q * s + c] = csub(x[q * s + c], acc[q]);
      }
    }
    __syncthreads();
    if (warp == 0) {
      // the block, from its last column: x_c final, then x_k -= L[c, k] x_c for b <= k < c
      for (int c = be - 1; c >= b; --c) {
        const int k = b + lane;
        const T l = (k < c) ? __ldg(G + (int64_t)k * ld + c) : CplxTraits<T>::zero();
        __syncwarp();
        if (k < c)
#pragma unroll
          for (int q = 0; q < RG; ++q) cfms(x[q * s + k], l, x[q * s + c]);
        __syncwarp();
      }
    }
    __syncthreads();
  }
  for (int c = threadIdx.x; c < s; c += blockDim.x)
#pragma unroll
    for (int q = 0; q < RG; ++q)
      if (rhs0 + q < cx.nrhs) write_solution(cx, first, c, rhs0 + q, x[q * s + c]);
}

template <typename T, int RG>
__global__ void __launch_bounds__(256) k_solve_bwd(const SolveTask* __restrict__ tasks, SolveCtx<T> cx, int phase,
                                                   int chunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (phase == 1 && cx.si == PSP_SI_NONE) bwd_tri_task<T, RG>(tasks[blockIdx.x], blockIdx.y * RG, cx, smem_raw);
  else bwd_task<T, RG>(tasks[blockIdx.x], blockIdx.y * RG, cx, smem_raw, phase, chunk);
}

// rhs group size so that the shared-memory footprint stays below ~200 KB
template <typename T>
static int pick_rg(int nrhs, size_t per_rhs_bytes) {
  int rg = 8;
  while (rg > 1 && (rg >= 2 * nrhs || per_rhs_bytes * rg > 200 * 1024)) rg >>= 1;
  return rg;
}

// ---------------------------------------------------------------------------
// The whole sweep of Alg. 1.5 in one cooperative launch, as a dataflow over the elimination trees.
// CTAs take tasks from one queue in topological order.  An up-the-tree task of a front waits until
// every task of its children has finished (one counter per front, which its children's tasks
// increment); a front without children waits for the previous panel solve of its problem's chain
// (the chains of a batch of independent problems are interleaved in the queue and run side by
// side), so every front does, through its descendants.  A down-the-tree task waits for its parent
// (the root: for its own up-the-tree tasks).  A task only waits on tasks earlier in the queue.  A
// CTA claims its tasks in queue order, one or two ahead of the task it runs; the earliest unfinished
// task is therefore the one some CTA runs (a CTA holding it only as a later task would be running an
// earlier unfinished one), every task it waits for has finished, and since every CTA of a
// cooperative launch is resident, the sweep progresses.  Each wait is bounded anyway: a CTA that
// gives up sets status[2] and stops; the others then give up at their next wait.
// ---------------------------------------------------------------------------
constexpr long long kWaitCycles = 4000000000LL;   // SM clock cycles: about two seconds at 2 GHz
constexpr long long kWaitSpins = 400000000LL;     // and a hard cap on polls, whatever the clock does

// a wait that gives up sets status[2] (cleared before every sweep) and the handle's sticky flag
// (cleared only when the host reads it)
__device__ __forceinline__ bool wait_count(const unsigned* p, unsigned target, int* status, int* sticky) {
  const long long t0 = clock64();
  long long it = 0;
  while (*(volatile const unsigned*)p < target) {
    if (*(volatile int*)(status + 2) != 0) return false;
    if (++it > kWaitSpins || clock64() - t0 > kWaitCycles) {
      atomicExch(status + 2, 1);
      if (sticky) atomicExch(sticky, 1);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// Warm L2 with the factor lines a task will stream, while its dependencies are still being
// waited for (the lines do not depend on them): up the tree rows [r0, r1) of the columns
// j < min(r1, s), down the tree columns [c0, c1) from below their diagonal to the end.
template <typename T>
__device__ __forceinline__ void prefetch_task(const SolveTask tk, const int dir, const SolveCtx<T>& cx) {
  const int sn = tk.sn;
  const int s = cx.sh.s[sn], ld = s + cx.sh.u[sn];
  const char* G = reinterpret_cast<const char*>(cx.G + cx.sh.g_off[sn]);
  constexpr int kLine = 128;
  if (dir == 0 || dir == kDirUpB) {
    const int ncol = min(tk.r1, s);
    const int64_t seg = (int64_t)(tk.r1 - tk.r0) * sizeof(T);
    const int lines = (int)((seg + kLine - 1) / kLine) + 1;   // the segment may straddle one more line
    for (int w = threadIdx.x; w < ncol * lines; w += blockDim.x) {
      const int j = w / lines, l = w % lines;
      const char* col = G + ((int64_t)j * ld + tk.r0) * sizeof(T);
      const char* a = col + (int64_t)l * kLine;
      if (a < col + seg) asm volatile("prefetch.L2 [%0];" ::"l"(a));
    }
  } else {
    const bool second = dir == kDirDownB && cx.si == PSP_SI_TWO;   // the second inverse after G
    const char* Gs = second ? G + second_inverse_offset(s, ld - s) * sizeof(T) : G;
    const int lds = second ? s : ld;
    for (int c = tk.r0; c < tk.r1; ++c) {
      const char* col = Gs + ((int64_t)c * lds + c + 1) * sizeof(T);
      const int64_t seg = (int64_t)(lds - c - 1) * sizeof(T);
      for (int64_t off = (int64_t)threadIdx.x * kLine; off < seg; off += (int64_t)blockDim.x * kLine)
        asm volatile("prefetch.L2 [%0];" ::"l"(col + off));
    }
  }
}

// tables cached in shared memory when they fit (a single problem: at most 3-4 shapes; batches
// and very deep sweeps read them from global memory instead)
constexpr int kMaxSweepShapes = 4, kMaxSweepSteps = 512, kMaxSweepPanels = 256;
constexpr int kSweepThreads = 256;

// one 16-byte asynchronous copy global -> shared (completed by cp_async_wait_all of the same thread)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T, int RG>
__global__ void __launch_bounds__(kSweepThreads) k_sweep(SweepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) QueueEntry s_q[2];   // the current task's queue entry and the next one's
  __shared__ int s_idx, s_ok;
  __shared__ SolveCtx<T> s_cx;      // this task's panel solve, filled by thread 0
  __shared__ ShapeDev s_shape[kMaxSweepShapes];
  __shared__ SweepStep s_step[kMaxSweepSteps];
  __shared__ PanelSweep s_panel[kMaxSweepPanels];
  // small per-sweep tables in shared memory when they fit; larger ones (batches of problems) are
  // read from global memory by thread 0
  const bool tab_smem = a.nshapes <= kMaxSweepShapes && a.nsteps <= kMaxSweepSteps && a.npanels <= kMaxSweepPanels;
  if (tab_smem) {
    for (int i = threadIdx.x; i < a.nshapes; i += blockDim.x) s_shape[i] = a.shapes[i];
    for (int i = threadIdx.x; i < a.nsteps; i += blockDim.x) s_step[i] = a.steps[i];
    for (int i = threadIdx.x; i < a.npanels; i += blockDim.x) s_panel[i] = a.panels[i];
  }
  unsigned* head = a.ctr;
  unsigned* step_done = a.ctr + kSweepStepCounters;
  const int nrg = (a.cx.nrhs + RG - 1) / RG;
  // Thread 0 holds the index of this CTA's current task and of its next one, and the next one's queue
  // entry is copied into the other shared-memory slot asynchronously, so that taking a task costs no
  // dependent global load.  Claiming two ahead (claim_ahead 2), the task after the next one is claimed
  // while the current one waits and runs, and the next one's entry is copied meanwhile; claiming one
  // ahead, the next task is claimed as the current one starts waiting and its entry copied once the
  // wait is over, so a CTA holds one task besides the one it runs, not two.
  const bool two_ahead = a.claim_ahead > 1;
  int cur = 0, nxt = 0, buf = 0;
  if (threadIdx.x == 0) {
    cur = (int)atomicAdd(head, 1u);
    if (two_ahead) nxt = (int)atomicAdd(head, 1u);
    if (cur < a.nqueue) s_q[0] = a.queue[cur];
    s_cx = a.cx;   // fields common to every task; thread 0 sets the per-task ones below
  }
  for (;;) {
    if (threadIdx.x == 0) {
      s_idx = cur;
      if (cur < a.nqueue) {
        const QueueEntry& e = s_q[buf];
        const SweepStep sp = tab_smem ? s_step[e.step] : a.steps[e.step];
        const PanelSweep pi = tab_smem ? s_panel[sp.panel] : a.panels[sp.panel];
        SolveCtx<T>& cx = s_cx;
        cx.sh = tab_smem ? s_shape[pi.shape] : a.shapes[pi.shape];
        cx.G = a.factor + pi.gbase;
        cx.z0 = pi.z0;
        cx.z1 = pi.z1;
        cx.lead = pi.lead;
        cx.has_prev = pi.has_prev;
        cx.has_next = pi.has_next;
        cx.mode = sp.mode;
        if (a.nprobs > 1) {
          // the problem's own vector block, coupling tables and work vectors
          const ProblemSweep& pr = a.probs[sp.prob];
          cx.u = a.cx.u + pr.off1 * a.cx.nrhs;
          cx.N = pr.N;
          cx.nz = pr.nz;
          cx.s1n = pr.s1n;
          cx.s2n = pr.s2n;
          cx.s3h = pr.s3h;
          cx.inv_h2 = pr.inv_h2;
          cx.xf = a.cx.xf + (int64_t)sp.prob * a.cx.n_loc * a.cx.nrhs;
          cx.xb = a.cx.xb + (int64_t)sp.prob * a.cx.n_loc * a.cx.nrhs;
          cx.upd = a.cx.upd + (int64_t)sp.prob * a.cx.upd_ld * a.cx.nrhs;
        }
      }
    }
    __syncthreads();
    if (s_idx >= a.nqueue) break;
    const QueueEntry& e = s_q[buf];
    const SolveTask tk{e.sn, e.r0, e.r1};
    const int dir = e.dir, R = e.R;
    int after = 0;
    if (threadIdx.x == 0) {
      if (two_ahead) {
        after = (int)atomicAdd(head, 1u);   // the task after the next one (its index is read at the end)
        if (nxt < a.nqueue) {
          const char* src = reinterpret_cast<const char*>(a.queue + nxt);
          char* dst = reinterpret_cast<char*>(&s_q[buf ^ 1]);
          cp_async16(dst, src);
          cp_async16(dst + 16, src + 16);
          cp_async16(dst + 32, src + 32);
        }
      } else {
        nxt = (int)atomicAdd(head, 1u);   // the next task (its index is read after the wait)
      }
    }
    prefetch_task<T>(tk, dir, s_cx);
    if (threadIdx.x == 0) {
      const bool ok = e.wait < 0 || wait_count(a.ctr + e.wait, e.target, a.status, a.sticky);
      if (!two_ahead && nxt < a.nqueue) {
        const char* src = reinterpret_cast<const char*>(a.queue + nxt);
        char* dst = reinterpret_cast<char*>(&s_q[buf ^ 1]);
        cp_async16(dst, src);
        cp_async16(dst + 16, src + 16);
        cp_async16(dst + 32, src + 32);
      }
      __threadfence();
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    const bool tri = s_cx.si == PSP_SI_NONE;
    for (int g = 0; g < nrg; ++g) {
      if (dir == 0 && tri) fwd_tri_task<T, RG>(tk, g * RG, s_cx, smem_raw);
      else if (dir == 0 || dir == kDirUpB) fwd_task<T, RG>(tk, g * RG, s_cx, R, smem_raw, dir == 0 ? 0 : 1, a.chunk);
      else if (dir == kDirDownB && tri) bwd_tri_task<T, RG>(tk, g * RG, s_cx, smem_raw);
      else bwd_task<T, RG>(tk, g * RG, s_cx, smem_raw, dir == 1 ? 0 : 1, a.chunk);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      // completion counters of this task's front (and of its parent's children, up the tree) and step
      __threadfence();
      atomicAdd(a.ctr + e.done, 1u);
      if (e.kids >= 0) atomicAdd(a.ctr + e.kids, 1u);
      atomicAdd(step_done + e.step, 1u);
      cp_async_wait_all();   // the next task's entry has landed
      cur = nxt;
      if (two_ahead) nxt = after;
    }
    buf ^= 1;   // every thread: the next task's entry is in the other slot
  }
  if (threadIdx.x == 0) cp_async_wait_all();
}

template <typename T, int RG>
static int sweep_rg(const SweepArgs<T>& args, size_t smem, int max_per_sm, cudaStream_t st) {
  if (cudaFuncSetAttribute(k_sweep<T, RG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<T, RG>, kSweepThreads, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return -1;
  }
  per_sm = per_sm > max_per_sm ? max_per_sm : per_sm;
  SweepArgs<T> a = args;
  void* kargs[] = {&a};
  cudaError_t e =
      cudaLaunchCooperativeKernel((const void*)k_sweep<T, RG>, dim3(sms * per_sm), dim3(kSweepThreads), kargs, smem, st);
  return e == cudaSuccess ? 0 : (int)e;
}

// A CTA carries RG right-hand sides through each pass over a factor block (as many as nrhs, at most 8,
// or rhs_group when > 0), and the vectors of a task pass through shared memory in chunks sized so
// that a CTA keeps within kSweepSmem (several CTAs stay resident per SM: a CTA that waits on a
// dependency leaves the SM to the others).  Substitution tasks (fronts keeping L_TL) hold a front's
// whole vector, so for them RG shrinks until that fits.
constexpr size_t kSweepSmem = 64 * 1024;

template <typename T>
int launch_sweep(const SweepArgs<T>& args, int smax, int ldmax, int max_per_sm, int rhs_group, cudaStream_t st) {
  const size_t es = sizeof(T);
  int rg = 8;
  while (rg > 1 && rg >= 2 * args.cx.nrhs) rg >>= 1;
  if (rhs_group > 0)
    while (rg > 1 && rg > rhs_group) rg >>= 1;
  const int full = (ldmax > smax ? ldmax : smax);
  int chunk;
  if (args.cx.si == PSP_SI_NONE) {
    chunk = full;
    while (rg > 1 && ((size_t)chunk + 256) * rg * es > 200 * 1024) rg >>= 1;
  } else {
    chunk = (int)((kSweepSmem / (rg * es) - 256) / 256 * 256);
    if (chunk < 256) chunk = 256;
    if (chunk >= full) chunk = full;   // one chunk: every task's vector at once
  }
  SweepArgs<T> a = args;
  a.chunk = chunk;
  const size_t smem = ((size_t)chunk + 256) * rg * es;
  switch (rg) {
    case 8: return sweep_rg<T, 8>(a, smem, max_per_sm, st);
    case 4: return sweep_rg<T, 4>(a, smem, max_per_sm, st);
    case 2: return sweep_rg<T, 2>(a, smem, max_per_sm, st);
    default: return sweep_rg<T, 1>(a, smem, max_per_sm, st);
  }
}

template <typename T, int RG>
static void fwd_rg(const SolveTask* tasks, int ntasks, const SolveCtx<T>& cx, int R, int smax, int phase, cudaStream_t st) {
  const size_t smem = ((size_t)smax + 256) * RG * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_solve_fwd<T, RG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr_set = true;
  }
  dim3 grid(ntasks, (cx.nrhs + RG - 1) / RG);
  k_solve_fwd<T, RG><<<grid, 256, smem, st>>>(tasks, cx, R, phase, smax > 0 ? smax : 1);
}

template <typename T, int RG>
static void bwd_rg(const SolveTask* tasks, int ntasks, const SolveCtx<T>& cx, int ldmax, int phase, cudaStream_t st) {
  const size_t smem = ((size_t)ldmax + 256) * RG * sizeof(T);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_solve_bwd<T, RG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr_set = true;
  }
  dim3 grid(ntasks, (cx.nrhs + RG - 1) / RG);
  k_solve_bwd<T, RG><<<grid, 256, smem, st>>>(tasks, cx, phase, ldmax > 0 ? ldmax : 1);
}

template <typename T>
void launch_solve_fwd(const SolveTask* tasks, int ntasks, const SolveCtx<T>& cx, int R, int smax, int phase,
                      cudaStream_t st) {
  if (ntasks <= 0) return;
  const int rg = pick_rg<T>(cx.nrhs, ((size_t)smax + 256) * sizeof(T));
  switch (rg) {
    case 8: fwd_rg<T, 8>(tasks, ntasks, cx, R, smax, phase, st); break;
    case 4: fwd_rg<T, 4>(tasks, ntasks, cx, R, smax, phase, st); break;
    case 2: fwd_rg<T, 2>(tasks, ntasks, cx, R, smax, phase, st); break;
    default: fwd_rg<T, 1>(tasks, ntasks, cx, R, smax, phase, st); break;
  }
}

template <typename T>
void launch_solve_bwd(const SolveTask* tasks, int ntasks, const SolveCtx<T>& cx, int ldmax, int phase, cudaStream_t st) {
  if (ntasks <= 0) return;
  const int rg = pick_rg<T>(cx.nrhs, ((size_t)ldmax + 256) * sizeof(T));
  switch (rg) {
    case 8: bwd_rg<T, 8>(tasks, ntasks, cx, ldmax, phase, st); break;
    case 4: bwd_rg<T, 4>(tasks, ntasks, cx, ldmax, phase, st); break;
    case 2: bwd_rg<T, 2>(tasks, ntasks, cx, ldmax, phase, st); break;
    default: bwd_rg<T, 1>(tasks, ntasks, cx, ldmax, phase, st); break;
  }
}

template void launch_solve_fwd<double2>(const SolveTask*, int, const SolveCtx<double2>&, int, int, int, cudaStream_t);
template void launch_solve_fwd<float2>(const SolveTask*, int, const SolveCtx<float2>&, int, int, int, cudaStream_t);
template void launch_solve_bwd<double2>(const SolveTask*, int, const SolveCtx<double2>&, int, int, cudaStream_t);
template void launch_solve_bwd<float2>(const SolveTask*, int, const SolveCtx<float2>&, int, int, cudaStream_t);
template int launch_sweep<double2>(const SweepArgs<double2>&, int, int, int, int, cudaStream_t);
template int launch_sweep<float2>(const SweepArgs<float2>&, int, int, int, int, cudaStream_t);

}  // namespace psp

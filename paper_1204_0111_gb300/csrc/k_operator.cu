// 7-point Helmholtz operators with PML (Eq. (1.1), Eq. (1.5), §1.1): coefficients, the
// complex128 stencil matvec used by GMRES, and batched front assembly + extend-add (§2.2).
#include "cplx.cuh"
#include "psp_internal.h"

namespace psp {

// Row of the s1 s2 s3-scaled operator at box node (x, y, z):
//   a_1(x -+ 1/2) = s2 s3 / s1(x -+ 1/2), a_2, a_3 alike; off-diagonals -a/h^2,
//   diagonal sum(a)/h^2 - k2num / c^2 * s1 s2 s3.
// The BoxOp stores the reciprocal stretches at half-points (s?h fields hold 1/s there).
struct Row7 {
  double2 d, xm, xp, ym, yp, zm, zp;
};

__device__ __forceinline__ Row7 row7(const BoxOp& op, int x, int y, int z) {
  const double2 s1 = op.s1n[x], s2 = op.s2n[y], s3 = op.s3n[z];
  const double2 s23 = cmul(s2, s3), s13 = cmul(s1, s3), s12 = cmul(s1, s2);
  const double2 axm = cmul(s23, op.s1h[x]), axp = cmul(s23, op.s1h[x + 1]);
  const double2 aym = cmul(s13, op.s2h[y]), ayp = cmul(s13, op.s2h[y + 1]);
  const double2 azm = cmul(s12, op.s3h[z]), azp = cmul(s12, op.s3h[z + 1]);
  const double cc = op.c[((int64_t)op.cplane[z] * op.ny + y) * op.nx + x];
  const double2 mass = cmul(cscale(op.k2num, 1.0 / (cc * cc)), cmul(s12, s3));
  Row7 r;
  double2 sum = cadd(cadd(cadd(axm, axp), cadd(aym, ayp)), cadd(azm, azp));
  r.d = csub(cscale(sum, op.inv_h2), mass);
  r.xm = cscale(axm, -op.inv_h2);
  r.xp = cscale(axp, -op.inv_h2);
  r.ym = cscale(aym, -op.inv_h2);
  r.yp = cscale(ayp, -op.inv_h2);
  r.zm = cscale(azm, -op.inv_h2);
  r.zp = cscale(azp, -op.inv_h2);
  return r;
}

// y = Op x for nrhs vectors (column-major, ld = N); one thread per node.
__global__ void k_matvec(BoxOp op, const double2* __restrict__ x, double2* __restrict__ y, int nrhs, int64_t N) {
  const int64_t plane = (int64_t)op.nx * op.ny;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    const int xx = (int)(g % op.nx);
    const int yy = (int)((g / op.nx) % op.ny);
    const int zz = (int)(g / plane);
    const Row7 r = row7(op, xx, yy, zz);
    for (int q = 0; q < nrhs; ++q) {
      const double2* xv = x + q * N;
      double2 acc = cmul(r.d, xv[g]);
      if (xx > 0) cfma(acc, r.xm, xv[g - 1]);
      if (xx + 1 < op.nx) cfma(acc, r.xp, xv[g + 1]);
      if (yy > 0) cfma(acc, r.ym, xv[g - op.nx]);
      if (yy + 1 < op.ny) cfma(acc, r.yp, xv[g + op.nx]);
      if (zz > 0) cfma(acc, r.zm, xv[g - plane]);
      if (zz + 1 < op.nz) cfma(acc, r.zp, xv[g + plane]);
      y[q * N + g] = acc;
    }
  }
}

// b = s1 s2 s3 f (the right-hand side of the symmetrised system)
__global__ void k_scale_rhs(BoxOp op, const double2* __restrict__ f, double2* __restrict__ b, int nrhs, int64_t N) {
  const int64_t plane = (int64_t)op.nx * op.ny;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    const int xx = (int)(g % op.nx);
    const int yy = (int)((g / op.nx) % op.ny);
    const int zz = (int)(g / plane);
    const double2 s = cmul(cmul(op.s1n[xx], op.s2n[yy]), op.s3n[zz]);
    for (int q = 0; q < nrhs; ++q) b[q * N + g] = cmul(s, f[q * N + g]);
  }
}

static int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  return (int)(b < 1 ? 1 : b);
}

void launch_matvec(const BoxOp& op, const double2* x, double2* y, int nrhs, int64_t N, cudaStream_t st) {
  k_matvec<<<grid_for(N, 256), 256, 0, st>>>(op, x, y, nrhs, N);
}
void launch_scale_rhs(const BoxOp& op, const double2* f, double2* b, int nrhs, int64_t N, cudaStream_t st) {
  k_scale_rhs<<<grid_for(N, 256), 256, 0, st>>>(op, f, b, nrhs, N);
}

// ---------------------------------------------------------------------------
// Front assembly (§2.2): F_TL = H[S,S], F_BL = H[U,S], F_BR = 0, then the children's update
// matrices are added through the relative index maps (extend-add).  One CTA owns a chunk of
// the front's (s+u) columns, so no two CTAs touch the same entry; children are added one after
// the other, which fixes the summation order.  The same pass initialises W = I (s x s).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_assemble(const FrontTask<T>* __restrict__ fronts,
                                                  const ColTask* __restrict__ tasks, const ShapeDev* __restrict__ shapes,
                                                  const BoxOp* __restrict__ boxops, T* const* __restrict__ upd_ptr,
                                                  const int32_t* __restrict__ upd_tile,
                                                  const int32_t* __restrict__ panel_shape) {
  const ColTask tk = tasks[blockIdx.x];
  const FrontTask<T> ft = fronts[tk.front];
  const ShapeDev sh = shapes[panel_shape[ft.panel]];
  const BoxOp op = boxops[ft.panel];
  const int s = ft.s, u = ft.u, ld = s + u;
  const int c0 = tk.c0, c1 = tk.c1;
  const int first = sh.first[ft.sn];
  const int32_t* sel = sh.struct_elim + sh.struct_ptr[ft.sn];
  const T zero = CplxTraits<T>::zero();

  // 1. zero the owned columns; W (and W2) = identity (when inverses of L_TL are built)
  for (int c = c0; c < c1; ++c) {
    if (c < s) {
      T* col = ft.G + (int64_t)c * ld;
      for (int r = threadIdx.x; r < ld; r += blockDim.x) col[r] = zero;
      if (ft.W) {
        T* wc = ft.W + (int64_t)c * s;
        for (int r = threadIdx.x; r < s; r += blockDim.x) wc[r] = (r == c) ? CplxTraits<T>::one() : zero;
      }
      if (ft.W2) {
        T* wc = ft.W2 + (int64_t)c * s;
        for (int r = threadIdx.x; r < s; r += blockDim.x) wc[r] = (r == c) ? CplxTraits<T>::one() : zero;
      }
    } else {
      // the lower part of column c - s of the packed update matrix
      for (int r = c - s + threadIdx.x; r < u; r += blockDim.x) ft.U[upd_index(r, c - s, u, ft.ut)] = zero;
    }
  }
  __syncthreads();

  // 2. original entries H[r, j], j in S (column), elim(r) >= elim(j)
  const int cs1 = c1 < s ? c1 : s;
  for (int w = threadIdx.x; w < (cs1 - c0) * 7; w += blockDim.x) {
    const int c = c0 + w / 7, which = w % 7;
    if (c >= cs1) continue;
    const int node = sh.order[first + c];
    const int x = node % sh.nx, y = (node / sh.nx) % sh.ny, z = node / (sh.nx * sh.ny);
    int nx = x, ny = y, nz = z;
    switch (which) {
      case 1: nx = x - 1; break;
      case 2: nx = x + 1; break;
      case 3: ny = y - 1; break;
      case 4: ny = y + 1; break;
      case 5: nz = z - 1; break;
      case 6: nz = z + 1; break;
      default: break;
    }
    if (nx < 0 || nx >= sh.nx || ny < 0 || ny >= sh.ny || nz < 0 || nz >= sh.nz) continue;
    const int rnode = nx + sh.nx * (ny + sh.ny * nz);
    const int e = sh.elim[rnode];
    if (e < first + c) continue;
    int pos;
    if (e < first + s) {
      pos = e - first;
    } else {
      int lo = 0, hi = u;  // lower_bound in struct(S)
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (sel[mid] < e) lo = mid + 1; else hi = mid;
      }
      pos = s + lo;
    }
    const Row7 r7 = row7(op, x, y, z);
    double2 v;
    switch (which) {
      case 0: v = r7.d; break;
      case 1: v = r7.xm; break;
      case 2: v = r7.xp; break;
      case 3: v = r7.ym; break;
      case 4: v = r7.yp; break;
      case 5: v = r7.zm; break;
      default: v = r7.zp; break;
    }
    ft.G[(int64_t)c * ld + pos] = CplxTraits<T>::from(v);
  }
  __syncthreads();

  // 3. extend-add of each child's update matrix (lower triangle), child by child
  for (int ci = sh.child_ptr[ft.sn]; ci < sh.child_ptr[ft.sn + 1]; ++ci) {
    const int ch = sh.child_idx[ci];
    const int uc = sh.u[ch];
    const int32_t* rel = sh.rel + sh.struct_ptr[ch];
    const T* Uc = upd_ptr[ft.gfid - ft.sn + ch];
    const int utc = upd_tile[ft.gfid - ft.sn + ch];
    // child columns b whose target column rel[b] lies in [c0, c1): a contiguous range
    int b0 = 0, b1 = uc;
    {
      int lo = 0, hi = uc;
      while (lo < hi) { int mid = (lo + hi) >> 1; if (rel[mid] < c0) lo = mid + 1; else hi = mid; }
      b0 = lo;
      lo = b0; hi = uc;
      while (lo < hi) { int mid = (lo + hi) >> 1; if (rel[mid] < c1) lo = mid + 1; else hi = mid; }
      b1 = lo;
    }
    // one warp per child column (the columns land in distinct target columns, so the warps never
    // touch the same entry), four independent entries in flight per lane
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int b = b0 + warp; b < b1; b += nw) {
      const int tc = rel[b];
      for (int a0 = b + lane; a0 < uc; a0 += 4 * 32) {
        T* dst[4];
        T val[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int a = a0 + 32 * t;
          dst[t] = nullptr;
          if (a < uc) {
            const int ra = rel[a];
            dst[t] = tc < s ? ft.G + (int64_t)tc * ld + ra : ft.U + upd_index(ra - s, tc - s, u, ft.ut);
            val[t] = Uc[upd_index(a, b, uc, utc)];
          }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (dst[t]) *dst[t] = cadd(*dst[t], val[t]);
      }
    }
    __syncthreads();
  }
}

template <typename T>
void launch_assemble_impl(const FrontTask<T>* fronts, const ColTask* tasks, int ntasks, const ShapeDev* shapes,
                          const BoxOp* boxops, T* const* upd_ptr, const int32_t* upd_tile, const int32_t* panel_shape,
                          cudaStream_t st) {
  if (ntasks <= 0) return;
  k_assemble<T><<<ntasks, 256, 0, st>>>(fronts, tasks, shapes, boxops, upd_ptr, upd_tile, panel_shape);
}

template void launch_assemble_impl<double2>(const FrontTask<double2>*, const ColTask*, int, const ShapeDev*,
                                            const BoxOp*, double2* const*, const int32_t*, const int32_t*,
                                            cudaStream_t);
template void launch_assemble_impl<float2>(const FrontTask<float2>*, const ColTask*, int, const ShapeDev*,
                                           const BoxOp*, float2* const*, const int32_t*, const int32_t*,
                                           cudaStream_t);

}  // namespace psp

// Complex128 building blocks of right-preconditioned restarted GMRES(k) (§2.4): batched inner
// products with a fixed two-stage reduction (no atomics, so every run sums in the same order and
// the Krylov recurrence is reproducible), multi-vector updates, and the Hessenberg least-squares
// by complex Givens rotations, one thread per column.  A column is one right-hand side of one
// problem; columns may differ in length (independent problems of a batch).
#include "cplx.cuh"
#include "psp_internal.h"

namespace psp {

constexpr int kDotBlocks = 152 * 2;    // most partial blocks per column
constexpr int64_t kDotMinChunk = 1024;   // fewest elements per partial block

// blocks that column `len` is cut into: a function of its own length only, so a column sums in
// the same order whatever other columns share the launch
__device__ __host__ __forceinline__ int dot_blocks_for(int64_t len) {
  int64_t b = (len + kDotMinChunk - 1) / kDotMinChunk;
  return (int)(b < 1 ? 1 : (b > kDotBlocks ? kDotBlocks : b));
}

int multidot_blocks(int64_t maxlen) { return dot_blocks_for(maxlen); }

// partial[(b * nvec + i) * ncol + c] = sum_{g in slice b of column c} conj(V_i[c][g]) * w[c][g]
__global__ void __launch_bounds__(256) k_dot_partial(const double2* __restrict__ V, int64_t ldv_vec,
                                                     const double2* __restrict__ w, const ColSpan* __restrict__ cols,
                                                     int ncol, double2* __restrict__ partial) {
  __shared__ double2 red[256];
  const int b = blockIdx.x, i = blockIdx.y, c = blockIdx.z;
  const ColSpan cs = cols[c];
  const int nb = dot_blocks_for(cs.len);
  double2 acc = make_double2(0.0, 0.0);
  if (b < nb) {
    const double2* v = V + i * ldv_vec + cs.off;
    const double2* ww = w + cs.off;
    const int64_t chunk = (cs.len + nb - 1) / nb;
    const int64_t g0 = b * chunk, g1 = min(cs.len, g0 + chunk);
    for (int64_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) cfma(acc, cconj(v[g]), ww[g]);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[((int64_t)b * gridDim.y + i) * ncol + c] = red[0];
}

__global__ void k_dot_final(const double2* __restrict__ partial, int nblk, int nvec, int ncol, double2* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nvec * ncol) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) acc = cadd(acc, partial[(int64_t)b * nvec * ncol + t]);
  out[t] = acc;
}

void launch_multidot(const double2* V, int64_t ldv_vec, int nvec, const double2* w, const ColSpan* cols, int ncol,
                     int64_t maxlen, double2* partial, double2* out, cudaStream_t st) {
  const int nblk = dot_blocks_for(maxlen);
  dim3 grid(nblk, nvec, ncol);
  k_dot_partial<<<grid, 256, 0, st>>>(V, ldv_vec, w, cols, ncol, partial);
  const int t = nvec * ncol;
  k_dot_final<<<(t + 127) / 128, 128, 0, st>>>(partial, nblk, nvec, ncol, out);
}

static unsigned elementwise_blocks(int64_t maxlen) {
  int64_t blocks = (maxlen + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  return (unsigned)(blocks < 1 ? 1 : blocks);
}

// w[c] += sign * sum_i h[i * ncol + c] * V_i[c]
__global__ void k_multiaxpy(const double2* __restrict__ V, int64_t ldv_vec, int nvec, const double2* __restrict__ h,
                            double2* __restrict__ w, const ColSpan* __restrict__ cols, int ncol, double sign) {
  const int c = blockIdx.y;
  const ColSpan cs = cols[c];
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < cs.len; g += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < nvec; ++i) cfma(acc, h[i * ncol + c], V[i * ldv_vec + cs.off + g]);
    double2* p = w + cs.off + g;
    *p = make_double2(p->x + sign * acc.x, p->y + sign * acc.y);
  }
}

void launch_multiaxpy(const double2* V, int64_t ldv_vec, int nvec, const double2* h, double2* w, const ColSpan* cols,
                      int ncol, int64_t maxlen, double sign, cudaStream_t st) {
  dim3 grid(elementwise_blocks(maxlen), ncol);
  k_multiaxpy<<<grid, 256, 0, st>>>(V, ldv_vec, nvec, h, w, cols, ncol, sign);
}

// y[c] = alpha_c x[c] (mode 0), y[c] = x[c] - y[c] (mode 1), y[c] += alpha_c x[c] (mode 2)
__global__ void k_axpby(const double2* __restrict__ x, double2* __restrict__ y, const ColSpan* __restrict__ cols,
                        const double2* alpha, int mode) {
  const int c = blockIdx.y;
  const ColSpan cs = cols[c];
  const double2 a = alpha ? alpha[c] : make_double2(1.0, 0.0);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < cs.len; g += (int64_t)gridDim.x * blockDim.x) {
    const double2 xv = x[cs.off + g];
    double2* p = y + cs.off + g;
    if (mode == 0) *p = cmul(a, xv);
    else if (mode == 1) *p = csub(xv, *p);
    else cfma(*p, a, xv);
  }
}

void launch_axpby_batch(const double2* x, double2* y, const ColSpan* cols, int ncol, int64_t maxlen,
                        const double2* alpha, int alpha_mode, cudaStream_t st) {
  dim3 grid(elementwise_blocks(maxlen), ncol);
  k_axpby<<<grid, 256, 0, st>>>(x, y, cols, alpha, alpha_mode);
}

// ---- Hessenberg least squares (one thread per right-hand side) ----
// column j of H is h1 + h2 (two Gram-Schmidt passes); nrm = ||w||^2 (stored in .x)
__global__ void k_arnoldi_step(LsqState L, int j, const double2* __restrict__ h1, const double2* __restrict__ h2,
                               const double2* __restrict__ nrm2) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= L.nrhs) return;
  const int k = L.k, ldh = k + 1;
  double2* H = L.H + (int64_t)r * ldh * k + (int64_t)j * ldh;
  double* cs = L.cs + (int64_t)r * k;
  double2* sn = L.sn + (int64_t)r * k;
  double2* g = L.g + (int64_t)r * (k + 1);
  if (!L.active[r]) {
    L.scl[r] = make_double2(0.0, 0.0);
    return;
  }
  for (int i = 0; i <= j; ++i) H[i] = cadd(h1[i * L.nrhs + r], h2[i * L.nrhs + r]);
  const double hn = sqrt(fmax(nrm2[r].x, 0.0));
  H[j + 1] = make_double2(hn, 0.0);
  L.scl[r] = make_double2(hn > 0.0 ? 1.0 / hn : 0.0, 0.0);
  for (int i = 0; i < j; ++i) {  // earlier rotations
    const double2 t = cadd(cscale(H[i], cs[i]), cmul(sn[i], H[i + 1]));
    H[i + 1] = csub(cscale(H[i + 1], cs[i]), cmul(cconj(sn[i]), H[i]));
    H[i] = t;
  }
  // new rotation zeroing H[j+1]: c = |a| / rho, s = (a / |a|) conj(b) / rho
  const double2 a = H[j], b = H[j + 1];
  const double aa = sqrt(cabs2(a)), bb = sqrt(cabs2(b));
  double c;
  double2 s;
  if (bb == 0.0) {
    c = 1.0;
    s = make_double2(0.0, 0.0);
  } else if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
  } else {
    const double rho = hypot(aa, bb);
    c = aa / rho;
    s = cscale(cmul(cscale(a, 1.0 / aa), cconj(b)), 1.0 / rho);
  }
  cs[j] = c;
  sn[j] = s;
  H[j] = cadd(cscale(a, c), cmul(s, b));
  H[j + 1] = make_double2(0.0, 0.0);
  g[j + 1] = cneg(cmul(cconj(s), g[j]));
  g[j] = cscale(g[j], c);
  L.resid[r] = sqrt(cabs2(g[j + 1]));
}

// y_r = R^{-1} g over the first jr[r] columns (back substitution); zeros beyond
__global__ void k_backsolve(LsqState L, const int* __restrict__ jr, double2* __restrict__ y) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= L.nrhs) return;
  const int k = L.k, ldh = k + 1, n = jr[r];
  const double2* H = L.H + (int64_t)r * ldh * k;
  const double2* g = L.g + (int64_t)r * (k + 1);
  for (int i = k - 1; i >= n; --i) y[i * L.nrhs + r] = make_double2(0.0, 0.0);
  for (int i = n - 1; i >= 0; --i) {
    double2 v = g[i];
    for (int c = i + 1; c < n; ++c) v = csub(v, cmul(H[(int64_t)c * ldh + i], y[c * L.nrhs + r]));
    y[i * L.nrhs + r] = cdiv(v, H[(int64_t)i * ldh + i]);
  }
}

// start of a cycle: beta = ||r||, V_0 = r / beta, g = (beta, 0, ...)
__global__ void k_cycle_start(LsqState L, const double2* __restrict__ nrm2) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= L.nrhs) return;
  const double beta = sqrt(fmax(nrm2[r].x, 0.0));
  double2* g = L.g + (int64_t)r * (L.k + 1);
  for (int i = 0; i <= L.k; ++i) g[i] = make_double2(0.0, 0.0);
  g[0] = make_double2(beta, 0.0);
  L.scl[r] = make_double2((L.active[r] && beta > 0.0) ? 1.0 / beta : 0.0, 0.0);
}

void launch_arnoldi_step(const LsqState& L, int j, const double2* h1, const double2* h2, const double2* nrm2,
                         cudaStream_t st) {
  k_arnoldi_step<<<(L.nrhs + 63) / 64, 64, 0, st>>>(L, j, h1, h2, nrm2);
}
void launch_backsolve(const LsqState& L, const int* jr, double2* y, cudaStream_t st) {
  k_backsolve<<<(L.nrhs + 63) / 64, 64, 0, st>>>(L, jr, y);
}
void launch_cycle_start(const LsqState& L, const double2* nrm2, cudaStream_t st) {
  k_cycle_start<<<(L.nrhs + 63) / 64, 64, 0, st>>>(L, nrm2);
}

}  // namespace psp

// C ABI and host orchestration of the sweeping preconditioner: panel plan and PML tables
// (§1.1), batched multifrontal setup of every panel (Alg. 1.4, §2.1-§2.2), the sweep (Alg. 1.5)
// and GMRES(k) (§2.4).  All arithmetic of the path runs in the kernels of this library; the host
// only plans (symbolic analysis, memory layout, task lists) and sequences launches.
#include <algorithm>
#include <climits>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <new>
#include <stdexcept>
#include <thread>
#include <tuple>
#include <type_traits>
#include <string>
#include <vector>

#include "cplx.cuh"
#include "psp_internal.h"

namespace psp {

static thread_local std::string g_last_error;

struct Error {
  psp_status st;
  std::string msg;
};

#define PSP_CK(call)                                                                                       \
  do {                                                                                                     \
    cudaError_t e_ = (call);                                                                               \
    if (e_ != cudaSuccess)                                                                                 \
      throw Error{e_ == cudaErrorMemoryAllocation ? PSP_ERR_OOM : PSP_ERR_CUDA,                          \
                  std::string(#call) + ": " + cudaGetErrorString(e_) + " (line " + std::to_string(__LINE__) + ")"}; \
  } while (0)

// Device allocator of a handle: the caller's callbacks (psp_options.dev_alloc / dev_free) or, when
// they are not given, cudaMalloc / cudaFree.
struct Allocator {
  void* (*alloc)(size_t, void*) = nullptr;
  void (*free)(void*, void*) = nullptr;
  void* ctx = nullptr;
};
// The allocator of the handle whose entry point is running on this thread (set by AllocScope).
static thread_local const Allocator* g_alloc = nullptr;
struct AllocScope {
  const Allocator* prev;
  explicit AllocScope(const Allocator* a) : prev(g_alloc) { g_alloc = a; }
  ~AllocScope() { g_alloc = prev; }
};

static void* dev_alloc(size_t b, const Allocator* A) {
  void* p = nullptr;
  if (A && A->alloc) {
    p = A->alloc(b, A->ctx);
    if (!p) throw Error{PSP_ERR_OOM, "the caller's dev_alloc returned NULL for " + std::to_string(b) + " bytes"};
  } else {
    PSP_CK(cudaMalloc(&p, b));
  }
  return p;
}
static void dev_free(void* p, const Allocator* A) {
  if (!p) return;
  if (A && A->free) {
    cudaDeviceSynchronize();   // the caller's allocator need not be stream-ordered: no work may still use p
    A->free(p, A->ctx);
  } else {
    cudaFree(p);
  }
}

// Owning device allocation; freed with the allocator it was made with.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  const Allocator* A = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes), A(o.A) { o.p = nullptr; o.bytes = 0; }
  ~DevBuf() { release(); }
  void release() {
    dev_free(p, A);
    p = nullptr;
    bytes = 0;
  }
  void alloc(size_t b) {
    release();
    if (b == 0) b = 16;
    A = g_alloc;
    p = dev_alloc(b, A);
    bytes = b;
  }
  void ensure(size_t b) {
    if (b > bytes) alloc(b);
  }
  template <typename U> U* as() const { return static_cast<U*>(p); }
};

template <typename U>
static void upload(DevBuf& d, const std::vector<U>& h) {
  d.alloc(std::max<size_t>(h.size() * sizeof(U), 16));
  if (!h.empty()) PSP_CK(cudaMemcpy(d.p, h.data(), h.size() * sizeof(U), cudaMemcpyHostToDevice));
}
// Stream-ordered upload: the copy from pageable memory is staged before the call returns, and it
// does not wait for work already queued on the stream.
// A stream for host-to-device uploads of tables built on the host: a copy from pageable memory may
// wait for the work already on the stream it is issued on, so uploads issued on the compute stream
// would hold the host until the device caught up; join() makes the compute stream wait for them.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t e = nullptr;
  SideStream() {
    PSP_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    PSP_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  SideStream(const SideStream&) = delete;
  SideStream& operator=(const SideStream&) = delete;
  ~SideStream() {
    if (e) cudaEventDestroy(e);
    if (s) cudaStreamDestroy(s);
  }
  void join(cudaStream_t st) {
    PSP_CK(cudaEventRecord(e, s));
    PSP_CK(cudaStreamWaitEvent(st, e, 0));
  }
};

template <typename U>
static void upload_async(DevBuf& d, const std::vector<U>& h, cudaStream_t st) {
  d.alloc(std::max<size_t>(h.size() * sizeof(U), 16));
  if (!h.empty()) PSP_CK(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(U), cudaMemcpyHostToDevice, st));
}

// true for device (or managed) memory, false for host memory; device memory of a device other than
// the current one is an argument error
static bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeDevice) {
    int cur = -1;
    PSP_CK(cudaGetDevice(&cur));
    if (a.device != cur)
      throw Error{PSP_ERR_ARG, "a pointer is memory of device " + std::to_string(a.device) + ", not of the current device " +
                                   std::to_string(cur)};
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// PML tables.  sigma(xi) = C/(g h) * t^2 with t = max(0, ((g+1) h - dist)/(g h)) measured to each
// PML-carrying wall; stretch s = 1 + i sigma/omega (real omega).  Half-point k sits at xi = k - 1/2;
// the tables keep 1/s there.
// ---------------------------------------------------------------------------
static double sigma_side(double dist, int gam, double C, double h) {
  if (gam <= 0) return 0.0;
  double t = ((gam + 1) * h - dist) / (gam * h);
  if (t <= 0.0) return 0.0;
  return C / (gam * h) * t * t;
}
static double sigma_axis(double xi, int n, int gam, double C, double h, bool lo, bool hi) {
  double s = 0.0;
  if (lo) s += sigma_side((xi + 1.0) * h, gam, C, h);
  if (hi) s += sigma_side((n - xi) * h, gam, C, h);
  return s;
}
static double2 stretch(double sig, double omega) { return make_double2(1.0, sig / omega); }
static double2 inv_stretch(double sig, double omega) { return cinv(stretch(sig, omega)); }

// Per-kernel accounting: launch counts and algorithmic work always, CUDA-event timing on request.
struct KStat {
  int64_t launches = 0;
  double flops = 0, bytes = 0, ms = 0;
  double extra = 0;   // executed flops beyond the algorithmic count (selective inversion)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};
struct Stats {
  bool timing = false;  // master switch (off inside the allocation-free apply)
  int mode = 0;         // 0 none, 1 every kernel, 2 setup kernels only
  std::map<std::string, KStat> k;
  std::vector<cudaEvent_t> pool;
  int64_t npending = 0;
  cudaEvent_t get() {
    if (pool.empty()) {
      cudaEvent_t e;
      PSP_CK(cudaEventCreate(&e));
      return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  template <class F>
  void run(const char* name, cudaStream_t st, int nlaunch, double flops, double bytes, F&& launch, bool setup = false,
           double extra = 0) {
    KStat& s = k[name];
    s.launches += nlaunch;
    s.flops += flops;
    s.bytes += bytes;
    s.extra += extra;
    if (!timing || mode == 0 || (mode == 2 && !setup)) {
      launch();
      return;
    }
    cudaEvent_t e0 = get(), e1 = get();
    PSP_CK(cudaEventRecord(e0, st));
    launch();
    PSP_CK(cudaEventRecord(e1, st));
    s.pending.push_back({e0, e1});
    if (++npending > 16384) collect(8192);
  }
  // resolve the oldest pending pairs (all when keep == 0)
  void collect(int64_t keep_at_most = 0) {
    for (auto& kv : k) {
      auto& v = kv.second.pending;
      size_t n = v.size();
      if (keep_at_most > 0) n = n > (size_t)keep_at_most / 2 ? n - keep_at_most / 2 : 0;
      for (size_t i = 0; i < n; ++i) {
        float ms = 0.f;
        PSP_CK(cudaEventSynchronize(v[i].second));
        PSP_CK(cudaEventElapsedTime(&ms, v[i].first, v[i].second));
        kv.second.ms += ms;
        pool.push_back(v[i].first);
        pool.push_back(v[i].second);
      }
      v.erase(v.begin(), v.begin() + n);
      npending -= (int64_t)n;
    }
    if (npending < 0) npending = 0;
  }
  // host-side phase of setup/solve (wall time, recorded as "host:<phase>")
  void host(const std::string& phase, double ms) {
    KStat& s = k["host:" + phase];
    s.ms += ms;
  }
  ~Stats() {
    for (auto& kv : k)
      for (auto& pr : kv.second.pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
      }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

}  // namespace psp

using namespace psp;

struct psp_ctx_s {
  Allocator allocator;   // first member: destroyed after every buffer made with it
  // problem
  int nx = 0, ny = 0, nz = 0;
  int64_t N = 0;
  double h = 0, omega = 0, alpha = 0, C = 0;
  int gamma = 0, depth = 0, pad = 0, leaf = 64, prec = 0, faces = 63, aux_mode = 0;
  // panels
  int m = 0;
  std::vector<int> z0, z1, lead, shape_of;
  std::vector<int64_t> sn_base;
  int64_t nfronts = 0;
  // panels whose auxiliary problems H_i are identical share one factorisation: owner[i] is the first
  // such panel (i itself when H_i is distinct); only owners are factored
  std::vector<int> owner;
  bool factor_every_panel = false;
  int64_t nfronts_factored = 0;
  int distinct_panels = 0;
  std::vector<Shape> shapes;
  std::vector<ShapeDev> shdev;
  std::vector<DevBuf> shape_bufs;
  DevBuf d_shapes, d_panel_shape;
  // operators
  DevBuf d_c, d_gtab, d_ptab, d_boxops;
  BoxOp opA{}, opJ{};
  const double2 *s1n = nullptr, *s2n = nullptr, *s3hi = nullptr;
  // factors
  DevBuf d_factor;
  int64_t factor_elems = 0;
  size_t elem_bytes = 16;
  std::vector<int64_t> panel_fbase;
  // solve plan
  struct LevelPlan {
    int64_t fwd_off = 0;
    int nfwd = 0, R = 64, smax = 0;
    int64_t bwd_off = 0;
    int nbwd = 0, ldmax = 0;
    // second phases of the fronts (factors that keep L_BL): up rows r >= s, down columns
    int64_t fwdB_off = 0, bwdB_off = 0;
    int nfwdB = 0, nbwdB = 0;
    double entries = 0;   // factor entries read by one direction of this level
    double vec = 0;       // vector entries gathered / written by one direction
  };
  std::vector<std::vector<LevelPlan>> splan;
  DevBuf d_stasks;
  // persistent sweep plan
  struct SweepPlan {
    DevBuf steps, queue;
    std::vector<SweepStep> hsteps;
    int nsteps = 0, nqueue = 0;
    int64_t nfront_steps = 0;                 // fronts summed over the steps
    double entries = 0, vec = 0;              // algorithmic factor entries / vector words per sweep
  };
  SweepPlan plans[3];              // 0: Alg. 1.5 over the handle's panels; 1: its forward part; 2: its backward part
  DevBuf d_sweep_panels, d_sweep_sync;
  size_t sweep_sync_words = 0;     // counters of the largest plan (one sweep runs at a time per handle)
  int sweep_smax = 0, sweep_ldmax = 0;   // the widest front's s and s + u (vector staging of the sweep)
  // block of panels [range_begin, range_end) this handle factors and sweeps (all of them unless the
  // handle is one block of a multi-GPU sweep)
  int range_begin = 0, range_count = 0, range_end = 0;
  bool partial = false;
  int64_t max_nloc = 0, max_upd = 0;
  // apply workspaces
  DevBuf ws_xf, ws_xb, ws_upd;
  int ws_nrhs = 0;
  DevBuf stage_in, stage_out;
  DevBuf d_status;
  // gmres workspace
  DevBuf gm;
  int gm_nrhs = 0, gm_k = 0;
  int zero_pivot_front = -1;
  double min_pivot_abs = INFINITY;   // smallest |d_jj| of the factorisation (pivot monitor)
  // residual history of the last solve: [kind][row][col], kind 0 Arnoldi estimates per iteration,
  // kind 1 true residuals per restart cycle
  std::vector<std::vector<double>> hist[2];
  int hist_cols = 0;
  bool has_history = false;
  int device = -1;          // CUDA device current at setup; every later call must run with it current
  bool use_tc = true;
  bool diag_fp64 = false;   // complex64: diagonal blocks factored and applied in complex128
  int tc_min_dim = 64;
  int sweep_level_tasks = 608, sweep_ctas_per_sm = 8, sweep_rhs_group = 0, solve_rhs_group = 0, sweep_min_rows = 8;
  int sweep_max_rows = 256;
  int sweep_claim_ahead = 1;   // tasks a sweep CTA holds besides the one it runs
  int gmres_basis = 0;   // 0 auto, 1 keep z_j, 2 V only
  int si_mode = 0;       // psp_si_mode: what the factor of each front keeps (selective inversion, §2.2)
  bool test_sweep_stall = false;
  bool persistent_sweep = true;
  int64_t upd_arena_elems = 0;
  int64_t temp_budget_elems = 0;   // cap on setup temporaries per level group (0: what the device has free)
  // problems: one, or the independent problems of a batch (psp_setup_batch) with their panels
  // concatenated; a batched vector holds problem q's N_q x nrhs block at off1_q * nrhs
  struct Prob {
    int64_t N = 0, off1 = 0;
    int panel0 = 0, m = 0, nz = 0;
    double h = 0;
    BoxOp opA{}, opJ{};
    const double2 *s1n = nullptr, *s2n = nullptr, *s3hi = nullptr;
  };
  std::vector<Prob> probs;
  std::vector<std::unique_ptr<psp_ctx_s>> subs;   // a batch's problems: their wave speeds and tables
  std::vector<BoxOp> h_boxops;                    // per panel, uploaded to d_boxops
  DevBuf d_sweep_probs, d_cols;
  int cols_nrhs = 0;
  Stats stats;
};

namespace psp {

static int64_t pad16(int64_t n) { return (n + 15) / 16 * 16; }

// sum_{j=0}^{n-1} clamp(a + j, 0, k)
static double sum_clamped(int64_t a, int64_t n, int64_t k) {
  if (n <= 0 || k <= 0) return 0.0;
  const int64_t j0 = std::clamp<int64_t>(1 - a, 0, n);   // first j with a + j >= 1
  const int64_t j1 = std::clamp<int64_t>(k - a, j0, n);  // first j with a + j >= k
  return (double)(j1 - j0) * a + 0.5 * ((double)j1 * (j1 - 1) - (double)j0 * (j0 - 1)) + (double)(n - j1) * k;
}

// useful complex multiply-adds of a GEMM task: written C entries times structurally non-zero k
template <typename T>
static double gemm_cmacs(const GemmTask<T>& g) {
  if (g.flags & GF_C_LOWER) {   // lower tiles carry no triangular operand
    double total = 0;
    const int64_t nn = std::min(g.n, g.m);
    total = (double)g.k * ((double)nn * g.m - 0.5 * (double)nn * (nn - 1));
    return total;
  }
  if (g.flags & GF_B_UNIT_LOWER_NT) return (double)g.m * sum_clamped((int64_t)g.ng0 - g.kg0 + 1, g.n, g.k);
  if (g.flags & GF_B_UNIT_LOWER_NN) return (double)g.m * sum_clamped((int64_t)g.kg0 + g.k - g.ng0 - (g.n - 1), g.n, g.k);
  return (double)g.m * g.n * g.k;
}

static double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// `while_device_runs` is host work done after the last launch is enqueued, before waiting for them.
template <typename T>
static void factor_all(psp_ctx_s* X, cudaStream_t st, const std::function<void()>& while_device_runs) {
  auto tp = std::chrono::steady_clock::now();
  const int nb = 32;
  const double tiny = sizeof(T) == 16 ? 1e-300 : 1e-30;
  // --- levels and memory plan ---
  // Fronts are batched by depth from the root, deepest first: level lv holds the fronts of depth
  // L - 1 - lv of every panel, so each child sits exactly one level below its parent.  The update
  // matrices made at one level are all consumed (extend-added) by the next, so two arenas used
  // alternately hold every update matrix.
  int L = 0;
  for (auto& sh : X->shapes) L = std::max(L, sh.ndepths);
  std::vector<std::vector<std::vector<int>>> depth_sns(X->shapes.size());
  for (size_t si = 0; si < X->shapes.size(); ++si) {
    const Shape& sh = X->shapes[si];
    depth_sns[si].assign(sh.ndepths, {});
    for (int sn = 0; sn < sh.nsn; ++sn) depth_sns[si][sh.depth[sn]].push_back(sn);
  }
  std::vector<int64_t> uoff(X->nfronts, -1);
  std::vector<std::vector<std::pair<int, int>>> lev_fronts(L);  // (panel, sn)
  for (int lv = 0; lv < L; ++lv)
    for (int p = 0; p < X->m; ++p) {
      if (X->owner[p] != p) continue;   // shares the factorisation of an identical panel
      const int si = X->shape_of[p];
      const int d = L - 1 - lv;
      if (d < (int)depth_sns[si].size())
        for (int sn : depth_sns[si][d]) lev_fronts[lv].push_back({p, sn});
    }
  // selective inversion (§2.2): 0 extended (G = [inv(L_TL); L_BL inv(L_TL)]), 1 the paper's
  // (G = [inv(L_TL); L_BL]), 2 none (G = [L_TL; L_BL], right-looking LDL^T over all s + u rows)
  const int si = X->si_mode;
  const bool tc_ok = std::is_same<T, float2>::value && X->use_tc && si != PSP_SI_NONE;
  auto use_tc = [&](int64_t s_, int64_t u_) { return tc_ok && s_ >= X->tc_min_dim && u_ >= X->tc_min_dim; };
  const int64_t TBLK = tc_block_bytes() / (int64_t)sizeof(T);   // packed block in T elements
  auto nrb = [](int64_t r) { return (r + 127) / 128; };
  auto nkb16 = [](int64_t k) { return (k + 15) / 16; };
  auto packed_elems = [&](int64_t s_, int64_t u_) {   // F_BL, Z D^-1, Z (u x s) and two inv(L) (s x s)
    return TBLK * (3 * nrb(u_) * nkb16(s_) + 2 * nrb(s_) * nkb16(s_));
  };
  auto front_temp = [&](int64_t s_, int64_t u_) {     // W (s x s), Z (u x s), Z D^-1 or packed operands,
    if (si == PSP_SI_NONE) return (int64_t)0;         // the second inverse under construction (s x s)
    return pad16(s_ * s_) + pad16(u_ * s_) + (si == PSP_SI_TWO ? pad16(s_ * s_) : 0) +
           (use_tc(s_, u_) ? packed_elems(s_, u_) : si == PSP_SI_EXTENDED ? pad16(u_ * s_) : 0);
  };
  int64_t arena[2] = {0, 0}, temp_level_max = 0, temp_front_max = 16;
  for (int lv = 0; lv < L; ++lv) {
    int64_t slab = 0, tsum = 0;
    for (auto [p, sn] : lev_fronts[lv]) {
      const Shape& sh = X->shapes[X->shape_of[p]];
      const int64_t s = sh.s[sn], u = sh.u[sn];
      if (u > 0) {
        uoff[X->sn_base[p] + sn] = slab;
        slab += pad16(upd_packed_elems((int)u, use_tc(s, u) ? 128 : 64));
      }
      const int64_t t = front_temp(s, u);
      tsum += t;
      temp_front_max = std::max(temp_front_max, t);
    }
    arena[lv & 1] = std::max(arena[lv & 1], slab);
    temp_level_max = std::max(temp_level_max, tsum);
  }
  X->upd_arena_elems = arena[0] + arena[1];
  X->stats.host("plan_memory", ms_since(tp));
  tp = std::chrono::steady_clock::now();
  DevBuf d_upd, d_temp;
  d_upd.alloc((size_t)std::max<int64_t>(X->upd_arena_elems, 16) * sizeof(T));
  // per-front temporaries of one group of a level; a level whose temporaries exceed what the device
  // has left is processed in several groups
  int64_t temp_budget = temp_level_max;
  {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
      const double avail = 0.8 * ((double)free_b - 2.0e9);
      const int64_t cap = (int64_t)std::max(0.0, avail / (double)sizeof(T));
      if (X->temp_budget_elems > 0) temp_budget = std::min(temp_budget, X->temp_budget_elems);
      temp_budget = std::max(temp_front_max, std::min(temp_budget, cap));
    } else {
      cudaGetLastError();
    }
  }
  d_temp.alloc((size_t)std::max<int64_t>(temp_budget, 16) * sizeof(T));
  X->stats.host("alloc_work", ms_since(tp));
  tp = std::chrono::steady_clock::now();
  std::vector<std::vector<std::pair<int, int>>> groups;   // (panel, sn) lists, in level order
  for (int lv = 0; lv < L; ++lv) {
    int64_t run = 0;
    bool fresh = true;   // every level starts a new group
    for (auto [p, sn] : lev_fronts[lv]) {
      const Shape& sh = X->shapes[X->shape_of[p]];
      const int64_t t = front_temp(sh.s[sn], sh.u[sn]);
      if (fresh || run + t > temp_budget) {
        groups.emplace_back();
        run = 0;
        fresh = false;
      }
      groups.back().push_back({p, sn});
      run += t;
    }
  }
  // odd levels use the second arena
  for (int lv = 1; lv < L; lv += 2)
    for (auto [p, sn] : lev_fronts[lv]) {
      int64_t& o = uoff[X->sn_base[p] + sn];
      if (o >= 0) o += arena[0];
    }
  T* ubase = d_upd.as<T>();
  T* tbase = d_temp.as<T>();
  T* fbase = X->d_factor.as<T>();
  std::vector<T*> upd_ptr(X->nfronts, nullptr);
  std::vector<int32_t> upd_tile(X->nfronts, 64);   // tile size of each front's packed update matrix
  for (int64_t i = 0; i < X->nfronts; ++i)
    if (uoff[i] >= 0) upd_ptr[i] = ubase + uoff[i];
  for (int p = 0; p < X->m; ++p) {
    const Shape& sh = X->shapes[X->shape_of[p]];
    for (int sn = 0; sn < sh.nsn; ++sn)
      if (use_tc(sh.s[sn], sh.u[sn])) upd_tile[X->sn_base[p] + sn] = 128;
  }
  DevBuf d_upd_ptr, d_upd_tile;
  upload(d_upd_ptr, upd_ptr);
  upload(d_upd_tile, upd_tile);

  // --- task lists ---
  std::vector<FrontTask<T>> fronts;
  std::vector<ColTask> ctasks;
  std::vector<int> dlist;
  std::vector<GemmTask<T>> gtasks;
  std::vector<unsigned char*> packs;     // per front: base of its packed operands (tensor-core fronts)
  std::vector<TcPackTask> ptasks;
  std::vector<TcGemmTask> ttasks;
  enum Kind { ASSEMBLE, DIAG, PRIGHT, PLEFT, GEMM, COPY, TCGEMM, TCPACK, SCALE, RSOLVE };
  struct Launch {
    Kind kind;
    int64_t front_off;
    int64_t off;
    int count;
    int kb;
    double flops = 0, bytes = 0;
    double extra = 0;   // selective-inversion flops (not part of the algorithmic count)
  };
  std::vector<Launch> launches;
  const double es = sizeof(T);
  // work of the gemm tasks [g0, end): algorithmic flops, selective-inversion flops, bytes
  auto gemm_work = [&](int64_t g0, double& fl, double& ex, double& by) {
    fl = 0;
    ex = 0;
    by = 0;
    for (size_t i = g0; i < gtasks.size(); ++i) {
      (gtasks[i].flags & GF_SI ? ex : fl) += 8.0 * gemm_cmacs(gtasks[i]);
      by += es * ((double)gtasks[i].m * gtasks[i].k + (double)gtasks[i].n * gtasks[i].k + 2.0 * gtasks[i].m * gtasks[i].n);
    }
  };

  auto tiles_lower = [&](T* C, int ldc, int M, auto&& emit) {
    for (int tj = 0; tj < M; tj += 64)
      for (int ti = tj; ti < M; ti += 64) emit(C, ldc, ti, tj, std::min(64, M - ti), std::min(64, M - tj));
  };

  // Each group's tasks are uploaded and its launches enqueued as soon as the group is planned, so
  // the host plans the next group while the device factors this one.  Task arrays go to
  // stream-ordered device chunks, one per group and array, freed after the final synchronisation.
  int* status = X->d_status.as<int>();
  // status: [0] 1 + front of a zero pivot, [1] tensor-core wait gave up, [2] sweep wait gave up (sticky),
  // [4..5] ~bits of the smallest |pivot| (0: none yet)
  PSP_CK(cudaMemsetAsync(status, 0, 8 * sizeof(int), st));
  static const char* names[] = {"k_assemble", "k_diag_ldlt", "k_panel_right", "k_panel_left", "k_gemm", "k_copy_linv",
                                "k_tc_gemm", "k_tc_pack", "k_scale_zd", "k_panel_rsolve"};
  // task arrays go up on a side stream, so that the next group's planning overlaps the device's work
  SideStream up;
  std::vector<void*> chunks;
  const Allocator* chunk_alloc = g_alloc && g_alloc->alloc ? g_alloc : nullptr;
  struct ChunkGuard {
    std::vector<void*>& c;
    cudaStream_t s;
    cudaStream_t up;
    const Allocator* A;
    ~ChunkGuard() {
      // copies still in flight on the side stream (an error between an upload and its join) end
      // before their chunks are released
      if (!c.empty()) cudaStreamSynchronize(up);
      if (A && !c.empty()) cudaStreamSynchronize(s);   // the caller's free is not stream-ordered
      for (void* p : c) {
        if (A) dev_free(p, A);
        else cudaFreeAsync(p, s);
      }
    }
  } chunk_guard{chunks, st, up.s, chunk_alloc};
  // copies v[done, size) to a new device chunk (the copy from pageable memory is staged before the
  // call returns, so the vector may grow afterwards); returns the chunk and advances done
  auto upload_tail = [&](const auto& v, size_t& done) {
    using E = typename std::decay_t<decltype(v)>::value_type;
    const size_t n = v.size() - done;
    E* d = nullptr;
    if (n > 0) {
      if (chunk_alloc) d = static_cast<E*>(dev_alloc(n * sizeof(E), chunk_alloc));
      else PSP_CK(cudaMallocAsync(reinterpret_cast<void**>(&d), n * sizeof(E), up.s));
      chunks.push_back(d);
      PSP_CK(cudaMemcpyAsync(d, v.data() + done, n * sizeof(E), cudaMemcpyHostToDevice, up.s));
    }
    return d;
  };
  size_t up_f = 0, up_c = 0, up_d = 0, up_g = 0, up_p = 0, up_t = 0;
  double plan_ms = 0, enqueue_ms = 0;
  auto enqueue_group = [&](size_t lb) {
    const size_t f0 = up_f, c0 = up_c, d0 = up_d, g0 = up_g, p0 = up_p, t0 = up_t;
    const FrontTask<T>* F = upload_tail(fronts, up_f);
    const ColTask* CT = upload_tail(ctasks, up_c);
    const int* DL = upload_tail(dlist, up_d);
    const GemmTask<T>* GT = upload_tail(gtasks, up_g);
    const TcPackTask* PT = upload_tail(ptasks, up_p);
    const TcGemmTask* TT = upload_tail(ttasks, up_t);
    up.join(st);   // the group's kernels after its task arrays
    up_f = fronts.size();
    up_c = ctasks.size();
    up_d = dlist.size();
    up_g = gtasks.size();
    up_p = ptasks.size();
    up_t = ttasks.size();
    for (size_t li = lb; li < launches.size(); ++li) {
      const Launch& l = launches[li];
      if (l.count <= 0) continue;
      const bool wide = X->prec == PSP_PREC_C64 && X->diag_fp64;
      const FrontTask<T>* Fl = F + (l.front_off - (int64_t)f0);
      X->stats.run(names[l.kind], st, 1, l.flops, l.bytes, [&] {
        switch (l.kind) {
          case ASSEMBLE:
            launch_assemble_impl<T>(Fl, CT + (l.off - (int64_t)c0), l.count, X->d_shapes.as<ShapeDev>(),
                                    X->d_boxops.as<BoxOp>(), d_upd_ptr.as<T*>(), d_upd_tile.as<int32_t>(),
                                    X->d_panel_shape.as<int32_t>(), st);
            break;
          case DIAG: launch_diag_ldlt<T>(Fl, DL + (l.off - (int64_t)d0), l.count, l.kb, tiny, status, wide, st); break;
          case PRIGHT: launch_panel_right<T>(Fl, CT + (l.off - (int64_t)c0), l.count, l.kb, wide, st); break;
          case PLEFT: launch_panel_left<T>(Fl, CT + (l.off - (int64_t)c0), l.count, l.kb, wide, st); break;
          case GEMM: launch_gemm<T>(GT + (l.off - (int64_t)g0), l.count, st); break;
          case COPY: launch_copy_linv<T>(Fl, CT + (l.off - (int64_t)c0), l.count, st); break;
          case TCGEMM: launch_tc_gemm(TT + (l.off - (int64_t)t0), l.count, status, st); break;
          case TCPACK: launch_tc_pack(PT + (l.off - (int64_t)p0), l.count, st); break;
          case SCALE: launch_scale_zd<T>(Fl, CT + (l.off - (int64_t)c0), l.count, st); break;
          case RSOLVE: launch_panel_rsolve<T>(Fl, CT + (l.off - (int64_t)c0), l.count, l.kb, wide, st); break;
        }
      }, true, l.extra);
    }
    PSP_CK(cudaGetLastError());
  };

  for (const auto& grp : groups) {
    const size_t lb = launches.size();
    const int64_t f0 = (int64_t)fronts.size();
    int smax = 0;
    int64_t toff = 0;
    for (auto [p, sn] : grp) {
      const Shape& sh = X->shapes[X->shape_of[p]];
      FrontTask<T> ft{};
      ft.s = sh.s[sn];
      ft.u = sh.u[sn];
      ft.panel = p;
      ft.sn = sn;
      ft.gfid = X->sn_base[p] + sn;
      ft.G = fbase + X->panel_fbase[p] + sh.g_off[sn];
      ft.U = upd_ptr[ft.gfid];
      ft.ut = upd_tile[ft.gfid];
      ft.W = ft.Z = ft.ZD = ft.W2 = nullptr;
      ft.ldzd = ft.u;
      packs.push_back(nullptr);
      if (si != PSP_SI_NONE) {
        ft.W = tbase + toff;
        toff += pad16((int64_t)ft.s * ft.s);
        ft.Z = tbase + toff;
        toff += pad16((int64_t)ft.u * ft.s);
        if (use_tc(ft.s, ft.u)) {
          packs.back() = reinterpret_cast<unsigned char*>(tbase + toff);
          toff += packed_elems(ft.s, ft.u);
        } else if (si == PSP_SI_EXTENDED) {
          ft.ZD = tbase + toff;
          toff += pad16((int64_t)ft.u * ft.s);
        }
        if (si == PSP_SI_PAPER || si == PSP_SI_TWO) {   // L_BL = Z D^{-1} is the factor's bottom block
          ft.ZD = ft.G + ft.s;
          ft.ldzd = ft.s + ft.u;
        }
        if (si == PSP_SI_TWO) {
          ft.W2 = tbase + toff;
          toff += pad16((int64_t)ft.s * ft.s);
        }
      }
      fronts.push_back(ft);
      smax = std::max(smax, ft.s);
    }
    const int nf = (int)(fronts.size() - f0);
    // GEMM tiles are emitted largest front first: a launch's tiles start in order, one CTA per SM,
    // so the long tiles start early and the short ones fill the tail
    std::vector<int> ord(nf);
    for (int f = 0; f < nf; ++f) ord[f] = f;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
      const auto& a = fronts[f0 + x];
      const auto& b = fronts[f0 + y];
      return (double)a.s * (a.s + a.u) * (a.s + a.u) > (double)b.s * (b.s + b.u) * (b.s + b.u);
    });
    // assembly: column chunks of 32 over the full front width
    {
      const int64_t c0 = (int64_t)ctasks.size();
      for (int f = 0; f < nf; ++f) {
        const auto& ft = fronts[f0 + f];
        for (int c = 0; c < ft.s + ft.u; c += 32) ctasks.push_back({f, c, std::min(c + 32, ft.s + ft.u)});
      }
      Launch la{ASSEMBLE, f0, c0, (int)(ctasks.size() - c0), 0};
      for (int f = 0; f < nf; ++f) {
        const auto& ft = fronts[f0 + f];
        const Shape& sh = X->shapes[X->shape_of[ft.panel]];
        double ea = 0;
        for (int c = sh.child_ptr[ft.sn]; c < sh.child_ptr[ft.sn + 1]; ++c) {
          const double uc = sh.u[sh.child_idx[c]];
          ea += uc * (uc + 1) / 2;
        }
        la.flops += 2.0 * ea;
        la.bytes += es * (2.0 * ea + (double)(ft.s + ft.u) * ft.s + (double)ft.s * ft.s + 0.5 * ft.u * (ft.u + 1.0));
      }
      launches.push_back(la);
    }
    // blocked LDL^T of F_TL with the inverse of L_TL built alongside in W; without selective
    // inversion the blocked factorisation runs over all s + u rows, so F_BL becomes L_BL directly
    const int nblk = (smax + nb - 1) / nb;
    for (int kb = 0; kb < nblk; ++kb) {
      const int o = kb * nb;
      const int64_t d0 = (int64_t)dlist.size();
      Launch ld{DIAG, f0, d0, 0, kb};
      for (int f = 0; f < nf; ++f)
        if (fronts[f0 + f].s > o) {
          dlist.push_back(f);
          const double bs = std::min(nb, fronts[f0 + f].s - o);
          ld.flops += 8.0 * bs * bs * bs / 3;
          ld.bytes += es * bs * bs;
        }
      ld.count = (int)(dlist.size() - d0);
      launches.push_back(ld);
      const int64_t pr0 = (int64_t)ctasks.size();
      for (int f = 0; f < nf; ++f) {
        const auto& ft = fronts[f0 + f];
        if (ft.s <= o) continue;
        // rows below the diagonal block: the rest of F_TL, and without inversion all of F_BL too (its
        // rows start at s, which the last block's o + nb may pass)
        const int rend = si == PSP_SI_NONE ? ft.s + ft.u : ft.s;
        for (int r = std::min(o + nb, ft.s); r < rend; r += 64) ctasks.push_back({f, r, std::min(r + 64, rend)});
      }
      Launch lr{PRIGHT, f0, pr0, (int)(ctasks.size() - pr0), kb};
      for (int64_t t = pr0; t < (int64_t)ctasks.size(); ++t) {
        const double rows = ctasks[t].c1 - ctasks[t].c0, bs = std::min(nb, fronts[f0 + ctasks[t].front].s - o);
        lr.flops += 8.0 * rows * bs * (bs + 1) / 2;
        lr.bytes += es * 2 * rows * bs;
      }
      launches.push_back(lr);
      const int64_t pl0 = (int64_t)ctasks.size();
      for (int f = 0; f < nf && si != PSP_SI_NONE; ++f) {
        const auto& ft = fronts[f0 + f];
        if (ft.s <= o) continue;
        const int cend = std::min(ft.s, o + nb);
        for (int c = 0; c < cend; c += 64) ctasks.push_back({f, c, std::min(c + 64, cend)});
      }
      Launch lp{PLEFT, f0, pl0, (int)(ctasks.size() - pl0), kb};
      for (int64_t t = pl0; t < (int64_t)ctasks.size(); ++t) {
        const double cols = ctasks[t].c1 - ctasks[t].c0, bs = std::min(nb, fronts[f0 + ctasks[t].front].s - o);
        lp.extra += 8.0 * cols * bs * (bs - 1) / 2;   // block row of inv(L): selective inversion
        lp.bytes += es * 2 * cols * bs;
      }
      launches.push_back(lp);
      const int64_t g0 = (int64_t)gtasks.size();
      for (int f : ord) {
        const auto& ft = fronts[f0 + f];
        if (ft.s <= o + nb) continue;
        const int ld = ft.s + ft.u;
        const int bs = std::min(nb, ft.s - o);
        const int t0 = o + nb;  // first row/col of the trailing block
        // F_TL trailing update: F(r, c) -= L(r, kb) D_kb L(c, kb)^T, lower
        tiles_lower(ft.G, ld, ft.s - t0, [&](T*, int, int ti, int tj, int mm, int nn) {
          GemmTask<T> g{};
          g.C = ft.G + (int64_t)(t0 + tj) * ld + (t0 + ti);
          g.ldc = ld;
          g.A = ft.G + (int64_t)o * ld + (t0 + ti);
          g.lda = ld;
          g.B = ft.G + (int64_t)o * ld + (t0 + tj);
          g.ldb = ld;
          g.d = ft.G + (int64_t)o * ld + o;
          g.ldd = ld + 1;
          g.m = mm; g.n = nn; g.k = bs;
          g.flags = GF_D_MUL | GF_NEG | (ti == tj ? GF_C_LOWER : 0);
          gtasks.push_back(g);
        });
        if (si == PSP_SI_NONE) {
          // F_BL trailing update: F_BL(r, c) -= L_BL(r, kb) D_kb L(c, kb)^T, full tiles
          for (int tj = 0; tj < ft.s - t0; tj += 64)
            for (int ti = 0; ti < ft.u; ti += 64) {
              GemmTask<T> g{};
              g.C = ft.G + (int64_t)(t0 + tj) * ld + (ft.s + ti);
              g.ldc = ld;
              g.A = ft.G + (int64_t)o * ld + (ft.s + ti);
              g.lda = ld;
              g.B = ft.G + (int64_t)o * ld + (t0 + tj);
              g.ldb = ld;
              g.d = ft.G + (int64_t)o * ld + o;
              g.ldd = ld + 1;
              g.m = std::min(64, ft.u - ti);
              g.n = std::min(64, ft.s - t0 - tj);
              g.k = bs;
              g.flags = GF_D_MUL | GF_NEG;
              gtasks.push_back(g);
            }
          continue;   // no inverse of L_TL is built
        }
        // W(r, c) -= L(r, kb) W(kb, c) for rows below the block, columns up to its end
        const int cend = o + bs;
        for (int tj = 0; tj < cend; tj += 64)
          for (int ti = t0; ti < ft.s; ti += 64) {
            GemmTask<T> g{};
            g.C = ft.W + (int64_t)tj * ft.s + ti;
            g.ldc = ft.s;
            g.A = ft.G + (int64_t)o * ld + ti;
            g.lda = ld;
            g.B = ft.W + (int64_t)tj * ft.s + o;  // B(n, k) = W[o + k, tj + n]
            g.ldb = ft.s;
            g.m = std::min(64, ft.s - ti);
            g.n = std::min(64, cend - tj);
            g.k = bs;
            g.kg0 = o;              // W is unit lower: B(n, k) = W[o + k, tj + n] vanishes for o + k < tj + n
            g.ng0 = tj;
            g.flags = GF_NEG | GF_B_NN | GF_B_UNIT_LOWER_NN | GF_SI;
            gtasks.push_back(g);
          }
      }
      Launch lg{GEMM, f0, g0, (int)(gtasks.size() - g0), kb};
      gemm_work(g0, lg.flops, lg.extra, lg.bytes);
      launches.push_back(lg);
    }
    // The two-inverse form: the second inverse X of L_TL row by row, X L_TL = I, by block columns from
    // the last: X(:, kb) := X(:, kb) L_kk^{-1}, then X(:, j) -= X(:, kb) L(kb, j) for the blocks j < kb
    // (X is unit lower: only rows from the block's first row down take part).
    if (si == PSP_SI_TWO) {
      for (int kb = nblk - 1; kb >= 0; --kb) {
        const int o = kb * nb;
        const int64_t r0 = (int64_t)ctasks.size();
        for (int f = 0; f < nf; ++f) {
          const auto& ft = fronts[f0 + f];
          if (ft.s <= o) continue;
          for (int r = o; r < ft.s; r += 64) ctasks.push_back({f, r, std::min(r + 64, ft.s)});
        }
        Launch lr{RSOLVE, f0, r0, (int)(ctasks.size() - r0), kb};
        for (int64_t q = r0; q < (int64_t)ctasks.size(); ++q) {
          const double rows = ctasks[q].c1 - ctasks[q].c0, bs = std::min(nb, fronts[f0 + ctasks[q].front].s - o);
          lr.extra += 8.0 * rows * bs * (bs - 1) / 2;
          lr.bytes += es * 2 * rows * bs;
        }
        launches.push_back(lr);
        if (kb == 0) break;
        const int64_t g0 = (int64_t)gtasks.size();
        for (int f : ord) {
          const auto& ft = fronts[f0 + f];
          if (ft.s <= o) continue;
          const int ld = ft.s + ft.u;
          const int bs = std::min(nb, ft.s - o);
          for (int tj = 0; tj < o; tj += 64)
            for (int ti = o; ti < ft.s; ti += 64) {
              GemmTask<T> g{};
              g.C = ft.W2 + (int64_t)tj * ft.s + ti;
              g.ldc = ft.s;
              g.A = ft.W2 + (int64_t)o * ft.s + ti;   // A(m, k) = X[ti + m, o + k]
              g.lda = ft.s;
              g.B = ft.G + (int64_t)tj * ld + o;      // B(n, k) = L[o + k, tj + n]
              g.ldb = ld;
              g.m = std::min(64, ft.s - ti);
              g.n = std::min(64, o - tj);
              g.k = bs;
              g.flags = GF_NEG | GF_B_NN | GF_SI;
              gtasks.push_back(g);
            }
        }
        Launch lg{GEMM, f0, g0, (int)(gtasks.size() - g0), kb};
        gemm_work(g0, lg.flops, lg.extra, lg.bytes);
        launches.push_back(lg);
      }
    }
    // inv(L_TL) into F_TL's strict lower part (and the second inverse after G)
    if (si != PSP_SI_NONE) {
      const int64_t c0 = (int64_t)ctasks.size();
      for (int f = 0; f < nf; ++f) {
        const auto& ft = fronts[f0 + f];
        for (int c = 0; c < ft.s; c += 16) ctasks.push_back({f, c, std::min(c + 16, ft.s)});
      }
      Launch lc{COPY, f0, c0, (int)(ctasks.size() - c0), 0};
      for (int f = 0; f < nf; ++f) lc.bytes += es * (double)fronts[f0 + f].s * (fronts[f0 + f].s - 1);
      launches.push_back(lc);
    }
    // Z = F_BL inv(L_TL)^T (= F_BL L^{-T}), then F_BR -= Z D^{-1} Z^T (lower) and M_BL = Z D^{-1} inv(L_TL).
    // Fronts with s, u >= 96 (complex64) run them on tcgen05 tiles of 128 x 128 from packed operands;
    // the others on 64 x 64 CUDA-core tiles.
    auto emit_z = [&](const FrontTask<T>& ft) {
      const int ld = ft.s + ft.u;
      for (int tj = 0; tj < ft.s; tj += 64)
        for (int ti = 0; ti < ft.u; ti += 64) {
          GemmTask<T> g{};
          const int j1 = std::min(tj + 64, ft.s);
          g.C = ft.Z + (int64_t)tj * ft.u + ti;
          g.ldc = ft.u;
          g.A = ft.G + ft.s + ti;  // F_BL rows, k from 0
          g.lda = ld;
          g.B = ft.G + tj;         // B(n, k) = Linv[tj + n, k]
          g.ldb = ld;
          g.m = std::min(64, ft.u - ti);
          g.n = j1 - tj;
          g.k = j1;
          g.kg0 = 0;
          g.ng0 = tj;
          g.flags = GF_BETA0 | GF_B_UNIT_LOWER_NT;
          gtasks.push_back(g);
        }
    };
    auto emit_schur_m = [&](const FrontTask<T>& ft) {
      const int ld = ft.s + ft.u;
      for (int tj = 0; tj < ft.u; tj += 64)
        for (int ti = tj; ti < ft.u; ti += 64) {
          GemmTask<T> g{};
          g.C = ft.U + upd_index(ti, tj, ft.u, 64);   // the packed 64 x 64 tile (ti, tj)
          g.ldc = 64;
          g.m = std::min(64, ft.u - ti);
          g.n = std::min(64, ft.u - tj);
          g.k = ft.s;
          g.flags = GF_NEG | (ti == tj ? GF_C_LOWER : 0);
          if (si == PSP_SI_NONE) {   // F_BR -= L_BL D L_BL^T
            g.A = ft.G + ft.s + ti;
            g.lda = ld;
            g.B = ft.G + ft.s + tj;
            g.ldb = ld;
            g.d = ft.G;
            g.ldd = ld + 1;
            g.flags |= GF_D_MUL;
          } else {                   // F_BR -= (Z D^{-1}) Z^T
            g.A = ft.ZD + ti;
            g.lda = ft.ldzd;
            g.B = ft.Z + tj;
            g.ldb = ft.u;
          }
          gtasks.push_back(g);
        }
      if (si != PSP_SI_EXTENDED) return;
      for (int tj = 0; tj < ft.s; tj += 64)
        for (int ti = 0; ti < ft.u; ti += 64) {
          GemmTask<T> g{};
          g.C = ft.G + (int64_t)tj * ld + ft.s + ti;
          g.ldc = ld;
          g.A = ft.ZD + (int64_t)tj * ft.u + ti;  // A(i, k) = (Z D^-1)[ti + i, tj + k]
          g.lda = ft.u;
          g.B = ft.G + (int64_t)tj * ld + tj;     // B(n, k) = Linv[tj + k, tj + n]
          g.ldb = ld;
          g.m = std::min(64, ft.u - ti);
          g.n = std::min(64, ft.s - tj);
          g.k = ft.s - tj;
          g.kg0 = tj;
          g.ng0 = tj;
          g.flags = GF_BETA0 | GF_B_NN | GF_B_UNIT_LOWER_NN | GF_SI;   // M_BL = Z D^-1 inv(L)
          gtasks.push_back(g);
        }
    };
    // packed operands of a tensor-core front: F_BL | Z D^-1 | Z (u x s each) | inv(L) | inv(L)^T (s x s)
    struct Packed { unsigned char *bl, *zd, *z, *l, *lt; int64_t ku; };
    auto packed_of = [&](int f) {
      const auto& ft = fronts[f0 + f];
      const int64_t bb = tc_block_bytes();
      const int64_t uu = nrb(ft.u) * nkb16(ft.s) * bb, ss = nrb(ft.s) * nkb16(ft.s) * bb;
      unsigned char* b = packs[f0 + f];
      return Packed{b, b + uu, b + 2 * uu, b + 3 * uu, b + 3 * uu + ss, nkb16(ft.s)};
    };
    auto pack = [&](const T* src, const T* d, unsigned char* dst, int ld_, int ldd_, int R, int K, int mode) {
      for (int rb = 0; rb < nrb(R); ++rb)
        for (int kb = 0; kb < nkb16(K); ++kb) {
          TcPackTask t{};
          t.src = reinterpret_cast<const float2*>(src);
          t.d = reinterpret_cast<const float2*>(d);
          t.dst = dst + ((int64_t)rb * nkb16(K) + kb) * tc_block_bytes();
          t.ld = ld_;
          t.ldd = ldd_;
          t.r0 = rb * 128;
          t.k0 = kb * 16;
          t.R = R;
          t.K = K;
          t.mode = mode;
          ptasks.push_back(t);
        }
    };
    auto tc_work = [&](double& fl, double& by, int64_t t0) {
      fl = 0;
      by = 0;
      for (size_t i = t0; i < ttasks.size(); ++i) by += 2.0 * ttasks[i].nkb * tc_block_bytes();
      (void)fl;
    };
    for (int phase = si == PSP_SI_NONE ? 1 : 0; phase < 2; ++phase) {
      if (phase == 1 && si != PSP_SI_NONE) {
        // Z D^{-1} once per front: of the CUDA-core fronts (extended form), or of every front into the
        // factor's bottom block (L_BL, the paper's form)
        const int64_t c0 = (int64_t)ctasks.size();
        Launch ls{SCALE, f0, c0, 0, 0};
        for (int f : ord) {
          const auto& ft = fronts[f0 + f];
          if (ft.u == 0 || (packs[f0 + f] && si == PSP_SI_EXTENDED)) continue;
          for (int c = 0; c < ft.s; c += 16) ctasks.push_back({f, c, std::min(c + 16, ft.s)});
          ls.bytes += 2.0 * es * ft.u * ft.s;
        }
        ls.count = (int)(ctasks.size() - c0);
        if (ls.count > 0) launches.push_back(ls);
      }
      // CUDA-core fronts
      {
        const int64_t g0 = (int64_t)gtasks.size();
        for (int f : ord) {
          const auto& ft = fronts[f0 + f];
          if (ft.u == 0 || packs[f0 + f]) continue;
          if (phase == 0) emit_z(ft);
          else emit_schur_m(ft);
        }
        if ((int64_t)gtasks.size() > g0) {
          Launch lg{GEMM, f0, g0, (int)(gtasks.size() - g0), -1};
          gemm_work(g0, lg.flops, lg.extra, lg.bytes);
          launches.push_back(lg);
        }
      }
      // tensor-core fronts: pack, then tiles
      const int64_t p0 = (int64_t)ptasks.size(), t0 = (int64_t)ttasks.size();
      double tflops = 0, tflops_si = 0;
      for (int f : ord) {
        const auto& ft = fronts[f0 + f];
        if (ft.u == 0 || !packs[f0 + f]) continue;
        const int ld = ft.s + ft.u;
        const Packed P = packed_of(f);
        const int64_t bb = tc_block_bytes();
        if (phase == 0) {
          pack(ft.G + ft.s, nullptr, P.bl, ld, 0, ft.u, ft.s, TC_PACK_PLAIN);
          pack(ft.G, nullptr, P.l, ld, 0, ft.s, ft.s, TC_PACK_UNIT_LOWER);
          if (si == PSP_SI_EXTENDED) pack(ft.G, nullptr, P.lt, ld, 0, ft.s, ft.s, TC_PACK_UNIT_LOWER_T);
          for (int tj = 0; tj < ft.s; tj += 128)
            for (int ti = 0; ti < ft.u; ti += 128) {
              const int j1 = std::min(tj + 128, ft.s);
              TcGemmTask t{};
              t.A = P.bl + (int64_t)(ti / 128) * P.ku * bb;
              t.B = P.l + (int64_t)(tj / 128) * P.ku * bb;
              t.C = reinterpret_cast<float2*>(ft.Z + (int64_t)tj * ft.u + ti);
              t.ldc = ft.u;
              t.m = std::min(128, ft.u - ti);
              t.n = j1 - tj;
              t.kb0 = 0;
              t.nkb = (int)nkb16(j1);
              t.flags = GF_BETA0;
              ttasks.push_back(t);
              GemmTask<T> sh{};
              sh.m = t.m; sh.n = t.n; sh.k = j1; sh.kg0 = 0; sh.ng0 = tj; sh.flags = GF_B_UNIT_LOWER_NT;
              tflops += 8.0 * gemm_cmacs(sh);
            }
        } else {
          pack(ft.Z, ft.G, P.zd, ft.u, ld + 1, ft.u, ft.s, TC_PACK_PLAIN);
          pack(ft.Z, nullptr, P.z, ft.u, 0, ft.u, ft.s, TC_PACK_PLAIN);
          for (int tj = 0; tj < ft.u; tj += 128)
            for (int ti = tj; ti < ft.u; ti += 128) {
              TcGemmTask t{};
              t.A = P.zd + (int64_t)(ti / 128) * P.ku * bb;
              t.B = P.z + (int64_t)(tj / 128) * P.ku * bb;
              t.C = reinterpret_cast<float2*>(ft.U + upd_index(ti, tj, ft.u, 128));   // packed 128 x 128 tile
              t.ldc = 128;
              t.m = std::min(128, ft.u - ti);
              t.n = std::min(128, ft.u - tj);
              t.kb0 = 0;
              t.nkb = (int)nkb16(ft.s);
              t.flags = GF_NEG | (ti == tj ? GF_C_LOWER : 0);
              ttasks.push_back(t);
              GemmTask<T> sh{};
              sh.m = t.m; sh.n = t.n; sh.k = ft.s; sh.flags = (ti == tj ? GF_C_LOWER : 0);
              tflops += 8.0 * gemm_cmacs(sh);
            }
          for (int tj = 0; tj < ft.s && si == PSP_SI_EXTENDED; tj += 128)
            for (int ti = 0; ti < ft.u; ti += 128) {
              TcGemmTask t{};
              t.A = P.zd + (int64_t)(ti / 128) * P.ku * bb;
              t.B = P.lt + (int64_t)(tj / 128) * P.ku * bb;
              t.C = reinterpret_cast<float2*>(ft.G + (int64_t)tj * ld + ft.s + ti);
              t.ldc = ld;
              t.m = std::min(128, ft.u - ti);
              t.n = std::min(128, ft.s - tj);
              t.kb0 = tj / 16;
              t.nkb = (int)(nkb16(ft.s) - tj / 16);
              t.flags = GF_BETA0;
              ttasks.push_back(t);
              GemmTask<T> sh{};
              sh.m = t.m; sh.n = t.n; sh.k = ft.s - tj; sh.kg0 = tj; sh.ng0 = tj; sh.flags = GF_B_UNIT_LOWER_NN;
              tflops_si += 8.0 * gemm_cmacs(sh);   // M_BL: selective inversion
            }
        }
      }
      if ((int64_t)ptasks.size() > p0) {
        Launch lp{TCPACK, f0, p0, (int)(ptasks.size() - p0), -1};
        lp.bytes = (double)(ptasks.size() - p0) * (tc_block_bytes() + 128.0 * 16 * sizeof(T));
        launches.push_back(lp);
        Launch lt{TCGEMM, f0, t0, (int)(ttasks.size() - t0), -1};
        double fl_unused = 0;
        tc_work(fl_unused, lt.bytes, t0);
        lt.flops = tflops;
        lt.extra = tflops_si;
        launches.push_back(lt);
      }
    }
    plan_ms += ms_since(tp);
    tp = std::chrono::steady_clock::now();
    enqueue_group(lb);
    enqueue_ms += ms_since(tp);
    tp = std::chrono::steady_clock::now();
  }

  X->stats.host("plan_tasks", plan_ms);
  X->stats.host("enqueue_setup", enqueue_ms);
  while_device_runs();
  tp = std::chrono::steady_clock::now();
  PSP_CK(cudaStreamSynchronize(st));
  X->stats.host("wait_setup", ms_since(tp));
  int hs[8];
  PSP_CK(cudaMemcpy(hs, status, sizeof(hs), cudaMemcpyDeviceToHost));
  {
    unsigned long long nb;
    std::memcpy(&nb, hs + 4, sizeof(nb));
    const unsigned long long bits = ~nb;
    double mp;
    std::memcpy(&mp, &bits, sizeof(mp));
    X->min_pivot_abs = nb == 0 ? INFINITY : mp;
  }
  if (hs[1] != 0) throw Error{PSP_ERR_TIMEOUT, "a tensor-core GEMM gave up waiting for its MMAs"};
  if (hs[0] != 0) {
    X->zero_pivot_front = hs[0] - 1;
    throw Error{PSP_ERR_ZERO_PIVOT, "zero pivot in front " + std::to_string(hs[0] - 1)};
  }
}

// ---------------------------------------------------------------------------
// Solve plan: per shape and level, forward row tasks and backward column tasks.
// ---------------------------------------------------------------------------
static void plan_solve(psp_ctx_s* X, cudaStream_t st) {
  SideStream side;   // the tables go up while the device still factors
  std::vector<SolveTask> tasks;
  X->splan.assign(X->shapes.size(), {});
  for (size_t si = 0; si < X->shapes.size(); ++si) {
    const Shape& sh = X->shapes[si];
    X->splan[si].resize(sh.nlevels);
    for (int lv = 0; lv < sh.nlevels; ++lv) {
      auto& P = X->splan[si][lv];
      int64_t rows = 0, cols = 0;
      for (int sn : sh.level_sns[lv]) {
        rows += sh.s[sn] + sh.u[sn];
        cols += sh.s[sn];
        P.smax = std::max(P.smax, (int)sh.s[sn]);
        P.ldmax = std::max(P.ldmax, (int)(sh.s[sn] + sh.u[sn]));
      }
      for (int sn : sh.level_sns[lv]) {
        const double ss = sh.s[sn], uu = sh.u[sn];
        P.entries += ss * (ss - 1) / 2 + uu * ss;
        P.vec += 2 * ss + 2 * uu;
      }
      // rows per up task and columns per down task: sweep_max_rows (64 .. 256), halved while the
      // level has fewer than sweep_level_tasks tasks, but not below sweep_min_rows (a task gathers
      // its front's vector for every right-hand side, so narrow tasks over wide fronts gather much and
      // stream little, and at the bottom of the tree, where tasks far outnumber CTAs, one task per
      // front gathers once)
      const int rmin = std::max(8, std::min(64, X->sweep_min_rows));
      int R = X->sweep_max_rows;
      while (R > rmin && rows / R < X->sweep_level_tasks) R >>= 1;
      P.R = R;
      int Cc = X->sweep_max_rows;
      while (Cc > rmin && cols / Cc < X->sweep_level_tasks) Cc >>= 1;
      // extended factors: one pass per front and direction over all s + u rows; factors keeping L_BL:
      // up, rows r < s (one whole-front substitution task without inversion) then rows r >= s; down,
      // columns for L_BL^T then columns for the triangle (one whole-front task without inversion)
      const bool two = X->si_mode != PSP_SI_EXTENDED, tri = X->si_mode == PSP_SI_NONE;
      auto rows_of = [&](int sn, int a, int b, int step) {
        for (int r = a; r < b; r += step) tasks.push_back({sn, r, std::min(r + step, b)});
      };
      P.fwd_off = (int64_t)tasks.size();
      for (int sn : sh.level_sns[lv]) {
        const int s_ = sh.s[sn], ld_ = s_ + sh.u[sn];
        if (!two) rows_of(sn, 0, ld_, R);
        else if (tri) tasks.push_back({sn, 0, s_});
        else rows_of(sn, 0, s_, R);
      }
      P.nfwd = (int)(tasks.size() - P.fwd_off);
      P.fwdB_off = (int64_t)tasks.size();
      if (two)
        for (int sn : sh.level_sns[lv]) rows_of(sn, sh.s[sn], sh.s[sn] + sh.u[sn], R);
      P.nfwdB = (int)(tasks.size() - P.fwdB_off);
      P.bwd_off = (int64_t)tasks.size();
      for (int sn : sh.level_sns[lv]) rows_of(sn, 0, sh.s[sn], Cc);
      P.nbwd = (int)(tasks.size() - P.bwd_off);
      P.bwdB_off = (int64_t)tasks.size();
      if (two)
        for (int sn : sh.level_sns[lv]) {
          if (tri) tasks.push_back({sn, 0, (int)sh.s[sn]});
          else rows_of(sn, 0, sh.s[sn], Cc);
        }
      P.nbwdB = (int)(tasks.size() - P.bwdB_off);
    }
  }
  upload_async(X->d_stasks, tasks, side.s);

  // per shape: tasks per front, up and down
  std::vector<int> front_base(X->shapes.size() + 1, 0), ntask_up, ntask_down, ntask_upA, ntask_downA;
  std::vector<double> shape_entries(X->shapes.size(), 0.0), shape_vec(X->shapes.size(), 0.0);
  std::vector<int> shape_tasks(X->shapes.size(), 0);
  for (size_t si = 0; si < X->shapes.size(); ++si) {
    const Shape& sh = X->shapes[si];
    front_base[si] = (int)ntask_up.size();
    ntask_up.resize(ntask_up.size() + sh.nsn, 0);
    ntask_down.resize(ntask_down.size() + sh.nsn, 0);
    ntask_upA.resize(ntask_upA.size() + sh.nsn, 0);
    ntask_downA.resize(ntask_downA.size() + sh.nsn, 0);
    for (const auto& P : X->splan[si]) {
      for (int t = 0; t < P.nfwd; ++t) ntask_upA[front_base[si] + tasks[P.fwd_off + t].sn]++;
      for (int t = 0; t < P.nbwd; ++t) ntask_downA[front_base[si] + tasks[P.bwd_off + t].sn]++;
      for (int t = 0; t < P.nfwdB; ++t) ntask_up[front_base[si] + tasks[P.fwdB_off + t].sn]++;
      for (int t = 0; t < P.nbwdB; ++t) ntask_down[front_base[si] + tasks[P.bwdB_off + t].sn]++;
      shape_entries[si] += 2 * P.entries;
      shape_vec[si] += 2 * P.vec;
      shape_tasks[si] += P.nfwd + P.nbwd + P.nfwdB + P.nbwdB;
    }
  }
  for (size_t f = 0; f < ntask_up.size(); ++f) {   // totals: both phases
    ntask_up[f] += ntask_upA[f];
    ntask_down[f] += ntask_downA[f];
  }
  front_base[X->shapes.size()] = (int)ntask_up.size();
  X->sweep_smax = 0;
  X->sweep_ldmax = 0;
  for (const auto& sp : X->splan)
    for (const auto& P : sp) {
      X->sweep_smax = std::max(X->sweep_smax, P.smax);
      X->sweep_ldmax = std::max(X->sweep_ldmax, P.ldmax);
    }

  // Persistent sweep plans: panel solves in Alg. 1.5 order and one task queue in topological order.
  // Plan 0 is the whole Alg. 1.5 over the handle's panels; plans 1 and 2 are its forward and its
  // backward part alone (a block of panels of a multi-GPU sweep runs them between plane hand-offs).
  // The chains of a batch's problems are interleaved step by step; each step follows the previous
  // step of its own problem.
  size_t sync_words = 0;
  for (int pi = 0; pi < 3; ++pi) {
    psp_ctx_s::SweepPlan& SP = X->plans[pi];
    std::vector<SweepStep> steps;
    std::vector<int> step_prev;
    const int np = (int)X->probs.size();
    std::vector<std::vector<SweepStep>> chain(np);
    size_t longest = 0;
    for (int q = 0; q < np; ++q) {
      const auto& pr = X->probs[q];
      const int last = pr.panel0 + pr.m;
      const int b = pr.panel0 + (X->partial ? X->range_begin : 0), e = X->partial ? pr.panel0 + X->range_end : last;
      if (pi != 2)
        for (int i = b; i < e; ++i) chain[q].push_back({i, 0, q});
      if (pi != 1)
        for (int i = std::min(e, last - 1) - 1; i >= b; --i) chain[q].push_back({i, 1, q});
      longest = std::max(longest, chain[q].size());
    }
    std::vector<int> lastq(np, -1);
    for (size_t t = 0; t < longest; ++t)
      for (int q = 0; q < np; ++q)
        if (t < chain[q].size()) {
          step_prev.push_back(lastq[q]);
          lastq[q] = (int)steps.size();
          steps.push_back(chain[q][t]);
        }
    std::vector<int> step_front(steps.size() + 1, 0), step_tasks(steps.size(), 0);
    SP.entries = 0;
    SP.vec = 0;
    for (size_t k = 0; k < steps.size(); ++k) {
      const int si = X->shape_of[steps[k].panel];
      step_front[k + 1] = step_front[k] + X->shapes[si].nsn;
      step_tasks[k] = shape_tasks[si];
      SP.entries += shape_entries[si];
      SP.vec += shape_vec[si];
    }
    const int64_t nfs = step_front[steps.size()];
    // counter words: head | status[4] | step_done[nsteps] | done_up[nfs] | done_down[nfs] | kids_up[nfs]
    const int64_t o_step = kSweepStepCounters, o_up = o_step + (int64_t)steps.size(), o_down = o_up + nfs,
                  o_kids = o_down + nfs, words = o_kids + nfs;
    if (words > INT_MAX) throw Error{PSP_ERR_ARG, "sweep plan too large"};
    std::vector<QueueEntry> queue;
    for (size_t k = 0; k < steps.size(); ++k) {
      const int si = X->shape_of[steps[k].panel];
      const Shape& sh = X->shapes[si];
      const int fb = front_base[si], sfb = step_front[k];
      const int prev = step_prev[k];
      // a front without children waits for the previous panel solve of its chain (the tasks of a
      // front with children wait for those, which waited for it)
      const unsigned prev_target =
          prev >= 0 ? (unsigned)step_tasks[prev] + (X->test_sweep_stall && prev == 0 ? 1u : 0u) : 0u;
      auto entry = [&](const SolveTask& tk, int dir, int R) {
        QueueEntry e{};
        e.step = (int)k;
        e.sn = tk.sn;
        e.r0 = tk.r0;
        e.r1 = tk.r1;
        e.dir = (short)dir;
        e.R = (short)R;
        const int sn = tk.sn, par = sh.parent[sn];
        const bool up = dir == 0 || dir == kDirUpB;
        e.done = (int)((up ? o_up : o_down) + sfb + sn);
        e.kids = up && par >= 0 ? (int)(o_kids + sfb + par) : -1;
        e.wait = -1;
        if (dir == 0) {
          unsigned kids = 0;
          for (int c = sh.child_ptr[sn]; c < sh.child_ptr[sn + 1]; ++c) kids += (unsigned)ntask_up[fb + sh.child_idx[c]];
          if (kids > 0) {
            e.wait = (int)(o_kids + sfb + sn);
            e.target = kids;
          } else if (prev >= 0) {
            e.wait = (int)(o_step + prev);
            e.target = prev_target;
          }
        } else if (dir == kDirUpB) {   // the front's own first phase up
          e.wait = (int)(o_up + sfb + sn);
          e.target = (unsigned)ntask_upA[fb + sn];
        } else if (dir == kDirDownB) {   // the front's own first phase down
          e.wait = (int)(o_down + sfb + sn);
          e.target = (unsigned)ntask_downA[fb + sn];
        } else if (par >= 0) {   // down: the parent's down tasks
          e.wait = (int)(o_down + sfb + par);
          e.target = (unsigned)ntask_down[fb + par];
        } else {   // the root, down: its own up tasks
          e.wait = (int)(o_up + sfb + sn);
          e.target = (unsigned)ntask_up[fb + sn];
        }
        queue.push_back(e);
      };
      const auto& plan = X->splan[si];
      for (size_t lv = 0; lv < plan.size(); ++lv) {
        for (int t = 0; t < plan[lv].nfwd; ++t) entry(tasks[plan[lv].fwd_off + t], 0, plan[lv].R);
        for (int t = 0; t < plan[lv].nfwdB; ++t) entry(tasks[plan[lv].fwdB_off + t], kDirUpB, plan[lv].R);
      }
      for (int lv = (int)plan.size() - 1; lv >= 0; --lv) {
        for (int t = 0; t < plan[lv].nbwd; ++t) entry(tasks[plan[lv].bwd_off + t], 1, 0);
        for (int t = 0; t < plan[lv].nbwdB; ++t) entry(tasks[plan[lv].bwdB_off + t], kDirDownB, 0);
      }
    }
    SP.hsteps = steps;
    SP.nsteps = (int)steps.size();
    SP.nqueue = (int)queue.size();
    upload_async(SP.steps, steps, side.s);
    upload_async(SP.queue, queue, side.s);
    SP.nfront_steps = nfs;
    sync_words = std::max(sync_words, (size_t)words);
  }
  std::vector<ProblemSweep> pss;
  for (const auto& pr : X->probs) {
    ProblemSweep p{};
    p.off1 = pr.off1;
    p.N = pr.N;
    p.s1n = pr.s1n;
    p.s2n = pr.s2n;
    p.s3h = pr.s3hi;
    p.inv_h2 = 1.0 / (pr.h * pr.h);
    p.nz = pr.nz;
    pss.push_back(p);
  }
  upload_async(X->d_sweep_probs, pss, side.s);
  X->sweep_sync_words = sync_words;
  X->d_sweep_sync.alloc(X->sweep_sync_words * 4);
  side.join(st);
  PSP_CK(cudaMemsetAsync(X->d_sweep_sync.p, 0, X->sweep_sync_words * 4, st));
}

// work vectors of one sweep: per problem (a batch's chains run side by side) a box vector pair of
// max_nloc x nrhs and update vectors of max_upd x nrhs
template <typename T>
static void ensure_apply_ws(psp_ctx_s* X, int nrhs) {
  if (X->ws_nrhs >= nrhs) return;
  const size_t np = X->probs.size();
  X->ws_xf.alloc((size_t)X->max_nloc * nrhs * np * sizeof(T));
  X->ws_xb.alloc((size_t)X->max_nloc * nrhs * np * sizeof(T));
  X->ws_upd.alloc((size_t)X->max_upd * nrhs * np * sizeof(T));
  X->ws_nrhs = nrhs;
}

// Alg. 1.5 (plan 0), or its forward (plan 1) or backward (plan 2) part over the handle's panels, on a
// device block u (N x nrhs, in place), with the box and update-vector work vectors given by the
// caller.  `timed` allows CUDA-event timing of the launches.
template <typename T>
static void apply_core(psp_ctx_s* X, double2* u, int nrhs, T* xf, T* xb, T* upd, bool timed, cudaStream_t st,
                       int plan_index = 0) {
  const psp_ctx_s::SweepPlan& SP = X->plans[plan_index];
  SolveCtx<T> cx{};
  const int np = (int)X->probs.size();
  // problem q's vectors and work vectors
  auto set_problem = [&](int q) {
    const auto& pr = X->probs[q];
    cx.xf = xf + (int64_t)q * X->max_nloc * nrhs;
    cx.xb = xb + (int64_t)q * X->max_nloc * nrhs;
    cx.upd = upd + (int64_t)q * X->max_upd * nrhs;
    cx.u = u + pr.off1 * nrhs;
    cx.N = pr.N;
    cx.nz = pr.nz;
    cx.s1n = pr.s1n;
    cx.s2n = pr.s2n;
    cx.s3h = pr.s3hi;
    cx.inv_h2 = 1.0 / (pr.h * pr.h);
  };
  cx.nrhs = nrhs;
  cx.si = X->si_mode;
  cx.upd_ld = X->max_upd;
  cx.n_loc = X->max_nloc;
  set_problem(0);
  // the persistent sweep offsets problem q's pointers itself: hand it the bases
  cx.xf = xf;
  cx.xb = xb;
  cx.upd = upd;
  cx.u = u;
  const SolveTask* tasks = X->d_stasks.as<SolveTask>();
  const bool was_timing = X->stats.timing;
  if (!timed) X->stats.timing = false;
  auto runT = [&](int q, int i, int mode) {
    const auto& pr = X->probs[q];
    set_problem(q);
    const int si = X->shape_of[i];
    cx.sh = X->shdev[si];
    cx.G = X->d_factor.as<T>() + X->panel_fbase[i];
    cx.z0 = X->z0[i];
    cx.z1 = X->z1[i];
    cx.lead = X->lead[i];
    cx.mode = mode;
    cx.has_prev = i > pr.panel0;
    cx.has_next = i < pr.panel0 + pr.m - 1;
    const auto& plan = X->splan[si];
    const int nl = (int)plan.size();
    const double es = sizeof(T);
    for (int lv = 0; lv < nl; ++lv) {
      const auto& P = plan[lv];
      X->stats.run("k_solve_fwd", st, 1, 8.0 * P.entries * nrhs, P.entries * es + P.vec * es * nrhs, [&] {
        launch_solve_fwd<T>(tasks + P.fwd_off, P.nfwd, cx, P.R, P.smax, 0, st);
        launch_solve_fwd<T>(tasks + P.fwdB_off, P.nfwdB, cx, P.R, P.smax, 1, st);
      });
    }
    for (int lv = nl - 1; lv >= 0; --lv) {
      const auto& P = plan[lv];
      X->stats.run("k_solve_bwd", st, 1, 8.0 * P.entries * nrhs, P.entries * es + P.vec * es * nrhs, [&] {
        launch_solve_bwd<T>(tasks + P.bwd_off, P.nbwd, cx, P.ldmax, 0, st);
        launch_solve_bwd<T>(tasks + P.bwdB_off, P.nbwdB, cx, P.ldmax, 1, st);
      });
    }
  };
  try {
    // one cooperative launch for the whole sweep when the device allows it
    SweepArgs<T> sa{};
    sa.cx = cx;
    sa.nshapes = (int)X->shapes.size();
    sa.nsteps = SP.nsteps;
    sa.npanels = X->m;
    sa.steps = SP.steps.as<SweepStep>();
    sa.panels = X->d_sweep_panels.as<PanelSweep>();
    sa.shapes = X->d_shapes.as<ShapeDev>();
    sa.factor = X->d_factor.as<T>();
    sa.queue = SP.queue.as<QueueEntry>();
    sa.nqueue = SP.nqueue;
    sa.claim_ahead = X->sweep_claim_ahead;
    sa.nprobs = np;
    sa.probs = X->d_sweep_probs.as<ProblemSweep>();
    unsigned* sync = X->d_sweep_sync.as<unsigned>();
    sa.ctr = sync;
    sa.status = reinterpret_cast<int*>(sync + 1);
    sa.sticky = X->d_status.as<int>() + 2;
    const size_t words = kSweepStepCounters + (size_t)SP.nsteps + 3 * (size_t)SP.nfront_steps;
    int rc = -1;
    if (SP.nsteps == 0) rc = 0;   // an empty part (the backward part of a block holding the last panel alone)
    else if (X->persistent_sweep) {
      // queue head and completion counters start at zero; status[2] is cleared too
      PSP_CK(cudaMemsetAsync(sync, 0, words * 4, st));
      const double es = sizeof(T);
      X->stats.run("k_sweep", st, 1, 8.0 * SP.entries * nrhs, SP.entries * es + SP.vec * es * nrhs,
                   [&] { rc = launch_sweep<T>(sa, X->sweep_smax, X->sweep_ldmax, X->sweep_ctas_per_sm, X->sweep_rhs_group, st); });
      if (rc > 0) throw Error{PSP_ERR_CUDA, std::string("sweep launch: ") + cudaGetErrorString((cudaError_t)rc)};
    }
    if (rc != 0) {
      // one launch per tree level: mode 0 u_i := T_i (u_i - J_{i,i-1} u_{i-1}); mode 1 u_i -= T_i J_{i+1,i}^T u_{i+1}
      for (const SweepStep& sp : SP.hsteps) runT(sp.prob, sp.panel, sp.mode);
    }
  } catch (...) {
    X->stats.timing = was_timing;
    throw;
  }
  X->stats.timing = was_timing;
  PSP_CK(cudaGetLastError());
}

template <typename T>
static void apply_impl(psp_ctx_s* X, double2* u, int nrhs, cudaStream_t st) {
  ensure_apply_ws<T>(X, nrhs);
  apply_core<T>(X, u, nrhs, X->ws_xf.as<T>(), X->ws_xb.as<T>(), X->ws_upd.as<T>(), true, st);
}

// work-vector layout of apply_core inside one caller-provided buffer
static size_t round256(size_t b) { return (b + 255) / 256 * 256; }

size_t apply_workspace_bytes(const psp_ctx_s* X, int nrhs) {
  const size_t e = X->elem_bytes, np = X->probs.size();
  return 2 * round256((size_t)X->max_nloc * nrhs * np * e) + round256((size_t)X->max_upd * nrhs * np * e);
}

psp_status apply_with_workspace(psp_ctx_s* X, double2* u, int nrhs, void* ws, cudaStream_t st) {
  if (X->partial) return set_error(PSP_ERR_STATE, "the handle holds one block of panels; use psp_sweep_part");
  try {
    char* p = static_cast<char*>(ws);
    const size_t e = X->elem_bytes;
    const size_t bx = round256((size_t)X->max_nloc * nrhs * X->probs.size() * e);
    if (X->prec == PSP_PREC_C64)
      apply_core<float2>(X, u, nrhs, (float2*)p, (float2*)(p + bx), (float2*)(p + 2 * bx), false, st);
    else
      apply_core<double2>(X, u, nrhs, (double2*)p, (double2*)(p + bx), (double2*)(p + 2 * bx), false, st);
  } catch (const Error& err) {
    g_last_error = err.msg;
    return err.st;
  } catch (const std::exception& ex) {
    g_last_error = ex.what();
    return PSP_ERR_STATE;
  }
  return PSP_OK;
}

psp_status set_error(psp_status s, const char* msg) {
  g_last_error = msg;
  return s;
}

int64_t handle_points(const psp_ctx_s* X) { return X->d_factor.p ? X->N : -1; }
int handle_device(const psp_ctx_s* X) { return X->device; }

// the handle's device must be current (its factors and tables live there)
static void check_device(const psp_ctx_s* X) {
  int cur = -1;
  PSP_CK(cudaGetDevice(&cur));
  if (cur != X->device)
    throw Error{PSP_ERR_ARG, "the handle was set up on device " + std::to_string(X->device) + ", but device " +
                                 std::to_string(cur) + " is current"};
}

// reads and clears the handle's sticky flag of a sweep wait that gave up (the stream is synchronised)
static bool sweep_gave_up(psp_ctx_s* X, cudaStream_t st) {
  int flag = 0;
  PSP_CK(cudaMemcpyAsync(&flag, X->d_status.as<int>() + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
  PSP_CK(cudaStreamSynchronize(st));
  if (flag) PSP_CK(cudaMemsetAsync(X->d_status.as<int>() + 2, 0, sizeof(int), st));
  return flag != 0;
}

static void apply_dispatch(psp_ctx_s* X, double2* u, int nrhs, cudaStream_t st) {
  if (X->prec == PSP_PREC_C64) apply_impl<float2>(X, u, nrhs, st);
  else apply_impl<double2>(X, u, nrhs, st);
}

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
// Panel plan (§1.1, Alg. 1.4): panel 0 = planes [0, gamma + d), then d planes each, the last one
// taking the remainder; lead = planes of the auxiliary box before the panel's own (the pad, or all
// planes below in exact mode, none for panel 0).
static void panel_plan(int nz, int gamma, int depth, int pad, int aux_mode, std::vector<int>& z0, std::vector<int>& z1,
                       std::vector<int>& lead) {
  z0.clear();
  z1.clear();
  lead.clear();
  const int first = std::min(gamma + depth, nz);
  z0.push_back(0);
  z1.push_back(first);
  for (int z = first; z < nz; z += depth) {
    z0.push_back(z);
    z1.push_back(std::min(z + depth, nz));
  }
  for (size_t i = 0; i < z0.size(); ++i)
    lead.push_back(z0[i] == 0 ? 0 : aux_mode == PSP_AUX_EXACT ? z0[i] : pad);
}

// algorithmic setup flops of one factored box: per front LDL^T of F_TL (s^3/3), F_BL L^{-T} (u s^2/2)
// and the Schur update (u(u+1)/2 s) complex multiply-adds, 8 flops each
static double shape_setup_flops(const Shape& sh) {
  double cm = 0;
  for (int f = 0; f < sh.nsn; ++f) {
    const double s = sh.s[f], u = sh.u[f];
    cm += s * s * s / 3 + u * s * s / 2 + u * (u + 1) / 2 * s;
  }
  return 8.0 * cm;
}

// One problem's own part of setup: wave speed, PML tables, panel plan, shapes and box operators
// (kept on the host in X->h_boxops); no factor storage yet.
static void build_problem(psp_ctx_s* X, const double* c, cudaStream_t st) {
  auto t_start = std::chrono::steady_clock::now();
  const int nx = X->nx, ny = X->ny, nz = X->nz;
  X->N = (int64_t)nx * ny * nz;
  // wave speed (host or device input)
  X->d_c.alloc(X->N * sizeof(double));
  PSP_CK(cudaMemcpyAsync(X->d_c.p, c, X->N * sizeof(double), cudaMemcpyDefault, st));

  // global stretch tables: s1n, 1/s1h, s2n, 1/s2h, s3n, 1/s3h
  const bool f[6] = {bool(X->faces & 1), bool(X->faces & 2), bool(X->faces & 4),
                     bool(X->faces & 8), bool(X->faces & 16), bool(X->faces & 32)};
  const int dims[3] = {nx, ny, nz};
  std::vector<double2> gt;
  int64_t goff[6];
  for (int a = 0; a < 3; ++a) {
    const int n = dims[a];
    goff[2 * a] = (int64_t)gt.size();
    for (int i = 0; i < n; ++i)
      gt.push_back(stretch(sigma_axis(i, n, X->gamma, X->C, X->h, f[2 * a], f[2 * a + 1]), X->omega));
    goff[2 * a + 1] = (int64_t)gt.size();
    for (int k = 0; k <= n; ++k)
      gt.push_back(inv_stretch(sigma_axis(k - 0.5, n, X->gamma, X->C, X->h, f[2 * a], f[2 * a + 1]), X->omega));
  }
  panel_plan(nz, X->gamma, X->depth, X->pad, X->aux_mode, X->z0, X->z1, X->lead);
  X->m = (int)X->z0.size();
  // the block of panels this handle factors and sweeps
  X->range_end = X->range_count > 0 ? X->range_begin + X->range_count : X->m;
  if (X->range_begin < 0 || X->range_begin >= X->m || X->range_end > X->m)
    throw Error{PSP_ERR_ARG, "panel block [" + std::to_string(X->range_begin) + ", " + std::to_string(X->range_end) +
                                 ") is not within the " + std::to_string(X->m) + " panels"};
  X->partial = X->range_begin > 0 || X->range_end < X->m;
  // per-panel tables: s3 nodes, 1/s3 half-points, c plane map (device-global layout appended to gt)
  std::vector<int32_t> cplane_all;
  std::vector<int64_t> p_s3n(X->m), p_s3h(X->m), p_cpl(X->m);
  std::map<std::tuple<int, int, int>, int> shape_idx;
  std::vector<int> shape_depth;   // box depth of each distinct shape (same index as X->shapes)
  X->shapes.clear();
  X->shape_of.assign(X->m, 0);
  for (int i = 0; i < X->m; ++i) {
    const int z0 = X->z0[i], z1 = X->z1[i];
    const int lead = X->lead[i];
    const int D = lead + (z1 - z0);
    p_s3n[i] = (int64_t)gt.size();
    for (int k = 0; k < D; ++k) {
      double sig;
      if (z0 == 0 || X->aux_mode == PSP_AUX_EXACT) {
        sig = sigma_axis(k + (z0 - lead), nz, X->gamma, X->C, X->h, f[4], f[5]);
      } else {
        sig = sigma_side((k + 1.0) * X->h, X->pad, X->C, X->h);
        if (k >= lead) sig += sigma_axis(z0 + k - lead, nz, X->gamma, X->C, X->h, f[4], f[5]);
      }
      gt.push_back(stretch(sig, X->omega));
    }
    p_s3h[i] = (int64_t)gt.size();
    for (int k = 0; k <= D; ++k) {
      const double xi = k - 0.5;
      double sig;
      if (z0 == 0 || X->aux_mode == PSP_AUX_EXACT) {
        sig = sigma_axis(xi + (z0 - lead), nz, X->gamma, X->C, X->h, f[4], f[5]);
      } else {
        sig = sigma_side((xi + 1.0) * X->h, X->pad, X->C, X->h);
        if (xi >= lead - 0.5) sig += sigma_axis(z0 + xi - lead, nz, X->gamma, X->C, X->h, f[4], f[5]);
      }
      gt.push_back(inv_stretch(sig, X->omega));
    }
    p_cpl[i] = (int64_t)cplane_all.size();
    for (int k = 0; k < D; ++k) cplane_all.push_back(k < lead && X->aux_mode != PSP_AUX_EXACT ? z0 : z0 - lead + k);
    auto key = std::make_tuple(nx, ny, D);
    auto it = shape_idx.find(key);
    if (it == shape_idx.end()) {
      const int idx = (int)X->shapes.size();
      shape_idx[key] = idx;
      X->shapes.emplace_back();
      shape_depth.push_back(D);
      X->shape_of[i] = idx;
    } else {
      X->shape_of[i] = it->second;
    }
  }
  // the distinct shapes' symbolic analyses are independent: build them on a few host threads.  A
  // worker catches what build_shape throws (a consistency error, bad_alloc); the first one is
  // rethrown here after every thread has joined, so it reaches the ABI as a status.
  {
    const int ns = (int)X->shapes.size();
    const int nthreads = std::max(1, std::min(ns, 8));
    std::vector<std::exception_ptr> errs(nthreads);
    auto worker = [&](int t) {
      try {
        for (int si = t; si < ns; si += nthreads) build_shape(X->shapes[si], nx, ny, shape_depth[si], X->leaf);
      } catch (...) {
        errs[t] = std::current_exception();
      }
    };
    std::vector<std::thread> pool;
    try {
      for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker, t);
    } catch (...) {
      for (auto& th : pool) th.join();
      throw;
    }
    worker(0);
    for (auto& th : pool) th.join();
    for (auto& e : errs)
      if (e) std::rethrow_exception(e);
  }
  // identical auxiliary problems (§3: a model invariant along the sweep direction needs O(1)
  // distinct panel factorisations): same box depth and pad, bitwise the same x3-stretch tables and
  // the same wave speed on every plane the box uses
  X->owner.resize(X->m);
  for (int i = 0; i < X->m; ++i) X->owner[i] = i >= X->range_begin && i < X->range_end ? i : -1;   // -1: not factored here
  if (!X->factor_every_panel && X->aux_mode == PSP_AUX_MOVING_PML && X->range_end - X->range_begin > 1) {
    const int64_t plane = (int64_t)nx * ny;
    std::vector<double> hc((size_t)X->N);
    PSP_CK(cudaMemcpyAsync(hc.data(), c, X->N * sizeof(double), cudaMemcpyDefault, st));   // c: host or device
    PSP_CK(cudaStreamSynchronize(st));
    auto depth_of = [&](int i) { return X->lead[i] + X->z1[i] - X->z0[i]; };
    auto mix = [](uint64_t h, uint64_t w) { return (h ^ (w + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2))) * 0x100000001b3ull; };
    auto words = [&](uint64_t h, const void* p, size_t bytes) {
      const unsigned char* b = static_cast<const unsigned char*>(p);
      for (size_t o = 0; o + 8 <= bytes; o += 8) {
        uint64_t w;
        std::memcpy(&w, b + o, 8);
        h = mix(h, w);
      }
      return h;
    };
    auto same = [&](int i, int j) {
      const int D = depth_of(i);
      if (D != depth_of(j) || X->lead[i] != X->lead[j]) return false;
      if (std::memcmp(&gt[p_s3n[i]], &gt[p_s3n[j]], D * sizeof(double2)) ||
          std::memcmp(&gt[p_s3h[i]], &gt[p_s3h[j]], (D + 1) * sizeof(double2)))
        return false;
      for (int k = 0; k < D; ++k)
        if (std::memcmp(&hc[cplane_all[p_cpl[i] + k] * plane], &hc[cplane_all[p_cpl[j] + k] * plane],
                        plane * sizeof(double)))
          return false;
      return true;
    };
    std::map<uint64_t, std::vector<int>> seen;
    for (int i = std::max(1, X->range_begin); i < X->range_end; ++i) {
      const int D = depth_of(i);
      uint64_t h = mix(mix(1469598103934665603ull, D), X->lead[i]);
      h = words(h, &gt[p_s3n[i]], D * sizeof(double2));
      h = words(h, &gt[p_s3h[i]], (D + 1) * sizeof(double2));
      for (int k = 0; k < D; ++k) h = words(h, &hc[cplane_all[p_cpl[i] + k] * plane], plane * sizeof(double));
      auto& cands = seen[h];
      for (int j : cands)
        if (same(i, j)) {
          X->owner[i] = j;
          break;
        }
      if (X->owner[i] == i) cands.push_back(i);
    }
  }
  // global plane map (identity) for the full-domain operators
  const int64_t gcpl = (int64_t)cplane_all.size();
  for (int k = 0; k < nz; ++k) cplane_all.push_back(k);

  upload(X->d_gtab, gt);
  upload(X->d_ptab, cplane_all);
  const double2* G = X->d_gtab.as<double2>();
  const int32_t* CP = X->d_ptab.as<int32_t>();
  X->s1n = G + goff[0];
  X->s2n = G + goff[2];
  X->s3hi = G + goff[5];
  auto make_op = [&](int bz, double2 k2num, const int32_t* cpl, const double2* s3n, const double2* s3h) {
    BoxOp op{};
    op.nx = nx; op.ny = ny; op.nz = bz;
    op.inv_h2 = 1.0 / (X->h * X->h);
    op.k2num = k2num;
    op.c = X->d_c.as<double>();
    op.cplane = cpl;
    op.s1n = G + goff[0]; op.s1h = G + goff[1];
    op.s2n = G + goff[2]; op.s2h = G + goff[3];
    op.s3n = s3n; op.s3h = s3h;
    return op;
  };
  const double2 k2A = make_double2(X->omega * X->omega, 0.0);
  const double2 k2J = make_double2(X->omega * X->omega - X->alpha * X->alpha, 2.0 * X->omega * X->alpha);
  X->opA = make_op(nz, k2A, CP + gcpl, G + goff[4], G + goff[5]);
  X->opJ = make_op(nz, k2J, CP + gcpl, G + goff[4], G + goff[5]);
  X->h_boxops.assign(X->m, BoxOp{});
  for (int i = 0; i < X->m; ++i)
    X->h_boxops[i] = make_op(X->lead[i] + X->z1[i] - X->z0[i], k2J, CP + p_cpl[i], G + p_s3n[i], G + p_s3h[i]);
  psp_ctx_s::Prob pr;
  pr.N = X->N;
  pr.off1 = 0;
  pr.panel0 = 0;
  pr.m = X->m;
  pr.nz = nz;
  pr.h = X->h;
  pr.opA = X->opA;
  pr.opJ = X->opJ;
  pr.s1n = X->s1n;
  pr.s2n = X->s2n;
  pr.s3hi = X->s3hi;
  X->probs.assign(1, pr);
  X->stats.host("symbolic_tables", ms_since(t_start));
}

// Shared part of setup, over every panel of the handle (one problem or a batch): device shapes and
// operators, factor storage, the solve plan, and the batched factorisation.
static void finish_setup(psp_ctx_s* X, cudaStream_t st) {
  auto t_start = std::chrono::steady_clock::now();
  upload(X->d_boxops, X->h_boxops);
  // factor blocks per front: G ((s + u) x s), and in the two-inverse form the second inverse of L_TL
  // (s x s) right after it, each padded to 16 elements
  for (auto& sh : X->shapes) {
    int64_t go = 0;
    for (int f = 0; f < sh.nsn; ++f) {
      sh.g_off[f] = go;
      go += second_inverse_offset(sh.s[f], sh.u[f]);
      if (X->si_mode == PSP_SI_TWO) go += ((int64_t)sh.s[f] * sh.s[f] + 15) / 16 * 16;
    }
    sh.g_total = go;
  }

  // shapes to the device
  X->shape_bufs.clear();
  X->shdev.clear();
  X->max_nloc = 0;
  X->max_upd = 0;
  for (auto& sh : X->shapes) {
    X->max_nloc = std::max<int64_t>(X->max_nloc, (int64_t)sh.nx * sh.ny * sh.nz);
    X->max_upd = std::max<int64_t>(X->max_upd, sh.upd_total);
    // pack all arrays of the shape into one buffer
    std::vector<char> blob;
    auto put = [&](const void* src, size_t bytes) {
      size_t off = (blob.size() + 15) / 16 * 16;
      blob.resize(off + bytes);
      if (bytes) std::memcpy(blob.data() + off, src, bytes);
      return off;
    };
    size_t o_order = put(sh.order.data(), sh.order.size() * 4);
    size_t o_elim = put(sh.elim.data(), sh.elim.size() * 4);
    size_t o_first = put(sh.first.data(), sh.first.size() * 4);
    size_t o_s = put(sh.s.data(), sh.s.size() * 4);
    size_t o_u = put(sh.u.data(), sh.u.size() * 4);
    size_t o_cp = put(sh.child_ptr.data(), sh.child_ptr.size() * 4);
    size_t o_ci = put(sh.child_idx.data(), sh.child_idx.size() * 4);
    size_t o_sp = put(sh.struct_ptr.data(), sh.struct_ptr.size() * 8);
    size_t o_se = put(sh.struct_elim.data(), sh.struct_elim.size() * 4);
    size_t o_rel = put(sh.rel.data(), sh.rel.size() * 4);
    size_t o_pp = put(sh.pull_ptr.data(), sh.pull_ptr.size() * 8);
    size_t o_pl = put(sh.pull.data(), sh.pull.size() * 4);
    size_t o_go = put(sh.g_off.data(), sh.g_off.size() * 8);
    size_t o_uo = put(sh.upd_off.data(), sh.upd_off.size() * 8);
    size_t o_par = put(sh.parent.data(), sh.parent.size() * 4);
    DevBuf b;
    b.alloc(blob.size());
    PSP_CK(cudaMemcpy(b.p, blob.data(), blob.size(), cudaMemcpyHostToDevice));
    char* base = b.as<char>();
    ShapeDev d{};
    d.nx = sh.nx; d.ny = sh.ny; d.nz = sh.nz; d.nsn = sh.nsn;
    d.order = (const int32_t*)(base + o_order);
    d.elim = (const int32_t*)(base + o_elim);
    d.first = (const int32_t*)(base + o_first);
    d.s = (const int32_t*)(base + o_s);
    d.u = (const int32_t*)(base + o_u);
    d.child_ptr = (const int32_t*)(base + o_cp);
    d.child_idx = (const int32_t*)(base + o_ci);
    d.struct_ptr = (const int64_t*)(base + o_sp);
    d.struct_elim = (const int32_t*)(base + o_se);
    d.rel = (const int32_t*)(base + o_rel);
    d.pull_ptr = (const int64_t*)(base + o_pp);
    d.pull = (const int32_t*)(base + o_pl);
    d.g_off = (const int64_t*)(base + o_go);
    d.upd_off = (const int64_t*)(base + o_uo);
    d.parent = (const int32_t*)(base + o_par);
    X->shdev.push_back(d);
    X->shape_bufs.push_back(std::move(b));
  }
  upload(X->d_shapes, X->shdev);
  std::vector<int32_t> ps(X->shape_of.begin(), X->shape_of.end());
  upload(X->d_panel_shape, ps);

  // front ids and factor slabs
  X->sn_base.assign(X->m, 0);
  X->panel_fbase.assign(X->m, 0);
  int64_t nf = 0, fe = 0;
  X->nfronts_factored = 0;
  X->distinct_panels = 0;
  for (int i = 0; i < X->m; ++i) {
    const Shape& sh = X->shapes[X->shape_of[i]];
    X->sn_base[i] = nf;
    nf += sh.nsn;
    if (X->owner[i] == i) {
      X->panel_fbase[i] = fe;
      fe += sh.g_total;
      X->nfronts_factored += sh.nsn;
      X->distinct_panels += 1;
    } else if (X->owner[i] >= 0) {
      X->panel_fbase[i] = X->panel_fbase[X->owner[i]];   // the owner comes first
    } else {
      X->panel_fbase[i] = 0;                              // outside this handle's block: never read
    }
  }
  X->nfronts = nf;
  X->factor_elems = fe;
  X->elem_bytes = X->prec == PSP_PREC_C64 ? 8 : 16;
  {
    std::vector<PanelSweep> ps(X->m);
    for (const auto& pr : X->probs)
      for (int i = pr.panel0; i < pr.panel0 + pr.m; ++i) {
        ps[i].gbase = X->panel_fbase[i];
        ps[i].shape = X->shape_of[i];
        ps[i].z0 = X->z0[i];
        ps[i].z1 = X->z1[i];
        ps[i].lead = X->lead[i];
        ps[i].has_prev = i > pr.panel0;
        ps[i].has_next = i < pr.panel0 + pr.m - 1;
      }
    upload(X->d_sweep_panels, ps);
  }
  X->stats.host("device_tables", ms_since(t_start));
  auto ta = std::chrono::steady_clock::now();
  X->d_factor.alloc((size_t)fe * X->elem_bytes);
  X->d_status.alloc(8 * sizeof(int));
  X->stats.host("alloc_factors", ms_since(ta));
  // the sweep's plan is host work the device does not need for the factorisation: it runs while
  // the device factors
  auto planner = [X, st] {
    auto t0 = std::chrono::steady_clock::now();
    plan_solve(X, st);
    X->stats.host("plan_solve", ms_since(t0));
  };
  if (X->prec == PSP_PREC_C64) factor_all<float2>(X, st, planner);
  else factor_all<double2>(X, st, planner);
}

static void setup_impl(psp_ctx_s* X, const double* c, cudaStream_t st) {
  build_problem(X, c, st);
  finish_setup(X, st);
}

// A batch: every problem's own tables, then its panels appended to the handle's panel list.
static void setup_batch_impl(psp_ctx_s* B, int nprob, const double* const* c, cudaStream_t st) {
  B->m = 0;
  B->N = 0;
  B->probs.clear();
  B->owner.clear();
  for (int q = 0; q < nprob; ++q) {
    psp_ctx_s* X = B->subs[q].get();
    build_problem(X, c[q], st);
    const int shape0 = (int)B->shapes.size();
    for (auto& sh : X->shapes) B->shapes.push_back(std::move(sh));
    X->shapes.clear();
    psp_ctx_s::Prob pr = X->probs[0];
    pr.off1 = B->N;
    pr.panel0 = B->m;
    B->probs.push_back(pr);
    for (int i = 0; i < X->m; ++i) {
      B->owner.push_back(B->m + X->owner[i]);
      B->z0.push_back(X->z0[i]);
      B->z1.push_back(X->z1[i]);
      B->lead.push_back(X->lead[i]);
      B->shape_of.push_back(shape0 + X->shape_of[i]);
      B->h_boxops.push_back(X->h_boxops[i]);
    }
    B->m += X->m;
    B->N += X->N;
    for (auto& kv : X->stats.k)
      if (kv.first.rfind("host:", 0) == 0) B->stats.host(kv.first.substr(5).c_str(), kv.second.ms);
  }
  B->nx = B->subs[0]->nx;
  B->ny = B->subs[0]->ny;
  B->nz = B->subs[0]->nz;
  B->h = B->subs[0]->h;
  B->opA = B->subs[0]->opA;
  B->opJ = B->subs[0]->opJ;
  finish_setup(B, st);
}

// ---------------------------------------------------------------------------
// GMRES(k), right preconditioned, x0 = 0, complex128 (§2.4, §3)
// ---------------------------------------------------------------------------
// store_z: keep z_j = M^{-1} v_j for every Krylov vector and update x += Z y at the end of a cycle;
// otherwise keep one work vector and form x += M^{-1} (V y) with one more application per cycle
// (right preconditioning: both give x0 + M^{-1} V y), which halves the vectors kept per right-hand side.
static void solve_impl(psp_ctx_s* X, const double2* f, double2* x, int nrhs_in, double tol, int k, int maxit,
                       psp_solve_info* info, cudaStream_t st, bool store_z,
                       std::vector<std::vector<double>>* hist_est = nullptr,
                       std::vector<std::vector<double>>* hist_true = nullptr) {
  // GMRES columns: right-hand side r of problem q is column q * nrhs + r, the span
  // [off1_q nrhs + r N_q, + N_q) of every vector block; all columns iterate in lockstep but each
  // has its own Krylov basis, Hessenberg matrix and convergence test
  const int np = (int)X->probs.size();
  const int nrhs = np * nrhs_in;        // columns
  const int64_t NT = X->N * nrhs_in;    // elements of one vector block
  int64_t maxlen = 0;
  if (X->cols_nrhs != nrhs_in) {
    std::vector<ColSpan> cols;
    for (const auto& pr : X->probs)
      for (int r = 0; r < nrhs_in; ++r) cols.push_back({pr.off1 * nrhs_in + r * pr.N, pr.N});
    upload(X->d_cols, cols);
    X->cols_nrhs = nrhs_in;
  }
  for (const auto& pr : X->probs) maxlen = std::max(maxlen, pr.N);
  const ColSpan* cols = X->d_cols.as<ColSpan>();
  const int K = k;
  // workspace layout (double2 elements)
  const int64_t nV = (int64_t)(K + 1) * NT, nZ = (store_z ? (int64_t)K : 1) * NT, nW = NT;
  const int64_t nB = nW;
  const int64_t nH = (int64_t)(K + 1) * K * nrhs, nSn = (int64_t)K * nrhs, nG = (int64_t)(K + 1) * nrhs;
  const int64_t nPart = (int64_t)multidot_blocks(maxlen) * (K + 1) * nrhs, nDot = (int64_t)(K + 1) * nrhs;
  const int64_t total = nV + nZ + nW + nB + nH + nSn + nG + nPart + 3 * nDot + 3 * nrhs + (int64_t)K * nrhs + 64;
  X->gm.ensure((size_t)total * sizeof(double2) + (size_t)(K + 8) * nrhs * sizeof(double) + 4 * nrhs * sizeof(int));
  double2* base = X->gm.as<double2>();
  double2* V = base;
  double2* Z = V + nV;
  double2* w = Z + nZ;
  double2* b = w + nW;
  double2* Hm = b + nB;
  double2* sn = Hm + nH;
  double2* g = sn + nSn;
  double2* part = g + nG;
  double2* h1 = part + nPart;
  double2* h2 = h1 + nDot;
  double2* nrm = h2 + nDot;
  double2* scl = nrm + nDot;
  double2* ybuf = scl + 3 * nrhs;
  double* cs = reinterpret_cast<double*>(ybuf + (int64_t)K * nrhs + 64);
  double* resid = cs + (int64_t)K * nrhs;
  int* active = reinterpret_cast<int*>(resid + 8 * nrhs);
  int* jr = active + nrhs;

  LsqState Ls{};
  Ls.H = Hm; Ls.cs = cs; Ls.sn = sn; Ls.g = g; Ls.resid = resid; Ls.scl = scl; Ls.active = active;
  Ls.k = K; Ls.nrhs = nrhs;
  const int64_t ldv_vec = NT;

  Stats& S = X->stats;
  const double vb = 16.0 * NT;   // bytes of one vector block
  auto matvec = [&](const double2* in, double2* out) {
    for (const auto& pr : X->probs) {
      const int64_t o = pr.off1 * nrhs_in;
      S.run("k_matvec", st, 1, 8.0 * 7 * pr.N * nrhs_in, 8.0 * pr.N + 32.0 * pr.N * nrhs_in,
            [&] { launch_matvec(pr.opA, in + o, out + o, nrhs_in, pr.N, st); });
    }
  };
  auto multidot = [&](const double2* Vv, int64_t ldvv, int nvec, const double2* ww, double2* out) {
    S.run("k_dot_partial+k_dot_final", st, 2, 8.0 * NT * nvec, (nvec + 1) * vb,
          [&] { launch_multidot(Vv, ldvv, nvec, ww, cols, nrhs, maxlen, part, out, st); });
  };
  auto multiaxpy = [&](const double2* Vv, int nvec, const double2* hh, double2* ww, double sign) {
    S.run("k_multiaxpy", st, 1, 8.0 * NT * nvec, (nvec + 2) * vb,
          [&] { launch_multiaxpy(Vv, ldv_vec, nvec, hh, ww, cols, nrhs, maxlen, sign, st); });
  };
  auto axpby = [&](const double2* xx, double2* yy, const double2* al, int mode) {
    S.run("k_axpby", st, 1, 8.0 * NT, 3 * vb, [&] { launch_axpby_batch(xx, yy, cols, nrhs, maxlen, al, mode, st); });
  };
  auto small = [&](const char* nm, auto&& fn) { S.run(nm, st, 1, 0.0, 0.0, fn); };

  auto t0 = std::chrono::steady_clock::now();
  for (const auto& pr : X->probs) {
    const int64_t o = pr.off1 * nrhs_in;
    S.run("k_scale_rhs", st, 1, 6.0 * pr.N * nrhs_in, 32.0 * pr.N * nrhs_in,
          [&] { launch_scale_rhs(pr.opA, f + o, b + o, nrhs_in, pr.N, st); });
  }
  // ||b||
  std::vector<double> bnorm(nrhs), rel(nrhs, 1.0), hres(nrhs), est(nrhs, 1.0);
  std::vector<int> act(nrhs, 1), its(nrhs, 0), restarts(nrhs, 0), jrh(nrhs, 0);
  multidot(b, 0, 1, b, nrm);
  std::vector<double2> hn(nrhs);
  PSP_CK(cudaMemcpyAsync(hn.data(), nrm, nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st));
  PSP_CK(cudaStreamSynchronize(st));
  for (int r = 0; r < nrhs; ++r) {
    bnorm[r] = std::sqrt(std::max(hn[r].x, 0.0));
    if (bnorm[r] == 0.0) { act[r] = 0; rel[r] = 0.0; }
  }
  PSP_CK(cudaMemsetAsync(x, 0, nW * sizeof(double2), st));
  PSP_CK(cudaMemcpyAsync(w, b, nW * sizeof(double2), cudaMemcpyDeviceToDevice, st));  // r = b - A*0
  int applies = 0, total_it = 0;
  bool any = std::any_of(act.begin(), act.end(), [](int a) { return a != 0; });
  while (any && total_it < maxit) {
    PSP_CK(cudaMemcpyAsync(active, act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
    // V_0 = r / ||r||
    multidot(w, 0, 1, w, nrm);
    small("k_cycle_start", [&] { launch_cycle_start(Ls, nrm, st); });
    axpby(w, V, scl, 0);
    for (int r = 0; r < nrhs; ++r) jrh[r] = 0;
    int j = 0;
    for (; j < K && total_it < maxit; ++j) {
      double2* Vj = V + (int64_t)j * ldv_vec;
      double2* Zj = store_z ? Z + (int64_t)j * ldv_vec : Z;
      PSP_CK(cudaMemcpyAsync(Zj, Vj, nW * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      apply_dispatch(X, Zj, nrhs_in, st);   // z_j = M^{-1} v_j
      ++applies;
      matvec(Zj, w);  // w = A z_j
      // classical Gram-Schmidt, twice
      multidot(V, ldv_vec, j + 1, w, h1);
      multiaxpy(V, j + 1, h1, w, -1.0);
      multidot(V, ldv_vec, j + 1, w, h2);
      multiaxpy(V, j + 1, h2, w, -1.0);
      multidot(w, 0, 1, w, nrm);
      small("k_arnoldi_step", [&] { launch_arnoldi_step(Ls, j, h1, h2, nrm, st); });
      axpby(w, V + (int64_t)(j + 1) * ldv_vec, scl, 0);
      PSP_CK(cudaMemcpyAsync(hres.data(), resid, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
      if (sweep_gave_up(X, st)) throw Error{PSP_ERR_TIMEOUT, "a dependency wait of the sweep gave up"};
      ++total_it;
      bool all_done = true;
      for (int r = 0; r < nrhs; ++r) {
        if (!act[r]) continue;
        its[r]++;
        jrh[r] = j + 1;
        est[r] = hres[r] / bnorm[r];
        if (est[r] < tol) act[r] = 0;   // converged within the cycle (estimate)
        else all_done = false;
      }
      if (hist_est) hist_est->push_back(est);
      PSP_CK(cudaMemcpyAsync(active, act.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
      if (all_done) { ++j; break; }
    }
    // x += M^{-1} V y for every rhs that iterated in this cycle (y is zero beyond a column's own
    // count; only the vectors some column reached are read)
    PSP_CK(cudaMemcpyAsync(jr, jrh.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
    small("k_backsolve", [&] { launch_backsolve(Ls, jr, ybuf, st); });
    const int jmax = *std::max_element(jrh.begin(), jrh.end());
    if (jmax > 0) {
      if (store_z) {
        multiaxpy(Z, jmax, ybuf, x, 1.0);
      } else {
        PSP_CK(cudaMemsetAsync(Z, 0, nW * sizeof(double2), st));
        multiaxpy(V, jmax, ybuf, Z, 1.0);
        apply_dispatch(X, Z, nrhs_in, st);
        ++applies;
        axpby(Z, x, nullptr, 2);
      }
    }
    // true residual r = b - A x
    matvec(x, w);
    axpby(b, w, nullptr, 1);
    multidot(w, 0, 1, w, nrm);
    PSP_CK(cudaMemcpyAsync(hn.data(), nrm, nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st));
    PSP_CK(cudaStreamSynchronize(st));
    any = false;
    for (int r = 0; r < nrhs; ++r) {
      if (bnorm[r] == 0.0) continue;
      if (jrh[r] > 0) restarts[r]++;
      rel[r] = std::sqrt(std::max(hn[r].x, 0.0)) / bnorm[r];
      act[r] = rel[r] >= tol ? 1 : 0;
      if (act[r]) any = true;
    }
    if (hist_true) hist_true->push_back(rel);
  }
  auto t1 = std::chrono::steady_clock::now();
  const double relmax = *std::max_element(rel.begin(), rel.end());
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iterations = *std::max_element(its.begin(), its.end());
    info->restarts = *std::max_element(restarts.begin(), restarts.end());
    info->converged = relmax < tol;
    info->applies = applies;
    info->relres_max = relmax;
    info->solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    info->status_front = -1;
  }
  if (!(relmax < tol)) throw Error{PSP_ERR_NOT_CONVERGED, "GMRES reached maxit with relative residual " + std::to_string(relmax)};
}

}  // namespace psp

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void psp_default_options(psp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->pml_C = 4.0;
  o->alpha = 2.0 * M_PI;
  o->pad_depth = -1;
  o->leaf_size = 64;
  o->precision = PSP_PREC_C128;
  o->pml_faces = 63;
  o->aux_mode = PSP_AUX_MOVING_PML;
}

const char* psp_status_string(psp_status s) {
  switch (s) {
    case PSP_OK: return "ok";
    case PSP_ERR_ARG: return "invalid argument";
    case PSP_ERR_OOM: return "out of memory";
    case PSP_ERR_CUDA: return "CUDA error";
    case PSP_ERR_ZERO_PIVOT: return "zero pivot";
    case PSP_ERR_NOT_CONVERGED: return "not converged";
    case PSP_ERR_TIMEOUT: return "device wait timed out";
    case PSP_ERR_STATE: return "invalid handle state";
  }
  return "unknown status";
}

const char* psp_last_error(void) { return g_last_error.c_str(); }

static psp_status fail(psp_status s, const std::string& m) {
  g_last_error = m;
  return s;
}

#define PSP_TRY try {
#define PSP_CATCH                                                          \
  }                                                                        \
  catch (const Error& e) { return fail(e.st, e.msg); }                     \
  catch (const std::bad_alloc&) { return fail(PSP_ERR_OOM, "host allocation failed"); } \
  catch (const std::exception& e) { return fail(PSP_ERR_STATE, e.what()); }

static psp_status check_options(const psp_options* opt, psp_options* o) {
  psp_default_options(o);
  if (opt) *o = *opt;
  if (o->collect_stats < 0 || o->collect_stats > 2) return fail(PSP_ERR_ARG, "bad collect_stats");
  if (o->leaf_size < 1 || o->pml_faces < 0 || o->pml_faces > 63 ||
      (o->precision != PSP_PREC_C128 && o->precision != PSP_PREC_C64) ||
      (o->aux_mode != PSP_AUX_MOVING_PML && o->aux_mode != PSP_AUX_EXACT) || !(o->alpha >= 0) || !(o->pml_C >= 0) ||
      o->gmres_basis < 0 || o->gmres_basis > 2 || o->panel_begin < 0 || o->panel_count < 0 ||
      (o->dev_alloc == nullptr) != (o->dev_free == nullptr) || o->selective_inversion < 0 || o->selective_inversion > 3 ||
      o->c64_diag_fp64 < 0 || o->c64_diag_fp64 > 1 || o->sweep_claim_ahead > 2)
    return fail(PSP_ERR_ARG, "bad options");
  return PSP_OK;
}

static psp_status check_problem(const psp_grid* g, const double* c, double omega, int pml_gamma, int panel_depth) {
  if (!g || !c) return fail(PSP_ERR_ARG, "grid or c is NULL");
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || !(g->h > 0)) return fail(PSP_ERR_ARG, "bad grid");
  if ((int64_t)g->nx * g->ny * g->nz > (int64_t)1 << 31) return fail(PSP_ERR_ARG, "grid too large");
  if (!(omega > 0) || pml_gamma < 0 || panel_depth < 1) return fail(PSP_ERR_ARG, "bad omega, gamma or panel depth");
  return PSP_OK;
}

// handle-wide settings from the options
static void init_options(psp_ctx_s* X, const psp_options& o) {
  X->allocator.alloc = o.dev_alloc;
  X->allocator.free = o.dev_free;
  X->allocator.ctx = o.alloc_ctx;
  X->alpha = o.alpha; X->C = o.pml_C;
  X->leaf = o.leaf_size; X->prec = o.precision; X->faces = o.pml_faces; X->aux_mode = o.aux_mode;
  X->stats.timing = o.collect_stats != 0;
  X->stats.mode = o.collect_stats;
  X->use_tc = o.tensor_cores != 0;
  X->diag_fp64 = o.c64_diag_fp64 != 0;
  X->tc_min_dim = o.tc_min_dim > 0 ? o.tc_min_dim : 64;
  // measured on lens100: both precisions' sweeps are fastest at about 608 tasks per level
  X->sweep_level_tasks = o.sweep_level_tasks > 0 ? o.sweep_level_tasks : 608;
  X->sweep_ctas_per_sm = o.sweep_ctas_per_sm > 0 ? o.sweep_ctas_per_sm : 8;
  X->sweep_rhs_group = o.sweep_rhs_group > 0 ? o.sweep_rhs_group : 0;
  X->sweep_min_rows = o.sweep_min_rows > 0 ? o.sweep_min_rows : 8;
  X->sweep_max_rows = o.sweep_max_rows > 0 ? std::min(256, std::max(64, o.sweep_max_rows)) : 256;
  X->sweep_claim_ahead = o.sweep_claim_ahead > 0 ? o.sweep_claim_ahead : 1;
  X->solve_rhs_group = o.solve_rhs_group > 0 ? o.solve_rhs_group : 0;
  X->gmres_basis = o.gmres_basis;
  X->si_mode = o.selective_inversion;
  X->factor_every_panel = o.factor_every_panel != 0;
  X->range_begin = o.panel_begin;
  X->range_count = o.panel_count;
  X->test_sweep_stall = o.test_sweep_stall == 1;
  X->temp_budget_elems = o.setup_temp_mb > 0 ? ((int64_t)o.setup_temp_mb << 20) / (o.precision == PSP_PREC_C64 ? 8 : 16) : 0;
}

static void init_problem(psp_ctx_s* X, const psp_grid* g, double omega, int pml_gamma, int panel_depth,
                         const psp_options& o) {
  X->nx = g->nx; X->ny = g->ny; X->nz = g->nz; X->h = g->h;
  X->omega = omega;
  X->gamma = pml_gamma; X->depth = panel_depth;
  X->pad = o.pad_depth < 0 ? pml_gamma : o.pad_depth;
  init_options(X, o);
}

psp_status psp_setup(const psp_grid* g, const double* c, double omega, int pml_gamma, int panel_depth,
                     const psp_options* opt, void* stream, psp_handle* out) {
  if (!out) return fail(PSP_ERR_ARG, "out is NULL");
  *out = nullptr;
  psp_status cs = check_problem(g, c, omega, pml_gamma, panel_depth);
  if (cs != PSP_OK) return cs;
  psp_options o;
  cs = check_options(opt, &o);
  if (cs != PSP_OK) return cs;
  psp_ctx_s* X = nullptr;
  try {
    X = new psp_ctx_s();
  } catch (...) {
    return fail(PSP_ERR_OOM, "host allocation failed");
  }
  init_problem(X, g, omega, pml_gamma, panel_depth, o);
  *out = X;
  PSP_TRY
  AllocScope scope(&X->allocator);
  PSP_CK(cudaGetDevice(&X->device));
  setup_impl(X, c, (cudaStream_t)stream);
  return PSP_OK;
  PSP_CATCH
}

psp_status psp_setup_batch(int nprob, const psp_grid* grids, const double* const* c, const double* omega,
                           const int* pml_gamma, const int* panel_depth, const psp_options* opt, void* stream,
                           psp_handle* out) {
  if (!out) return fail(PSP_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (nprob < 1 || !grids || !c || !omega || !pml_gamma || !panel_depth) return fail(PSP_ERR_ARG, "bad batch arguments");
  int64_t total = 0;
  for (int q = 0; q < nprob; ++q) {
    psp_status cs = check_problem(grids + q, c[q], omega[q], pml_gamma[q], panel_depth[q]);
    if (cs != PSP_OK) return cs;
    total += (int64_t)grids[q].nx * grids[q].ny * grids[q].nz;
  }
  if (total > (int64_t)1 << 31) return fail(PSP_ERR_ARG, "batch too large");
  psp_options o;
  psp_status cs = check_options(opt, &o);
  if (cs != PSP_OK) return cs;
  if (o.panel_begin != 0 || o.panel_count != 0) return fail(PSP_ERR_ARG, "a batch handle holds every panel of its problems");
  psp_ctx_s* B = nullptr;
  try {
    B = new psp_ctx_s();
    for (int q = 0; q < nprob; ++q) {
      B->subs.emplace_back(new psp_ctx_s());
      init_problem(B->subs.back().get(), grids + q, omega[q], pml_gamma[q], panel_depth[q], o);
    }
  } catch (...) {
    delete B;
    return fail(PSP_ERR_OOM, "host allocation failed");
  }
  init_problem(B, grids, omega[0], pml_gamma[0], panel_depth[0], o);
  *out = B;
  PSP_TRY
  AllocScope scope(&B->allocator);
  PSP_CK(cudaGetDevice(&B->device));
  setup_batch_impl(B, nprob, c, (cudaStream_t)stream);
  return PSP_OK;
  PSP_CATCH
}

psp_status psp_batch_layout(psp_handle X, int* nprob, int64_t* points, int capacity) {
  if (!X || capacity < 0 || (capacity > 0 && !points)) return fail(PSP_ERR_ARG, "bad layout arguments");
  if (nprob) *nprob = (int)X->probs.size();
  for (int q = 0; q < capacity && q < (int)X->probs.size(); ++q) points[q] = X->probs[q].N;
  return PSP_OK;
}

static const char* kPartialMsg = "the handle holds one block of panels; apply its part with psp_sweep_part";

psp_status psp_apply(psp_handle X, const double* rhs, double* out, int nrhs, void* stream) {
  if (!X || !rhs || !out || nrhs < 1) return fail(PSP_ERR_ARG, "bad apply arguments");
  if (!X->d_factor.p) return fail(PSP_ERR_STATE, "handle has no factorisation");
  if (X->partial) return fail(PSP_ERR_STATE, kPartialMsg);
  PSP_TRY
  check_device(X);
  AllocScope scope(&X->allocator);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)X->N * nrhs * sizeof(double2);
  const bool dev_out = is_device_pointer(out);
  (void)is_device_pointer(rhs);
  double2* u;
  if (dev_out) {
    u = reinterpret_cast<double2*>(out);
  } else {
    X->stage_out.ensure(bytes);
    u = X->stage_out.as<double2>();
  }
  if ((const void*)rhs != (const void*)u) PSP_CK(cudaMemcpyAsync(u, rhs, bytes, cudaMemcpyDefault, st));
  apply_dispatch(X, u, nrhs, st);
  if (!dev_out) {
    PSP_CK(cudaMemcpyAsync(out, u, bytes, cudaMemcpyDeviceToHost, st));
    PSP_CK(cudaStreamSynchronize(st));
    if (sweep_gave_up(X, st)) return fail(PSP_ERR_TIMEOUT, "a dependency wait of the sweep gave up; out is incomplete");
  }
  return PSP_OK;
  PSP_CATCH
}

psp_status psp_matvec(psp_handle X, int which, const double* x, double* y, int nrhs, void* stream) {
  if (!X || !x || !y || nrhs < 1 || (which != 0 && which != 1)) return fail(PSP_ERR_ARG, "bad matvec arguments");
  PSP_TRY
  check_device(X);
  AllocScope scope(&X->allocator);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)X->N * nrhs * sizeof(double2);
  const double2* xd = reinterpret_cast<const double2*>(x);
  if (!is_device_pointer(x)) {
    X->stage_in.ensure(bytes);
    PSP_CK(cudaMemcpyAsync(X->stage_in.p, x, bytes, cudaMemcpyHostToDevice, st));
    xd = X->stage_in.as<double2>();
  }
  const bool dev_out = is_device_pointer(y);
  double2* yd = reinterpret_cast<double2*>(y);
  if (!dev_out) {
    X->stage_out.ensure(bytes);
    yd = X->stage_out.as<double2>();
  }
  if ((const void*)xd == (const void*)yd) return fail(PSP_ERR_ARG, "matvec cannot run in place");
  for (const auto& pr : X->probs) {
    const int64_t o = pr.off1 * nrhs;
    X->stats.run("k_matvec", st, 1, 8.0 * 7 * pr.N * nrhs, 8.0 * pr.N + 32.0 * pr.N * nrhs,
                 [&] { launch_matvec(which == 0 ? pr.opA : pr.opJ, xd + o, yd + o, nrhs, pr.N, st); });
  }
  PSP_CK(cudaGetLastError());
  if (!dev_out) {
    PSP_CK(cudaMemcpyAsync(y, yd, bytes, cudaMemcpyDeviceToHost, st));
    PSP_CK(cudaStreamSynchronize(st));
  }
  return PSP_OK;
  PSP_CATCH
}

psp_status psp_solve(psp_handle X, const double* f, double* u, int nrhs, double tol, int k, int maxit,
                     psp_solve_info* info, void* stream) {
  if (!X || !f || !u || nrhs < 1 || !(tol > 0) || k < 1 || maxit < 1) return fail(PSP_ERR_ARG, "bad solve arguments");
  if (!X->d_factor.p) return fail(PSP_ERR_STATE, "handle has no factorisation");
  if (X->partial) return fail(PSP_ERR_STATE, kPartialMsg);
  PSP_TRY
  check_device(X);
  AllocScope scope(&X->allocator);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)X->N * nrhs * sizeof(double2);
  const double2* fd = reinterpret_cast<const double2*>(f);
  if (!is_device_pointer(f)) {
    X->stage_in.ensure(bytes);
    PSP_CK(cudaMemcpyAsync(X->stage_in.p, f, bytes, cudaMemcpyHostToDevice, st));
    fd = X->stage_in.as<double2>();
  }
  const bool dev_out = is_device_pointer(u);
  double2* ud = reinterpret_cast<double2*>(u);
  if (!dev_out) {
    X->stage_out.ensure(bytes);
    ud = X->stage_out.as<double2>();
  }
  // Right-hand sides per GMRES run: all of them when their Krylov bases (V and Z, 2k + 1 vectors)
  // fit the free device memory, else groups that do.  The columns iterate independently, so the
  // groups give the same result.  (Batches keep one run: their columns interleave problems.)
  // When not all of them fit with z_j = M^{-1} v_j kept (2k + 1 vectors each), GMRES keeps V only
  // (k + 2 vectors each, one more application per cycle) if that needs fewer sweep passes.
  // The runs get balanced sizes: a sweep carries up to `width` right-hand sides per pass over the
  // factors, so of the run counts the memory allows, the one needing the fewest passes is taken
  // (32 columns with room for 10 per run: four runs of 8, not 10, 10, 10 and 2).
  int width = 8;
  if (X->sweep_rhs_group > 0)
    while (width > 1 && width > X->sweep_rhs_group) width >>= 1;
  auto plan_runs = [&](int cap, int* best_passes) {
    int best_r = nrhs, best_p = INT_MAX;
    for (int r = (nrhs + cap - 1) / cap; r <= nrhs; ++r) {
      const int q = nrhs / r, rem = nrhs % r;
      const int p = rem * ((q + width) / width) + (r - rem) * ((q + width - 1) / width);
      if (p < best_p) {
        best_p = p;
        best_r = r;
      }
      if (q <= width) break;   // one pass per run already: more runs only add passes
    }
    *best_passes = best_p;
    return best_r;
  };
  int runs = 1;
  bool store_z = true;
  if (X->probs.size() == 1) {
    const int cap = X->solve_rhs_group > 0 ? std::min(nrhs, X->solve_rhs_group) : nrhs;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
      const double ws = (2.0 * X->max_nloc + X->max_upd) * (double)X->elem_bytes;
      const double vec = (double)X->N * sizeof(double2);
      const double held = (double)X->gm.bytes + X->ws_xf.bytes + X->ws_xb.bytes + X->ws_upd.bytes;
      const double avail = (double)free_b + held - 2.0e9;
      auto fit = [&](double per_rhs) { return std::max(1, std::min(cap, (int)(avail / per_rhs))); };
      int pz = 0, pv = 0;
      const int rz = plan_runs(fit((2.0 * k + 6) * vec + ws), &pz), rv = plan_runs(fit((k + 7.0) * vec + ws), &pv);
      store_z = X->gmres_basis == 1 || (X->gmres_basis == 0 && pv >= pz);
      runs = store_z ? rz : rv;
    } else {
      cudaGetLastError();
      int p = 0;
      runs = plan_runs(cap, &p);
      store_z = X->gmres_basis != 2;
    }
  } else {
    store_z = X->gmres_basis != 2;
  }
  psp_status rs = PSP_OK;
  psp_solve_info agg{};
  agg.converged = 1;
  agg.status_front = -1;
  agg.min_pivot_abs = X->min_pivot_abs;
  const int ncols = nrhs * (int)X->probs.size();
  for (int kind = 0; kind < 2; ++kind) X->hist[kind].clear();
  X->hist_cols = ncols;
  X->has_history = true;
  // a group's history rows go into its columns; a column that stopped repeats its last value
  auto merge = [&](std::vector<std::vector<double>>& dst, const std::vector<std::vector<double>>& src, int c0, int nc) {
    for (size_t r = 0; r < src.size(); ++r) {
      if (dst.size() <= r) dst.push_back(dst.empty() ? std::vector<double>(ncols, 1.0) : dst.back());
      for (int c = 0; c < nc; ++c) dst[r][c0 + c] = src[r][c];
    }
    for (size_t r = src.size(); r < dst.size() && !src.empty(); ++r)
      for (int c = 0; c < nc; ++c) dst[r][c0 + c] = src.back()[c];
  };
  for (int run = 0, r0 = 0; run < runs; ++run) {
    const int ng = nrhs / runs + (run < nrhs % runs ? 1 : 0);
    psp_solve_info gi{};
    std::vector<std::vector<double>> he, ht;
    try {
      solve_impl(X, fd + (int64_t)r0 * X->N, ud + (int64_t)r0 * X->N, ng, tol, k, maxit, &gi, st, store_z, &he, &ht);
    } catch (const Error& e) {
      if (e.st != PSP_ERR_NOT_CONVERGED) throw;
      rs = fail(e.st, e.msg);
    }
    // columns of this run: one per right-hand side (single-problem handles run in groups)
    merge(X->hist[0], he, r0, (int)(he.empty() ? ng : he[0].size()));
    merge(X->hist[1], ht, r0, (int)(ht.empty() ? ng : ht[0].size()));
    agg.iterations = std::max(agg.iterations, gi.iterations);
    agg.restarts = std::max(agg.restarts, gi.restarts);
    agg.converged = agg.converged && gi.converged;
    agg.applies += gi.applies;
    agg.relres_max = std::max(agg.relres_max, gi.relres_max);
    agg.solve_ms += gi.solve_ms;
    agg.groups += 1;
    r0 += ng;
  }
  if (info) *info = agg;
  if (!dev_out) {
    PSP_CK(cudaMemcpyAsync(u, ud, bytes, cudaMemcpyDeviceToHost, st));
    PSP_CK(cudaStreamSynchronize(st));
  }
  return rs;
  PSP_CATCH
}

psp_status psp_solve_history(psp_handle X, int kind, double* buf, int capacity, int* rows, int* cols) {
  if (!X || (kind != 0 && kind != 1) || capacity < 0) return fail(PSP_ERR_ARG, "bad history arguments");
  if (!X->has_history) return fail(PSP_ERR_STATE, "no solve has run on this handle");
  const auto& H = X->hist[kind];
  if (rows) *rows = (int)H.size();
  if (cols) *cols = X->hist_cols;
  if (!buf) return PSP_OK;
  if ((int64_t)capacity < (int64_t)H.size() * X->hist_cols) return fail(PSP_ERR_ARG, "history buffer too small");
  for (size_t r = 0; r < H.size(); ++r)
    std::memcpy(buf + r * X->hist_cols, H[r].data(), X->hist_cols * sizeof(double));
  return PSP_OK;
}

psp_status psp_symbolic_export(psp_handle X, int panel, int32_t* buf, size_t* len) {
  if (!X || !len || panel < 0 || panel >= X->m) return fail(PSP_ERR_ARG, "bad panel");
  const Shape& sh = X->shapes[X->shape_of[panel]];
  size_t n = 5;
  for (int f = 0; f < sh.nsn; ++f) n += 3 + sh.s[f] + sh.u[f];
  if (!buf) {
    *len = n;
    return PSP_OK;
  }
  if (*len < n) return fail(PSP_ERR_ARG, "buffer too small");
  size_t p = 0;
  buf[p++] = sh.nx; buf[p++] = sh.ny; buf[p++] = sh.nz; buf[p++] = X->lead[panel]; buf[p++] = sh.nsn;
  for (int f = 0; f < sh.nsn; ++f) {
    buf[p++] = sh.s[f];
    buf[p++] = sh.u[f];
    buf[p++] = sh.parent[f];
    for (int e = sh.first[f]; e < sh.first[f] + sh.s[f]; ++e) buf[p++] = sh.order[e];
    for (int64_t a = sh.struct_ptr[f]; a < sh.struct_ptr[f + 1]; ++a) buf[p++] = sh.order[sh.struct_elim[a]];
  }
  *len = n;
  return PSP_OK;
}

psp_status psp_info(psp_handle X, int* panels, int64_t* fronts, int64_t* factor_bytes) {
  if (!X) return fail(PSP_ERR_ARG, "NULL handle");
  if (panels) *panels = X->m;
  if (fronts) *fronts = X->nfronts_factored;
  if (factor_bytes) *factor_bytes = X->factor_elems * (int64_t)X->elem_bytes;
  return PSP_OK;
}

psp_status psp_export_front(psp_handle X, int panel, int sn, double* buf, int* s, int* u) {
  if (!X || panel < 0 || panel >= X->m) return fail(PSP_ERR_ARG, "bad panel");
  const Shape& sh = X->shapes[X->shape_of[panel]];
  if (sn < 0 || sn >= sh.nsn) return fail(PSP_ERR_ARG, "bad supernode");
  if (X->owner.empty() || X->owner[panel] < 0) return fail(PSP_ERR_ARG, "the panel is outside this handle's block");
  if (s) *s = sh.s[sn];
  if (u) *u = sh.u[sn];
  if (!buf) return PSP_OK;
  PSP_TRY
  check_device(X);
  const int64_t n = (int64_t)(sh.s[sn] + sh.u[sn]) * sh.s[sn];
  const char* src = X->d_factor.as<char>() + (X->panel_fbase[panel] + sh.g_off[sn]) * (int64_t)X->elem_bytes;
  if (X->elem_bytes == 16) {
    PSP_CK(cudaMemcpy(buf, src, n * 16, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> tmp(2 * n);
    PSP_CK(cudaMemcpy(tmp.data(), src, n * 8, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < 2 * n; ++i) buf[i] = tmp[i];
  }
  return PSP_OK;
  PSP_CATCH
}

psp_status psp_export_second_inverse(psp_handle X, int panel, int sn, double* buf, int* s) {
  if (!X || panel < 0 || panel >= X->m) return fail(PSP_ERR_ARG, "bad panel");
  const Shape& sh = X->shapes[X->shape_of[panel]];
  if (sn < 0 || sn >= sh.nsn) return fail(PSP_ERR_ARG, "bad supernode");
  if (X->owner.empty() || X->owner[panel] < 0) return fail(PSP_ERR_ARG, "the panel is outside this handle's block");
  if (X->si_mode != PSP_SI_TWO || !X->d_factor.p) return fail(PSP_ERR_STATE, "the handle keeps no second inverse");
  if (s) *s = sh.s[sn];
  if (!buf) return PSP_OK;
  PSP_TRY
  check_device(X);
  const int64_t n = (int64_t)sh.s[sn] * sh.s[sn];
  const int64_t off = X->panel_fbase[panel] + sh.g_off[sn] + second_inverse_offset(sh.s[sn], sh.u[sn]);
  const char* src = X->d_factor.as<char>() + off * (int64_t)X->elem_bytes;
  if (X->elem_bytes == 16) {
    PSP_CK(cudaMemcpy(buf, src, n * 16, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> tmp(2 * n);
    PSP_CK(cudaMemcpy(tmp.data(), src, n * 8, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < 2 * n; ++i) buf[i] = tmp[i];
  }
  return PSP_OK;
  PSP_CATCH
}

psp_status psp_stats(psp_handle X, psp_kernel_stat* out, int capacity, int* count, int reset) {
  if (!X || capacity < 0 || (capacity > 0 && !out)) return fail(PSP_ERR_ARG, "bad stats arguments");
  PSP_TRY
  X->stats.collect();
  int i = 0;
  for (auto& kv : X->stats.k) {
    if (i < capacity) {
      psp_kernel_stat& r = out[i];
      std::memset(&r, 0, sizeof(r));
      std::strncpy(r.name, kv.first.c_str(), sizeof(r.name) - 1);
      r.launches = kv.second.launches;
      r.total_ms = kv.second.ms;
      r.flops = kv.second.flops;
      r.bytes = kv.second.bytes;
      r.extra_flops = kv.second.extra;
    }
    ++i;
  }
  if (count) *count = i;
  if (reset)
    for (auto& kv : X->stats.k) {
      kv.second.launches = 0;
      kv.second.ms = kv.second.flops = kv.second.bytes = kv.second.extra = 0;
    }
  return PSP_OK;
  PSP_CATCH
}

psp_status psp_tune_sweep(psp_handle X, int nrhs, int reps, void* stream, psp_sweep_tuning* out) {
  if (!X || nrhs < 1 || reps < 1) return fail(PSP_ERR_ARG, "bad tuning arguments");
  if (!X->d_factor.p) return fail(PSP_ERR_STATE, "handle has no factorisation");
  PSP_TRY
  check_device(X);
  AllocScope scope(&X->allocator);
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf u;
  const size_t bytes = (size_t)X->N * nrhs * sizeof(double2);
  u.alloc(bytes);
  PSP_CK(cudaMemsetAsync(u.p, 0x3f, bytes, st));   // a fixed, finite, normal pattern
  cudaEvent_t e0, e1;
  PSP_CK(cudaEventCreate(&e0));
  PSP_CK(cudaEventCreate(&e1));
  struct Sched { int lt, cps, rg, mr, xr, ca; };
  int timed = 0;
  auto time_one = [&](const Sched& c) {
    if (c.lt != X->sweep_level_tasks || c.mr != X->sweep_min_rows || c.xr != X->sweep_max_rows) {
      X->sweep_level_tasks = c.lt;
      X->sweep_min_rows = c.mr;
      X->sweep_max_rows = c.xr;
      plan_solve(X, st);
    }
    X->sweep_ctas_per_sm = c.cps;
    X->sweep_rhs_group = c.rg;
    X->sweep_claim_ahead = c.ca;
    apply_dispatch(X, u.as<double2>(), nrhs, st);
    PSP_CK(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) apply_dispatch(X, u.as<double2>(), nrhs, st);
    PSP_CK(cudaEventRecord(e1, st));
    PSP_CK(cudaEventSynchronize(e1));
    float ms = 0;
    PSP_CK(cudaEventElapsedTime(&ms, e0, e1));
    ++timed;
    return (double)ms / reps;
  };
  const bool was_timing = X->stats.timing;
  X->stats.timing = false;
  Sched best{X->sweep_level_tasks, X->sweep_ctas_per_sm, X->sweep_rhs_group, X->sweep_min_rows, X->sweep_max_rows,
             X->sweep_claim_ahead};
  double best_ms = 0, initial_ms = 0;
  try {
    best_ms = initial_ms = time_one(best);
    auto consider = [&](Sched c) {
      const double ms = time_one(c);
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    };
    for (int xr : {64, 128, 256})
      if (xr != best.xr) consider({best.lt, best.cps, best.rg, best.mr, xr, best.ca});
    for (int lt : {152, 304, 608, 1216, 2432})
      if (lt != best.lt) consider({lt, best.cps, best.rg, best.mr, best.xr, best.ca});
    for (int cps : {2, 3, 4, 6, 8})
      if (cps != best.cps) consider({best.lt, cps, best.rg, best.mr, best.xr, best.ca});
    if (nrhs > 1)
      for (int rg : {1, 2, 4, 8})
        if (rg <= nrhs && rg != best.rg) consider({best.lt, best.cps, rg, best.mr, best.xr, best.ca});
    for (int mr : {8, 16, 32, 64})
      if (mr != best.mr) consider({best.lt, best.cps, best.rg, mr, best.xr, best.ca});
    for (int ca : {1, 2})
      if (ca != best.ca) consider({best.lt, best.cps, best.rg, best.mr, best.xr, ca});
  } catch (...) {
    X->stats.timing = was_timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  X->stats.timing = was_timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best.lt != X->sweep_level_tasks || best.mr != X->sweep_min_rows || best.xr != X->sweep_max_rows) {
    X->sweep_level_tasks = best.lt;
    X->sweep_min_rows = best.mr;
    X->sweep_max_rows = best.xr;
    plan_solve(X, st);
  }
  X->sweep_ctas_per_sm = best.cps;
  X->sweep_rhs_group = best.rg;
  X->sweep_claim_ahead = best.ca;
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->sweep_level_tasks = best.lt;
    out->sweep_ctas_per_sm = best.cps;
    out->sweep_rhs_group = best.rg;
    out->sweep_min_rows = best.mr;
    out->sweep_max_rows = best.xr;
    out->sweep_claim_ahead = best.ca;
    out->candidates = timed;
    out->initial_ms = initial_ms;
    out->best_ms = best_ms;
  }
  return PSP_OK;
  PSP_CATCH
}

psp_status psp_sweep_part(psp_handle X, double* u, int nrhs, int direction, void* stream) {
  if (!X || !u || nrhs < 1 || (direction != 0 && direction != 1)) return fail(PSP_ERR_ARG, "bad sweep-part arguments");
  if (!X->d_factor.p) return fail(PSP_ERR_STATE, "handle has no factorisation");
  if (X->probs.size() != 1) return fail(PSP_ERR_STATE, "psp_sweep_part takes single-problem handles");
  PSP_TRY
  check_device(X);
  AllocScope scope(&X->allocator);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)X->N * nrhs * sizeof(double2);
  const bool dev = is_device_pointer(u);
  double2* ud = reinterpret_cast<double2*>(u);
  if (!dev) {
    X->stage_out.ensure(bytes);
    ud = X->stage_out.as<double2>();
    PSP_CK(cudaMemcpyAsync(ud, u, bytes, cudaMemcpyHostToDevice, st));
  }
  const int plan = direction == 0 ? 1 : 2;
  if (X->prec == PSP_PREC_C64) {
    ensure_apply_ws<float2>(X, nrhs);
    apply_core<float2>(X, ud, nrhs, X->ws_xf.as<float2>(), X->ws_xb.as<float2>(), X->ws_upd.as<float2>(), true, st, plan);
  } else {
    ensure_apply_ws<double2>(X, nrhs);
    apply_core<double2>(X, ud, nrhs, X->ws_xf.as<double2>(), X->ws_xb.as<double2>(), X->ws_upd.as<double2>(), true, st,
                        plan);
  }
  if (!dev) {
    PSP_CK(cudaMemcpyAsync(u, ud, bytes, cudaMemcpyDeviceToHost, st));
    PSP_CK(cudaStreamSynchronize(st));
    if (sweep_gave_up(X, st)) return fail(PSP_ERR_TIMEOUT, "a dependency wait of the sweep gave up; u is incomplete");
  }
  return PSP_OK;
  PSP_CATCH
}

psp_status psp_plan_panels(const psp_grid* g, int pml_gamma, int panel_depth, const psp_options* opt, int* z0, int* z1,
                           double* cost, int capacity, int* m) {
  if (!g || !m || capacity < 0 || (capacity > 0 && (!z0 || !z1))) return fail(PSP_ERR_ARG, "bad plan arguments");
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || pml_gamma < 0 || panel_depth < 1) return fail(PSP_ERR_ARG, "bad grid");
  psp_options o;
  psp_status cs = check_options(opt, &o);
  if (cs != PSP_OK) return cs;
  PSP_TRY
  const int pad = o.pad_depth < 0 ? pml_gamma : o.pad_depth;
  std::vector<int> a, b, lead;
  panel_plan(g->nz, pml_gamma, panel_depth, pad, o.aux_mode, a, b, lead);
  *m = (int)a.size();
  std::map<int, double> flops_of_depth;   // box depth -> setup flops of its factorisation
  for (int i = 0; i < (int)a.size() && i < capacity; ++i) {
    z0[i] = a[i];
    z1[i] = b[i];
    if (cost) {
      const int D = lead[i] + b[i] - a[i];
      auto it = flops_of_depth.find(D);
      if (it == flops_of_depth.end()) {
        Shape sh;
        build_shape(sh, g->nx, g->ny, D, o.leaf_size);
        it = flops_of_depth.emplace(D, shape_setup_flops(sh)).first;
      }
      cost[i] = it->second;
    }
  }
  return PSP_OK;
  PSP_CATCH
}

psp_status psp_check_status(psp_handle X, void* stream) {
  if (!X) return fail(PSP_ERR_ARG, "NULL handle");
  if (!X->d_status.p) return PSP_OK;
  PSP_TRY
  check_device(X);
  if (sweep_gave_up(X, (cudaStream_t)stream))
    return fail(PSP_ERR_TIMEOUT, "a dependency wait of a sweep gave up since the last check");
  return PSP_OK;
  PSP_CATCH
}

psp_status psp_tune_setup(psp_handle X, int nrhs, int expected_applies, void* stream, psp_setup_tuning* out) {
  if (!X || nrhs < 1 || expected_applies < 0) return fail(PSP_ERR_ARG, "bad tuning arguments");
  if (!X->d_factor.p) return fail(PSP_ERR_STATE, "handle has no factorisation");
  if (X->partial) return fail(PSP_ERR_STATE, kPartialMsg);
  PSP_TRY
  check_device(X);
  AllocScope scope(&X->allocator);
  cudaStream_t st = (cudaStream_t)stream;
  struct Cand { int si, tc; };
  std::vector<Cand> cands;
  const bool tc = X->prec == PSP_PREC_C64 && X->use_tc;
  for (int si : {PSP_SI_EXTENDED, PSP_SI_PAPER, PSP_SI_NONE})
    if (tc && si != PSP_SI_NONE)
      for (int t : {32, 64, 128}) cands.push_back({si, t});
    else
      cands.push_back({si, X->tc_min_dim});
  const Cand initial{X->si_mode, X->tc_min_dim};
  DevBuf u;
  const size_t bytes = (size_t)X->N * nrhs * sizeof(double2);
  u.alloc(bytes);
  cudaEvent_t e0, e1;
  PSP_CK(cudaEventCreate(&e0));
  PSP_CK(cudaEventCreate(&e1));
  struct EventGuard {
    cudaEvent_t a, b;
    ~EventGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } eg{e0, e1};
  const bool was_timing = X->stats.timing;
  X->stats.timing = false;
  struct TimingGuard {
    psp_ctx_s* X;
    bool was;
    ~TimingGuard() { X->stats.timing = was; }
  } tg{X, was_timing};
  // setup (host and device, the factorisation synchronises) and one application after a warm one
  auto time_one = [&](const Cand& c, double& setup_ms, double& apply_ms) {
    X->si_mode = c.si;
    X->tc_min_dim = c.tc;
    const auto t0 = std::chrono::steady_clock::now();
    finish_setup(X, st);
    setup_ms = ms_since(t0);
    PSP_CK(cudaMemsetAsync(u.p, 0x3f, bytes, st));   // a fixed, finite, normal pattern
    apply_dispatch(X, u.as<double2>(), nrhs, st);
    PSP_CK(cudaEventRecord(e0, st));
    apply_dispatch(X, u.as<double2>(), nrhs, st);
    PSP_CK(cudaEventRecord(e1, st));
    PSP_CK(cudaEventSynchronize(e1));
    float ms = 0;
    PSP_CK(cudaEventElapsedTime(&ms, e0, e1));
    apply_ms = ms;
  };
  Cand best = initial;
  double best_total = 0, initial_total = 0, best_setup = 0, best_apply = 0;
  int tried = 0;
  for (const Cand& c : cands) {
    double sm = 0, am = 0;
    time_one(c, sm, am);
    ++tried;
    const double total = sm + (double)expected_applies * am;
    if (c.si == initial.si && c.tc == initial.tc) initial_total = total;
    if (tried == 1 || total < best_total) {
      best_total = total;
      best = c;
      best_setup = sm;
      best_apply = am;
    }
  }
  if (X->si_mode != best.si || X->tc_min_dim != best.tc) {   // keep the factorisation of the best choice
    X->si_mode = best.si;
    X->tc_min_dim = best.tc;
    finish_setup(X, st);
  }
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->selective_inversion = best.si;
    out->tc_min_dim = best.tc;
    out->candidates = tried;
    out->setup_ms = best_setup;
    out->apply_ms = best_apply;
    out->initial_total_ms = initial_total;
    out->best_total_ms = best_total;
  }
  return PSP_OK;
  PSP_CATCH
}

psp_status psp_destroy(psp_handle X) {
  if (!X) return PSP_OK;
  delete X;
  return PSP_OK;
}

}  // extern "C"

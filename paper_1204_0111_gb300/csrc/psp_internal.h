// Internal declarations shared by the translation units of libpsp.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "psp.h"

struct psp_ctx_s;

namespace psp {

// sweep with caller-provided work vectors (defined in psp_api.cu)
size_t apply_workspace_bytes(const psp_ctx_s* X, int nrhs);
psp_status apply_with_workspace(psp_ctx_s* X, double2* u, int nrhs, void* ws, cudaStream_t st);
int64_t handle_points(const psp_ctx_s* X);   // N, or -1 when the handle has no factorisation
int handle_device(const psp_ctx_s* X);       // CUDA device the handle was set up on
psp_status set_error(psp_status s, const char* msg);

// ---------------------------------------------------------------------------
// Symbolic analysis of one auxiliary-problem box (nx x ny x depth): the
// supernodal nested-dissection tree of §2.1 (separator-tree figure), postorder.
// ---------------------------------------------------------------------------
struct Shape {
  int nx = 0, ny = 0, nz = 0;  // box extents (nz = depth of the auxiliary problem)
  int leaf = 0;
  int nsn = 0;
  std::vector<int32_t> order;       // elimination index -> box node id
  std::vector<int32_t> elim;        // box node id -> elimination index
  std::vector<int32_t> first;       // nsn + 1: elimination index of each supernode's first node
  std::vector<int32_t> s, u;        // supernode size, |struct(S)|
  std::vector<int32_t> parent;      // -1 for the root
  std::vector<int32_t> child_ptr, child_idx;
  std::vector<int64_t> struct_ptr;  // nsn + 1 offsets into struct_elim / rel
  std::vector<int32_t> struct_elim; // struct(S) as sorted elimination indices
  std::vector<int32_t> rel;         // position of each struct entry in the parent's front rows
  std::vector<int32_t> height;      // leaves 0, parent = 1 + max(children)
  int nlevels = 0;
  std::vector<std::vector<int32_t>> level_sns;
  std::vector<int32_t> depth;       // root 0, child = parent + 1
  int ndepths = 0;
  // solve-side pull map: for each front row position p of S u struct(S), up to two
  // offsets (within the per-panel update-vector slab) of children's update entries
  std::vector<int64_t> pull_ptr;    // nsn + 1, = sum (s + u)
  std::vector<int32_t> pull;        // 2 per position, -1 = none
  // per-panel layouts
  std::vector<int64_t> g_off;       // G block offset within a panel's factor slab (elements)
  int64_t g_total = 0;
  std::vector<int64_t> upd_off;     // update-vector offset within the panel's update slab
  int64_t upd_total = 0;
};

void build_shape(Shape& sh, int nx, int ny, int nz, int leaf);

// ---------------------------------------------------------------------------
// Device views
// ---------------------------------------------------------------------------
struct ShapeDev {
  int nx, ny, nz, nsn;
  const int32_t* order;
  const int32_t* elim;
  const int32_t* first;
  const int32_t* s;
  const int32_t* u;
  const int32_t* child_ptr;
  const int32_t* child_idx;
  const int64_t* struct_ptr;
  const int32_t* struct_elim;
  const int32_t* rel;
  const int64_t* pull_ptr;
  const int32_t* pull;
  const int64_t* g_off;
  const int64_t* upd_off;
  const int32_t* parent;
};

// 7-point operator on a box: -sum_j d_j(a_j d_j u) - k2num / c^2 * s1 s2 s3 u (Eq. (1.1)/(1.5),
// s1 s2 s3-scaled).  Stretch tables are complex; half[k] sits between node k-1 and node k.
struct BoxOp {
  int nx, ny, nz;
  double inv_h2;
  double2 k2num;            // omega^2 (A) or (omega + i alpha)^2 (J)
  const double* c;          // global wave speed, nx*ny*nz_global
  const int32_t* cplane;    // box plane -> global plane whose c is used
  const double2* s1n;
  const double2* s1h;
  const double2* s2n;
  const double2* s2h;
  const double2* s3n;
  const double2* s3h;
};

// One panel's auxiliary problem (Alg. 1.4) as seen by the apply kernels.
struct PanelDev {
  int z0, z1, lead;         // global planes [z0, z1); lead pad (or exact-mode) planes before them
  int shape;
  int64_t sn_base;          // global front id of supernode 0
};

enum GemmFlags : int {
  GF_BETA0 = 1,           // C = alpha * A B^T (do not read C)
  GF_C_LOWER = 2,         // write only local row >= local col (diagonal tiles)
  GF_B_NN = 4,            // B(n,k) = B[k + n ldb]   (default NT: B[n + k ldb])
  GF_B_UNIT_LOWER_NT = 8, // B(n,k) is T[n,k] of a unit lower T stored with D on its diagonal
  GF_B_UNIT_LOWER_NN = 16,// B(n,k) is T[k,n] of a unit lower T stored with D on its diagonal
  GF_D_MUL = 32,          // scale A(:,k) by d(k)
  GF_D_DIV = 64,          // scale A(:,k) by 1/d(k)
  GF_NEG = 128,           // alpha = -1 (else +1)
  GF_SI = 256             // selective-inversion work (inv(L_TL), M_BL): host accounting only, kernels ignore it
};

// C(m x n) (+)= alpha * A(m x k) * diag(d)^{+-1} * B(n x k)^T ; pointers already offset.
template <typename T>
struct GemmTask {
  T* C;
  const T* A;
  const T* B;
  const T* d;
  int ldc, lda, ldb, ldd;
  int m, n, k;
  int kg0, ng0;   // global k / n index of the first element (for the unit-lower masks)
  int flags;
  int pad_;
};

// Update matrices F_BR (u x u, symmetric) keep only their lower tiles: tiles of ut x ut (ut = 64 for
// fronts whose products run on CUDA cores, 128 for tensor-core fronts), tile (I, J), I >= J, stored
// column of tiles after column of tiles, each tile column-major with leading dimension ut.
__host__ __device__ __forceinline__ int64_t upd_tile_offset(int64_t I, int64_t J, int64_t ntiles, int ut) {
  return (J * ntiles - J * (J - 1) / 2 + (I - J)) * (int64_t)ut * ut;
}
__host__ __device__ __forceinline__ int64_t upd_index(int r, int c, int u, int ut) {   // r >= c; ut 64 or 128
  const int sh = ut == 128 ? 7 : 6;
  const int nt = (u + ut - 1) >> sh;
  return upd_tile_offset(r >> sh, c >> sh, nt, ut) + ((int64_t)(c & (ut - 1)) << sh) + (r & (ut - 1));
}
__host__ __device__ __forceinline__ int64_t upd_packed_elems(int u, int ut) {
  const int64_t nt = (u + ut - 1) / ut;
  return nt * (nt + 1) / 2 * (int64_t)ut * ut;
}

// A front in a level batch.
template <typename T>
struct FrontTask {
  T* G;        // (s+u) x s, ld = s+u
  T* U;        // u x u update (F_BR) in lower tiles of ut x ut (upd_index); nullptr for the root
  T* W;        // s x s work: inv(L_TL) under construction
  T* Z;        // u x s work: F_BL L^{-T}
  T* ZD;       // u x s: Z D^{-1}, leading dimension ldzd (a work block for the extended selective
               // inversion of CUDA-core fronts, G's bottom block when L_BL itself is stored; else nullptr)
  T* W2;       // s x s work: the second inverse of L_TL under construction (two-inverse form), else nullptr
  int s, u;
  int panel, sn;
  int64_t gfid;
  int ut, ldzd;   // tile size of U; leading dimension of ZD
};

// elements from a front's G block to its second inverse of L_TL (two-inverse form): G padded to 16
__host__ __device__ __forceinline__ int64_t second_inverse_offset(int64_t s, int64_t u) {
  return ((s + u) * s + 15) / 16 * 16;
}

struct ColTask {   // a chunk of columns / rows of one front
  int front;       // index into the level's FrontTask array
  int c0, c1;
};

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
void launch_matvec(const BoxOp& op, const double2* x, double2* y, int nrhs, int64_t N, cudaStream_t st);
void launch_scale_rhs(const BoxOp& op, const double2* f, double2* b, int nrhs, int64_t N, cudaStream_t st);

template <typename T>
void launch_assemble_impl(const FrontTask<T>* fronts, const ColTask* tasks, int ntasks, const ShapeDev* shapes,
                          const BoxOp* boxops, T* const* upd_ptr, const int32_t* upd_tile, const int32_t* panel_shape,
                          cudaStream_t st);
template <typename T>
void launch_diag_ldlt(const FrontTask<T>* fronts, const int* list, int nlist, int kb, double tiny, int* status, bool wide,
                      cudaStream_t st);
template <typename T>
void launch_panel_right(const FrontTask<T>* fronts, const ColTask* tasks, int ntasks, int kb, bool wide, cudaStream_t st);
template <typename T>
void launch_panel_left(const FrontTask<T>* fronts, const ColTask* tasks, int ntasks, int kb, bool wide, cudaStream_t st);
template <typename T>
void launch_panel_rsolve(const FrontTask<T>* fronts, const ColTask* tasks, int ntasks, int kb, bool wide, cudaStream_t st);
template <typename T>
void launch_gemm(const GemmTask<T>* tasks, int ntasks, cudaStream_t st);
// tensor-core path (complex64): operands packed once per front into TF32 planes, then tiles
enum TcPackMode { TC_PACK_PLAIN = 0, TC_PACK_UNIT_LOWER = 1, TC_PACK_UNIT_LOWER_T = 2 };
struct TcPackTask {        // one 128-row x 16-k block of a packed operand
  const float2* src;       // column-major source, ld
  const float2* d;         // PLAIN only: divide column k by d[k * ldd] (nullptr: no scaling)
  void* dst;               // 48 KB destination block
  int ld, ldd;
  int r0, k0;              // first row / k of the block
  int R, K;                // source extents (rows, k); outside -> 0
  int mode;                // TcPackMode: PLAIN X[r, k]; UNIT_LOWER T[r, k]; UNIT_LOWER_T T[k, r]
  int pad_;
};
struct TcGemmTask {        // one 128 x 128 tile of C (+)= +-A B^T from packed blocks
  const unsigned char* A;  // packed A row block (k-blocks contiguous)
  const unsigned char* B;  // packed B row block
  float2* C;
  int ldc, m, n;
  int kb0, nkb;            // k-blocks [kb0, kb0 + nkb)
  int flags;               // GF_NEG, GF_BETA0, GF_C_LOWER
};
void launch_tc_pack(const TcPackTask* tasks, int ntasks, cudaStream_t st);
void launch_tc_gemm(const TcGemmTask* tasks, int ntasks, int* status, cudaStream_t st);
int tc_block_k();
int64_t tc_block_bytes();
int tc_gemm_tile();
template <typename T>
void launch_copy_linv(const FrontTask<T>* fronts, const ColTask* tasks, int ntasks, cudaStream_t st);
template <typename T>
void launch_scale_zd(const FrontTask<T>* fronts, const ColTask* tasks, int ntasks, cudaStream_t st);

// ---- multifrontal solve of one panel (Alg. 1.3 inside Alg. 1.5) ----
struct SolveTask {  // rows [r0, r1) of front sn (forward) or columns [r0, r1) of S (backward)
  int sn, r0, r1;
};

template <typename T>
struct SolveCtx {
  ShapeDev sh;
  const T* G;              // this panel's factor slab
  T* xf;                   // box vector after L^{-1} and D^{-1} (elimination order), ld = n_loc
  T* xb;                   // box vector after L^{-T}
  T* upd;                  // children's update vectors, ld = upd_ld
  double2* u;              // global vector block, ld = N
  int64_t N, n_loc, upd_ld;
  int nrhs;
  int z0, z1, lead, nz;    // panel planes, pad planes, global plane count
  int mode;                // 0: forward sweep (u_i := T_i(u_i - J_{i,i-1} u_{i-1})); 1: backward (u_i -= T_i J^T u_{i+1})
  int has_prev, has_next;
  int si;                  // psp_si_mode of the factors (what G keeps)
  const double2* s1n;      // global stretch tables for the plane coupling J_{i+1,i}
  const double2* s2n;
  const double2* s3h;
  double inv_h2;
};

// phase 0: the single pass (extended factors) or first phase of a front; phase 1: its second phase
template <typename T>
void launch_solve_fwd(const SolveTask* tasks, int ntasks, const SolveCtx<T>& cx, int R, int smax, int phase,
                      cudaStream_t st);
template <typename T>
void launch_solve_bwd(const SolveTask* tasks, int ntasks, const SolveCtx<T>& cx, int ldmax, int phase, cudaStream_t st);

// ---- the whole sweep in one cooperative launch ----
struct SweepStep {      // one panel solve of Alg. 1.5, in order
  int panel, mode;      // mode 0: forward sweep (assign), 1: backward sweep (subtract)
  int prob;             // problem of a batch (0 for a single problem)
};
// per problem of a batch: where its vectors sit and its coupling tables
struct ProblemSweep {
  int64_t off1;         // offset of the problem's block in a batched vector, per right-hand side
  int64_t N;            // points of the problem
  const double2* s1n;
  const double2* s2n;
  const double2* s3h;
  double inv_h2;
  int nz, pad_;
};
struct PanelSweep {
  int64_t gbase;        // factor slab offset (elements)
  int shape, z0, z1, lead, has_prev, has_next;
};
struct LevelSweep {
  int64_t fwd_off, bwd_off;
  int nfwd, nbwd, R, pad_;
};
// one entry of the sweep's task queue (topological order: panel solves in Alg. 1.5 order; inside
// one, the up-the-tree tasks level by level, then the down-the-tree tasks from the root).  An entry
// carries its one dependency and the counters it signals, so that a CTA takes a task with a single
// 48-byte read.  Counters are words of the sweep's counter array (zeroed before every sweep):
//   [0] dequeue head, [1, 5) status, then per step the tasks completed, then per step and front the
//   up tasks completed, the down tasks completed and the up tasks of the front's children completed.
struct QueueEntry {
  int step;                     // panel solve index
  int sn, r0, r1;               // the task: rows (up) or columns (down) [r0, r1) of front sn
  int wait;                     // counter the task waits for (-1: none) ...
  unsigned target;              // ... until it reaches this count
  int done;                     // counter of the front's own completed tasks (this direction)
  int kids;                     // counter of the parent's children's completed up tasks (-1: none)
  short dir;                    // 0 up the tree, 1 down the tree; 2 / 3 the second phase up / down of a front
                                // whose factor keeps L_BL (the first phase is then 0 / 1)
  short R;                      // rows per up-the-tree task
  int pad_[3];
};
static_assert(sizeof(QueueEntry) == 48, "queue entries are copied as three 16-byte words");
// second phases of a front (factors that keep L_BL rather than L_BL inv(L_TL))
constexpr int kDirUpB = 2, kDirDownB = 3;
constexpr int kSweepStepCounters = 5;   // first word of the per-step counters
template <typename T>
struct SweepArgs {
  SolveCtx<T> cx;               // fields common to every panel (vectors, sizes, coupling tables); for a batch
                                // (nprobs > 1) the vector and work-vector bases, offset per problem
  int nshapes, nsteps, npanels; // sizes of the three tables below (kept in shared memory)
  const SweepStep* steps;
  const PanelSweep* panels;
  const ShapeDev* shapes;
  const T* factor;
  const QueueEntry* queue;
  int nqueue;
  unsigned* ctr;                // counter array (layout above)
  int* status;                  // status[2] set when a wait gave up (= ctr + 1)
  int* sticky;                  // also set then; kept until the host reads it (psp_check_status)
  // batches of independent problems (nprobs > 1): each problem's steps form their own chain
  int nprobs;
  const ProblemSweep* probs;    // per problem; cx's vectors and work vectors are offset per problem
  int chunk;                    // vector entries a task stages in shared memory at a time (set by launch_sweep)
  int claim_ahead;              // 2: a CTA holds the two tasks after the one it runs; 1: the next one only
};
// returns 0 on success, -1 when a cooperative launch is not possible, else a cudaError_t; smax / ldmax:
// the widest front's s and s + u
template <typename T>
int launch_sweep(const SweepArgs<T>& args, int smax, int ldmax, int max_per_sm, int rhs_group, cudaStream_t st);

// ---- GMRES helpers (complex128) ----
// A block of vectors holds ncol columns (right-hand sides, and problems of a batch); column c of
// every vector of the block is the span [off, off + len).
struct ColSpan {
  int64_t off, len;
};
// out[i * ncol + c] = sum_g conj(V_i[c][g]) w[c][g], V_i = V + i * ldv_vec; fixed two-stage order
void launch_multidot(const double2* V, int64_t ldv_vec, int nvec, const double2* w, const ColSpan* cols, int ncol,
                     int64_t maxlen, double2* partial, double2* out, cudaStream_t st);
int multidot_blocks(int64_t maxlen);   // partial blocks per column (size partial as blocks * nvec * ncol)
// w[c] += sign * sum_i h[i * ncol + c] V_i[c]
void launch_multiaxpy(const double2* V, int64_t ldv_vec, int nvec, const double2* h, double2* w, const ColSpan* cols,
                      int ncol, int64_t maxlen, double sign, cudaStream_t st);
// y[c] = alpha_c x[c] (mode 0), y[c] = x[c] - y[c] (mode 1), y[c] += alpha_c x[c] (mode 2)
void launch_axpby_batch(const double2* x, double2* y, const ColSpan* cols, int ncol, int64_t maxlen,
                        const double2* alpha, int alpha_mode, cudaStream_t st);

// Hessenberg least-squares state, one column block per right-hand side
struct LsqState {
  double2* H;        // (k+1) x k per rhs, column-major, ld = k+1
  double* cs;        // k per rhs
  double2* sn;       // k per rhs
  double2* g;        // k+1 per rhs
  double* resid;     // |g_{j+1}| per rhs
  double2* scl;      // scale of the next basis vector per rhs (0 when inactive)
  const int* active; // 1 while the rhs iterates
  int k, nrhs;
};
void launch_arnoldi_step(const LsqState& L, int j, const double2* h1, const double2* h2, const double2* nrm2,
                         cudaStream_t st);
void launch_backsolve(const LsqState& L, const int* jr, double2* y, cudaStream_t st);
void launch_cycle_start(const LsqState& L, const double2* nrm2, cudaStream_t st);

}  // namespace psp

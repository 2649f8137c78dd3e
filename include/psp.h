/*
 * psp.h - C ABI of the GB300 (sm_103a) moving-PML sweeping preconditioner.
 *
 * Poulson, Engquist, Li, Ying, "A parallel sweeping preconditioner for
 * heterogeneous 3D Helmholtz equations" (arXiv:1204.0111).
 *
 * Problem (§1, Eq. (1.1)): the Helmholtz operator A = -Laplacian - omega^2/c(x)^2
 * on the interior grid nx x ny x nz (spacing h, node (i1,i2,i3) at
 * ((i1+1)h, (i2+1)h, (i3+1)h), unknown index i1 + i2 nx + i3 nx ny), second
 * order 7-point differences, PML of pml_gamma points on the faces selected by
 * psp_options.pml_faces, homogeneous Dirichlet beyond.  The library works with
 * the symmetric form multiplied through by s1 s2 s3 (s_j = 1 + i sigma_j/omega):
 *     A_s u = s1 s2 s3 f,
 * which is complex symmetric (§1.1).  The preconditioner is built from the
 * damped operator J of Eq. (1.5) (omega -> omega + i alpha in the mass term).
 *
 * Conventions for every entry point:
 *  - Complex vectors are interleaved (re, im) doubles.  A block of nrhs vectors
 *    of length N = nx ny nz is column-major: vector r starts at element r*N.
 *  - Pointers may be DEVICE pointers (cudaMalloc'd / torch CUDA tensors) or
 *    HOST pointers; the library inspects each pointer and stages host data
 *    through device memory itself (on the given stream, synchronising it
 *    before returning host results).  The caller keeps ownership of all
 *    buffers it passes; the library owns everything behind a psp_handle.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work is
 *    ordered on it.  Calls returning host data synchronise the stream.
 *  - No exception or abort crosses the ABI: every call returns a psp_status.
 *    psp_last_error() returns a thread-local message for the last failure.
 *    A handle stays destroyable after any error.
 *  - A handle must not be used from two host threads at once.
 *  - A handle belongs to the CUDA device that was current when it was set up: every later call
 *    must run with that device current and pass device pointers of that device (or host
 *    pointers); otherwise it returns PSP_ERR_ARG.
 *  - The sweep's dependency waits are bounded (about two seconds).  A wait that gives up leaves
 *    that application's output incomplete and raises a flag that stays set until it is reported:
 *    by psp_apply with a host `out` (which synchronises), by psp_solve, or by psp_check_status.
 *    Calls that only enqueue work on device pointers return before the sweep has run and cannot
 *    report it themselves.
 */
#ifndef PSP_H
#define PSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct psp_ctx_s* psp_handle;

typedef enum {
  PSP_OK = 0,
  PSP_ERR_ARG = 1,            /* invalid argument (size, NULL pointer, option out of range) */
  PSP_ERR_OOM = 2,            /* device or host allocation failed */
  PSP_ERR_CUDA = 3,           /* a CUDA runtime call failed; see psp_last_error() */
  PSP_ERR_ZERO_PIVOT = 4,     /* an unpivoted LDL^T pivot fell below the threshold */
  PSP_ERR_NOT_CONVERGED = 5,  /* GMRES hit maxit before reaching tol */
  PSP_ERR_TIMEOUT = 6,        /* a bounded device wait gave up */
  PSP_ERR_STATE = 7           /* handle not in a state that allows the call */
} psp_status;

typedef struct {
  int nx, ny, nz; /* interior points per axis, >= 1 */
  double h;       /* grid spacing, > 0 */
} psp_grid;

typedef enum {
  PSP_PREC_C128 = 0,  /* fronts and sweeps in complex128 (FP64 CUDA cores) */
  PSP_PREC_C64 = 1    /* fronts and sweeps in complex64; GMRES and matvec stay complex128 */
} psp_precision;

/* What the factor of each front keeps (§2.2): after the partial LDL^T of the front
   F = [F_TL F_BL^T; F_BL F_BR], L_TL D L_TL^T = F_TL and L_BL = F_BL L_TL^{-T} D^{-1}. */
typedef enum {
  PSP_SI_EXTENDED = 0, /* G = [inv(L_TL); L_BL inv(L_TL)]: selective inversion extended to the bottom block, so
                          each front is one matrix-vector product per sweep direction (default) */
  PSP_SI_PAPER = 1,    /* G = [inv(L_TL); L_BL]: the paper's selective inversion; each front takes two dependent
                          products per direction, and setup skips the u s^2 / 2 products of L_BL inv(L_TL) */
  PSP_SI_NONE = 2,     /* G = [L_TL; L_BL]: no inversion; the sweep solves with L_TL by substitution, one CTA
                          per front (complex64 fronts stay on CUDA cores) */
  PSP_SI_TWO = 3       /* the paper's G = [inv(L_TL); L_BL] plus a second inverse of L_TL (§2.2, last
                          paragraph: one inverse by columns, one by rows).  The first is built column by
                          column (forward substitution, L X = I) and applied up the tree as inv(L_TL) w;
                          the second row by row (backward substitution, X L = I) and applied down the
                          tree as inv(L_TL)^T t, so each direction applies an inverse whose vectors were
                          computed by a backward-stable solve.  s x s more factor storage per front */
} psp_si_mode;

typedef enum {
  PSP_AUX_MOVING_PML = 0, /* H_i = PML pad + panel (Alg. 1.4): the preconditioner */
  PSP_AUX_EXACT = 1       /* H_i = all planes below the panel's top (Fig. 2 middle): M = J exactly */
} psp_aux_mode;

/* Options; psp_default_options() fills the defaults shown. */
typedef struct {
  double pml_C;       /* PML amplitude "C" (§3) of the stretch sigma = (C / (gamma h)) t^2, default 4.0;
                         a wave of speed c decays by exp(-C / (3 c)) across the layer, so in media
                         faster than 1 pass the amplitude times the fastest speed */
  double alpha;       /* damping of Eq. (1.5), default 2*pi */
  int pad_depth;      /* artificial PML planes prefixed to each panel (Alg. 1.4); -1 = pml_gamma */
  int leaf_size;      /* nested-dissection leaf: boxes with nx*ny*depth <= leaf are leaves; default 64 */
  int precision;      /* psp_precision, default PSP_PREC_C128 */
  int pml_faces;      /* bit mask x-lo 1, x-hi 2, y-lo 4, y-hi 8, z-lo 16, z-hi 32; default 63 */
  int aux_mode;       /* psp_aux_mode, default PSP_AUX_MOVING_PML */
  int collect_stats;  /* CUDA-event timing of launches (psp_stats): 0 none (default), 1 every kernel,
                         2 the setup kernels only (a few hundred launches per setup) */
  int tensor_cores;   /* complex64 path: 1 (default) runs the Schur update and the selective-inversion
                         multiplies on tcgen05 tensor cores, 0 keeps them on CUDA cores */
  int tc_min_dim;     /* complex64 path: fronts with s >= tc_min_dim and u >= tc_min_dim take the tensor
                         cores, the others CUDA cores; <= 0 selects the default (64) */
  int sweep_level_tasks; /* sweep schedule: tasks a tree level is split into at least (row / column
                            blocks of 8..64); <= 0 selects the default (608) */
  int sweep_ctas_per_sm; /* sweep schedule: resident CTAs per SM of the persistent sweep (capped by
                            occupancy); <= 0 selects the default (8) */
  int setup_temp_mb;   /* cap, in MiB, on the per-front temporaries of one batch of fronts during setup
                          (a level whose fronts need more is factored in several batches); <= 0: up
                          to 80 % of the device memory left after the factors and update matrices */
  int sweep_rhs_group; /* sweep schedule: most right-hand sides (1, 2, 4 or 8) one CTA carries through a
                          pass over a factor block; <= 0: as many as the application has, at most 8 (the
                          task's vector is staged through 64 KB of shared memory in chunks) */
  int solve_rhs_group; /* psp_solve: most right-hand sides per GMRES run; <= 0: as many as fit the free
                          device memory (single-problem handles) */
  int sweep_min_rows;   /* sweep schedule: fewest rows (up) / columns (down) of a front per task, 8 .. 64;
                           <= 0 selects the default (8).  Each task gathers its front's vector for every
                           right-hand side, so with many right-hand sides wider tasks gather less */
  int test_sweep_stall; /* tests only: 1 makes one dependency of the persistent sweep impossible to
                           meet, so its bounded wait (about 2 s) gives up; psp_solve then returns
                           PSP_ERR_TIMEOUT and the device stays usable.  0 (default): off */
  int gmres_basis;      /* psp_solve: 1 keeps z_j = M^{-1} v_j for every Krylov vector (2k + 1 vectors per
                           right-hand side); 2 keeps V only and forms x += M^{-1}(V y) with one more
                           application per restart cycle (k + 2 vectors); 0 (default): 1 when every
                           right-hand side fits in one run, else whichever needs fewer runs */
  int factor_every_panel; /* 0 (default): panels whose auxiliary problems are identical (same depth and
                             pad, bitwise the same x3-stretch and wave speed on every plane, as in a
                             model invariant along x3, §3) share one factorisation; 1: factor each */
  int panel_begin;      /* first panel of the block this handle factors and sweeps (one GPU's share of a
                           multi-GPU sweep, see psp_sweep_part), default 0 */
  int panel_count;      /* panels in that block; 0 (default): through the last panel.  A handle holding
                           a proper block takes psp_sweep_part, not psp_apply / psp_solve */
  /* Device memory of the handle (factors, update matrices, work vectors, tables): when both are
     given, every allocation the library makes for this handle calls dev_alloc(bytes, alloc_ctx) and
     every release dev_free(ptr, alloc_ctx), so a framework's allocator can own that memory; NULL
     (default): cudaMalloc / cudaFree.  dev_alloc returns device memory of the current device aligned
     to 256 bytes, or NULL, which the call reports as PSP_ERR_OOM.  It is called from the thread
     that calls the library, outside any kernel; memory is handed back with dev_free only after the
     work using it has finished.  One given without the other is PSP_ERR_ARG. */
  void* (*dev_alloc)(size_t bytes, void* ctx);
  void (*dev_free)(void* ptr, void* ctx);
  void* alloc_ctx;
  int selective_inversion; /* psp_si_mode, default PSP_SI_EXTENDED */
  int c64_diag_fp64;    /* complex64 factors only: 1 factors each 32 x 32 diagonal block of F_TL, and
                           solves against it (the rows of L_BL and the block rows of inv(L_TL), §2.2),
                           in complex128 arithmetic, rounding to complex64 only when storing; the
                           products between blocks stay complex64.  0 (default): all complex64 */
  int sweep_max_rows;   /* sweep schedule: most rows (up the tree) or columns (down) of a front per task,
                           64 .. 256: a level whose fronts outnumber the CTAs takes whole fronts of up
                           to this many rows per task, gathering each front's vector once; <= 0
                           selects the default (256) */
  int sweep_claim_ahead; /* sweep schedule: queue tasks a CTA of the persistent sweep holds besides the
                            one it runs, 1 or 2.  2 claims the task after next while a task waits and
                            runs, so the next one's queue entry is in shared memory when it is done;
                            1 claims the next task only as a task starts waiting, so a task claimed by
                            a busy CTA waits behind one task rather than two (measured faster on
                            most workloads).  <= 0 selects the default (1).  The results do not
                            depend on it */
} psp_options;

/* Per-solve report filled by psp_solve (host struct). */
typedef struct {
  int iterations;      /* total inner GMRES iterations, max over right-hand sides */
  int restarts;        /* restart cycles, max over right-hand sides */
  int converged;       /* 1 if every right-hand side reached tol */
  int applies;         /* preconditioner applications issued */
  double relres_max;   /* max over rhs of the true ||b - A_s u|| / ||b||, b = s1 s2 s3 f */
  double solve_ms;     /* wall time of the solve (host clock, stream synchronised) */
  int status_front;    /* front id of a zero pivot, -1 if none */
  int groups;          /* GMRES runs the right-hand sides were solved in (1 unless their Krylov bases
                          did not fit the free device memory together) */
  double min_pivot_abs; /* smallest |d_jj| of the handle's LDL^T factorisation (the pivot monitor of the
                           unpivoted factorisation, §2.5: the solver does no pivoting) */
  int reserved[4];
} psp_solve_info;

void psp_default_options(psp_options* opt);

/*
 * psp_setup - Alg. 1.4 (§1.1): plan the m panels (panel 0 = planes [0, gamma+d),
 * then d planes each, the last one taking the remainder), form every PML-padded
 * auxiliary problem H_i, and factor all of them with the supernodal
 * nested-dissection multifrontal LDL^T of §2.1-§2.2 (unpivoted, complex symmetric),
 * followed by selective inversion of every front (§2.2).
 *
 *   g            grid (host struct)
 *   c            wave speed c(x) > 0, N doubles, x fastest (host or device)
 *   omega        angular frequency > 0
 *   pml_gamma    PML points gamma >= 0 on each selected face
 *   panel_depth  planes per panel d >= 1
 *   opt          options or NULL for defaults
 *   out          receives the new handle (owned by the library until psp_destroy)
 * Errors: PSP_ERR_ARG, PSP_ERR_OOM, PSP_ERR_CUDA, PSP_ERR_ZERO_PIVOT (|d| < 1e-300
 * for complex128, < 1e-30 for complex64; *out is still set and must be destroyed).
 * The c array is copied; the caller may free it after the call returns.
 */
psp_status psp_setup(const psp_grid* g, const double* c, double omega, int pml_gamma, int panel_depth,
                     const psp_options* opt, void* stream, psp_handle* out);

/*
 * psp_setup_batch - psp_setup for nprob independent problems (own grid, c, omega, gamma and panel
 * depth each; one options struct for all, pad_depth < 0 meaning each problem's own gamma) in one
 * handle.  The panels of every problem are factored together: each tree level of all problems'
 * fronts is one batch of launches (§2.1: the panels' factorisations are independent), and each
 * application runs the problems' sweeps (Alg. 1.5) side by side in one persistent launch.
 *
 *   grids, c, omega, pml_gamma, panel_depth   arrays of nprob entries; c[q] as for psp_setup
 *   out          receives the handle
 * The handle's vectors are batched: with nrhs right-hand sides per problem, a vector block holds
 * problem 0's N_0 x nrhs block (column per right-hand side, x fastest), then problem 1's, and so
 * on (psp_batch_layout gives the N_q).  psp_apply, psp_apply_noalloc, psp_matvec and psp_solve take
 * such blocks (their nrhs is per problem); psp_solve runs one GMRES(k) per problem and right-hand
 * side, in lockstep.  Panel indices of psp_symbolic_export and psp_export_front count all
 * problems' panels in order.  Errors as for psp_setup, PSP_ERR_ARG for a bad entry of any array.
 */
psp_status psp_setup_batch(int nprob, const psp_grid* grids, const double* const* c, const double* omega,
                           const int* pml_gamma, const int* panel_depth, const psp_options* opt, void* stream,
                           psp_handle* out);

/*
 * psp_batch_layout - the number of problems of a handle (1 for psp_setup) and, in points[0 ..
 * capacity), each problem's point count N_q.  Errors: PSP_ERR_ARG for a NULL handle or a
 * negative capacity, or points NULL with capacity > 0.
 */
psp_status psp_batch_layout(psp_handle h, int* nprob, int64_t* points, int capacity);

/*
 * psp_apply - Alg. 1.5: out = M^{-1} rhs, a forward sweep u_i := T_i u_i,
 * u_{i+1} -= J_{i+1,i} u_i and a backward sweep u_i -= T_i(J_{i+1,i}^T u_{i+1}),
 * with T_i the Alg. 1.3 application of the factored H_i (extend by zero over the
 * pad, multifrontal solve, keep the panel's planes).  rhs and out are nrhs
 * complex vectors of length N (host or device); out may alias rhs.
 * With a host `out` the call synchronises the stream and returns PSP_ERR_TIMEOUT if a dependency
 * wait of the sweep gave up; with a device `out` it returns once the work is enqueued, and a give-up
 * is reported by the next psp_solve or psp_check_status.
 */
psp_status psp_apply(psp_handle h, const double* rhs, double* out, int nrhs, void* stream);

/*
 * psp_apply_noalloc - the same result as psp_apply, computed without allocating device memory.
 * The paper has no counterpart; this entry point exists for callers that cannot allocate while
 * they run: a process whose framework allocator already holds the free device memory (a cudaMalloc
 * would fail although the caller has room), a process held to a fixed device-memory budget, or a
 * loop timed as one stream-ordered region in which a cudaMalloc would synchronise the device.
 * psp_apply grows its work vectors on demand; this call never calls cudaMalloc, cudaFree or any
 * other allocating routine.
 *  - Work vectors (two box vectors per panel and the fronts' update vectors, per right-hand side)
 *    live in one file-scope device array of 16 MiB that every GPU context loading the library
 *    reserves until the process exits.  When a problem needs more for the given nrhs the call
 *    returns PSP_ERR_ARG with the size it needs; use psp_apply then.
 *  - rhs and out are DEVICE pointers of the handle's device (N x nrhs, as for psp_apply; out may
 *    alias rhs).  Host pointers are rejected with PSP_ERR_ARG: staging them would need an allocation.
 *  - The first call in a CUDA context of a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; a context created anew on the device (after
 *    cudaDeviceReset, for instance) gets its first call too.  Make that first call before any stream
 *    capture.
 *  - Like psp_apply with device pointers, the call only enqueues the sweep: a dependency wait that
 *    gives up is reported by the next psp_solve or psp_check_status.
 *  - Every call shares the one array, which keeps the last call's contents.  Nothing in it has to
 *    start at zero: the sweep writes each work entry before it reads it.  Calls that overlap on the
 *    GPU (other streams, handles or host threads) race on the array and give wrong results.
 */
psp_status psp_apply_noalloc(psp_handle h, const double* rhs, double* out, int nrhs, void* stream);

/*
 * psp_matvec - y = A_s x (which = 0) or y = J_s x (which = 1), the 7-point
 * operators of Eq. (1.1) / Eq. (1.5) in the symmetric s1 s2 s3-scaled form.
 */
psp_status psp_matvec(psp_handle h, int which, const double* x, double* y, int nrhs, void* stream);

/*
 * psp_solve - right-preconditioned restarted GMRES(k) (§2.4) for A_s u = s1 s2 s3 f
 * with x0 = 0 (§3), in complex128, preconditioned by psp_apply.  Stops when every
 * right-hand side has a true relative residual < tol or after maxit inner
 * iterations.  f: nrhs unscaled sources; u: nrhs solutions (host or device).
 * info (host, may be NULL) receives the report.
 * Returns PSP_ERR_NOT_CONVERGED (u holds the last iterate) if maxit is reached.
 */
psp_status psp_solve(psp_handle h, const double* f, double* u, int nrhs, double tol, int k, int maxit,
                     psp_solve_info* info, void* stream);

/*
 * psp_solve_history - the residual history of the handle's last psp_solve, one column per
 * right-hand side (per problem and right-hand side for a batch), row-major rows x cols:
 *   kind 0: the Arnoldi estimate |g_{j+1}| / ||b|| after each inner GMRES iteration;
 *   kind 1: the true relative residual ||b - A_s u|| / ||b|| at the end of each restart cycle.
 * A column that stopped earlier than others (converged, or solved in another GMRES run) repeats its
 * last value.  Call with buf = NULL for the sizes.  Errors: PSP_ERR_ARG (kind, or capacity below
 * rows x cols), PSP_ERR_STATE (no solve yet).
 */
psp_status psp_solve_history(psp_handle h, int kind, double* buf, int capacity, int* rows, int* cols);

/*
 * psp_symbolic_export - the nested-dissection tree of panel `panel`'s auxiliary
 * problem (§2.1 separator tree, postorder), for bit-exact comparison.
 * Layout of the int32 stream: [nx, ny, depth, lead, nsn, then for each supernode:
 * s, u, parent, then s node ids, then u struct node ids] with node id
 * x + nx*y + nx*ny*k in the box (k = 0 is the bottom pad plane).
 * Call with buf = NULL to get the length in *len (int32 count).
 */
psp_status psp_symbolic_export(psp_handle h, int panel, int32_t* buf, size_t* len);

/* Number of panels m, fronts factored (panels that share a factorisation count once), and bytes of
   factor storage (any pointer may be NULL). */
psp_status psp_info(psp_handle h, int* panels, int64_t* fronts, int64_t* factor_bytes);

/*
 * psp_export_front - copy the factor of one front (panel, supernode) to host memory:
 * the (s+u) x s column-major block G the handle keeps (psp_si_mode, D on the top block's
 * diagonal): [inv(L_TL); L_BL inv(L_TL)], [inv(L_TL); L_BL] or [L_TL; L_BL], as complex128
 * (converted if the handle is complex64).
 * Call with buf = NULL to get s and u.
 */
psp_status psp_export_front(psp_handle h, int panel, int supernode, double* buf, int* s, int* u);

/*
 * psp_export_second_inverse - for a handle in the form PSP_SI_TWO, copy one front's second inverse of
 * L_TL (built row by row, X L_TL = I) to host memory: s x s column-major, complex128, unit lower (the
 * diagonal and the upper part are written as stored: one and zero).  Call with buf = NULL to get s.
 * Errors: PSP_ERR_ARG (bad panel or supernode, a front outside the handle's block of panels),
 * PSP_ERR_STATE (the handle is not in the form PSP_SI_TWO or has no factorisation).
 */
psp_status psp_export_second_inverse(psp_handle h, int panel, int supernode, double* buf, int* s);

/*
 * Per-kernel accounting of one handle (setup, applies, matvecs and solves issued through it).
 * Launch counts and algorithmic work are always kept; total_ms is filled for the kernels that the
 * handle's collect_stats selects (CUDA events around each such launch, on the launch stream).
 * flops: useful real floating-point operations (a complex multiply-add counts 8) of the plain
 * multifrontal method (LDL^T of F_TL, F_BL L^{-T}, the Schur update, the solves); extra_flops: the
 * further flops the kernel executes for selective inversion (inv(L_TL) and M_BL = L_BL inv(L_TL),
 * §2.2); bytes: the algorithmic HBM bytes (matrix entries read once, vectors read/written once).
 * Copies min(capacity, kinds) records into out, sets *count to the number of kernel kinds,
 * synchronises the device, and zeroes the counters when reset != 0.
 */
typedef struct {
  char name[40];
  int64_t launches;
  double total_ms;
  double flops;
  double bytes;
  double extra_flops;
} psp_kernel_stat;

psp_status psp_stats(psp_handle h, psp_kernel_stat* out, int capacity, int* count, int reset);

/*
 * psp_tune_sweep - the paper has no counterpart: an autotuner for the schedule of the persistent
 * sweep (the GPU's counterpart of the paper's choice of process grids, §2.1).  On this handle it
 * times psp_apply with nrhs right-hand sides (per problem of a batch) under candidate schedules
 * and keeps the fastest: the tasks a tree level is split into (152 .. 2432), the resident CTAs per
 * SM (2, 3, 4, 6, 8), the cap on rows / columns per task (64 .. 256), the floor on rows per task
 * (8 .. 64), the queue tasks a CTA holds ahead (1, 2) and, for nrhs > 1, the right-hand sides per
 * CTA pass (1 .. 8).  It searches one
 * coordinate at a time, starting from the handle's current schedule, timing `reps` applications
 * (CUDA events on `stream`) per candidate after one untimed one.  Results do not change beyond
 * rounding (the schedule only regroups the same sums).  The work vectors are the handle's own; the
 * call allocates one N x nrhs block for its input and synchronises the stream.
 *   out   receives the chosen schedule and the times (may be NULL)
 * Errors: PSP_ERR_ARG (nrhs < 1, reps < 1), PSP_ERR_STATE (no factorisation), PSP_ERR_CUDA.
 */
typedef struct {
  int sweep_level_tasks;
  int sweep_ctas_per_sm;
  int sweep_rhs_group;    /* 0: the default grouping */
  int candidates;         /* schedules timed */
  double initial_ms;      /* one application under the schedule the handle had */
  double best_ms;         /* one application under the chosen schedule */
  int sweep_min_rows;     /* floor on rows / columns per task */
  int sweep_max_rows;     /* cap on rows / columns per task */
  int sweep_claim_ahead;  /* tasks a CTA holds besides the one it runs */
  int reserved[1];
} psp_sweep_tuning;

psp_status psp_tune_sweep(psp_handle h, int nrhs, int reps, void* stream, psp_sweep_tuning* out);

/*
 * psp_tune_setup - the paper has no counterpart: an autotuner for what the setup builds.  The paper
 * weighs selective inversion's dearer setup against its faster solves (§2.2, §3 Table 2); this call
 * measures that trade on the handle's own problem.  It re-factors the handle under each candidate
 * (the forms PSP_SI_EXTENDED, PSP_SI_PAPER and PSP_SI_NONE; the two-inverse form is a choice for
 * accuracy, not speed, and is not among them; for complex64 tensor-core fronts tc_min_dim 32 / 64 / 128),
 * timing the setup (host clock, the factorisation synchronises) and one application to nrhs
 * right-hand sides (CUDA events on `stream`, after an untimed one), and keeps the candidate with
 * the least setup_ms + expected_applies x apply_ms; the handle ends factored that way.  Results
 * change only by rounding (the forms apply the same preconditioner).  Costs one factorisation per
 * candidate.
 * Errors: PSP_ERR_ARG, PSP_ERR_STATE (no factorisation, or a block handle), PSP_ERR_CUDA.
 */
typedef struct {
  int selective_inversion;  /* chosen psp_si_mode */
  int tc_min_dim;           /* chosen tensor-core threshold (complex64) */
  int candidates;           /* configurations timed */
  double setup_ms;          /* setup of the chosen configuration */
  double apply_ms;          /* one application of the chosen configuration */
  double initial_total_ms;  /* setup + expected_applies x apply under the handle's configuration before */
  double best_total_ms;     /* the same for the chosen one */
  int reserved[4];
} psp_setup_tuning;

psp_status psp_tune_setup(psp_handle h, int nrhs, int expected_applies, void* stream, psp_setup_tuning* out);

/*
 * psp_sweep_part - one half of Alg. 1.5 restricted to the handle's block of panels [b, e)
 * (psp_options.panel_begin / panel_count), for a sweep whose panels are spread over several GPUs
 * (§2: the panel factorisations are independent, the panel solves run in sequence).  u holds nrhs
 * global vectors (N x nrhs, host or device) and is updated in place:
 *   direction 0 (forward):  for i = b .. e-1:  u_i := T_i (u_i - J_{i,i-1} u_{i-1})
 *                           (for b > 0 it reads plane z0(b) - 1, the previous block's last plane,
 *                           which must hold that block's forward result)
 *   direction 1 (backward): for i = min(e, m-1) - 1 .. b:  u_i -= T_i J_{i+1,i}^T u_{i+1}
 *                           (for e < m it reads plane z0(e), the next block's first plane, which must
 *                           hold that block's final result)
 * Running the blocks' forward parts in order, then their backward parts in reverse order, handing
 * those single planes between them, gives psp_apply's result on each block's planes.  Planes
 * outside the reads above and the block's own are neither read nor written.
 * Errors as for psp_apply; PSP_ERR_STATE for a batch handle.
 */
psp_status psp_sweep_part(psp_handle h, double* u, int nrhs, int direction, void* stream);

/*
 * psp_plan_panels - the paper has no counterpart: host-only planning, no GPU needed.  The panel
 * plan psp_setup would make (§1.1, Alg. 1.4) for this grid, gamma, depth and options: *m panels,
 * panel i holding the global planes [z0[i], z1[i]), and (cost != NULL) the algorithmic flops of
 * factoring its auxiliary problem (8 per complex multiply-add of the LDL^T, the F_BL solve and the
 * Schur updates of its nested-dissection fronts), for partitioning the panels over GPUs.  Entries
 * beyond `capacity` are not written.  Errors: PSP_ERR_ARG.
 */
psp_status psp_plan_panels(const psp_grid* g, int pml_gamma, int panel_depth, const psp_options* opt, int* z0, int* z1,
                           double* cost, int capacity, int* m);

/*
 * psp_check_status - the paper has no counterpart: synchronises `stream` and reports whether a
 * bounded dependency wait of any sweep on this handle gave up since setup or the last report
 * (PSP_ERR_TIMEOUT, after which the flag is cleared), else PSP_OK.  The device stays usable.
 */
psp_status psp_check_status(psp_handle h, void* stream);

psp_status psp_destroy(psp_handle h);
const char* psp_status_string(psp_status s);
const char* psp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PSP_H */

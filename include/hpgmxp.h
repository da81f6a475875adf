/*
 * hpgmxp.h -- C ABI of the HPG-MxP GMRES-IR solve path on one GB300 GPU.
 *
 * The library solves A x = b for the 27-point-stencil matrix of the HPG-MxP
 * benchmark (arXiv 2507.11512, Sec. 2-3) with restarted GMRES(m), CGS2
 * orthogonalisation and Givens rotations (Algorithm 3), right-preconditioned
 * by one geometric-multigrid V-cycle (Fig. 1) whose smoother is multicolour
 * symmetric Gauss-Seidel (eqs. (1)-(2), Sec. 3.2.1), inside an FP64
 * iterative-refinement loop.  Every step runs in the library's CUDA kernels.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - Every call returns an int status: HPG_OK (0) or a negative HPG_ERR_*
 *   code.  hpg_status_string() names a code; hpg_last_error() gives the
 *   message of the most recent failure on the calling thread.
 * - Pointers named "device" must point to memory of the current CUDA device
 *   (cudaMalloc'd, or a torch tensor's data_ptr()); the library never frees
 *   them.  The problem handle owns all memory the library allocates and
 *   hpg_destroy() releases it.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Work is enqueued on it; calls that return results to the host
 *   (hpg_gmres_ir_solve's info) synchronise that stream.
 * - Grid point (i, j, k), 0 <= i < nx etc., has NATURAL index
 *   i + nx * (j + ny * k).  Internally every level stores rows in
 *   COLOUR-BLOCKED order: colour c = ((i+1)&1) + 2((j+1)&1) + 4((k+1)&1)
 *   (so points with all coordinates even are colour 7), blocks c = 0..7 in
 *   order, each block lexicographic over (i>>1, j>>1, k>>1) and padded to a
 *   multiple of 32 rows.  hpg_spmv and hpg_mg_vcycle take vectors in this
 *   storage order (length n_store, padding entries zero); hpg_permute
 *   converts.  hpg_gmres_ir_solve takes natural order.
 * - Not thread-safe per handle: calls on one handle must not overlap.
 */
#ifndef HPGMXP_H
#define HPGMXP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HPG_API __attribute__((visibility("default")))
#else
#define HPG_API
#endif

/* ----------------------------------------------------------- status codes */
#define HPG_OK                  0
#define HPG_ERR_INVALID        -1  /* bad argument (size, pointer, option)      */
#define HPG_ERR_CUDA           -2  /* a CUDA runtime call or kernel failed        */
#define HPG_ERR_NOT_CONVERGED  -3  /* maxit reached before ||r||/||b|| < tol      */
#define HPG_ERR_BREAKDOWN      -4  /* singular Hessenberg (H_kk = H_k+1,k = 0)    */
#define HPG_ERR_NAN            -5  /* a residual norm became NaN or Inf           */
#define HPG_ERR_ALLOC          -6  /* device allocation failed                    */
#define HPG_ERR_STATE          -7  /* call out of order (e.g. no hierarchy yet)   */
#define HPG_ERR_UNSUPPORTED    -8  /* option not built into this library          */
#define HPG_ERR_TIMEOUT        -9  /* a device-side wait ran out of its limit     */

/* -------------------------------------------------------------- precisions */
typedef enum {
  HPG_FP64 = 0,   /* IEEE binary64                                    */
  HPG_FP32 = 1,   /* IEEE binary32                                    */
  HPG_BF16 = 2,   /* bfloat16 storage (Krylov basis only), FP32 math  */
  HPG_FP16 = 3    /* binary16 storage (Krylov basis only), FP32 math  */
} hpg_prec;

typedef struct hpg_problem hpg_problem_t;

/* Stencil parameters (Sec. 3).  beta: nonsymmetric option; the off-diagonal
 * at grid offset d = (dx,dy,dz) of the neighbour is -1 + beta*(dx+dy+dz)/3
 * (beta = 0 is the paper's benchmarked symmetric matrix; |beta| <= 1 keeps
 * every row weakly diagonally dominant).  theta: NULL, or nx*ny*nz FP64
 * per-cell diagonal scales in natural order (host or device memory; copied):
 * a_ii = 26 * theta_i.  Coarse levels inject theta: theta_c(I) = theta(2I). */
typedef struct {
  double beta;
  const double* theta;
} hpg_stencil_params;

/* Geometry of one level (filled by hpg_level_info). */
typedef struct {
  int nx, ny, nz;
  int64_t n;             /* grid points nx*ny*nz                              */
  int64_t n_store;       /* rows in storage order, padding included            */
  int64_t nnz;           /* structural non-zeros (padding slots excluded)      */
  int64_t colour_offset[9]; /* storage start of colour block c; [8] = n_store  */
  int64_t colour_count[8];  /* grid points of colour c                         */
} hpg_level_desc;

/* Result of a solve. */
typedef struct {
  int iterations;        /* total inner (Arnoldi) steps over all restarts       */
  int restarts;          /* restart cycles completed                            */
  int converged;         /* 1 if ||b - A x||_2 / ||b||_2 < tol (FP64)           */
  int status;            /* same value the call returns                         */
  double rel_residual;   /* final ||b - A x||_2 / ||b||_2, FP64                 */
  double rho0;           /* ||b||_2                                             */
  int kernel_launches;   /* kernels the device ran for this solve (graph-launched
                            kernels counted per execution)                      */
  int graph_launches;    /* CUDA graph launches this solve made (1 or 0)        */
} hpg_solve_info;

/* Creates a problem on the current CUDA device: the fine-level 27-point
 * ELLPACK matrix (Sec. 3.2.2; slot-major column-index array shared by an FP64
 * and an FP32 value array), generated on the device in storage order.
 * Padding slots (neighbours outside the grid, Dirichlet truncation, Sec. 2)
 * hold column = own row and value 0.
 * nx, ny, nz >= 1 and nx*ny*nz*27 < 2^31.  p may be NULL (beta = 0).
 * Returns HPG_ERR_INVALID for bad sizes, HPG_ERR_ALLOC / HPG_ERR_CUDA on
 * device failure; *out is NULL on failure.  Synchronous. */
HPG_API int hpg_setup_problem(int nx, int ny, int nz,
                              const hpg_stencil_params* p,
                              hpg_problem_t** out);

/* Builds the geometric multigrid hierarchy (Sec. 2, Fig. 1; Sec. 3 injection
 * restriction eq. (3), P = R^T): levels = min(levels, 1 + the number of
 * times 2 divides nx, ny and nz together), each coarse level re-discretising
 * the stencil on the 2x coarser grid; pre/post = symmetric Gauss-Seidel sweeps
 * before/after the coarse correction (>= 0; the coarsest level always does
 * one sweep).  May be called again to rebuild (this drops the batch buffers
 * and tuned shapes of the many-right-hand-side entry points; HPG_ERR_STATE
 * while a multi-system batch uses the problem).  Synchronous. */
HPG_API int hpg_build_mg_hierarchy(hpg_problem_t* h, int levels,
                                   int pre_sweeps, int post_sweeps);

/* Number of levels built (1 before hpg_build_mg_hierarchy). */
HPG_API int hpg_num_levels(const hpg_problem_t* h, int* levels);

/* Geometry of `level` (0 = finest). */
HPG_API int hpg_level_info(const hpg_problem_t* h, int level,
                           hpg_level_desc* out);

/* Reorders a vector of `level` between natural order (length n) and storage
 * order (length n_store).  direction 0: natural -> storage (padding entries
 * written as 0); 1: storage -> natural.  in_prec / out_prec: HPG_FP64 or
 * HPG_FP32 (converting on the way).  in and out are device pointers and must
 * not overlap.  Asynchronous on `stream`. */
HPG_API int hpg_permute(hpg_problem_t* h, int level, int direction,
                        hpg_prec in_prec, const void* in,
                        hpg_prec out_prec, void* out, void* stream);

/* y = A_level x (Sec. 3.2.2 ELLPACK SpMV; Algorithm 3 "SpMV to get next basis
 * vector").  prec HPG_FP64: FP64 values and vectors; HPG_FP32: FP32 values,
 * vectors and accumulation.  x, y: device, storage order, length n_store,
 * must not overlap.  Asynchronous on `stream`. */
HPG_API int hpg_spmv(hpg_problem_t* h, int level, hpg_prec prec,
                     const void* x, void* y, void* stream);

/* z = M^{-1} r: one V-cycle from z = 0 starting at `level` (Fig. 1 applied
 * recursively; Sec. 3.2.4 residual fused with restriction): per level
 * `pre` symmetric multicolour Gauss-Seidel sweeps (forward colours 0..7,
 * backward 7..0), fused residual-restriction to the coarse-coincident points,
 * recursion, prolongation z_{f_c(i)} += z^c_i, `post` sweeps; the coarsest
 * level does one sweep.  prec HPG_FP64 or HPG_FP32 (values, vectors and
 * arithmetic).  r, z: device, storage order, length n_store, must not
 * overlap.  Requires hpg_build_mg_hierarchy.  Asynchronous on `stream`. */
HPG_API int hpg_mg_vcycle(hpg_problem_t* h, int level, hpg_prec prec,
                          const void* r, void* z, void* stream);

/* `sweeps` symmetric multicolour Gauss-Seidel sweeps on `level` (eqs. (1)-(2),
 * Sec. 3.2.1 -- the smoother of the V-cycle, launched exactly as the V-cycle
 * launches it): each sweep updates the colours 0..7, then 7..0, with
 * z_i <- (r_i - sum_{j != i} a_ij z_j) / a_ii for every row i of the colour;
 * a colour phase that would repeat the previous one on unchanged data (at the
 * forward/backward turn and between sweeps) is skipped, which changes no value.
 * z_is_zero != 0: z enters as 0 and its contents are never read (the first
 * forward sweep omits the zero terms); otherwise z holds the initial iterate.
 * sweeps = 0 leaves z unchanged (or zeroes it when z_is_zero).  prec HPG_FP64
 * or HPG_FP32.  r, z: device, storage order, length n_store, must not
 * overlap; padding rows of z stay 0 if they enter 0.  Requires
 * hpg_build_mg_hierarchy.  HPG_ERR_INVALID for a bad level, precision,
 * sweep count or pointer.  Asynchronous on `stream`. */
HPG_API int hpg_mg_smooth(hpg_problem_t* h, int level, hpg_prec prec,
                          const void* r, void* z, int sweeps, int z_is_zero,
                          void* stream);

/* Allocation-free V-cycle.  The paper has no counterpart: this is an entry
 * point for callers that cannot allocate device memory when they call --
 * code running inside a CUDA stream capture (cudaMalloc is not allowed there),
 * real-time loops that must not stall on the allocator, or memory-pool owners
 * that forbid allocations outside their pool.  It computes what hpg_mg_vcycle
 * computes with one kernel launch per colour phase and transfer (the same
 * kernels, order and results as hpg_mg_vcycle with the default options; it
 * ignores HPG_OPT_COARSE_CLUSTER and always launches the phases), but the
 * coarse levels' work vectors (restricted residuals and corrections of levels
 * level+1 .. last) live in one static device array of
 * HPG_NOALLOC_SCRATCH_BYTES bytes that the library declares at file scope:
 * every GPU that loads the library holds it until the process exits.
 * - The caller passes r and z as for hpg_mg_vcycle (device, storage order,
 *   length n_store of `level`); the handle's hierarchy supplies the matrices.
 * - Needs 2 * sizeof(prec) * (sum of n_store over the coarse levels) bytes;
 *   larger requests return HPG_ERR_INVALID with the sizes in hpg_last_error()
 *   (the coarse levels of the 128^3 grid need 4.8 MB in FP64 and fit; those
 *   of the 320^3 grid need 37 MB in FP32 and are rejected).
 * - The call allocates and frees nothing (no cudaMalloc / cudaFree, no
 *   allocating library routine); it zeroes the part of the array it uses with
 *   cudaMemsetAsync on `stream`.
 * - The first call on a device looks up the array's device address once
 *   (cudaGetSymbolAddress, with that device current); make that first call
 *   before any stream capture.  The address is kept for the life of the
 *   process: a device reset (cudaDeviceReset) before a later call is not
 *   supported.
 * - All calls share the one array: calls that overlap on the GPU (other
 *   streams, other threads, other handles) race on it and give wrong results.
 * Asynchronous on `stream`. */
#define HPG_NOALLOC_SCRATCH_BYTES (32u << 20)
HPG_API int hpg_mg_vcycle_noalloc(hpg_problem_t* h, int level, hpg_prec prec,
                                  const void* r, void* z, void* stream);

/* GMRES-IR (Algorithm 3): restarted right-preconditioned GMRES(restart) with
 * CGS2 and Givens rotations.  The outer residual r = b - A x, its norm, the
 * convergence test ||r||/||b|| < tol, the update x += M^{-1} Q t and the
 * Hessenberg least-squares run in FP64; `inner` (HPG_FP32 or HPG_FP64) is the
 * precision of the V-cycle and the Arnoldi SpMV; `basis` the storage of the
 * Krylov basis Q: HPG_FP64 with inner = HPG_FP64 (plain FP64 GMRES,
 * Algorithm 2), or with inner = HPG_FP32 one of HPG_FP32, HPG_BF16, HPG_FP16.
 * A BF16/FP16 basis (the low-precision basis of Sec. 5's outlook) stores each
 * vector as u_j = q_j / max_i |q_ij| with one FP32 scale sigma_j =
 * max_i |q_ij| (so q_j = sigma_j u_j, |u_j| <= 1: no overflow, no vector
 * flushed to zero); CGS2 reads it with FP32 arithmetic, the V-cycle is
 * applied to the dequantised vector, and the FP64 refinement recovers the
 * accuracy the basis loses (more inner steps may be needed).  Other
 * combinations return HPG_ERR_UNSUPPORTED.  b: FP64, natural order, n entries; x: FP64, natural order,
 * in: initial guess, out: solution.  b and x may be device or host pointers
 * (host buffers are staged through device memory).  restart in [1, 64],
 * maxit >= 0 (total inner steps), tol > 0.  Returns HPG_OK on convergence,
 * HPG_ERR_NOT_CONVERGED when maxit is reached (x holds the last iterate),
 * HPG_ERR_NAN / HPG_ERR_BREAKDOWN on numerical failure.  b = 0 returns x = 0.
 * info may be NULL.  Synchronises `stream`. */
HPG_API int hpg_gmres_ir_solve(hpg_problem_t* h, const double* b, double* x,
                               double tol, int restart, int maxit,
                               hpg_prec inner, hpg_prec basis,
                               hpg_solve_info* info, void* stream);

/* Gradient of a scalar loss L(x) with respect to the per-cell diagonal scales
 * theta of hpg_stencil_params, for x = A(theta)^{-1} b (the adjoint method;
 * the paper has no differentiable solve -- this serves a torch.autograd
 * wrapper of hpg_gmres_ir_solve).  Only a_ii = 26 theta_i depends on
 * theta_i, so with lambda = A(theta)^{-T} dL/dx (a solve on the handle made
 * with beta -> -beta: A(beta)^T = A(-beta)),
 *   grad_i = dL/dtheta_i = -26 lambda_i x_i,  computed as (-26 lambda_i) x_i.
 * lambda, x, grad: device, FP64, natural order, nx*ny*nz entries of h's
 * fine grid; grad may alias neither input.  dL/db is lambda itself.
 * HPG_ERR_INVALID for a NULL handle or pointer.  Asynchronous on `stream`. */
HPG_API int hpg_diag_scale_gradient(hpg_problem_t* h, const double* lambda,
                                    const double* x, double* grad, void* stream);

/* ------------------------------------------------- many right-hand sides
 * The paper solves one right-hand side; these entry points solve R of them
 * (R = nrhs in {1, 2, 4, 8}) together, so that every matrix entry read from
 * memory serves R rows of work (the multigrid and SpMV kernels are
 * bandwidth-bound, Sec. 4).  Each right-hand side is solved by its own
 * GMRES-IR (Algorithm 3: its own basis, Hessenberg matrix, rotations and
 * convergence test, FP32 inner solve and basis, FP64 refinement); the R
 * solves advance in lockstep and a converged one is frozen while the others
 * continue.  Layout of a storage-order R-vector of a level: [n_store][nrhs],
 * the nrhs values of a storage row contiguous (FP32).  Natural-order inputs
 * and outputs: nrhs vectors of n = nx*ny*nz values, vector r at offset r*n.
 * All pointers are device pointers; no call allocates memory the caller must
 * free.  The per-handle buffers these calls allocate are freed by
 * hpg_destroy. */

/* Y = A_level X for nrhs FP32 right-hand sides (storage-order R-vectors);
 * column r equals hpg_spmv of column r bit for bit.  X, Y must not overlap.
 * Asynchronous on `stream`. */
HPG_API int hpg_spmv_batch(hpg_problem_t* h, int level, int nrhs, const float* X,
                           float* Y, void* stream);

/* Z = M^{-1} R for nrhs FP32 right-hand sides (storage-order R-vectors): the
 * V-cycle of hpg_mg_vcycle, phase for phase; column r equals the FP32
 * hpg_mg_vcycle of column r bit for bit.  Requires hpg_build_mg_hierarchy.
 * R, Z must not overlap.  Asynchronous on `stream`. */
HPG_API int hpg_mg_vcycle_batch(hpg_problem_t* h, int level, int nrhs,
                                const float* R, float* Z, void* stream);

/* FP32 nrhs-vectors between natural order (direction 0: in natural, out
 * storage, padding rows 0) and storage order (direction 1).  Asynchronous. */
HPG_API int hpg_permute_batch(hpg_problem_t* h, int level, int direction, int nrhs,
                              const float* in, float* out, void* stream);

/* GMRES-IR for nrhs right-hand sides of one problem (see above).  B: FP64,
 * natural order, nrhs vectors of n; X: FP64, same layout, in: initial
 * guesses, out: solutions.  tol, restart (1..64), maxit (inner steps of each
 * right-hand side) as for hpg_gmres_ir_solve.  infos: NULL or nrhs entries.
 * Returns HPG_OK when every right-hand side converged, else the first
 * failure (HPG_ERR_NOT_CONVERGED, HPG_ERR_NAN, HPG_ERR_BREAKDOWN).  One CUDA
 * graph launch per call (host-driven in the eager and profiling modes).
 * Synchronises `stream`. */
HPG_API int hpg_gmres_ir_solve_batch(hpg_problem_t* h, int nrhs, const double* B,
                                     double* X, double tol, int restart, int maxit,
                                     hpg_solve_info* infos, void* stream);

/* Launch shape of the multi-right-hand-side kernels of `level`: kind 0 the
 * Gauss-Seidel phases, kind 1 the SpMV; lpr lanes per row (1, 2 or nrhs; 0 =
 * default 1) and block threads (64, 128, 256; 0 = default).  Every shape
 * gives the same results.  hpg_batch_tune sets them by timing. */
HPG_API int hpg_batch_set_shape(hpg_problem_t* h, int level, int kind, int nrhs, int lpr,
                                int block);
HPG_API int hpg_batch_get_shape(const hpg_problem_t* h, int level, int kind, int nrhs,
                                int* lpr, int* block);

/* Times every launch shape of the multi-right-hand-side Gauss-Seidel sweep
 * on each level and of the level-0 SpMV for nrhs right-hand sides and keeps
 * the fastest (the autotuner; a few milliseconds per level).  Synchronises
 * `stream`. */
HPG_API int hpg_batch_tune(hpg_problem_t* h, int nrhs, void* stream);

/* Several problems (each its own grid, stencil and hierarchy; no handle
 * twice) solved by ONE launch of one CUDA graph that holds every problem's
 * batched GMRES-IR as an independent branch.  hpg_batch_create allocates the
 * problems' batch buffers for nrhs and restart and captures the graph (tune
 * the problems first: the graph keeps the shapes it was captured with);
 * while the batch exists the problems' batch buffers belong to it (batched
 * solves of the same problems with another nrhs or restart are refused).
 * hpg_batch_solve: B[i], X[i] as for hpg_gmres_ir_solve_batch for problem
 * i; infos: NULL or nsys * nrhs entries (problem-major).  hpg_batch_destroy
 * releases the graph (the problems stay).  Destroy a batch before any of its
 * problems: while it exists, hpg_destroy, hpg_build_mg_hierarchy and
 * hpg_set_option on those problems return HPG_ERR_STATE. */
typedef struct hpg_batch hpg_batch_t;
HPG_API int hpg_batch_create(hpg_problem_t* const* hs, int nsys, int nrhs, int restart,
                             hpg_batch_t** out);
HPG_API int hpg_batch_solve(hpg_batch_t* b, const double* const* B, double* const* X,
                            double tol, int maxit, hpg_solve_info* infos, void* stream);
HPG_API int hpg_batch_destroy(hpg_batch_t* b);

/* Autotuner of a batch: lanes per row (1, 2 or nrhs) of the
 * multi-right-hand-side kernels chosen by timing whole batch solves of B from
 * x0 = 0 (X as for hpg_batch_solve, overwritten) with each candidate applied to
 * every problem and level, then the graph is recaptured with the fastest.
 * Under a batch the problems' kernels run concurrently, so the per-problem
 * timing of hpg_batch_tune does not predict it.  times_ms: NULL or 3 floats,
 * the measured solve times of lanes per row 1, 2, nrhs (fewer for nrhs < 4).
 * Synchronises `stream`. */
HPG_API int hpg_batch_tune_solve(hpg_batch_t* b, const double* const* B, double* const* X,
                                 double tol, int maxit, float* times_ms, void* stream);

/* ------------------------------------------------------------ profiling
 * Measurement support, not a step of the method (the paper profiles its
 * kernels with rocprof and rocprofiler-compute, Sec. 4.3).  While enabled,
 * every kernel the handle launches is bracketed by two CUDA events on its
 * own stream; the report aggregates per (kernel class, level, precision)
 * the launches, the summed event durations and the summed algorithmic DRAM
 * bytes of the library's byte model (matrix slots, vectors read and written
 * once).  Enabling adds two event records per launch. */
typedef struct {
  const char* name;      /* kernel class (static string)                 */
  int level;             /* multigrid level (0 for vector kernels)       */
  int prec;              /* hpg_prec of the kernel's data                */
  long long launches;
  double total_ms;       /* summed CUDA-event durations                  */
  double bytes;          /* summed algorithmic DRAM bytes                */
} hpg_kernel_stat;

/* Enables (1) or disables (0) profiling and clears recorded launches. */
HPG_API int hpg_set_profiling(hpg_problem_t* h, int enable);

/* Waits for the recorded launches, writes up to `capacity` aggregated rows
 * to out, sets *count to the number of rows available, and clears the
 * records.  HPG_ERR_INVALID on NULL handle / count. */
HPG_API int hpg_profile_report(hpg_problem_t* h, hpg_kernel_stat* out, int capacity,
                               int* count);

/* Execution of hpg_gmres_ir_solve.  HPG_EXEC_GRAPH (default): the whole solve
 * runs as one CUDA graph with conditional WHILE / IF nodes (one launch, one
 * host synchronisation).  HPG_EXEC_EAGER: the same kernels driven from the
 * host, one synchronisation per inner step (for tools that cannot look into
 * conditional graphs).  Both give bitwise-identical results.  Enabling
 * profiling implies eager execution. */
#define HPG_EXEC_GRAPH 0
#define HPG_EXEC_EAGER 1
HPG_API int hpg_set_execution(hpg_problem_t* h, int mode);

/* Implementation options (not steps of the method; results are the same).
 * HPG_OPT_COARSE_CLUSTER (default 0): run the part of a V-cycle from the
 * first level with at most 300000 storage rows down to the coarsest (and back)
 * as one kernel on one thread-block cluster (up to 16 CTAs, hardware cluster
 * barrier between colour phases); 0: one kernel launch per colour phase /
 * transfer on every level.  HPG_OPT_PDL (default 1): programmatic dependent
 * launch between the solve's kernels.  HPG_OPT_GS_PIPELINE: on levels whose
 * matrix streams from memory, a symmetric Gauss-Seidel sweep may run as one
 * kernel in which a tile of a colour phase starts as soon as the tiles of the
 * previous phase within one grid plane of it are done (bounded waits; a wait
 * that runs out makes the solve return HPG_ERR_TIMEOUT) instead of one launch
 * per colour phase; same results.  0: never; 1 (default): FP64 sweeps only
 * (measured faster on GB300 for FP64, slower for FP32); 2: always.  Setting
 * an option drops captured solve graphs (single- and many-right-hand-side).
 * HPG_ERR_INVALID for an unknown option; HPG_ERR_STATE while a multi-system
 * batch uses the problem (its graph keeps the options it was captured
 * with: destroy the batch, set the option, create it again). */
#define HPG_OPT_COARSE_CLUSTER 1
#define HPG_OPT_PDL 2
#define HPG_OPT_GS_PIPELINE 3
/* HPG_OPT_GS_HALO (default 0): on levels whose matrix streams from memory,
 * FP32 Gauss-Seidel phases that read every slot run TMA-tiled: a CTA moves
 * its rows' 27 value and 26 index slices, their r and the part of z its rows
 * can touch into shared memory with bulk asynchronous copies completing on
 * one mbarrier, then computes from shared memory; same results (measured
 * slower than the default on GB300).  Its copy wait is bounded: if it runs
 * out the solve returns HPG_ERR_TIMEOUT. */
#define HPG_OPT_GS_HALO 4
/* HPG_OPT_COARSE_CTA (default 0): the coarsest level's symmetric sweep of a
 * V-cycle runs in one CTA (z in shared memory, a block barrier between colour
 * phases) when every colour block has at most 512 rows and the level's vector
 * fits in 64 KB; 0: one launch per colour phase there too.  Same results
 * (measured slower than the default on GB300).  Ignored while
 * HPG_OPT_GS_PIPELINE is 3.
 * HPG_OPT_PDL_ROWS (default 16384): Gauss-Seidel phases of levels whose
 * matrix does not stream from memory, up to this many rows per phase, let
 * the next kernel launch as soon as they start (their own matrix loads then
 * overlap the previous phase); larger phases let it launch only as their
 * blocks exit.  Multi-right-hand-side phases (the *_batch calls and batched
 * solves) up to this many rows are launched programmatically and let the
 * next kernel launch as soon as they start; larger ones start after the
 * previous kernel has completed.  Same results: kernels read the vectors an
 * earlier kernel wrote only after the grid-dependency wait, through coherent
 * loads. */
#define HPG_OPT_COARSE_CTA 5
#define HPG_OPT_PDL_ROWS 6
HPG_API int hpg_set_option(hpg_problem_t* h, int option, int value);

/* Failure-detection test support (not a step of the method): the next
 * pipelined sweep on `level` starts its tile queue at `tiles`, so the tiles
 * below never run and the waits of the tiles after them on those run out
 * (each wait is bounded, under a second); that sweep then abandons its
 * remaining tiles and records the error, and the solve that contains it (or
 * the next solve on this handle, for a sweep run through hpg_mg_smooth /
 * hpg_mg_vcycle) returns HPG_ERR_TIMEOUT.  The device stays usable.  Only
 * levels that have a pipelined sweep (HPG_OPT_GS_PIPELINE) are accepted.
 * Synchronous. */
HPG_API int hpg_inject_stall(hpg_problem_t* h, int level, int tiles);

/* Frees everything the handle owns (NULL is accepted).  A problem that a
 * multi-system batch still uses (hpg_batch_create) is not freed: the call
 * returns HPG_ERR_STATE; destroy the batch first (hpg_batch_destroy). */
HPG_API int hpg_destroy(hpg_problem_t* h);

/* Static string naming a status code. */
HPG_API const char* hpg_status_string(int status);

/* Message of the last failure on the calling thread ("" if none). */
HPG_API const char* hpg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HPGMXP_H */

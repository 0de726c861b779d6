/*
 * hz.h -- C ABI of the GB300 (sm_103a) matrix-free two-level deflation +
 * CSLP-preconditioned Krylov solver for the 2-D finite-difference Helmholtz
 * equation  -Lap u - k(x,y)^2 u = b  (Chen, Dwarka, Vuik, arXiv 2308.06152).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - A grid has nx * ny nodes, spacing h, node (i, j) at flat index
 *    j * nx + i (x fastest).  Vectors are complex128 (interleaved re, im
 *    doubles, i.e. double2) laid out [nrhs][ny][nx]; nrhs vectors are
 *    stored back to back.
 *  - Under HZ_BC_DIRICHLET the boundary nodes are not unknowns: inputs there
 *    are ignored (read as 0) and outputs there are written as 0.
 *  - Every pointer named *_dev is device memory of the current CUDA device;
 *    *_host is host memory (pinned memory makes the copies asynchronous).
 *    The library never allocates device memory: all device storage is the
 *    caller's workspace (hz_workspace_bytes / hz_setup).  The caller keeps
 *    ownership of every buffer it passes and must keep the workspace and
 *    the k2 array alive until hz_destroy.
 *  - Work is issued on the stream given to hz_setup, in stream order.
 *    Entry points that return numbers on the host (hz_solve's info, J)
 *    synchronise that stream before returning.
 *  - Errors are return codes; nothing throws across the ABI.
 *    hz_last_error gives a one-line description of the last failure.
 */
#ifndef HZ_H_
#define HZ_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HZ_OK = 0,
  HZ_INVALID_ARG = 1,         /* null pointer, nrhs out of range, bad enum  */
  HZ_INVALID_GRID = 2,        /* too small, cannot be coarsened for
                                 deflation, or coarsest level too large     */
  HZ_WORKSPACE_TOO_SMALL = 3,
  HZ_NOT_CONVERGED = 4,       /* iteration cap reached; x holds the last
                                 iterate, info.relres its true residual     */
  HZ_BREAKDOWN = 5,           /* Arnoldi breakdown without convergence      */
  HZ_NAN = 6,                 /* NaN / Inf met in a residual norm           */
  HZ_TIMEOUT = 7,             /* a bounded pipeline wait inside a kernel ran
                                 out (the TMA-ring Gram-Schmidt kernels wait
                                 on mbarriers for at most 2 s each); the
                                 solve stopped, the solver stays usable    */
  HZ_CUDA_ERROR = 8
} hz_status;

typedef enum { HZ_BC_DIRICHLET = 0, HZ_BC_SOMMERFELD = 1 } hz_bc;

/* Deflation vectors Z (Sec. 3.2.1): none (plain CSLP preconditioner),
 * bilinear interpolation (A-DEF1) or the quadratic higher-order
 * interpolation (APD). */
typedef enum { HZ_Z_NONE = 0, HZ_Z_BILINEAR = 1, HZ_Z_HO = 2 } hz_zkind;

/* Coarse operator E = A_2h (Sec. 5.2): the Galerkin product R A_h Z
 * (str-Glk, Sec. 5.2.1, or its stored stencil, see hz_tuning), 2nd-order
 * re-discretisation (ReD-O2, Sec. 5.2.3), the Galerkin-derived 5x5
 * re-discretisation with 2nd-order rows on the two outer rings (ReD-Glk1)
 * or on the outer ring with ghost values on the second (ReD-Glk2, Sec.
 * 5.2.4), the 4th-order cross with ReD-O2 rows within one node of the
 * boundary (ReD-O4, Sec. 5.2.3, eq. Helmstencil Oh4 with the wavenumber
 * term read as -k^2), or the compact 4th-order 3x3 scheme with 4th-order
 * Sommerfeld ghosts (ReD-cmpO4, Sec. 5.2.5, gamma = 1). */
typedef enum {
  HZ_E_GALERKIN = 0, HZ_E_RED_O2 = 1, HZ_E_RED_GLK1 = 2, HZ_E_RED_GLK2 = 3,
  HZ_E_RED_O4 = 4, HZ_E_RED_CMPO4 = 5,
  HZ_E_RED_O6 = 6,  /* sixth-order cross (Sec. 5.2.3), ReD-O2 rows within two
                       nodes of the boundary                                */
  HZ_E_RED_9PT = 7  /* ReD-9ptO2 (Appendix B): the fitted compact 3x3
                       scheme, 2nd-order Sommerfeld ghosts                 */
} hz_ekind;

/* Arithmetic of the preconditioner (V-cycle, deflation, inner coarse
 * solve).  The outer flexible GMRES, its Arnoldi process, Givens updates,
 * residuals and solution update are always complex FP64.
 * HZ_PREC_MIXED_BF16 is HZ_PREC_MIXED_FP32 with the vectors of the V-cycle
 * hierarchy (level right-hand sides, iterates and smoothed iterates) stored
 * as BF16 pairs; the V-cycle's input and output and all arithmetic stay FP32. */
typedef enum {
  HZ_PREC_FP64 = 0, HZ_PREC_MIXED_FP32 = 1, HZ_PREC_MIXED_BF16 = 2
} hz_precision;

/* Outer Krylov iteration, both right-preconditioned by A-DEF1 and flexible
 * (variable inner tolerance, Sec. 6.3): FGMRES (Arnoldi + Givens, the
 * iterate formed at the end) or the preconditioned GCR of Sec. 3.3 / 6.3
 * (the iterate and residual updated every step; each step one CUDA graph
 * launch, one graph per step index for the first 128 steps).  Both store
 * two sets of outer_maxit FP64 vectors. */
typedef enum { HZ_OUTER_FGMRES = 0, HZ_OUTER_GCR = 1 } hz_outer;

/* Two-level preconditioner: A-DEF1 (APD with the higher-order Z), eq. ADEF1,
 * P = M^-1 (I - A Q) + Q; or the practical TLKM of Sec. 3.2.2,
 * P = (I - M^-1 A Q~ + Q~) M^-1 (gamma = 1), whose coarse system
 * I_h^2h I_2h^h M_2h^-1 A_2h v2 = v1 (Sec. 5.2, eq. TLKM CGP) is solved by
 * GMRES on that operator (R_Z Z after a V-cycle on M_2h after E). */
typedef enum { HZ_PRECOND_ADEF1 = 0, HZ_PRECOND_TLKM = 1 } hz_precond;

/* Scale of the deflation restriction R_Z.  CONSISTENT: R_Z = Z^T / 4, the
 * scale on which R_Z A Z matches the re-discretised coarse operators (those
 * of A_2h).  PRINTED: the unscaled Z^T that Sec. 3.2.1 prints (1/2 [1 2 1]
 * in 1-D; the higher-order restriction of eq. O4 matrix-free restriction,
 * stencil sum 4), with the re-discretised operators and the ReD-O2 rows of
 * ReD-Glk kept at the A_2h scale and the 5x5 ReD-Glk rows as printed (the
 * scale of Z^T A Z); this combination reproduces the outer iteration counts
 * the paper prints for re-discretised coarse operators.  The Galerkin E and
 * TLKM do not depend on the scale: with HZ_E_GALERKIN the library keeps
 * Z^T / 4 under either choice. */
typedef enum { HZ_DEFL_SCALE_CONSISTENT = 0, HZ_DEFL_SCALE_PRINTED = 1 } hz_defl_scale;

typedef struct {
  int nx, ny;                 /* nodes; each >= 3                            */
  double h;                   /* grid spacing                                */
  hz_bc bc;
  hz_zkind zkind;
  hz_ekind ekind;
  hz_precision prec;
  double beta1, beta2;        /* CSLP shift, default (1, -0.5) (Sec. 3.1),
                                 entering M = -Lap - (beta1 - i beta2) k^2 as
                                 the coefficient printed in Sec. 5.1;
                                 beta2 = +0.5 gives the sign of the Sec. 3.1
                                 definition, M = -Lap - (1 - 0.5i) k^2      */
  double jacobi_omega;        /* damped Jacobi weight, default 0.8 (Sec. 3.1)*/
  int min_coarse_intervals;   /* coarsening stop rule, default 2 (Sec. 4)    */
  double coarse_tol;          /* inner coarse-solve tolerance (Sec. 6.3)     */
  int coarse_maxit;           /* inner iteration cap (= its basis size),
                                 1..3000                                    */
  int outer_maxit;            /* outer FGMRES cap (= its basis size),
                                 1..3000                                    */
  int nrhs_max;               /* right-hand sides per hz_solve call          */
  int inner_basis_fp16;       /* mixed precisions only: store the inner
                                 coarse-solve Krylov basis as FP16 pairs
                                 (arithmetic stays FP32); 0 = FP32 basis   */
  int outer_solver;           /* HZ_OUTER_FGMRES (default) or HZ_OUTER_GCR  */
  int preconditioner;         /* HZ_PRECOND_ADEF1 (default) or HZ_PRECOND_TLKM
                                 (needs zkind != HZ_Z_NONE)                 */
  int deflation_levels;       /* 0 or 1 (default): the paper's two-level
                                 method.  D = 2 .. 23: multilevel deflation
                                 (the multilevel direction of Sec. 1 / 7,
                                 our reading): the coarse system of every
                                 level l < D is solved by flexible GMRES
                                 preconditioned by A-DEF1 built from it,
                                 deflating to level l + 1 (ReD-Glk2 below
                                 level 1); level D by V-cycle-preconditioned
                                 GMRES; every level to coarse_tol with
                                 coarse_maxit iterations at most.  Needs
                                 deflation vectors, A-DEF1 and D coarsenings
                                 (HZ_INVALID_GRID otherwise); each level's
                                 loop is a WHILE node nested in its parent's
                                 in the CUDA graph; not in groups.          */
  int no_cuda_graph;          /* 0 (default): each outer iteration of hz_solve
                                 runs as one CUDA graph launch whose inner
                                 coarse-solve loop is a device-side WHILE
                                 node; 1: the same kernels issued one by one
                                 with a host completion check every 4 inner
                                 iterations.  Results are the same.         */
  int deflation_scaling;      /* hz_defl_scale; default CONSISTENT.  PRINTED
                                 needs deflation_levels <= 1.             */
  int restart;                /* FGMRES only: 0 (default) no restart; m in
                                 1 .. outer_maxit: after every m iterations
                                 the iterate is formed and the Arnoldi process
                                 starts again from the true residual b - A x
                                 (GMRES(m)); the stopping test keeps ||b||;
                                 outer_maxit still caps the total           */
} hz_desc;

typedef struct {
  int outer_iters;            /* outer FGMRES iterations of this RHS         */
  int inner_iters_total;      /* inner coarse-solve iterations, summed       */
  int inner_iters_max;        /* largest single coarse solve                 */
  double relres;              /* true ||b - A x|| / ||b|| after the solve    */
  hz_status status;
} hz_solve_info;

typedef struct hz_solver hz_solver;

/* Operators exposed one by one (parity tests, benchmarks). */
typedef enum {
  HZ_OP_HELMHOLTZ = 0,     /* y = A_h x, level 0, FP64 (Sec. 2.1, Alg. 2)   */
  HZ_OP_CSLP = 1,          /* y = M_l x on level l (Sec. 3.1, 5.1)          */
  HZ_OP_VCYCLE = 2,        /* y = one V-cycle for M_l y = x from level l    */
  HZ_OP_RESTRICT_FW = 3,   /* y(level l+1) = full weighting of x(level l)   */
  HZ_OP_PROLONG_BILINEAR = 4, /* y(level l) = bilinear interp. of x(l+1)    */
  HZ_OP_RESTRICT_Z = 5,    /* y(level 1) = Z^T x / 4                        */
  HZ_OP_PROLONG_Z = 6,     /* y(level 0) = Z x(level 1)                     */
  HZ_OP_COARSE_E = 7,      /* y = E x on level 1 (Sec. 5.2)                 */
  HZ_OP_COARSE_SOLVE = 8,  /* y ~= E^-1 x by the inner CSLP-GMRES           */
  HZ_OP_PRECOND = 9        /* y = P_A-DEF1 x = M^-1 (x - A Q x) + Q x       */
} hz_op;

/* Fills *d with the paper's defaults for an nx x ny grid of spacing h. */
void hz_desc_default(hz_desc* d, int nx, int ny, double h);

/* Device workspace bytes hz_setup needs for *d (grows with nrhs_max,
 * outer_maxit and coarse_maxit).  Returns HZ_INVALID_GRID / HZ_INVALID_ARG
 * for descriptors hz_setup would reject. */
hz_status hz_workspace_bytes(const hz_desc* d, size_t* bytes);

/* Builds the level hierarchy (Sec. 4 coarsening, injected wavenumber), the
 * Jacobi diagonals and the inverted coarsest-level CSLP, all inside the
 * workspace, on stream `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream).  k2_dev: device FP64 [ny][nx], k(x,y)^2; it is copied.
 * workspace_dev must be 256-byte aligned.  *out receives a host handle. */
hz_status hz_setup(const hz_desc* d, const double* k2_dev,
                   void* workspace_dev, size_t workspace_bytes,
                   void* cuda_stream, hz_solver** out);

/* Solves A x = b for nrhs right-hand sides (nrhs <= nrhs_max) by flexible
 * GMRES right-preconditioned with A-DEF1 (eq. ADEF1), stopping each RHS when
 * its least-squares residual falls below tol * ||b|| (Sec. 6.3).  b_dev,
 * x_dev: device complex128 [nrhs][ny][nx].  If use_x0 is nonzero x_dev holds
 * the initial guess, otherwise it is ignored.  info_host: array of nrhs
 * records, or NULL.  Returns HZ_OK when every RHS converged, else the first
 * failing status. */
hz_status hz_solve(hz_solver* s, const void* b_dev, void* x_dev, int nrhs,
                   double tol, int use_x0, hz_solve_info* info_host);

/* hz_solve without a host synchronisation (the paper has no counterpart):
 * the whole solve (start, the outer FGMRES loop as a device-side WHILE loop
 * holding the inner one, the update of x, the true residual and the report)
 * is one CUDA graph, captured on the first call for these buffers, nrhs,
 * tol and use_x0 (up to 4 are kept) and launched on the solver's stream;
 * the call returns as soon as it is enqueued.  info_dev: device memory for
 * nrhs hz_solve_info records, written by the graph's last kernel (status
 * HZ_TIMEOUT for every RHS if a bounded wait ran out).  x_dev and info_dev
 * are valid once the stream reaches the end of the solve.  Needs FGMRES
 * without restart and with CUDA graphs (HZ_INVALID_ARG otherwise); the
 * first call on new buffers must not be made during a stream capture. */
hz_status hz_solve_async(hz_solver* s, const void* b_dev, void* x_dev, int nrhs,
                         double tol, int use_x0, hz_solve_info* info_dev);

/* hz_solve with host buffers: copies b_host to the device, solves, copies
 * the solution back to x_host, all on the solver's stream. */
hz_status hz_solve_host(hz_solver* s, const void* b_host, void* x_host,
                        int nrhs, double tol, hz_solve_info* info_host);

/* Applies one operator of the method (see hz_op) to nrhs vectors.  x_dev and
 * y_dev are device complex128 full grids of the levels the operator maps
 * between.  Operators of the preconditioner run in the solver's precision
 * (inputs rounded, outputs widened under HZ_PREC_MIXED_FP32). */
hz_status hz_apply(hz_solver* s, hz_op op, int level, const void* x_dev,
                   void* y_dev, int nrhs);

/* Iteration counts of the most recent inner coarse solve, one per RHS. */
hz_status hz_last_inner_iters(hz_solver* s, int* iters_host, int nrhs);

/* Number of levels (finest = 0) and the node counts of level l. */
int hz_num_levels(const hz_solver* s);
hz_status hz_level_shape(const hz_solver* s, int level, int* nx, int* ny);

/* The paper solves forward problems only and has no counterpart of this
 * entry point; it builds on the paper's solver (the adjoint solve reuses it
 * unchanged, see below).
 * Adjoint gradient of J(m) = 1/2 sum_s ||S u_s - d_s||^2 with respect to the
 * squared slowness m, k^2 = omega^2 m (k^2 is the array given to hz_setup).
 * S samples u at the nrec flat node indices rec_idx_dev (device int32).
 * src_dev: device complex128 [nshots][ny][nx]; d_obs_dev: device complex128
 * [nshots][nrec].  Shots are processed in batches of nrhs_max: forward
 * solve, adjoint solve A x = conj(D^-1 S^T (S u - d)) with the same solver
 * (D A is symmetric, so A^H = D conj(A) D^-1), lam = D conj(x), then
 * grad_dev[n] = -sum_s Re(conj(lam_s,n) dA_nn/dm_n u_s,n).  grad_dev:
 * device FP64 [ny][nx], overwritten.  *J_host receives J.  info_host: 2 *
 * nshots records (forward then adjoint per shot) or NULL. */
hz_status hz_gradient(hz_solver* s, double omega, const void* src_dev,
                      int nshots, const int* rec_idx_dev, int nrec,
                      const void* d_obs_dev, double tol, double* J_host,
                      double* grad_dev, hz_solve_info* info_host);

/* Releases the host handle (the workspace stays the caller's).  Resource
 * handling only; the paper has no counterpart. */
hz_status hz_destroy(hz_solver* s);

/* Size of the fixed device scratch array used by
 * hz_coarse_galerkin_noalloc (32 MiB). */
#define HZ_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* y = (Z^T / 4) A_h Z x, the straightforward Galerkin coarse operator (the
 * same result as hz_apply with HZ_OP_COARSE_E on an FP64 solver set up with
 * HZ_E_GALERKIN), for callers that cannot allocate device memory: services
 * whose device-memory budget is fixed when they start, plug-ins running
 * inside a host framework that owns all device memory, and latency-critical
 * loops that must not block in an allocator.  The paper has no counterpart;
 * this entry point exists only for such callers.
 *
 * Nothing is allocated: the two fine-grid intermediates live in one
 * library-owned device array of HZ_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library keeps until the process exits.  The caller still
 * passes the inputs and the output:
 *   nx, ny      fine grid nodes (odd, >= 5); the coarse grid has
 *               ((nx+1)/2) x ((ny+1)/2) nodes
 *   h           fine spacing; bc, zkind (HZ_Z_BILINEAR or HZ_Z_HO)
 *   k2_dev      device FP64 [ny][nx] squared wavenumber of the fine grid
 *   x_dev/y_dev device complex128 [nrhs][ncy][ncx] coarse vectors
 *   cuda_stream cudaStream_t the work is issued on (NULL = default stream)
 * Returns HZ_WORKSPACE_TOO_SMALL when 2 * nrhs * nx * ny * 16 bytes exceed
 * HZ_NOALLOC_SCRATCH_BYTES (no work is issued), HZ_INVALID_ARG for bad
 * arguments, HZ_CUDA_ERROR if a launch fails, or, before any work is
 * issued, if a CUDA error is already pending on the calling thread (that
 * error is left pending for the caller).
 *
 * The first call on each device looks up the array's device address with
 * cudaGetSymbolAddress (with that device current); make that first call
 * before any stream capture begins.  The address is kept for the life of
 * the process: it assumes the device's primary context is not reset
 * (cudaDeviceReset) while the library is loaded.  All calls share the one array: calls
 * whose work overlaps on the GPU (other streams, other threads) race and
 * must be serialised by the caller.  No state carries over between calls:
 * every scratch entry read is written by the same call first. */
hz_status hz_coarse_galerkin_noalloc(int nx, int ny, double h, hz_bc bc,
                                     hz_zkind zkind, const double* k2_dev,
                                     const void* x_dev, void* y_dev, int nrhs,
                                     void* cuda_stream);

/* Grids of different sizes solved together (a batching extension: the
 * paper solves one grid at a time and has no counterpart).  Member g of
 * the group (up to HZ_MAX_GROUP solvers, each set up on its own grid and
 * workspace) solves nrhs[g] right-hand sides b_dev[g] -> x_dev[g] (layout
 * and x0 = 0 as hz_solve) to tol.  Every outer and inner Krylov iteration of
 * all members advances together: each member's stencil, transfer and
 * coarse-operator kernels run on its own grid, and the Gram-Schmidt kernels
 * of all members run as one persistent launch over a table of the members'
 * tiles, so small grids share the GPU instead of taking turns.  A member
 * that converged only skips its work.  Members must agree in precision class
 * (FP64 or mixed), inner-basis storage and deflation on/off (HZ_INVALID_ARG
 * otherwise, and for a repeated member); they run on members[0]'s stream.
 * Each outer iteration of the active members is one CUDA graph launch
 * (unless a member was set up with no_cuda_graph): in the graph every
 * member's own kernels run on a branch of their own, concurrently with the
 * other members', joined before each grouped Gram-Schmidt step, and the
 * inner coarse solves advance together in a device-side WHILE loop.  The
 * graphs are captured on first use within the call (one per set of active
 * members) and released before it returns.  info[g] (nrhs[g] entries) may
 * be null.  Returns the worst status over the members. */
#define HZ_MAX_GROUP 8
hz_status hz_solve_group(hz_solver* const* members, int count, const void* const* b_dev,
                         void* const* x_dev, const int* nrhs, double tol,
                         hz_solve_info* const* info);

/* hz_gradient for a group of grids: member g uses omega[g], nshots[g]
 * sources src_dev[g], receivers rec_idx_dev[g] (nrec[g]) and data
 * d_obs_dev[g], and receives J_host[g] and grad_dev[g] (its own grid).  Shot
 * batches of all members run their forward and adjoint solves together
 * through hz_solve_group. */
hz_status hz_gradient_group(hz_solver* const* members, int count, const double* omega,
                            const void* const* src_dev, const int* nshots,
                            const int* const* rec_idx_dev, const int* nrec,
                            const void* const* d_obs_dev, double tol, double* J_host,
                            double* const* grad_dev, hz_solve_info* const* info);

/* Kernel classes that hz_profile_* can time: the multi-vector dot product
 * and the multi-vector update of the Gram-Schmidt step (Alg. 1 inner loop),
 * which carry the basis traffic of both Krylov solvers, and the two fused
 * smoothing/transfer kernels at the top level of every V-cycle (Sec. 3.1;
 * their staged form, hz_tuning.vcycle_fused = 2, only). */
typedef enum {
  HZ_KC_NONE = 0, HZ_KC_MDOT = 1, HZ_KC_MAXPY = 2, HZ_KC_VCYCLE = 3
} hz_kernel_class;

/* Starts timing every launch of kernel class kc on the solver's stream:
 * CUDA events bracket each launch (at most max_launches are kept) and the
 * kernels add their algorithmic bytes (basis vectors and w read, w written,
 * per active RHS) to a counter in the workspace.  HZ_KC_NONE stops it. */
hz_status hz_profile_begin(hz_solver* s, hz_kernel_class kc, int max_launches);

/* Synchronises the stream and returns the launches timed, their summed
 * duration in ms and their summed algorithmic bytes; ends profiling.
 * HZ_INVALID_ARG if the event pool overflowed (totals then incomplete). */
hz_status hz_profile_end(hz_solver* s, long long* launches, double* ms_total,
                         double* alg_bytes);

/* Kernels launched by this library since it was loaded (all solvers),
 * including the kernels run inside the device-side loops of CUDA graphs
 * (read from the current device's counter). */
long long hz_kernel_launches(void);

/* Launch operations the host issued since the library was loaded: each
 * kernel launched directly and each CUDA graph launched counts one (a
 * graph's kernels count once, with the graph).  The paper has no
 * counterpart; it measures how much of the work runs from graphs. */
long long hz_host_launches(void);

/* Implementation choices that leave the method's arithmetic unchanged up to
 * rounding order.  hz_setup starts from hz_tuning_default; hz_autotune
 * times the candidates on the solver's own workspace and keeps the fastest;
 * hz_set_tuning sets them directly (e.g. from a cache of an earlier
 * tuning).  The paper has no counterpart: its CPU code has one kernel per
 * operation. */
typedef struct {
  int mdot_kernel;  /* multi-vector dot product of the Gram-Schmidt step:
                       0 register-pipelined (each block streams basis rows
                       through registers), 1 TMA ring (bulk copies into a
                       6-stage shared-memory ring, 8 consumer warps per SM),
                       2 TMA ring with 16 consumer warps                   */
  int maxpy_kernel; /* multi-vector update of the Gram-Schmidt step, the
                       same three choices                                  */
  int galerkin_apply; /* HZ_E_GALERKIN only: 0 the product R_Z (A_h (Z x))
                       on the fly each application (str-Glk, Sec. 5.2.1),
                       1 the product's 5x5 (higher-order Z) or 3x3 (bilinear
                       Z) stencil stored per coarse node at setup and applied
                       as a stencil (stcl-op-Glk, Table 1)                 */
  int e_rhs_per_block; /* stored-stencil E: right-hand sides that one block
                       walks through with its coefficients held in registers
                       (0 = all of them; else 1..1024)                     */
  int vcycle_fused; /* 0 the V-cycle's smoothing and transfers as separate
                       kernels; 1 pre-smoothing + residual + restriction and
                       prolongation + post-smoothing fused into one tiled
                       kernel each (the intermediate iterate stays in shared
                       memory), one block per tile and right-hand side;
                       2 the same fused kernels with each block walking over
                       vcycle_rhs_per_block right-hand sides, its tile's
                       coefficients held in registers and the input tiles
                       copied ahead into a ring of shared-memory stages;
                       the restriction kernel gives each thread one coarse
                       node and its 2 x 2 fine nodes                       */
  int vcycle_rhs_per_block; /* vcycle_fused = 2: right-hand sides per block
                       (0 = all of them; else 1..1024); levels with too few
                       tiles for two blocks per SM halve it (down to 1)    */
  int vcycle_tile;  /* vcycle_fused = 2, prolongation + post-smoothing:
                       0 = blocks of 32 x 8 fine nodes, one thread per fine
                       node; 1 = blocks of 64 x 16 fine nodes, one thread
                       per coarse cell and its 2 x 2 fine nodes            */
  int e_column_pairs; /* stored-stencil E: 0 one coarse node per thread;
                       1 two nodes of a column per thread, which share the
                       rows of x they read                                 */
} hz_tuning;

/* Candidates hz_autotune times, in the order of its ms[] output:
 * mdot_kernel 0, 1, 2; maxpy_kernel 0, 1, 2; galerkin_apply 0, 1;
 * e_rhs_per_block 0, 8, 4; vcycle_fused 0, 1; then vcycle_fused 2 with
 * (vcycle_rhs_per_block, vcycle_tile) = (4, 0), (8, 0), (16, 0), (4, 1),
 * (8, 1), (16, 1); e_column_pairs 1 (with the e_rhs_per_block picked). */
#define HZ_TUNE_CANDIDATES 20

void hz_tuning_default(hz_tuning* t);

/* Times the candidates on this solver's workspace and stream and keeps the
 * fastest of each (as hz_set_tuning; *best receives them if not null).
 * ms[HZ_TUNE_CANDIDATES], if not null, receives the time of one launch per
 * candidate (-1 where not applicable), each for nrhs right-hand sides: the
 * Gram-Schmidt dot and update kernels at Arnoldi column min(maxit - 1, 64)
 * of the inner solver (of the outer one without deflation) on synthetic
 * basis rows, then E (Galerkin E only) on the fly and stored, then the
 * stored stencil's RHS per block, then one V-cycle from level 1 (level 0
 * without deflation) unfused and fused.
 * Overwrites the iteration state in the workspace: call it between solves.
 * HZ_INVALID_ARG for nrhs outside 1..nrhs_max. */
hz_status hz_autotune(hz_solver* s, int nrhs, hz_tuning* best, double* ms);
/* HZ_INVALID_ARG for a null pointer or an out-of-range field. */
hz_status hz_get_tuning(const hz_solver* s, hz_tuning* t);
hz_status hz_set_tuning(hz_solver* s, const hz_tuning* t);

/* Fault drill (a test control; the paper has no counterpart).  The TMA-ring
 * Gram-Schmidt kernels (hz_tuning.mdot_kernel / maxpy_kernel 1 or 2) bound
 * every pipeline wait; a wait that runs out stops the kernel's work, sets a
 * flag the host reads after the launch, and the call returns HZ_TIMEOUT
 * with the solver still usable (the flag is cleared as it is reported).
 * This call sets the bound of those waits to wait_seconds (0 < w <= 2; 2 is
 * the default) and, with starve_copies nonzero, makes the kernels' producer
 * warp issue no copies, so that every consumer wait runs out with nothing in
 * flight: the way to check the timeout path without a fault.
 * hz_fault_drill(s, 0, 2.0) restores normal operation.  HZ_INVALID_ARG for a
 * null solver or a bound outside (0, 2]. */
hz_status hz_fault_drill(hz_solver* s, int starve_copies, double wait_seconds);

const char* hz_status_str(hz_status st);
const char* hz_last_error(const hz_solver* s);

#ifdef __cplusplus
}
#endif

#endif /* HZ_H_ */

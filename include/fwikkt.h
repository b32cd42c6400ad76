/*
 * fwikkt.h -- C ABI of the GB300 full-space Gauss-Newton FWI library.
 *
 * Method: Malovichko, Orazbayev & Khokhlov, "Iterative PDE-constrained
 * optimization for seismic full-waveform inversion" (arXiv:2204.06489).
 * Each Gauss-Newton step solves the KKT system of Sec. 4 (eq. KKT) with a
 * right-preconditioned flexible GMRES whose preconditioner is the
 * block-triangular matrix of Sec. 5 (eq. precond; eq. precond_approx with
 * inexact block solves).  The inexact Helmholtz block solves are BiCGStab
 * iterations preconditioned by a multigrid cycle of the shifted operator
 * (the shifted-Laplacian route named at the end of Sec. 5).
 *
 * Conventions shared by every call
 *   - Status: every int-returning call returns FWI_OK (0) or a negative
 *     FWI_E_* code; fwi_last_error() then describes the failure.  No call
 *     throws across the ABI.  Calls on one context are not thread-safe.
 *   - Units: SI; frequencies in Hz (omega = 2 pi f); gamma (squared slowness,
 *     Sec. 2) in s^2/m^2.  Complex numbers are interleaved (re, im) pairs.
 *   - Grids: an instance has nx x nz core nodes, npml absorbing nodes on every
 *     side (padded Nx = nx + 2 npml, Nz = nz + 2 npml), flat index j*Nx + i
 *     (x fast).  "Core" arrays are [nz][nx] row-major.
 *   - Blocks: one Helmholtz problem per (instance, frequency, source)
 *     (Sec. 2, eq. helmholtz_j), ordered instance-major, then frequency, then
 *     source.  A "field" buffer holds all blocks' padded grids back to back.
 *   - Scaling: the library solves the exactly rescaled system
 *     A' = h^2 A, lambda' = lambda / h^2, ds~ = ds / gamma_ref (see
 *     fwi_kkt_solve); results are returned in physical units.
 *   - Ownership: the context owns the device memory it allocates (released
 *     by fwi_destroy).  Host pointers are read or written only during the call.
 *     Device pointers (arguments documented as "device") must be valid CUDA
 *     device memory of the context's device, are accessed on the context's
 *     stream, and must stay valid until that stream has finished the call's work
 *     (every call below synchronises its stream before returning unless stated).
 */
#ifndef FWIKKT_H
#define FWIKKT_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FWI_OK 0
#define FWI_E_INVAL (-1)   /* bad argument or call order                      */
#define FWI_E_NOMEM (-2)   /* device allocation failed (before any launch)    */
#define FWI_E_CUDA (-3)    /* a CUDA runtime call or kernel launch failed     */
#define FWI_E_NOCONV (-4)  /* iteration cap reached; results and stats valid  */
#define FWI_E_NUMERIC (-5) /* NaN/Inf detected, or gamma <= 0                 */

/* ---- inner products of the FGMRES orthogonalisation (fwi_opts.arnoldi_dots) --
 * RUNS: FP32 products summed in FP32 runs of 64 per thread, runs summed in FP64.
 * FP64: every product formed and summed in FP64 (exact products of floats).
 * COMP: compensated dot product (Dot2 of Ogita, Rump & Oishi 2005): exact FP32
 *       product splitting and error-free sums per thread, as accurate as a dot
 *       product in twice the working precision; threads summed in FP64. */
#define FWI_DOT_RUNS 0
#define FWI_DOT_FP64 1
#define FWI_DOT_COMP 2
#define FWI_HBLOCK_MAX 8   /* pairs of the quasi-Newton H block */

/* ---- precision modes ---------------------------------------------------- */
#define FWI_C128 0        /* complex128 throughout ("plain FP64 GPU form")       */
#define FWI_C64_REFINE 1  /* complex64 bulk, FP64 dots / coarsest level / refinement */

typedef struct fwi_ctx fwi_ctx;

/* Grid of one instance (Sec. 2).  The absorbing layer has the quadratic
 * profile sigma(d) = sigma_max (d / (npml h))^2 with
 * sigma_max = 3 pml_c ln(1/pml_R) / (2 npml h) and X = 1 + i sigma / omega. */
typedef struct {
  int nx, nz;     /* core nodes                                    */
  int npml;       /* absorbing-layer nodes on each of the 4 sides  */
  double h;       /* grid spacing [m]                              */
  double pml_c;   /* reference velocity of the layer profile [m/s] */
  double pml_R;   /* target reflection coefficient (0 < R < 1)     */
} fwi_grid;

/* Solver options.  fwi_default_opts() fills the defaults given in brackets. */
typedef struct {
  int precision;          /* FWI_C64_REFINE | FWI_C128                  [C64_REFINE] */
  double eps;             /* regulariser weight on the relative model (s/gamma_ref);
                             the paper's L = eps I equals eps / gamma_ref^2     [1e-3] */
  int include_Ls_n;       /* keep the -L s_n term of the KKT right-hand side   [1]   */
  double tol;             /* target ||b - M xi|| / ||b|| of the KKT solve      [1e-6] */
  int restart;            /* FGMRES restart length (Sec. 6 uses 30)            [30]   */
  int max_outer;          /* cap on FGMRES iterations over all sweeps          [600]  */
  double sweep_tol;       /* c64 FGMRES tolerance per refinement sweep         [1e-3] */
  int max_refine;         /* cap on FP64 refinement sweeps                     [8]    */
  int inner_iters;        /* BiCGStab iterations per preconditioner block solve [4]  */
  double inner_tol;       /* > 0: stop a block's inner solve at this relative
                             residual (exact-preconditioner mode uses 1e-12)   [0]    */
  int mg_cycle;           /* cycle index on levels 1..mg_wdepth (2 = W)        [2]    */
  int mg_wdepth;          /* deepest level that repeats its correction; V below [2]  */
  int nu1, nu2;           /* pre / post Jacobi sweeps                          [2, 2] */
  double omega_jac;       /* Jacobi damping                                    [0.5]  */
  double shift_beta;      /* shifted operator omega^2 -> (1 + i beta) omega^2  [0.5]  */
  double sigma_cap;       /* clip sigma/omega of the shifted operator's layer  [1.0]  */
  int mg_levels;          /* 0 = automatic                                     [0]    */
  double fwd_tol;         /* forward/adjoint wavefield residual target (FP64)  [1e-9] */
  int fwd_iters;          /* BiCGStab iterations of the first forward refinement sweep;
                             doubled (up to 8x) after a sweep that gains < 20x [60]   */
  int max_fwd_refine;     /* cap on forward refinement sweeps                  [20]   */
  int use_graph;          /* replay the preconditioner from a CUDA graph       [1]    */
  int arnoldi_dots;       /* FGMRES inner products (orthogonalisation, norms) of complex64
                             vectors: FWI_DOT_RUNS, FWI_DOT_FP64 or FWI_DOT_COMP (see below);
                             complex128 vectors always use FP64                  [COMP] */
  int check_orth;         /* measure max |I - V^T V| of every FGMRES basis into
                             fwi_stats.orth_loss (diagnostics, costs extra dots) [0]   */
  int strip_rows;         /* rows per warp of the column-strip stencil kernels on level 0
                             (2..64; half as many on the coarser global levels) [16]  */
  int coarse_threads;     /* threads per CTA of the shared-memory coarse cycle (512 | 1024) [512] */
  int fwd_warm;           /* start the forward solve from the previous forward wavefields
                             of this context (same tolerance; 0: from zero)      [1]    */
  int outer_solver;       /* KKT Krylov method: 0 FGMRES(restart); 1 BiCGStab in the real
                             inner product (eight KKT-size vectors, no basis; the
                             memory-lean option of Sec. 7); outer_iters then counts
                             BiCGStab iterations (two preconditioner applications each) [0] */
  int inner_solver;       /* block solves inside the preconditioner: 0 BiCGStab with the
                             shifted-Laplacian multigrid cycle; 1 BiCGStab with ILU(0) of A';
                             2 one ILU(0) application as A~ (the paper's incomplete-LU
                             approximation, zero fill); forward/adjoint modelling always
                             uses 0 (fwi_inner_solve: 1 and 2 mean BiCGStab + ILU(0)) [0] */
  int hblock;             /* H block of the preconditioner (Sec. 5 after eq. precond):
                             0 the paper's L = eps I; 1 the L-BFGS inverse built from the
                             pairs of fwi_hblock_set with H_0 = (1/eps) I (no pairs: as 0) [0] */
} fwi_opts;

typedef struct {
  int outer_iters;        /* FGMRES iterations, all sweeps                      */
  int refinements;        /* FP64 refinement sweeps                             */
  int fwd_sweeps;         /* forward-solve refinement sweeps                    */
  long long inner_iters;  /* BiCGStab iterations x blocks                       */
  double rel_res;         /* final ||b - M xi|| / ||b|| recomputed in FP64 (max over instances) */
  double misfit;          /* data misfit 1/2 sum |W r|^2 at the step's model (sum over instances) */
  double t_setup_ms, t_forward_ms, t_solve_ms;
  double fwd_rel_res;     /* final max_b ||f_b - A u_b|| / ||f_b|| of the forward / adjoint solve */
  double orth_loss;       /* max |I - V^T V| over the FGMRES bases (with opts.check_orth), else 0 */
  int fwd_warm;           /* 1 if the forward solve started from the previous wavefields */
} fwi_stats;

/* Layout of the context's buffers (element counts). */
typedef struct {
  int n_instances;
  int n_blocks;               /* all instances                                     */
  long long field_elems;      /* complex elements of one field buffer (all blocks) */
  long long ctrl_elems;       /* real elements of the control (all instances' cores) */
  long long kkt_elems;        /* real elements of a packed KKT vector =
                                 4*field_elems + ctrl_elems, order [du | lambda | ds] */
} fwi_layout_info;

/* Fill *o with the defaults listed in fwi_opts. */
void fwi_default_opts(fwi_opts *o);

/* Create a context with n_instances independent problems on the current CUDA
 * device.  grids: host array [n_instances].  cuda_stream: a cudaStream_t on
 * which all work is queued; NULL makes the context create a private blocking
 * stream (ordered with the legacy default stream) on first device use, because
 * the legacy stream cannot be captured into a CUDA graph.  *out receives the
 * context (NULL on failure).  Makes no CUDA call.  Returns FWI_E_INVAL for bad
 * grid values. */
int fwi_create(fwi_ctx **out, int n_instances, const fwi_grid *grids, void *cuda_stream);

/* Sources and receivers of one instance (Sec. 2: point sources f_k, receivers
 * x_kj, observation operator Q by sampling at nodes).  All arrays are host:
 * freq_hz[n_freq]; src_ix, src_iz [n_src] core indices; src_amp [2*n_src]
 * complex amplitudes; rec_offsets [n_src+1] CSR offsets into rec_ix, rec_iz,
 * rec_weight (diagonal W; NULL = all 1).  Must be called once per instance
 * before fwi_set_model.  FWI_E_INVAL for indices outside the core. */
int fwi_set_survey(fwi_ctx *ctx, int inst, int n_freq, const double *freq_hz, int n_src,
                   const int *src_ix, const int *src_iz, const double *src_amp,
                   const int *rec_offsets, const int *rec_ix, const int *rec_iz,
                   const double *rec_weight);

/* Model gamma = 1/c^2 of one instance on the core, [nz][nx] FP64, host
 * (on_device = 0) or device (on_device = 1).  The first call also freezes the
 * absorbing layer's gamma (edge replication of this model) and, for
 * gamma_ref <= 0, sets gamma_ref = mean(gamma_core); later calls replace the
 * core only.  FWI_E_NUMERIC for gamma <= 0 or non-finite values. */
int fwi_set_model(fwi_ctx *ctx, int inst, const double *gamma_core, double gamma_ref,
                  int on_device);

/* Copy the current core model of one instance to gamma_core [nz][nx] (host). */
int fwi_get_model(fwi_ctx *ctx, int inst, double *gamma_core);

/* Observed data d of one instance: [n_freq][rec_total] complex (2 doubles per
 * entry), host or device.  rec_total = rec_offsets[n_src]. */
int fwi_set_observed(fwi_ctx *ctx, int inst, const double *d, int on_device);

/* Forward modelling of every block at the current models (Sec. 2, Au = f):
 * FP64-refined inner solves until ||f - A u|| / ||f|| <= opts->fwd_tol.
 * d_pred (host, nullable): predicted data Q u, all instances back to back,
 * [inst][n_freq][rec_total] complex.  misfit (host, nullable) [n_instances]:
 * 1/2 sum |W (d - Q u)|^2 (needs observed data).  The wavefields stay in the
 * context for fwi_kkt_solve / fwi_gradient. */
int fwi_forward(fwi_ctx *ctx, const fwi_opts *opts, double *d_pred, double *misfit,
                fwi_stats *stats);

/* Copy the forward wavefield of all blocks (field layout, complex128) into u
 * (device, 2*field_elems doubles).  Requires fwi_forward. */
int fwi_get_wavefields(fwi_ctx *ctx, double *u_device);

/* Misfit and its gradient with respect to the core gamma (Sec. 3: the
 * adjoint-state form of the gradient, -sum_b omega_b^2 Re(conj(u_b) lambda_b)
 * with A^H lambda_b = Q^T W^T W r_b).  Runs the forward solve first.
 * misfit (host) [n_instances]; grad (host or device) all instances' cores back
 * to back, FP64. */
int fwi_gradient(fwi_ctx *ctx, const fwi_opts *opts, double *misfit, double *grad,
                 int on_device, fwi_stats *stats);

/* One KKT solve (Sec. 4, eq. KKT; Sec. 5 preconditioner) at the current models
 * for all instances jointly, using the wavefields of the last fwi_forward.
 * ds (host or device, FP64): the model update of all instances' cores back to
 * back, s^2/m^2.  Stops when every instance's FP64 relative residual of the
 * rescaled system is <= opts->tol (FWI_E_NOCONV with ds and stats filled if
 * max_outer / max_refine are reached first). */
int fwi_kkt_solve(fwi_ctx *ctx, const fwi_opts *opts, double *ds, int on_device,
                  fwi_stats *stats);

/* One Gauss-Newton step (Sec. 3-5): set-up, forward modelling, KKT solve, and
 * the full step s <- s + ds (no line search).  ds as in fwi_kkt_solve
 * (nullable). */
int fwi_newton_step(fwi_ctx *ctx, const fwi_opts *opts, double *ds, int on_device,
                    fwi_stats *stats);

/* One reduced-space Gauss-Newton step (Sec. 3, "RSGN-CG": the normal equations
 * eq. normal_system_discrete_sum solved by conjugate gradients), the paper's
 * comparison method: set-up, forward modelling, CG on
 *   (eps I + Re(P~^H A'^{-H} Q^T W^T W Q A'^{-1} P~)) ds~ = b_s + Re(P~^H A'^{-H} Q^T W^T W r)
 * in the scaled variables of fwi_kkt_solve (same ds), one forward and one
 * adjoint refined block solve (to opts->fwd_tol) per CG iteration, stopping at
 * ||g - H ds~|| / ||g|| <= opts->tol or opts->max_outer iterations; then the
 * full step s <- s + ds.  ds as in fwi_kkt_solve (nullable);
 * stats->outer_iters = CG iterations.  FWI_E_NOCONV (with the step applied) at
 * the iteration cap or when a block solve misses fwd_tol; FWI_E_NUMERIC if
 * p^T H p is not positive. */
int fwi_rsgn_step(fwi_ctx *ctx, const fwi_opts *opts, double *ds, int on_device,
                  fwi_stats *stats);

/* Largest eigenvalue of the Gauss-Newton matrix Re(J~^H W^T W J~) at the
 * current models (Sec. 3, eq. normal_system_discrete2 without the eps I term,
 * in the scaled control ds~ of fwi_kkt_solve; J~ = Q A'^{-1} P~), by `iters`
 * power iterations from the constant vector: v_0 = 1/||1||,
 * w = G v_{k-1}, lambda_k = v_{k-1}^T w, v_k = w / ||w||; *lambda =
 * lambda_iters (a lower bound that rises towards the largest eigenvalue).
 * Each iteration makes one forward and one adjoint refined solve of every
 * block (opts->fwd_tol, opts->precision).  Needs fwi_forward.  With several
 * instances the matrix is block diagonal over them.  Used for the rule
 * eps = alpha * lambda_max that sets the regulariser from the data term.
 * FWI_E_NOCONV if a block solve missed fwd_tol (lambda still written). */
int fwi_normal_lambda_max(fwi_ctx *ctx, const fwi_opts *opts, int iters, double *lambda,
                          fwi_stats *stats);

/* Hessian-vector product of the reduced Gauss-Newton system at the current
 * models (Sec. 3, eq. normal_system_discrete_sum) in the scaled control of
 * fwi_kkt_solve (ds~ = ds / gamma_ref of each instance):
 *   hv = eps v + Re(J~^H W^T W J~) v,  eps = opts->eps (0: the Gauss-Newton part),
 * one forward and one adjoint refined block solve of every block
 * (opts->fwd_tol, opts->precision).  v, hv: ctrl_elems doubles, host
 * (on_device = 0) or device buffers.  Needs fwi_forward.  FWI_E_NOCONV if a
 * block solve missed fwd_tol (hv still written).  Used to build exact
 * curvature pairs (s, H s) for the quasi-Newton H block. */
int fwi_hessian_apply(fwi_ctx *ctx, const fwi_opts *opts, const double *v, double *hv, int on_device,
                      fwi_stats *stats);

/* Curvature pairs of the quasi-Newton H block (opts->hblock = 1; Sec. 5
 * after eq. precond and Sec. 7: the block-triangular preconditioner's
 * H ~ L may be replaced by L-BFGS).  S and Y: m x ctrl_elems doubles,
 * row-major, pair j = (S[j], Y[j]) in the scaled control, oldest first, with
 * Y[j] = H~ S[j] or a secant difference; every pair needs S[j]^T Y[j] > 0
 * (else FWI_E_INVAL and no pairs are kept).  0 <= m <= FWI_HBLOCK_MAX; m = 0
 * removes the pairs.  The pairs are copied (host or device source); they
 * belong to the control layout, so they stay valid across model updates and
 * are used until replaced.  The preconditioner then forms
 * z_s = B^{-1} (v2 + Re(P~^H z_lambda)), B^{-1} the L-BFGS inverse with
 * H_0 = (1/eps) I, in the compact representation of Byrd, Nocedal & Schnabel
 * (two kernels: 2m FP64 dot products and one update). */
int fwi_hblock_set(fwi_ctx *ctx, int m, const double *S, const double *Y, int on_device);

/* ---- operator-level entry points (device buffers, for checks and tools) ----
 * x, y: device field buffers in the given precision (float2 or double2
 * elements, field layout).  The operators use the current models and, where
 * stated, the last forward wavefields. */

/* y = A'_b x_b (adjoint = 0) or A'_b^H x_b (adjoint = 1) for every block: the
 * h^2-scaled 5-point PML Helmholtz operator (Sec. 2, eq.
 * helmholtz_preliminary).  precision: FWI_C128 (double2) or FWI_C64_REFINE
 * (float2). */
int fwi_apply_helmholtz(fwi_ctx *ctx, const void *x, void *y, int adjoint, int precision);

/* y = M xi, the rescaled KKT matrix (Sec. 4, eq. KKT) on packed real vectors
 * of kkt_elems elements (double or float).  Needs fwi_forward. */
int fwi_apply_kkt(fwi_ctx *ctx, const fwi_opts *opts, const void *xi, void *y, int precision);

/* z = P~^{-1} v, the block-triangular preconditioner (Sec. 5, eq.
 * precond_approx) with the inexact block solves of opts, packed vectors. */
int fwi_apply_precond(fwi_ctx *ctx, const fwi_opts *opts, const void *v, void *z,
                      int precision);

/* x = inexact solve A'_b x_b = b_b (adjoint: A'^H) for every block: BiCGStab
 * with multigrid preconditioning, opts->inner_iters iterations (or to
 * opts->inner_tol).  Field buffers. */
int fwi_inner_solve(fwi_ctx *ctx, const fwi_opts *opts, const void *b, void *x, int adjoint,
                    int precision);

/* x = one multigrid cycle for the shifted operator from x = 0 (field buffers). */
int fwi_mg_cycle(fwi_ctx *ctx, const fwi_opts *opts, const void *b, void *x, int precision);

/* Size of the static device array behind fwi_mg_cycle_noalloc (16 MiB). */
#define FWI_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)

/* Same result as fwi_mg_cycle, for callers that must not allocate device
 * memory during the call: code whose device memory is owned by another pool
 * or budget, and code that runs this cycle while other streams are busy, where
 * cudaMalloc / cudaFree would block (cudaFree waits for the whole device).
 * The paper has no counterpart; this is a service of the library.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *     The cycle's level buffers live in one file-scope __device__ array of
 *     FWI_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library keeps
 *     until the process exits.
 *   - Needs a context whose multigrid hierarchy was already built for the same
 *     options and models by an allocating call (fwi_mg_cycle or fwi_forward);
 *     otherwise FWI_E_INVAL.
 *   - Needs at most FWI_NOALLOC_SCRATCH_BYTES of level buffers (about
 *     2 x field_elems complex elements of the given precision); larger batches
 *     get FWI_E_INVAL with the required size in fwi_last_error.
 *   - The first call on each device (with that device current) looks up the
 *     array's device address; make that first call before any stream capture.
 *     The context's device (the device current at its first device use) must
 *     be the current device; otherwise FWI_E_INVAL.
 *   - Live stencil timing (fwi_stencil_timer) is suspended during the call.
 *   - Every call, on every context, shares the one array and leaves its
 *     contents behind; the cycle writes each buffer before reading it, so no
 *     clearing is needed.  Calls whose GPU work overlaps (different streams,
 *     threads or contexts on the same device) race on the array.
 * b, x: device field buffers as in fwi_mg_cycle; precision FWI_C128 or
 * FWI_C64_REFINE.  Synchronises the context's stream before returning. */
int fwi_mg_cycle_noalloc(fwi_ctx *ctx, const fwi_opts *opts, const void *b, void *x, int precision);

/* Sizes of the context's buffers. */
int fwi_get_layout(fwi_ctx *ctx, fwi_layout_info *info);

/* Number of CUDA kernels this library has launched in this process so far
 * (kernels replayed from a CUDA graph included).  Diagnostics only; the paper
 * has no counterpart. */
unsigned long long fwi_kernel_launches(void);

/* Number of cudaMalloc, cudaMallocHost, cudaFree and cudaFreeHost calls this
 * library has made in this process so far.  Diagnostics (it lets a caller
 * check that a call allocated nothing); the paper has no counterpart. */
unsigned long long fwi_memory_calls(void);

/* Live timing of the complex64 level-0 smoother kernel (two damped-Jacobi
 * sweeps of the shifted 5-point operator of Sec. 2 in one pass, every block):
 * while enabled, every launch of it that is not inside a CUDA graph is
 * bracketed by CUDA events on the context's stream, and the kernel counts the
 * grid nodes it processed (blocks whose inner solve has finished are
 * skipped).  Writes (nullable) the accumulated time (ms), the algorithmic
 * bytes (per processed node and sweep: x, b and the result, one complex
 * element each, so six elements per node for the two sweeps and five when the
 * first starts from zero), the launch count, and pass_bytes (per processed
 * node what the fused pass itself must move: b and the result, plus x unless
 * it starts from zero) since the last reset; then enable = 1 resets and turns
 * timing on, 0 resets and turns it off, -1 only reads.  Diagnostics; the
 * paper has no counterpart. */
int fwi_stencil_timer(fwi_ctx *ctx, int enable, double *ms, double *bytes, long long *launches,
                      double *pass_bytes);

/* Kernel profile (diagnostics; the paper has no counterpart).  While it is
 * enabled, every kernel this library launches directly (not inside a stream
 * capture or a CUDA graph) is bracketed by two CUDA events on its stream.
 * Per kernel and multigrid level (-1 where none applies) the profile sums the
 * launches, the event time and the algorithmic bytes each launch site states
 * (every operand read and result written once; a damped-Jacobi sweep counts
 * x, b and the result, so the two-sweep smoother counts six complex elements
 * per node, five when it starts from zero); it also sums the time between one
 * launch's end and the next launch's start ("gap": launch and host latency).
 * The call synchronises the context's stream, then, if buf is not NULL,
 * writes the profile as a NUL-terminated JSON object
 *   {"gap_ms": g, "gaps": n, "rows": [{"kernel": s, "level": l, "launches": n,
 *    "ms": t, "bytes": b}, ...]}
 * into buf (FWI_E_INVAL if buflen is too small; the message gives the size).
 * Then enable = 1 clears the profile and turns it on, 0 clears it and turns
 * it off, -1 changes nothing.  The profile is process-wide. */
int fwi_kernel_profile(fwi_ctx *ctx, int enable, char *buf, long long buflen);

/* Message of the last failure on this context ("" if none). NULL ctx: the
 * message of the last failed fwi_create. */
const char *fwi_last_error(const fwi_ctx *ctx);

/* Release the context and all device memory it owns. NULL is ignored. */
void fwi_destroy(fwi_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* FWIKKT_H */

/*
 * ww.h -- C ABI of the GB300 library for the Jacobian of the standing-water-
 * wave shooting map (Wilkening & Yu, "Overdetermined shooting methods for
 * computing standing water waves with spectral accuracy").
 *
 * The method: the 2 pi-periodic free-surface Euler equations (Sec. 2.1,
 * Eq. ww) are advanced from t = 0 to T/4 by classic RK4 together with the
 * variational equations of every Jacobian column (Sec. 3.3, Eq. q:qdot;
 * App. B, Eqs. l5a, l6a).  In each RK stage the boundary-integral matrices of
 * the base surface (Eq. K1K2, Sec. 2.2) are assembled once, A = 1/2 I + K is
 * factored (or inverted) once, and every column's Dirichlet data is solved
 * against it as one multi-right-hand-side solve (Sec. 3.3).
 *
 * Conventions for every entry point
 *  - All arrays are IEEE double.  Matrices are column-major with leading
 *    dimension N (the number of surface points).
 *  - Unless a name ends in _host, array arguments are DEVICE pointers (memory
 *    of the GPU the context was created on) owned by the caller; the library
 *    only reads inputs and writes outputs, and keeps no reference after the
 *    call returns.  Work is queued on the context's stream (ww_set_stream),
 *    and each call synchronises that stream before returning its status.
 *  - Every call returns WW_OK (0) or a negative WW_ERR_* code; the thread-local
 *    ww_last_error() string says why.  No call aborts or exits the process.
 *  - A context is not thread-safe; use one context per host thread/stream.
 *
 * Grid: alpha_j = 2 pi j / N, j = 0..N-1, N a power of two (16 <= N <= 4096).
 * The mean depth is absorbed into eta (bottom at y = 0, Sec. 2.1), so a
 * finite-depth surface must satisfy eta_j > 0; in deep water (h = INFINITY)
 * the mirror-image kernels K2, G2 are omitted.
 */
#ifndef WW_H
#define WW_H

#ifdef __cplusplus
extern "C" {
#endif

#define WW_OK                  0
#define WW_ERR_ARG            -1  /* bad argument (size, NULL pointer, layout)        */
#define WW_ERR_GEOMETRY       -2  /* surface at/below the bottom, or non-finite data   */
#define WW_ERR_NO_CONVERGENCE -3  /* iterative refinement missed refine_tol            */
#define WW_ERR_CUDA           -4  /* a CUDA runtime call failed                        */
#define WW_ERR_TIMEOUT        -5  /* a bounded device-side wait gave up                */
#define WW_ERR_ALLOC          -6  /* device or host allocation failed                  */

/* Arithmetic of the dense DtN linear algebra. */
#define WW_FP64  0  /* plain FP64: LU of A, triangular solves, G apply, all FP64 */
#define WW_MIXED 1  /* FP32-accurate approximate inverse of A on the tensor cores,
                       FP64-accurate residuals and G apply by exact bf16 splitting,
                       iterative refinement to refine_tol (Sec. 3.3 refinement
                       precedent: quad residuals + double solves, here FP64
                       residuals + FP32 solves) */

typedef struct {
    int N;              /* surface points, power of two in [16, 4096]                 */
    int n;              /* mode unknowns c_1..c_n (J has n+1 columns), 0 <= n <= 4096 */
    double g;           /* gravity                                                    */
    double tau;         /* surface tension sigma/rho (>= 0)                           */
    double h;           /* mean depth, or INFINITY for deep water                     */
    int steps;          /* RK4 steps from t = 0 to t = T/4 (>= 1)                     */
    const double *basis;/* HOST pointer: 2N x n column-major initial-data basis
                           (rows 0..N-1 eta, N..2N-1 phi), copied at ww_create;
                           NULL selects column k = (cos k x, 0)                       */
    int precision;      /* WW_FP64 or WW_MIXED                                        */
    double refine_tol;  /* WW_MIXED: relative residual target, 0 => 1e-13             */
    int max_refine;     /* WW_MIXED: most refinement corrections per solve, 0 => 4    */
} ww_problem;

typedef struct {
    int refine_iters_max;      /* most refinement corrections any solve needed      */
    double refine_resid_max;   /* largest final relative residual of any stage      */
    double ns_resid_max;       /* WW_MIXED: largest ||I - X A||_max seen            */
    int stages;                /* RK stages run by the last call                     */
    long long launches;        /* kernels launched by the last shoot / shoot_jacobian
                                  (graph kernel nodes x replays + outputs; -1 when
                                  the legacy stream forced direct launches)        */
    double refine_iters_mean;  /* WW_MIXED: mean refinement corrections per solve   */
    double refine_resid_measured;  /* WW_MIXED with ww_set_verify: largest MEASURED
                                  relative residual max_j max_i |R_ij| / (max|Psi_j| +
                                  max|M_j|) of the sampled solves, R = Psi - A M
                                  recomputed (7-digit FP64-accurate product) after
                                  the last correction; -1 when nothing was sampled */
    int verified_solves;       /* multi-column solves measured by the last call     */
    long long device_bytes;    /* device memory held by the context (all workspace)  */
    long long adjoint_bytes;   /* of which the objective_and_grad workspace (trajectory
                                  records, checkpoints, second operand copies)      */
} ww_stats;

/* How a context lays out its step program (no counterpart in the paper: the
 * knobs of the GB300 kernels; ww_autotune picks them by timing).  Every
 * schedule computes the same discrete map to the same accuracy. */
typedef struct {
    int overlap;   /* WW_MIXED: run the base chain one stage ahead of the columns on a
                      second branch of the step graph (1), or in line (0)              */
    int ns_every;  /* WW_MIXED with overlap: move the approximate inverse to every
                      stage's A (1); on even stages and when it drifted (0); or as 0
                      until a wide solve of an odd stage has needed three
                      corrections in this shot, then on every stage (2)                */
    int corr_bn;   /* WW_MIXED: column tile of the refinement corrections X R (32, 64, 128) */
    int inv_bn;    /* WW_MIXED: column tile of the inverse update's products (64, 128,
                      256; 256 needs N a multiple of 256)                               */
    int lu_nb;     /* WW_FP64: block size of the LU and triangular solves (32, 64)      */
    int inv_ctas;  /* WW_MIXED: CTAs per SM of the inverse update's products: 1 (one
                      CTA with a 4-deep operand ring) or 2 (two CTAs with 2-deep rings,
                      so that one's epilogue overlaps the other's main loop; inv_bn
                      64 or 128)                                                        */
    int prio;      /* WW_MIXED with overlap: the step graph runs the base chain's
                      kernels at a higher priority than the columns' (1: its blocks
                      go first when SMs free up), or all at the launching stream's
                      priority (0)                                                      */
} ww_schedule;

typedef struct ww_ctx ww_ctx;

/* Create a context for problem *p on the current CUDA device: validates the
 * sizes, allocates all device workspace (about 3 N^2 + 8 N (n+2) doubles in
 * WW_FP64; WW_MIXED adds FP32/bf16 copies of the N x N operators), uploads
 * the basis.  *ctx is NULL on failure. */
int ww_create(ww_ctx **ctx, const ww_problem *p);

/* Free everything ww_create allocated.  NULL is a no-op. */
void ww_destroy(ww_ctx *ctx);

/* Queue subsequent work on `stream` (a cudaStream_t; NULL = legacy default). */
int ww_set_stream(ww_ctx *ctx, void *stream);

/* Statistics of the last shoot / shoot_jacobian / dtn_apply call. */
int ww_get_stats(const ww_ctx *ctx, ww_stats *out);

/* Measured refinement residual (WW_MIXED; a diagnostic of the Sec. 3.3
 * refinement, which the paper runs with quad-precision residuals).  The
 * refinement stops when the residual left after its last correction,
 * extrapolated from the observed contraction, is below refine_tol.  With
 * every > 0 the library also MEASURES it on a sample: after the last
 * correction of every every-th multi-column solve of a call (stage 0,
 * every, 2 every, ... of a shoot_jacobian; dtn_apply solves count too) it
 * recomputes R = Psi - (1/2 I + K) M with the 7-digit product and records
 * the worst relative residual in ww_stats.refine_resid_measured.  0 (the
 * default) turns it off.  A change takes effect at the next call, whose
 * step program is captured again.  WW_ERR_ARG in WW_FP64 (no refinement). */
int ww_set_verify(ww_ctx *ctx, int every);

/* The context's schedule.  ww_create sets the default {1, 2, 64, 128, 64, 2, 1};
 * ww_set_schedule validates the fields (WW_ERR_ARG) and drops the captured
 * step programs, which the next call captures again. */
int ww_set_schedule(ww_ctx *ctx, const ww_schedule *s);
int ww_get_schedule(const ww_ctx *ctx, ww_schedule *s);

/* ww_autotune -- choose the context's schedule by timing.  Candidate
 * schedules (coordinate by coordinate: the stage program, then the tile of
 * the corrections, then the tile and the CTAs per SM of the inverse update in
 * WW_MIXED; the LU
 * block in WW_FP64) each run the initial data and probe_steps RK steps of the
 * Jacobian of the shot c (device, n+1 doubles) on the context's stream, timed
 * with CUDA events after one untimed step; the fastest is kept.  cache_path
 * (NULL: none) names a text file of earlier choices, one line per (N, n+1,
 * precision): a cached choice is taken without timing, and a new one is
 * appended.  *ms_per_step (may be NULL) receives the chosen schedule's probe
 * time per RK step (0 when it came from the cache).  The context's outputs
 * are not touched; its state afterwards is that of a partial shot. */
int ww_autotune(ww_ctx *ctx, const double *c, int probe_steps, const char *cache_path, double *ms_per_step);

/* Thread-local description of the last error (empty string if none). */
const char *ww_last_error(void);

/* Phase timing (a profiling aid; no counterpart in the paper).  When enabled,
 * shoot / shoot_jacobian record a CUDA event pair on the context's stream
 * around each phase below in every RK stage, and ww_get_timing returns, for
 * the last call, the summed milliseconds and the number of timed launches of
 * each phase.  Costs two event records per phase and stage. */
#define WW_PHASE_ASSEMBLY   0  /* K, G assembly kernel                          */
#define WW_PHASE_FACTOR     1  /* LU of A (FP64) / inverse update (MIXED)       */
#define WW_PHASE_SOLVE      2  /* multi-RHS solve of the n+1 columns            */
#define WW_PHASE_GAPPLY     3  /* G gamma for the n+1 columns                   */
#define WW_PHASE_COLRHS     4  /* variational RHS + RK update kernel            */
#define WW_PHASE_GAMMA      5  /* gamma = mu', H gamma for the n+1 columns      */
#define WW_PHASE_BASE       6  /* base-state chain (geometry .. base RHS)       */
#define WW_PHASE_GKERNEL    7  /* the single product kernel inside GAPPLY (the
                                  FP64 GEMM, or the MIXED Ozaki tensor-core GEMM
                                  without its operand split)                    */
#define WW_PHASE_INVERSE    8  /* MIXED: the two tensor-core products of the
                                  inverse update inside FACTOR (none in FP64)   */
#define WW_NPHASE           9
int ww_set_timing(ww_ctx *ctx, int enable);
int ww_get_timing(const ww_ctx *ctx, double *ms /* WW_NPHASE */, int *launches /* WW_NPHASE */);

/* dtn_setup -- Sec. 2.1 Eqs. (fred), (G); Sec. 2.2 Eq. (K1K2).
 * Assemble A = 1/2 I + K and G for the surface eta (device, N doubles; mean
 * depth included), and factor A (WW_FP64) or build its approximate inverse
 * (WW_MIXED).  Returns WW_ERR_GEOMETRY if eta is non-finite or, with finite
 * depth, min(eta) <= 0. */
int dtn_setup(ww_ctx *ctx, const double *eta);

/* dtn_apply -- the Dirichlet-to-Neumann operator of the surface given to the
 * last dtn_setup (Sec. 2.1, three steps: solve Eq. (fred) for mu, gamma = mu',
 * G phi = 1/2 H gamma + (1/2 pi) int G gamma, |xi'| = 1 on the uniform grid).
 * phi: device, N x nrhs column-major; Gphi: device, N x nrhs (may not alias
 * phi).  1 <= nrhs <= n + 2.  WW_ERR_ARG if dtn_setup was not called. */
int dtn_apply(ww_ctx *ctx, const double *phi, int nrhs, double *Gphi);

/* shoot -- Sec. 3.1 Eq. (f:phi).  c: device, n+1 doubles (c[0] = T, c[k] the
 * coefficient of basis column k).  Evolves q0 = (hbar + B_eta c, B_phi c) to
 * T/4 with `steps` RK4 steps (36th-order filter on every RHS and after every
 * step, Eq. filter) and writes r_i = phi(x_i, T/4)/sqrt(N) (device, N) and
 * f = r.r/2 (device, 1 double). */
int shoot(ww_ctx *ctx, const double *c, double *r, double *f);

/* shoot_jacobian -- Sec. 3.3 Eqs. (Jik), (q:qdot).  As shoot, and also
 * J (device, N x (n+1) column-major): column 0 = dr/dT (the variational
 * column forced by F(q)/T, exact for the discrete map), column k = dr/dc_k
 * (variational column started from basis column k).  All n+1 columns share
 * each stage's DtN setup. */
int shoot_jacobian(ww_ctx *ctx, const double *c, double *r, double *J, double *f);

/* shoot_jacobian_host -- shoot_jacobian with HOST arrays: copies c in, runs,
 * copies r, J, f out (pinned or pageable host memory). */
int shoot_jacobian_host(ww_ctx *ctx, const double *c, double *r, double *J, double *f);

/* shoot_jacobian_batch -- nshots independent shots (each its own context,
 * problem size, step count and schedule) in ONE graph launch on one GPU: the
 * batch graph holds, per shot, a branch [inputs, initial data, a WHILE node
 * whose body is the shot's captured RK step and a counter that ends the loop
 * after its `steps` steps, outputs], and the branches run concurrently, so
 * small shots fill the SMs that a large one leaves idle (the paper runs 2-3
 * jobs per GPU for the same reason, Sec. 4.6).  ctx[i], cvec[i], r[i], J[i],
 * f[i] as for shoot_jacobian (device arrays of shot i's sizes).  The
 * contexts must be distinct and each on a stream of its own (ww_create gives
 * one; the legacy default stream is rejected with WW_ERR_ARG).  The graph is
 * built on the first call with a given set of contexts and arrays and kept
 * for the next; it is launched on ctx[0]'s stream after the other shots'
 * streams, which wait for it in turn.  Returns when every shot is done; the
 * first failing shot's status is returned, its message naming the shot.
 * Results are bitwise those of shoot_jacobian on each context. */
int shoot_jacobian_batch(ww_ctx *const *ctx, int nshots, const double *const *cvec, double *const *r,
                         double *const *J, double *const *f);

/* objective_and_grad -- Sec. 3.2 Eqs. (adj), (nabla:f), App. C Eq. (adj2):
 * f (device, 1 double) and its gradient with respect to c (device, n+1
 * doubles; grad[0] = d f / d T) by the DISCRETE adjoint: one forward pass of
 * the base state that records every RK stage (6N doubles a stage, allocated
 * on the first call and kept with the context), then the transposed RK4
 * steps backward, each stage with its DtN assembled transposed (A^T, G^T) and
 * factored as in the forward form.  grad equals J^T r of shoot_jacobian up to
 * roundoff, at the cost of about two shots instead of n + 1 columns.
 * Errors as shoot; WW_ERR_ALLOC if the trajectory record does not fit (see
 * ww_set_checkpoint for the bounded-memory form). */
int objective_and_grad(ww_ctx *ctx, const double *c, double *f, double *grad);

/* ww_set_checkpoint -- memory of objective_and_grad (Sec. 3.2: the forward
 * solution is stored at mile-markers and recomputed between them when memory
 * is short).  every = 0 (the default) keeps the record of every RK stage of
 * the forward pass resident (6N doubles a stage).  every = K > 0 keeps the
 * base state (2N doubles) every K steps and the records of only K steps: the
 * backward sweep goes segment by segment from the last, and before each
 * segment (except the last) recomputes that segment's records forward from
 * its checkpoint: 24 N K + 2 N steps/K doubles instead of 24 N steps, so
 * K = sqrt(steps) makes the memory grow like sqrt(steps), for one more
 * forward pass of the base state (all segments but the last).  In
 * WW_FP64 the gradient is bitwise that of every = 0; in WW_MIXED each
 * recomputed segment restarts its approximate inverse, so the refined solves
 * round differently (agreement to ~1e-12 relative).  Takes effect at the next
 * objective_and_grad, which reallocates the workspace. */
int ww_set_checkpoint(ww_ctx *ctx, int every);

/* dtn_apply_static -- the same operator as dtn_setup followed by dtn_apply,
 * for callers that cannot allocate device memory when they need it: code
 * under a memory-pool or allocator policy that forbids cudaMalloc, plug-ins
 * of a host application that owns every allocation itself, and loops that
 * must not touch the allocator.  (The paper has no counterpart; it is an
 * interface convenience.)  The caller passes
 * only inputs and outputs -- eta (device, N), phi (device, N x nrhs,
 * column-major), Gphi (device, N x nrhs, must not alias phi), h (mean depth
 * or INFINITY) and a cudaStream_t (NULL = legacy default stream) -- and the
 * call allocates nothing: its workspace is one fixed array inside the
 * library, sized for N <= WW_STATIC_MAX_N and nrhs <= WW_STATIC_MAX_RHS
 * (1.7 MB, held by every GPU that loads the library until the process
 * exits).  Larger sizes return WW_ERR_ARG.  The first call on a device does
 * a one-time set-up there (it looks up the array's device address and sets a
 * kernel attribute), so make that first call before any stream capture.  The
 * call uploads small tables from host memory, then reads the status word
 * back and synchronises its stream before returning.  All calls share the
 * array, which keeps the last call's contents; calls that overlap on the GPU
 * (other threads, other streams) race on it and must be serialised by the
 * caller. */
#define WW_STATIC_MAX_N   256
#define WW_STATIC_MAX_RHS 64
int dtn_apply_static(const double *eta, const double *phi, int N, int nrhs, double h, double *Gphi, void *stream);

/* Time segments with adaptive meshes and a general explicit Runge-Kutta
 * scheme (Sec. 2.2, Eq. (xi); the paper's production runs use DOP853).  The
 * quarter period is split into segments; segment l covers the fraction
 * theta_l of T/4 with `steps` uniform steps of the tableau (a, b) on the
 * grid x_j = xi_l(alpha_j), alpha_j = 2 pi j / M_l, of the mesh of Eq. (xi):
 * xi' = 1 - P[A sin^4(alpha/2)] (centre = 1, refined near x = pi) or
 * 1 - P[A cos^4(alpha/2)] (centre = 0, near x = 0), A = 8 (1 - rho)/(5 + 3 rho),
 * P the mean-free part (rho = min xi' / max xi'; rho = 1 is the uniform grid).
 * On a mesh every x-derivative is d/dalpha over xi', the DtN carries Eq. (G)'s
 * 1/|xi'|, P removes the mean over x and the residual weights are
 * sqrt(xi'/M) (Eq. (f:phi)).  Between segments the state and every
 * variational column are carried over by trigonometric interpolation of the
 * old grid at xi_old^{-1}(xi_new(alpha'_j)). */
typedef struct {
    int steps;          /* uniform steps of the tableau in this segment (>= 1)             */
    double theta;       /* fraction of T/4 the segment covers (the fractions sum to 1)      */
    double rho;         /* mesh parameter, 0 < rho <= 1 (1: uniform)                        */
    int centre;         /* 1: refined near x = pi, 0: near x = 0                            */
    int stages;         /* stages s of the explicit tableau (1..16)                         */
    const double *a;    /* HOST, s x s row-major, strictly lower triangular (copied)        */
    const double *b;    /* HOST, s weights (copied)                                         */
} ww_segment;

/* ww_set_segment -- make the context (its N is the segment's M) a segment of
 * a segmented shot: uploads the mesh tables and the tableau and allocates the
 * stage right-hand sides (s (n + 2) 2N doubles).  NULL removes it.  N must be
 * a multiple of 32.  The context's uniform RK4 entry points are unaffected. */
int ww_set_segment(ww_ctx *ctx, const ww_segment *seg);

/* shoot_jacobian_segments -- Sec. 2.2 and Sec. 3.3 on segments: r, J and f
 * (device; r: M_last, J: M_last x (n+1) column-major, f: 1) of the segmented
 * shot from c (device, n+1; c[0] = T) through the contexts ctx[0..nseg), one
 * per segment in time order, each set up by ww_set_segment.  ctx[0] holds
 * the initial data (its basis) and must be uniform (rho = 1); all contexts
 * share n, g, tau, h and the form; the thetas sum to 1.  The variational
 * columns (the T column forced by F(q)/T in every segment) ride through the
 * respacing with the base state, so J is the derivative of the discrete map.
 * All work runs on ctx[0]'s stream.  Errors as shoot_jacobian. */
int shoot_jacobian_segments(ww_ctx *const *ctx, int nseg, const double *c, double *r, double *J, double *f);

/* objective_and_grad_segments -- Sec. 3.2's gradient (Eqs. (adj), (nabla:f))
 * of the segmented shot of Sec. 2.2: f (device, 1 double) and its gradient
 * with respect to c (device, n+1 doubles; grad[0] = d f / d T) by the
 * DISCRETE adjoint of the map shoot_jacobian_segments differentiates.  A
 * forward pass of the base state alone records every stage of every segment
 * (6 M_l doubles a stage, allocated by the first call and kept with each
 * segment's context); then, segment by segment from the last, the transposed
 * steps of the segment's tableau run backward, each stage with its DtN
 * assembled transposed on the segment's mesh (A^T, G^T) and factored in the
 * context's form, and the adjoint state goes back through the transposed
 * respacing between segments.  grad equals J^T r of shoot_jacobian_segments
 * up to roundoff, for about two base shots instead of n + 1 columns.
 * Contexts, stream and errors as shoot_jacobian_segments; WW_ERR_ALLOC if
 * the records do not fit. */
int objective_and_grad_segments(ww_ctx *const *ctx, int nseg, const double *c, double *f, double *grad);

/* Self-tests of the dense products (diagnostics; no counterpart in the
 * paper).  C = A B for column-major FP64 device arrays A (M x K, ld M),
 * B (K x Nn, ld K) and the output C (M x Nn, ld M, overwritten), through
 *   ww_selftest_f32gemm: the FP32-accurate product of 3 + 3 bf16 slices
 *                        (tensor cores; K a multiple of 64),
 *   ww_selftest_ozaki:   the FP64-accurate product of 7 + 7 exact bf16 digits
 *                        (tensor cores; K a multiple of 64),
 *   ww_selftest_dgemm:   the FP64 DGEMM of the plain form (CUDA cores).
 * The caller compares C with a product of its own.  They allocate their own
 * scratch, use the legacy default stream and synchronise the device;
 * WW_ERR_TIMEOUT if a bounded device wait expired. */
int ww_selftest_f32gemm(const double *A, const double *B, int M, int Nn, int K, double *C);
int ww_selftest_ozaki(const double *A, const double *B, int M, int Nn, int K, double *C);
int ww_selftest_dgemm(const double *A, const double *B, int M, int Nn, int K, double *C);

/* Self-test of the assembly's reciprocal (Newton-Raphson from the FP32
 * hardware reciprocal, two steps): *max_rel = max |r(d_i) - 1/d_i| / (1/d_i)
 * over the n positive normal doubles d (device array), against the division
 * operator.  Same conventions as the self-tests above. */
int ww_selftest_recip(const double *d, int n, double *max_rel);

#ifdef __cplusplus
}
#endif
#endif /* WW_H */

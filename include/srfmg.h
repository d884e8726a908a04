/*
 * srfmg.h -- C ABI of the GB300 (sm_103a) one-pass FMG-FAS solver with
 * segmental refinement (SR), after M. F. Adams, "A low memory, highly
 * concurrent multigrid algorithm".
 *
 * Problem (Sec. 4 of the paper): -u'' = f on (0,1) with u(0) = u(1) = 0,
 * discretised by cell-centred second order finite volumes on N = 2^M cells
 * (centres x_i = (i + 1/2)/N; the Dirichlet wall is an odd ghost cell).
 *
 * Method: one FMG cycle (Fig. 2) of FAS V(nu1, nu2)-cycles (Fig. 1) with the
 * tau correction of Eqs. 6-7; the finest n_sr_levels levels are SR levels
 * (Fig. 3): they are split into segments of segment_width cells with
 * buffer_width buffer cells per side, smoothed additively (block Jacobi), and
 * in the post-smoothing leg they are rebuilt from the coarse grid by the full
 * update of Eq. 5 and smoothed with the Kaczmarz compatible relaxation of
 * Fig. 5.  The finest level is never stored: it lives in on-chip memory only.
 * The smoother is the paper's lexicographic Gauss-Seidel (omega = 1, the
 * sweep direction reversed after every sweep within one smoothing call); tau
 * at segment edges is formed from the assembled level, as in the paper's
 * appendix program.  With n_sr_levels = 0 the same entry points run plain
 * FMG-FAS with every level stored.
 *
 * Conventions for every entry point:
 *   - No C++ types or exceptions cross this boundary.
 *   - Arguments are checked on the host before anything is enqueued; a bad
 *     argument returns SRFMG_EINVAL (or SRFMG_EUNSUPPORTED for a valid but
 *     not implemented option) and enqueues nothing.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  srfmg_solve is asynchronous on it.
 *   - The caller owns f and u; the handle owns its device workspace (the
 *     stored coarse levels, the seam buffer, the coarsest-grid inverse and
 *     the captured CUDA graphs).
 *   - A handle may be used from one host thread at a time.  Its calls share
 *     the handle's device workspace, so calls that use it (solves, adjoints,
 *     reconstructions) must be ordered on the GPU: enqueue them on one
 *     stream, or order their streams with events.
 *   - There is no CPU fallback: without a usable CUDA device srfmg_create
 *     returns SRFMG_ECUDA.
 */
#ifndef SRFMG_H
#define SRFMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct srfmg_plan *srfmg_handle;

typedef enum {
    SRFMG_OK = 0,
    SRFMG_EINVAL = 1,          /* invalid argument; nothing was enqueued */
    SRFMG_ENOMEM = 2,          /* device workspace allocation failed */
    SRFMG_ECUDA = 3,           /* a CUDA call failed; see srfmg_last_error */
    SRFMG_ETIMEOUT = 4,        /* a bounded device wait expired */
    SRFMG_ENONFINITE = 5,      /* non-finite value detected */
    SRFMG_EUNSUPPORTED = 6     /* valid option that this build does not implement */
} srfmg_status;

/* Operators.  SRFMG_OP_BRATU is the nonlinear -u'' + lambda e^u = f (lambda >= 0)
 * with the same discretisation, solved by the same FAS cycles (Sec. 2.2,
 * Eqs. 1-2: the coarse equation of a nonlinear operator; Fig. 1 with the
 * nonlinear smoother: pointwise Newton Gauss-Seidel).  SRFMG_OP_VARCOEF is
 * -(a u')' = f with a > 0 at the cell faces (fluxes a_{i+1/2} (u_{i+1} - u_i),
 * a wall face counted twice by the odd ghost; coarse faces take the
 * coefficient of the coinciding fine face), set by srfmg_set_coefficient.
 * Precisions: SRFMG_FP64 runs every step in FP64.  SRFMG_MIXED keeps the
 * accuracy-bearing quantities exact or rounded below FP64's unit and takes the
 * rest off GB300's narrow FP64 pipe: for SRFMG_OP_LAPLACE and SRFMG_OP_VARCOEF
 * the solution, residual, tau correction, restriction and interpolations are
 * 64-bit fixed-point integers (the variable coefficient's fluxes exact 128-bit
 * products, its Gauss-Seidel multipliers 31-bit), the coarsest solve FP64; for
 * SRFMG_OP_BRATU the solution, residual (with lambda e^u), tau correction,
 * interpolations and coarsest Newton solve are FP64 and the Newton Gauss-Seidel
 * correction recurrence FP32. */
typedef enum { SRFMG_OP_LAPLACE = 0, SRFMG_OP_VARCOEF = 1, SRFMG_OP_BRATU = 2 } srfmg_op;
typedef enum { SRFMG_FP64 = 0, SRFMG_MIXED = 1 } srfmg_precision;
typedef enum { SRFMG_SMOOTH_LEX = 0 } srfmg_smoother;
/* Where the tau correction of a segment's two edge coarse cells comes from
 * (SR levels; Fig. 3 forms tau from each segment's smoothed extended patch,
 * the paper's program from the assembled level, which the paper states has
 * the same semantics): SRFMG_TAU_ASSEMBLED (default) uses the neighbouring
 * segments' interior values, exchanged through a seam pass;
 * SRFMG_TAU_SEGMENT uses the segment's own buffer cells (fully local, no
 * exchange; at large N its rounding-level mismatch with the assembled
 * restriction grows like N^2). */
typedef enum { SRFMG_TAU_ASSEMBLED = 0, SRFMG_TAU_SEGMENT = 1 } srfmg_tau_edge;
/* The post-smoothing leg of the SR level (Fig. 3): SRFMG_POST_FULL_UPDATE
 * (default) rebuilds the level from the corrected coarse grid by the full
 * update of Eq. 5 and smooths with the Kaczmarz compatible relaxation of
 * Fig. 5, the paper's method; SRFMG_POST_FAS_RECOMPUTE applies the FAS
 * correction of Eq. 4 to the pre-smoothed level instead, which each segment
 * recomputes from the coarse iterate the pre-leg interpolated (kept), with the
 * neighbouring segments' pre-smoothed edge cells (b + 1 per side, kept) in its
 * buffer, and smooths without Kaczmarz: the result is that of stored-grid FAS
 * with the same segmented smoother, at the cost of a second pre-smoothing and
 * two coarse-level arrays.  SRFMG_POST_FAS_RECOMPUTE needs n_sr_levels = 1,
 * tau_edge = SRFMG_TAU_ASSEMBLED, n_vcycles = 0 and buffer_width <
 * segment_width. */
typedef enum { SRFMG_POST_FULL_UPDATE = 0, SRFMG_POST_FAS_RECOMPUTE = 1 } srfmg_post;

/* Solve parameters (the paper's problem statement and cycle type). */
typedef struct {
    int32_t op;                /* srfmg_op */
    int32_t precision;         /* srfmg_precision */
    int32_t log2_n;            /* M: N = 2^M fine cells, M0 < M <= 28 */
    int32_t log2_n_coarsest;   /* M0: coarsest level, solved exactly; 2 <= M0 <= 6 (default 2) */
    int32_t n_sr_levels;       /* number of SR levels: 0 (plain stored FMG-FAS), 1 or 2 (the finest
                                  levels; level M - l has segments of W >> l cells) */
    int32_t segment_width;     /* W: finest-level cells per segment; power of two, 16 <= W <= 4096, W <= N */
    int32_t buffer_width;      /* b: buffer cells per segment side; even, 2 <= b <= 64, b <= W */
    int32_t nu1, nu2;          /* V(nu1, nu2): 1 <= nu1, nu2 <= 4 */
    int32_t smoother;          /* srfmg_smoother */
    double lambda;             /* SRFMG_OP_BRATU: lambda >= 0, finite; must be 0 otherwise */
    int32_t batch;             /* independent problems of this size solved together, in
                                  [0, 65535] (0 means 1); see srfmg_solve */
    int32_t tau_edge;          /* srfmg_tau_edge (SR levels only; 0 without SR) */
    int32_t n_vcycles;         /* FAS V-cycles (Fig. 1, with the SR steps of Fig. 3 on the SR levels)
                                  after the FMG cycle, each from the current fine solution:
                                  0..16 (default 0).  Without SR they converge to the exact
                                  discrete solution (about a digit per cycle), which makes
                                  srfmg_adjoint and srfmg_coef_gradient the exact gradients
                                  of the solve; with SR they stop at the SR floor. */
    int32_t post_leg;          /* srfmg_post (SR levels only; 0 without SR) */
    /* CTA shape (no effect on the result, which is the same bits for every choice:
       the stored-level tiles compute their halo cells exactly like the tile that
       owns them, and the coarse tail runs the same sweeps on whole levels): */
    int32_t tail_level;        /* finest level of the one-block coarse tail: 0 (default:
                                  min(12, M - n_sr_levels)) or in [log2_n_coarsest, 12] */
    int32_t tile_cells;        /* cells per block of the stored-level passes on levels of
                                  at most 2^18 cells over the whole batch (latency-bound;
                                  larger ones take 2048): 0 (default 256) or a power of
                                  two in [64, 2048] */
    int32_t chain_down;        /* 0 or 1 (off), or 2 .. 4: on the stored levels of at most
                                  2^18 cells over the whole batch, the down passes of up to
                                  chain_down consecutive levels run as one launch that
                                  keeps them in shared memory (a wider halo instead of the
                                  launches in between); the same bits as without it.
                                  SRFMG_MIXED with SRFMG_OP_LAPLACE only. */
    int32_t chain_up;          /* the same for the up passes (0 or 1: off, or 2 .. 4) */
} srfmg_params;

/* Information about a created plan. */
typedef struct {
    int64_t workspace_bytes;   /* device memory owned by the handle */
    int32_t kernels_per_solve; /* kernel launches enqueued by one srfmg_solve */
    int32_t coarse_tail_level; /* finest level handled by the one-block coarse tail */
    int32_t n_segments;        /* segments on the finest level (0 without SR) */
    int32_t segment_width;     /* W of the plan (0 without SR) */
    int32_t buffer_width;      /* b of the plan (0 without SR) */
    int32_t batch;             /* problems solved together (>= 1) */
    int32_t reserved[4];
} srfmg_info;

/* Fill *p with the defaults for N = 2^log2_n: M0 = 2, one SR level,
 * W = min(4096, N/4) (at least 16), b = 8, V(1,1), FP64, lexicographic GS.
 * Returns SRFMG_EINVAL if p is NULL. */
srfmg_status srfmg_default_params(int32_t log2_n, srfmg_params *p);

/* Create a plan on CUDA device `device`: validates *p (Sec. 3/4 parameter
 * meanings above), allocates the device workspace and records the level
 * schedule (the FMG loop of Fig. 2 with the SR steps of Fig. 3).
 * On success *out is a new handle; on failure *out is NULL. */
srfmg_status srfmg_create(const srfmg_params *p, int device, srfmg_handle *out);

/* One FMG-FAS(-SR) solve (Figs. 2-4).
 * f: device pointer, N doubles, the right-hand side at the cell centres.
 * u: device pointer, N doubles, receives the solution at the cell centres.
 * With batch = B > 1 the plan solves B independent problems of N cells with
 * the same launches (each kernel's grid has one row per problem): f and u
 * then hold B * N doubles, problem k at offset k * N.
 * f and u must not overlap and must stay valid until the stream reaches the
 * end of the solve.  Enqueued asynchronously on `stream`; the launch sequence
 * is captured into a CUDA graph the first time a (f, u, stream) triple is seen
 * and replayed afterwards.  Errors: SRFMG_EINVAL for NULL or misaligned
 * (not 16-byte aligned) pointers, SRFMG_ECUDA if a launch fails. */
srfmg_status srfmg_solve(srfmg_handle h, const double *f, double *u, void *stream);

/* Number of functionals srfmg_solve_functionals returns per problem. */
#define SRFMG_NUM_FUNCTIONALS 5

/* An SR solve (n_sr_levels = 1) that collects functionals of the fine-grid
 * solution while its segments are swept (Fig. 3 computes a functional of the
 * fine grid in the post-smoothing leg; the paper's section on obtaining the
 * solution names this as one way to get quantities of interest without
 * storing the fine grid).  For each problem k, functionals[5 k ..] receives
 *   [0] h sum_i u_i          (the integral of u, midpoint rule, h = 1/N)
 *   [1] h sum_i u_i^2        (the squared L2 norm)
 *   [2] max_i |u_i|
 *   [3] h sum_i (u_i - u_ref_i)^2   (0 without u_ref)
 *   [4] max_i |u_i - u_ref_i|       (0 without u_ref)
 * each segment reducing its interior and one kernel reducing the segments,
 * both in a fixed order (the same bits on every run).
 * u: device pointer as in srfmg_solve, or NULL: the fine solution is then
 * never written to memory (the solve moves 8 bytes per cell less); the plan
 * still keeps the coarse solution for srfmg_reconstruct.  u_ref: device
 * pointer, N doubles per problem, or NULL.  functionals: device pointer,
 * 5 doubles per problem.  Alignment as in srfmg_solve for f and u, 8 bytes for
 * u_ref and functionals; no output may overlap another argument.
 * Asynchronous on `stream`, captured and replayed per pointer set like
 * srfmg_solve.  Errors: SRFMG_EUNSUPPORTED without an SR level; SRFMG_EINVAL
 * for NULL f or functionals, misalignment or overlap; SRFMG_ECUDA. */
srfmg_status srfmg_solve_functionals(srfmg_handle h, const double *f, double *u, const double *u_ref,
                                     double *functionals, void *stream);

/* PDE decompression on demand (the paper's section on obtaining the
 * solution): expand fine-grid segments [seg_begin, seg_begin + seg_count)
 * from the coarse solution u_{M-1} that the plan keeps after its last solve
 * (srfmg_solve, srfmg_solve_functionals or srfmg_adjoint), by that solve's
 * post-leg: the full update Pi u_{M-1} and the nu2 compatible-relaxation
 * iterations on each segment's extended patch (plans with
 * SRFMG_POST_FAS_RECOMPUTE return SRFMG_EUNSUPPORTED).  The result equals, bit for
 * bit, the same cells of that solve's u.  f: device pointer, the right-hand
 * side of that solve (N doubles per problem).  u_seg: device pointer,
 * seg_count * W doubles per problem (problem k at offset k * seg_count * W),
 * receives cells [seg_begin W, (seg_begin + seg_count) W).  One kernel on
 * `stream`, ordered after the solve by the caller (same stream or an event).
 * Errors: SRFMG_EUNSUPPORTED without an SR level; SRFMG_EINVAL for a plan that
 * has not solved yet, a segment range outside [0, n_segments), NULL or
 * misaligned pointers (f 16 bytes, u_seg 8 bytes) or overlap; SRFMG_ECUDA. */
srfmg_status srfmg_reconstruct(srfmg_handle h, const double *f, int32_t seg_begin, int32_t seg_count,
                               double *u_seg, void *stream);
/* (The handle keeps the captured graphs of up to four (f, u) pointer pairs;
 * the least recently used one is replaced.) */

/* The same solve from and to HOST memory: copies f (N doubles, B * N for a
 * batch) to a device staging buffer owned by the handle, solves, copies the
 * solution back into u and synchronises `stream` before returning.  Pinned host
 * buffers give the fastest copies; pageable ones work.  f and u may alias. */
srfmg_status srfmg_solve_host(srfmg_handle h, const double *f, double *u, void *stream);

/* Pipelined solves from and to HOST memory, for a stream of right-hand sides
 * (no counterpart in the paper: a way to feed the solver of Figs. 2-3 from host
 * memory): like srfmg_solve_host, but the call only enqueues and returns.  Each call
 * copies f into one of two device staging buffers of the plan (used in turn),
 * solves on `stream` into the matching solution buffer, and copies the
 * solution back into u; the copies run on two streams of the plan, so a
 * call's copy-in overlaps the previous call's solve and its copy-out the next
 * call's solve.  Ordering: the solves run in call order on `stream`, each
 * after the work enqueued on `stream` before it; a call's copy-in does not wait
 * for `stream` (f is read from host memory as it is when the call is made, and
 * must not be written by work still pending on the GPU).
 * srfmg_solve_host_join(h, stream) makes `stream` wait for every copy-out
 * enqueued so far; only after that stream reaches the join may u be read, and f
 * and u (host buffers) must stay valid and unchanged until then.  Pinned host
 * buffers are needed for the overlap (pageable ones work, without it).  The
 * first call allocates the staging buffers (4 x N doubles per problem).
 * Errors as srfmg_solve_host (SRFMG_EINVAL for NULL pointers). */
srfmg_status srfmg_solve_host_async(srfmg_handle h, const double *f, double *u, void *stream);
srfmg_status srfmg_solve_host_join(srfmg_handle h, void *stream);

/* Gradient of a loss L(u) through the solve (the paper has no adjoint; the
 * operator is the one of Sec. 4).  The discrete operator L of SRFMG_OP_LAPLACE
 * (cell-centred finite volumes with odd ghosts: tridiag(-1, 2, -1)/h^2 with 3 in
 * the wall rows) is symmetric, so the adjoint equation L^T lambda = dL/du is the
 * forward equation with dL/du as its right-hand side, and dL/df = lambda.
 * lambda is computed by the same FMG(-SR) solve as srfmg_solve (same plan,
 * precision and launch schedule), so it carries that solve's algebraic error
 * for the right-hand side dL/du (for a rough dL/du, such as a residual against
 * noisy data, of the order of 1e-4 relative at N = 2^14 after one FMG cycle).
 * dL_du: device pointer, N doubles (the gradient of L with respect to u at the
 * cell centres); dL_df: device pointer, N doubles, receives dL/df.  Pointers,
 * alignment, overlap, asynchrony and errors as in srfmg_solve (it is the same
 * call: it has its own captured graph for its pointer pair).  SRFMG_OP_VARCOEF
 * is symmetric as well; its gradient with respect to the coefficient follows
 * from u and dL/df by srfmg_coef_gradient.  Returns SRFMG_EUNSUPPORTED for
 * SRFMG_OP_BRATU. */
srfmg_status srfmg_adjoint(srfmg_handle h, const double *dL_du, double *dL_df, void *stream);

/* SRFMG_OP_VARCOEF: set the coefficient for the following solves.  log_a:
 * device pointer, 2^M + 1 doubles per problem (B * (2^M + 1) for a batch), the
 * natural logarithm of a at the faces x_j = j / N, j = 0..N.  Fills the plan's
 * face coefficients of every level (a = exp(log_a); coarse faces coincide
 * with fine faces and take their value) with one kernel on `stream`, and
 * checks on the device that the sweeps can take it exactly: every log_a finite
 * with |log_a| <= 700, and on every level of 128 or more cells adjacent faces
 * within a factor 1.5 of each other (|log a_{j+1} - log a_j| <= ln 1.5; the
 * Gauss-Seidel carry over 99 cells is exact to 2^-72 for multipliers
 * a_near / (a_near + a_far) <= 0.6); with SRFMG_MIXED also a contrast
 * max a / min a below 2^8 over the problem (the fixed-point face coefficients
 * then keep at least 52 bits).  With SRFMG_MIXED the call also forms the fixed-
 * point face coefficients and multipliers of every level.  The call
 * synchronises `stream` to read the check; log_a may be freed when it
 * returns.  Until the first call a = 1.
 * Errors: SRFMG_EINVAL for a NULL handle or pointer, a plan of another
 * operator, or a coefficient that fails the check (the plan's coefficient is
 * then reset to a = 1). */
srfmg_status srfmg_set_coefficient(srfmg_handle h, const double *log_a, void *stream);

/* SRFMG_OP_VARCOEF: gradient of a loss L with respect to the coefficient,
 * dL/dlog a, from the solution u of srfmg_solve and the adjoint state
 * lam = dL/df of srfmg_adjoint (the operator is symmetric, so lam solves
 * A lam = dL/du).  The derivative of the variable-coefficient operator of the
 * paper's Sec. 4 discretisation (the paper itself has no gradient): face f,
 * between cells f-1 and f, gives
 *   dL/dlog a_f = -a_f (u_f - u_{f-1}) (lam_f - lam_{f-1}) N^2,
 * the wall faces -2 a_0 u_0 lam_0 N^2 and -2 a_N u_{N-1} lam_{N-1} N^2, with
 * the plan's current coefficient (the one the solve used).  It is the gradient
 * of the discrete problem evaluated at the FMG-SR u and lam, so it carries
 * their algebraic error.  u, lam: device pointers, N doubles per problem;
 * dL_dloga: device pointer, N + 1 doubles per problem (B * (N + 1) for a
 * batch), not overlapping u or lam; all 8-byte aligned.  One kernel on
 * `stream`, asynchronous.  Errors: SRFMG_EINVAL for a NULL handle or pointer,
 * misalignment, overlap, or a plan of another operator. */
srfmg_status srfmg_coef_gradient(srfmg_handle h, const double *u, const double *lam, double *dL_dloga,
                                 void *stream);

/* Non-finite detection: the kernels that read f record an inf or NaN in it,
 * and a functionals solve records non-finite functionals, in the plan's
 * status word.  srfmg_check synchronises `stream`, reads and clears that word,
 * and returns SRFMG_ENONFINITE if anything was recorded since the last check
 * (the solves themselves run on and return SRFMG_OK), else SRFMG_OK.
 * Errors: SRFMG_EINVAL for a NULL handle; SRFMG_ECUDA. */
srfmg_status srfmg_check(srfmg_handle h, void *stream);

/* Plan information (workspace size, launches per solve, ...). */
srfmg_status srfmg_query(srfmg_handle h, srfmg_info *info);

/* Per-kernel timing: runs `nsolves` solves with individual launches (no
 * graph) and a CUDA event pair around every kernel on `stream`, synchronises,
 * and writes the average duration in milliseconds of each launch of one solve
 * to ms_per_launch[0 .. kernels_per_solve-1] (kernels_per_solve from
 * srfmg_query; `capacity` is the array length).  f and u as in srfmg_solve. */
srfmg_status srfmg_profile(srfmg_handle h, const double *f, double *u, void *stream,
                           int32_t nsolves, float *ms_per_launch, int32_t capacity);

/* Name of launch i of one solve, e.g. "sr_post L24" or "level_down L23";
 * NULL if i is out of range. */
const char *srfmg_launch_name(srfmg_handle h, int32_t i);

/* Allocation-free small solve (the paper has no counterpart; this entry point
 * exists for callers that cannot call cudaMalloc: code that runs while a CUDA
 * stream capture is open in global mode, code whose device memory is owned by
 * a caching allocator or a fixed pool, and loops that must not allocate after
 * start-up).  It runs plain FMG-FAS (every level stored, no SR level: Fig. 2
 * with the V-cycle of Fig. 1) for N = 2^log2_n <= SRFMG_NOALLOC_MAX_N cells in
 * one thread block, exactly as srfmg_solve does for such sizes with
 * n_sr_levels = 0, and allocates nothing: its one piece of scratch memory,
 * the inverse of the coarsest-level operator, lives in a static device array
 * of SRFMG_NOALLOC_MAX_COARSE^2 doubles (32 KiB) that every GPU which loads
 * the library holds until the process exits.
 *   log2_n: 2 <= log2_n_coarsest < log2_n <= 12; log2_n_coarsest <= 6;
 *   nu1, nu2 in [1, 4]; f, u: device pointers, N doubles each, 16-byte
 *   aligned, not overlapping; stream as in srfmg_solve.
 * Sizes beyond these limits return SRFMG_EINVAL and enqueue nothing; errors
 * are reported by the status code only (srfmg_last_error is not updated).
 * This entry point has no status word and no srfmg_check: an inf or NaN in f
 * is not detected and gives a non-finite u with SRFMG_OK.
 * The first call on a device (with that device current) does a synchronous
 * set-up: it looks up the static array's device address, raises the kernel's
 * shared-memory limit and uploads the inverse for log2_n_coarsest; a later
 * call with a different log2_n_coarsest uploads again.  Make the first call,
 * and any call that changes log2_n_coarsest, before any stream capture.  All
 * calls share the array and it keeps the last upload: calls with different
 * log2_n_coarsest whose kernels overlap on the GPU race.  Concurrent host
 * calls are serialised by a lock held until the kernel is enqueued, so a call
 * never launches with another call's table.  Nothing in the array has to
 * start at zero. */
#define SRFMG_NOALLOC_MAX_N 4096
#define SRFMG_NOALLOC_MAX_COARSE 64
srfmg_status srfmg_solve_small_noalloc(int32_t log2_n, int32_t log2_n_coarsest, int32_t nu1,
                                       int32_t nu2, const double *f, double *u, void *stream);

/* Autotuner for the SR segment layout (the paper leaves W and b free; Sec. 4
 * finds four buffer cells enough for one FMG cycle to stay at discretization
 * accuracy in every configuration studied, so only b >= 4 is admissible).
 * For the solve described by *base (n_sr_levels must be 1; segment_width and
 * buffer_width are ignored) it times every candidate (W, b) with W in
 * {256, 512, 1024, 2048, 4096}, W <= N/2, and b in {4, 8}, b <= W (candidate
 * k in that order; srfmg_autotune_candidate names it): a plan per candidate,
 * two warm-up solves of a zero right-hand side (the kernels have no data-
 * dependent control flow) and `reps` timed solves with CUDA events on a
 * stream of its own; it allocates and frees its own f and u.  *best receives
 * *base with the fastest (W, b); the result of a solve depends on (W, b), so a
 * caller that checks it replays the oracle with the same pair.  ms (optional,
 * capacity entries) receives the average milliseconds per solve of each
 * candidate; *ncand (optional) the number of candidates.  Synchronous.
 * Errors: SRFMG_EINVAL for NULL or invalid arguments (before any device
 * work), as srfmg_create/srfmg_solve otherwise. */
srfmg_status srfmg_autotune(const srfmg_params *base, int device, int32_t reps, srfmg_params *best,
                            float *ms, int32_t capacity, int32_t *ncand);
srfmg_status srfmg_autotune_candidate(const srfmg_params *base, int32_t k, int32_t *segment_width,
                                      int32_t *buffer_width);

/* Autotuner for the CTA shape of a plan (no counterpart in the paper; the
 * launch shapes leave the result unchanged, bit for bit): for the solve
 * described by *base (any SR layout; base's tail_level, tile_cells, chain_down
 * and chain_up are ignored) it times every candidate shape: tail_level in
 * {9, 10, 11, 12} (those in [log2_n_coarsest, min(12, M - n_sr_levels)], each
 * distinct coarse tail once) with tile_cells in {128, 256, 512} and no chained
 * passes (tail level major), then, for SRFMG_MIXED with SRFMG_OP_LAPLACE, the
 * two finest of those tails with tile_cells in {256, 512} and chain_down = 2,
 * chain_up in {3, 4}.  Candidate k (srfmg_autotune_shape_candidate writes
 * *base with its shape to *cand) is timed the same way as in srfmg_autotune,
 * and *best is *base with the fastest shape.  ms (optional, capacity entries)
 * and *ncand (optional) as in srfmg_autotune.  Synchronous.  Errors as
 * srfmg_autotune. */
srfmg_status srfmg_autotune_shape(const srfmg_params *base, int device, int32_t reps, srfmg_params *best,
                                  float *ms, int32_t capacity, int32_t *ncand);
srfmg_status srfmg_autotune_shape_candidate(const srfmg_params *base, int32_t k, srfmg_params *cand);

/* Independent problems of uneven sizes solved together (many problems with
 * N = 2^m cells for varying m; the paper solves one problem, this is the
 * data-parallel use of its solver on independent ones).  A group holds one
 * batched plan per distinct size (srfmg_params.batch = the number of problems
 * of that size, at most 65535 per plan; more are split over several plans)
 * and replays all of them as ONE CUDA graph in which every plan runs on a
 * branch of its own, so the launch chains of the sizes overlap on the GPU.
 *
 * Packed layout: the problems lie back to back, ordered by size (ascending)
 * and, within a size, in their given order.  It depends only on the sizes:
 * srfmg_group_offsets gives it without a device, so a caller can arrange its
 * data before creating the group. */
typedef struct srfmg_group *srfmg_group_handle;

/* offsets: host array of nprob + 1 int64; offsets[k] receives the first cell
 * of problem k in the packed arrays and offsets[nprob] the total number of
 * cells.  log2_n: host array of nprob sizes, each in [1, 28].  Pure host
 * function.  Errors: SRFMG_EINVAL for nprob < 1, NULL pointers or a size
 * outside [1, 28]. */
srfmg_status srfmg_group_offsets(int32_t nprob, const int32_t *log2_n, int64_t *offsets);

/* Create a group on `device`.  base: the settings every problem shares (op,
 * precision, log2_n_coarsest, n_sr_levels, nu1, nu2, smoother, lambda,
 * tau_edge, n_vcycles, and the segment layout below); base->log2_n and
 * base->batch are ignored.  log2_n: host array of nprob sizes.
 * Segment layout of each size (plans with SR levels): with tune = 0,
 * W = min(base->segment_width, max(16, N/4)) and b = min(base->buffer_width,
 * W); with tune > 0, srfmg_autotune picks (W, b) for each size and then
 * srfmg_autotune_shape its CTA shape (tail_level, tile_cells, chain_down, chain_up) (`tune` timed
 * solves per candidate, on a sample of min(count, max(1, 2^24 / N)) problems
 * of that size; needs n_sr_levels = 1).  Every size must make a valid plan
 * (srfmg_create's checks: N > 2^log2_n_coarsest, ...).  On success *out is a
 * new handle.  Errors: as srfmg_create and srfmg_autotune; SRFMG_EINVAL for
 * nprob < 1, NULL pointers or tune < 0. */
srfmg_status srfmg_group_create(const srfmg_params *base, int32_t nprob, const int32_t *log2_n, int32_t tune,
                                int device, srfmg_group_handle *out);

/* Solve every problem of the group.  f, u: device pointers to the packed
 * arrays (offsets[nprob] doubles each), 16-byte aligned, not overlapping.
 * Asynchronous on `stream`: the first call for an (f, u) pair captures the
 * launches of all plans into one CUDA graph (a fork from `stream` into one
 * branch per plan and a join back), later calls replay it; a new pair is
 * captured anew.  Each problem's result is the one a single srfmg_solve with
 * its size's parameters gives, bit for bit.  Errors: SRFMG_EINVAL for a NULL
 * handle or pointer, misalignment or overlap; SRFMG_ECUDA. */
srfmg_status srfmg_group_solve(srfmg_group_handle g, const double *f, double *u, void *stream);

/* The same from and to HOST memory (the packed layout), with device staging
 * buffers owned by the group: every plan's branch copies its part of f in,
 * solves it and copies its part of u out (launched directly, not from the
 * graph), so the copies of one size overlap the work of the others; then
 * `stream` is synchronised.  Pinned host buffers give the fastest copies and
 * the overlap; pageable ones work. */
srfmg_status srfmg_group_solve_host(srfmg_group_handle g, const double *f, double *u, void *stream);

/* The group's plans, by ascending size: *nplans (optional) and *total_cells
 * (optional) of the packed arrays. */
srfmg_status srfmg_group_query(srfmg_group_handle g, int32_t *nplans, int64_t *total_cells);

/* Plan i of the group (0 <= i < nplans): *plan (optional) is its handle, owned
 * by the group (valid until srfmg_group_destroy; do not destroy it), usable
 * with srfmg_query, srfmg_check, srfmg_profile, srfmg_set_coefficient and the
 * other per-plan calls on its part of the packed arrays; *log2_n, *count and
 * *offset (each optional) receive its size, its number of problems and the
 * first cell of its part.  Errors: SRFMG_EINVAL for a NULL handle or i out of
 * range. */
srfmg_status srfmg_group_member(srfmg_group_handle g, int32_t i, srfmg_handle *plan, int32_t *log2_n,
                                int32_t *count, int64_t *offset);

/* Release the group, its plans and its graph (synchronises the device first).
 * Accepts NULL. */
srfmg_status srfmg_group_destroy(srfmg_group_handle g);

/* Message of the last error on g (or of the last failed srfmg_group_create
 * when g is NULL); never NULL. */
const char *srfmg_group_last_error(srfmg_group_handle g);

/* Release the device workspace and graphs.  Synchronises the device first.
 * Accepts NULL (returns SRFMG_OK). */
srfmg_status srfmg_destroy(srfmg_handle h);

/* Message describing the last error on h (or the last creation error when h
 * is NULL).  Never NULL; owned by the library; valid until the next call on
 * the same handle. */
const char *srfmg_last_error(srfmg_handle h);

/* Arithmetic throughput of the device, measured (no counterpart in the paper:
 * the denominators of the arithmetic rooflines of this library's kernels).
 * Runs four short probe kernels on `device` (a grid of 8 blocks of 256
 * threads per SM, eight interleaved dependent chains per thread, CUDA events
 * on a stream of its own, best of five timed runs after one warm-up) and
 * writes to ops_per_s[0..3]:
 *   [0] 64-bit integer adds per second,
 *   [1] 64-bit integer operations per second in the rounding halving
 *       (x + y + 1) >> 1 of the fixed-point sweep (two adds and a shift),
 *   [2] FP64 flops per second (fused multiply-adds, two flops each),
 *   [3] FP32 flops per second (fused multiply-adds, two flops each).
 * Synchronous; allocates and frees a small device buffer.  Errors:
 * SRFMG_EINVAL for NULL ops_per_s or a bad device index, SRFMG_ECUDA,
 * SRFMG_ENOMEM. */
srfmg_status srfmg_alu_peaks(int device, double *ops_per_s);

/* Self-check of the exponential of the Bratu operator in SRFMG_MIXED (no
 * counterpart in the paper; the mixed residual and tau take e^u from a
 * table-driven method, Tang's, with about half of the FP64 work of exp):
 * writes to *max_rel the largest relative difference to CUDA's exp at n
 * evenly spaced points of [lo, hi].  Synchronous; allocates one word.  Errors:
 * SRFMG_EINVAL for NULL max_rel, n outside [1, 2^26], lo > hi or |lo|, |hi|
 * > 700 (checked before any device work), a bad device index; SRFMG_ECUDA,
 * SRFMG_ENOMEM. */
srfmg_status srfmg_exp_error(int device, double lo, double hi, int32_t n, double *max_rel);

/* Library version string, e.g. "srfmg 0.1 sm_103a". */
const char *srfmg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SRFMG_H */

/*
 * ftoep.h -- C ABI of libftoep: GB300 (sm_103a) solver for the linear systems of
 * L1-type Caputo finite-difference schemes (Liu, Cheng, Li, Wang, "Fast procedures
 * for Caputo fractional ordinary and partial differential equations").
 *
 * Problem statement (Sec. 3, Eq. 18 and Eq. 14 with the advection term replaced by
 * -u_xx; Sec. 2 for the scalar case):
 *
 *     D_t^g u(x,t) = u_xx(x,t) + f(x,t),   x in (0,L), t in (0,T],  u(0,t) = u(L,t) = 0,
 *     u(x,0) = u0(x)  [and u_t(x,0) = phi(x) when 1 < g < 2],
 *
 * or, without space (FTOEP_SPACE_NONE), D_t^g u = -lambda*u + f on (0,T].
 *
 * Discretisation: tau = T/N, h = L/(M+1), x_j = j*h (j = 1..M).
 *   FTOEP_L1_SUBDIFFUSION (0 < g < 1): Scheme 4, Eq. 19 (L1 formula of Lemma 2, Eq. 4),
 *       level t_n; left-hand first column a_0 = mu, a_j = mu*(G_j - G_{j-1}),
 *       mu = tau^-g/Gamma(2-g), G_k = (k+1)^(1-g) - k^(1-g).
 *   FTOEP_L1_HYPERBOLIC (1 < g < 2): Eq. 15/17 at t_{n-1/2} with c = tau^-g/Gamma(3-g),
 *       a_0 = c, a_1 = c(M_1 - 2M_0), a_j = c(M_{j-2} - 2M_{j-1} + M_j),
 *       M_k = (k+1)^(2-g) - k^(2-g); spatial term taken at level n.
 *   FTOEP_L1_HYPERBOLIC_CN (1 < g < 2): the same time terms (Eq. 15, the same first
 *       column a) with the spatial term averaged over levels n and n-1,
 *       (u_xx^n + u_xx^{n-1})/2, u^0 = u0: the Crank-Nicolson form of the scheme that
 *       Eq. 15 is taken from (Sun and Wu, cited for Eq. 15), O(tau^(3-g) + h^2).  In the
 *       difference form below only the diagonal changes: E + lambda_m tau (1 - I/2).
 *   Space: central second difference with Dirichlet zeros (Eq. 19).
 * With the unknowns of one spatial point ordered in time (the reordering of Sec. 3,
 * "U_i = (U_i^1, ..., U_i^N)"), the time operator is lower-triangular Toeplitz with
 * first column a (Sec. 3, the block A-hat).  The library diagonalises the spatial
 * operator with an orthonormal sine transform (eigenvalues
 * lambda_m = (4/h^2) sin^2(m pi/(2(M+1)))), so each mode solves (lambda_m I + T) u_m = r_m
 * exactly (a direct solve, not an iteration).  Internally the rows are solved for the
 * difference quotients v^n = (u^n - u^{n-1})/tau, the variables in which Eq. 4 and Eq. 15
 * are written: per mode the operator becomes E + lambda_m tau 1 (E lower-triangular
 * Toeplitz with first column scale*tau*G_j, resp. scale*tau*(M_j - M_{j-1}); 1 the
 * all-ones lower triangle), and u = u0 + tau * cumsum(v).  Same equations, same
 * solution; the history terms carry tau^(1-g) instead of tau^-g.
 *
 * Field layout (all field arguments): [M][N] row-major, double precision, time index
 * contiguous; element (j-1, n-1) is the value at x_j and time level n (t_n for the
 * sub-diffusion scheme, t_{n-1/2} for the source of the hyperbolic scheme).  A plan
 * with several problems uses their fields concatenated in problem order (problem p
 * starts at element offset sum_{q<p} M_q*N_q).
 *
 * Pointers: field pointers may be device memory or host memory (pinned or pageable);
 * the library detects which.  Host buffers are staged through the plan's device
 * workspace inside the call.  On the chain schedule (FTOEP_SCHED_CHAIN) the first
 * host-buffer solve also allocates device copies of the fields of the plan's largest
 * group when they fit in the free device memory with 1 GiB to spare: f then crosses the
 * host link once and u once per solve; otherwise (or with FTOEP_HOST_STAGED=1 in the
 * environment at plan creation) each problem passes through the staging arrays, f twice
 * and, for a mixed problem, u out twice and in once.  The caller keeps ownership of every
 * buffer it passes.
 *
 * Streams and errors: every call is ordered on the CUDA stream given to ftoep_create
 * and may return before the GPU work has finished.  Errors are returned as status
 * codes only; nothing aborts or throws across this interface.  No kernel of the library
 * waits for another block or launch (blocks synchronise only within themselves or their
 * hardware cluster), so no call can time out.  ftoep_last_error gives a message for the
 * last failure.
 *
 * Threads: a plan's workspace, counters and captured graphs are shared by its calls, so
 * calls on one plan must not overlap in time from different host threads; different
 * plans are independent.
 */
#ifndef FTOEP_H
#define FTOEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ftoep_plan_s* ftoep_plan;

typedef enum {
  FTOEP_OK = 0,
  FTOEP_EINVAL = 1,       /* bad argument (range, null pointer, size mismatch)        */
  FTOEP_ENOMEM = 2,       /* device or host allocation failed                          */
  FTOEP_ECUDA = 3,        /* a CUDA runtime call failed                                */
  FTOEP_ETIMEOUT = 4,     /* reserved: never returned (the library has no device-side
                             waits)                                                    */
  FTOEP_EUNSUPPORTED = 5  /* valid input that this build does not handle               */
} ftoep_status;

typedef enum {
  FTOEP_L1_SUBDIFFUSION = 0, /* 0 < gamma < 1, Eq. 4/19                                 */
  FTOEP_L1_HYPERBOLIC = 1,   /* 1 < gamma < 2, Eq. 15/17                                */
  FTOEP_L1_HYPERBOLIC_CN = 2 /* 1 < gamma < 2, Eq. 15 time terms, spatial term averaged */
} ftoep_kind;

typedef enum {
  FTOEP_SPACE_NONE = 0,              /* D^g u = -lambda u + f; every row independent   */
  FTOEP_SPACE_DIRICHLET_LAPLACIAN = 1 /* D^g u = u_xx + f with Dirichlet zeros          */
} ftoep_space;

typedef enum {
  FTOEP_FP64 = 0,  /* all arithmetic in double precision                               */
  FTOEP_MIXED = 1  /* float solve (sine transforms, block inverses, convolutions; the
                      running sums of the all-ones part in double), then one correction
                      sweep: residual with a float-float (~48-bit) Toeplitz product and the
                      spatial stencil in double, correction solved in float and added     */
} ftoep_precision;

/* One problem.  T: final time (> 0).  L: length of the space interval (> 0, ignored for
 * FTOEP_SPACE_NONE).  lambda: reaction coefficient for FTOEP_SPACE_NONE (>= 0).
 * N >= 1 time steps (N <= 2^22); M >= 1 interior points (rows, for FTOEP_SPACE_NONE).
 * Sine transform sizes: M+1 a power of two up to 4096 (double) / 8192 (mixed); any other
 * M+1 (chirp-z FFT) up to 4096; beyond: FTOEP_EUNSUPPORTED. */
typedef struct {
  int kind;       /* ftoep_kind      */
  int space;      /* ftoep_space     */
  int precision;  /* ftoep_precision */
  double gamma, T, L, lambda;
  int64_t N, M;
} ftoep_problem;

/* Schedules of the pair solves (ftoep_tuning.scheduler). */
typedef enum {
  FTOEP_SCHED_AUTO = 0,   /* library choice: chain for plans of several problems, else levels */
  FTOEP_SCHED_LEVELS = 1, /* one launch per time block and per cross-block level, all pairs
                             of a problem in each launch, problems on internal streams     */
  FTOEP_SCHED_CHAIN = 2   /* one persistent launch per solve for every pair of a group of
                             problems: each block runs one pair's whole time recursion, pairs
                             taken longest chain first from a work counter; groups of
                             problems sized to a memory budget (half the free device memory
                             at plan creation, at most 32 GiB of pair arrays)              */
} ftoep_scheduler;

/* Solver of the per-mode lower-triangular Toeplitz systems (ftoep_tuning.solver). */
typedef enum {
  FTOEP_SOLVER_AUTO = 0,      /* library choice: HALFSPLIT (its error follows the size of each
                                 time block's own values; see INVERSE)                       */
  FTOEP_SOLVER_HALFSPLIT = 1, /* time blocks of B levels solved by the block inverse, then the
                                 recursive half-split updates between blocks (Sec. 3: the
                                 fast direct method of the reordered systems)                 */
  FTOEP_SOLVER_INVERSE = 2,   /* the inverse-series solve: x = h_m * y over the whole padded
                                 length, h_m = T_m^-1 e_1 computed once per plan (by the
                                 half-split solve of a unit impulse, in double); each solve is
                                 one causal convolution of length 2 Np per mode pair.  Its
                                 rounding is normwise over the whole time axis (one FFT): the
                                 error of every level is about eps log2(2 Np) |h_m| |y| /
                                 |x| of the largest values, where the half split's stays
                                 with the size of each block's own values -- for a growing
                                 hyperbolic or mixed-precision solution the early levels lose
                                 relative accuracy                                           */
  FTOEP_SOLVER_INVERSE_MIXED_SUBDIFFUSION = 3
                              /* INVERSE for the mixed-precision sub-diffusion problems
                                 (FTOEP_L1_SUBDIFFUSION, FTOEP_MIXED), HALFSPLIT for the rest.
                                 In the mixed path the correction sweep removes the first
                                 solve's error; what remains is the correction's own normwise
                                 rounding, a float rounding of a correction of about the
                                 first solve's error, which the sub-diffusion inverse (positive
                                 and decreasing) keeps well inside the mixed bar.  The
                                 hyperbolic inverse oscillates and its float error can exceed
                                 what one correction removes.  The inverse spectra take 8 B
                                 per unknown x 2 Np/N of device memory beside the plan.       */
} ftoep_solver;

/* Optional tuning (NULL or 0 fields = library choice; ftoep_autotune picks fft_tile,
 * scheduler, streams and solver).
 * fft_tile: the time block length B (power of two, 16..4096; default 4096, capped at N
 *   rounded up to a power of two).  Every block of B levels is solved by a causal
 *   convolution with the per-mode inverse of the block operator (one FFT of length 2B);
 *   the half-split updates between blocks are circulant convolutions.
 * leaf, gemm_max_level: shape only the substitution that builds the per-mode block
 *   inverses once at plan creation (leaf: dense forward-substitution size, power of two
 *   <= 16; levels below gemm_max_level use dense products instead of FFTs).  The solves
 *   themselves do not depend on them (up to rounding of the block inverses).
 * scheduler: an ftoep_scheduler value.
 * streams: internal streams of a plan with several problems (1..8; default 4): the
 *   per-problem phases (sine transforms, time sums, residuals; with the levels schedule
 *   every launch) of different problems run concurrently on them.
 * solver: an ftoep_solver value.  INVERSE applies to problems with more than one time block
 *   and 2 Np above the shared-memory convolution length (8192 mixed, 4096 double); it costs
 *   P * 2 Np complex values of the solve precision per problem (P = ceil(M/2) mode pairs)
 *   and one double half-split solve at plan creation.  A mixed problem with INVERSE solves
 *   both float solves (first and correction) with it; its adjoint (double) uses the
 *   half-split.  ftoep_problem_solver reports the solver each problem got. */
typedef struct {
  int leaf, fft_tile, gemm_max_level, scheduler, streams, solver;
} ftoep_tuning;

/* Create a plan for nprob problems (1 <= nprob).  Computes the weights a_j of every
 * problem on the host (cancellation-free series, double result), uploads them, builds
 * the per-level kernel spectra and allocates the device workspace.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  On success *out owns all of it.
 * Errors: FTOEP_EINVAL (gamma outside the kind's range, N/M/T/L invalid, nprob < 1,
 * out NULL), FTOEP_EUNSUPPORTED (sizes beyond the limits above), FTOEP_ENOMEM, FTOEP_ECUDA. */
ftoep_status ftoep_create(ftoep_plan* out, const ftoep_problem* probs, int nprob,
                          const ftoep_tuning* tune, void* cuda_stream);

/* First column a_j (j = 0..N-1) of problem iprob's time operator (see top), and, if
 * dadgamma is not NULL, its derivative with respect to gamma.  a and dadgamma are
 * host or device buffers of N doubles.  Returns after the values are in place. */
ftoep_status ftoep_weights(ftoep_plan p, int iprob, double* a, double* dadgamma);

/* Solve every problem of the plan: u = A^-1 (f + initial-data terms), where A is the
 * space-time operator of the scheme (Eq. 20 and its hyperbolic analogue).
 * f, u: concatenated fields (see top); u0, phi: concatenated length-M vectors or NULL
 * (zero).  phi is only used by hyperbolic problems.  f and u must not overlap.
 * Device buffers: the second call with the same (f, u, u0, phi) pointers captures the
 * whole solve (all problems, internal streams) as one CUDA graph of the plan and later
 * calls replay it -- the buffers' contents may change between calls, the pointers name
 * the graph (the plan keeps the four most recent).  Host buffers and calls while
 * ftoep_profile is on run the kernels directly. */
ftoep_status ftoep_solve(ftoep_plan p, const double* f, double* u, const double* u0, const double* phi);

/* y = T x (transpose = 0) or y = T^T x (transpose = 1) for nlines independent lines of
 * length N of problem iprob, T the lower-triangular Toeplitz time operator with first
 * column a (no lambda, no spatial part).  Computed by circulant embedding of size 2N'
 * (N' = N rounded up to a power of two) and FFTs (Sec. 3.1, Eq. be1; the input is
 * padded with zeros).  x, y: [nlines][N] doubles, host or device; they may not overlap.
 * Always double precision. */
ftoep_status ftoep_matvec(ftoep_plan p, int iprob, const double* x, double* y, int64_t nlines, int transpose);

/* Adjoint of ftoep_solve for zero initial data.  g = dL/du (concatenated fields),
 * u = the result of ftoep_solve for the same plan.  Writes dldf = A^-T g (same layout)
 * and, if dldgamma is not NULL, dL/dgamma_p = -<dldf_p, (dA/dgamma) u_p> for every
 * problem p into the HOST array dldgamma[nprob] (this synchronises the stream).
 * The transposed time operator is solved by reversing time, applying the forward solve
 * and reversing back (J T^T J = T for Toeplitz T).  Always double precision. */
ftoep_status ftoep_adjoint(ftoep_plan p, const double* g, const double* u, double* dldf, double* dldgamma);

/* Kernel classes for the instrumentation calls below. */
typedef enum {
  FTOEP_K_BLOCK_SOLVE = 0,    /* in-block half-split solve (leaves, direct and FFT levels)  */
  FTOEP_K_CONV_SMEM = 1,      /* cross-block circulant convolution, one shared-memory FFT   */
  FTOEP_K_CONV_FOURSTEP = 2,  /* cross-block circulant convolution, three-kernel four-step  */
  FTOEP_K_SINE = 3,           /* sine transforms along space                                */
  FTOEP_K_OTHER = 4,          /* packing, time sums, reductions, spectra                    */
  FTOEP_K_RESIDUAL = 5,       /* mixed path: float-float residual product and residual      */
  FTOEP_K_CHAIN = 6,          /* persistent per-pair solve (block solves and every level)   */
  FTOEP_K_INVERSE = 7         /* inverse-series solve (one convolution of length 2 Np)       */
} ftoep_kernel_class;

/* Instrumentation (no counterpart in the paper).  ftoep_profile waits for the stream,
 * clears the per-class counters and switches CUDA-event timing of every subsequent
 * operation on (enable != 0) or off.  Kernel launches are always counted.
 * While timing is on, every problem's kernels run on the plan's stream one after another
 * (no internal streams, no graph), so the class times add up to the instrumented solve
 * and do not overlap.  ftoep_profile_read waits for the stream and returns, for one class,
 * the summed event time in milliseconds of the timed operations, the number of timed
 * operations (one operation = one launcher call: 1 kernel, or 3 for the four-step
 * convolution) and the number of kernels launched since the last ftoep_profile.  Any
 * output may be NULL. */
ftoep_status ftoep_profile(ftoep_plan p, int enable);
ftoep_status ftoep_profile_read(ftoep_plan p, int kclass, double* total_ms, int64_t* ops, int64_t* launches);

/* Plan-free, allocation-free variant of ftoep_matvec (the paper has no counterpart:
 * it exists for callers that cannot allocate device memory -- code running after its
 * memory budget is frozen by a host framework's caching allocator, plugins that may not
 * allocate, loops where cudaMalloc's blocking and device synchronisation are not
 * acceptable).  y = T x (transpose = 0) or T^T x (transpose = 1) for nlines lines of
 * length N, T lower-triangular Toeplitz with first column a (N doubles, e.g. from
 * ftoep_weights).  a, x, y: device (or managed) memory, [nlines][N]; host memory returns
 * FTOEP_EINVAL before any launch (nothing is staged); x and y may not overlap.  A CUDA error
 * pending from earlier work is reported as FTOEP_ECUDA and left in place.
 * Work is ordered on cuda_stream (a cudaStream_t, NULL = legacy default stream).
 * All intermediates live in one static device array of 16.8 MB compiled into the
 * library (held on every GPU that loads it until the process exits); hence N <= 32768,
 * larger N returns FTOEP_EINVAL.  Nothing is allocated or freed, ever.  The first call
 * on a device (with that device current) looks up the array's address and writes its
 * twiddle tables, synchronising the device once: make that first call before any stream
 * capture.  The array's address and tables belong to the device context of that first
 * call: a device reset (cudaDeviceReset) while the library is loaded is not supported.
 * Calls share the array, so calls whose GPU work overlaps in time race and must not be
 * issued.  Messages for failures: ftoep_last_error(NULL, ...). */
ftoep_status ftoep_matvec_noalloc(const double* a, int64_t N, const double* x, double* y, int64_t nlines,
                                  int transpose, void* cuda_stream);

/* Scheme 1 (Sec. 2, Eq. 7-9): the two-sided fractional ODE
 *     D_left^g u + D_right^g u + u = f  on (0, T),  u(0) = u(T) = 0,  0 < gamma < 1,
 * with the left L1 formula (Eq. 4) and the right one (Eq. 5) on tau = T/N: the symmetric
 * positive definite Toeplitz system A u = f of Eq. 9 of order N-1 (Theorem 1; first column
 * a_0 = 1 + 2 mu G_0, a_d = mu (G_d - G_{d-1}), mu = tau^-g / Gamma(2-g)), solved by the
 * conjugate gradient method of Sec. 2.3 with every product A w by circulant embedding
 * (Eq. 10, the input padded with zeros) and FFTs -- the paper's fast CG.  Double precision.
 * f, u: N-1 doubles (values at t_1 .. t_{N-1}), host or device; u holds the initial guess on
 * entry (zeros if none) and the solution on exit.  Stops when the recursively updated
 * residual satisfies ||r||_2 <= tol ||f||_2, or after maxit iterations.  *iters (nullable):
 * iterations done; *relres (nullable): ||f - A u||_2 / ||f||_2 of the returned u, from a fresh
 * product.  Allocates its device workspace and frees it before returning; ordered on
 * cuda_stream (a cudaStream_t, NULL = legacy default stream) and blocks until done.
 * Errors: FTOEP_EINVAL (gamma outside (0,1), N outside [2, 2^24], T <= 0, tol <= 0,
 * maxit < 1, f or u NULL), FTOEP_ENOMEM, FTOEP_ECUDA.  Message: ftoep_last_error(NULL, ...). */
ftoep_status ftoep_two_sided_cg(double gamma, double T, int64_t N, const double* f, double* u, double tol,
                                int maxit, int* iters, double* relres, void* cuda_stream);

/* Restarted GMRES(restart) of Sec. 3.2 (the method the paper accelerates with circulant
 * products) on the space-time system of problem iprob of the plan, with zero initial data:
 * the reordered system of Eq. 21 (I_M (x) T + K (x) I_N; T lower-triangular Toeplitz with the
 * plan's first column a (ftoep_weights), K the spatial operator: -(second difference) with
 * Dirichlet zeros, or lambda I without space; for FTOEP_L1_HYPERBOLIC_CN averaged over levels
 * n and n-1).  Every product: T by circulant embedding (Eq. be1, the input padded with zeros)
 * and FFTs, K by a stencil; Arnoldi with classical Gram-Schmidt applied twice; double
 * precision.  A comparison path for ftoep_solve (the direct solve of the same system).
 * f: right-hand side [M][N] (the problem's field layout), u: initial guess in, solution out;
 * host or device memory.  restart in [1, 64]; stops when the true residual of an iterate
 * (checked at every restart) or the Arnoldi estimate satisfies ||r||_2 <= tol ||f||_2, or
 * after maxit Arnoldi steps.  *iters (nullable): Arnoldi steps done; *relres (nullable):
 * ||f - A u||_2 / ||f||_2 of the returned u from a fresh product.  Allocates (restart + 1) M N
 * doubles of device workspace and frees it before returning (on an error path it is freed at
 * ftoep_destroy); runs on the plan's stream and blocks until done.  Errors: FTOEP_EINVAL
 * (plan NULL, iprob out of range, f or u NULL, restart outside [1, 64], tol <= 0, maxit < 1),
 * FTOEP_ENOMEM, FTOEP_ECUDA. */
ftoep_status ftoep_gmres(ftoep_plan p, int iprob, const double* f, double* u, int restart, double tol, int maxit,
                         int* iters, double* relres);

/* Advection schemes of Sec. 3 by the fast procedure (space order, Figure 2):
 *   scheme 2 (0 < gamma < 1, Eq. 12/13): D^g u + u_x = f with the L1 quotient at x_{i-1/2} as
 *     the average of the L1 formulas (Eq. 4, scale tau^-g/(2 Gamma(2-g))) of nodes i and i-1,
 *     u_x by (U_i - U_{i-1})/h, f at (x_{i-1/2}, t_n): per node the lower-triangular Toeplitz
 *     system A-tilde U_i = B U_{i-1} + F_i (A-tilde = c L1 + I/h, B = I/h - c L1);
 *   scheme 3 (1 < gamma < 2, Eq. 16/17): the time terms of Eq. 17 at node i with u_x by the
 *     upwind difference at level n, f at (x_i, t_{n-1/2}): A-tilde U_i = U_{i-1}/h + F_i
 *     (A-tilde = c W + I/h).
 * Grid: tau = T/N, h = L/M, nodes x_i = i h (i = 1..M), inflow value u(0, t) = 0 (a = 1).
 * The node systems share one operator, so U_i = G U_{i-1} + V_i with G = A-tilde^-1 B and
 * V_i = A-tilde^-1 F_i (lower-triangular Toeplitz matrices commute): V for all nodes by one
 * batched solve of the scalar problem (lambda = 2/h, resp. 1/h; precision FTOEP_FP64 or
 * FTOEP_MIXED), the first column of G by one more, and the recursion over i as a scan of
 * ceil(log2 M) rounds U_i += G^d U_{i-d} (d = 1, 2, 4, ...), each a batched circulant-
 * embedded product in double.  f, u: [M][N] doubles (row i-1 = node x_i), u0: length M or
 * NULL, phi: length M or NULL (scheme 3 only); host or device memory.  The initial-data
 * weights are those of Eq. 4 (the u0 weight G_{n-1}) and Eq. 17.  Creates and destroys an
 * internal plan; ordered on cuda_stream and blocks until done.  Errors: FTOEP_EINVAL (scheme
 * not 2 or 3, gamma outside the scheme's range, N or M < 1, T or L <= 0, NULL f or u, bad
 * precision), FTOEP_ENOMEM, FTOEP_ECUDA; message by ftoep_last_error(NULL, ...). */
ftoep_status ftoep_advection_sweep(int scheme, double gamma, double T, double L, int64_t N, int64_t M,
                                   const double* f, const double* u0, const double* phi, double* u, int precision,
                                   void* cuda_stream);

/* The solver a plan uses for problem iprob (FTOEP_SOLVER_HALFSPLIT or
 * FTOEP_SOLVER_INVERSE), after the library's choice and the tuning's rule.  Errors: FTOEP_EINVAL. */
ftoep_status ftoep_problem_solver(ftoep_plan p, int iprob, int* solver);

/* Autotuner (no counterpart in the paper).  Times ftoep_solve on synthetic fields for
 * every candidate tuning -- time-block length fft_tile in {1024, 2048, 4096} of the
 * half-split solver (the inverse-series solves are the caller's choice: they trade accuracy
 * or device memory for time) x scheduler in {levels, chain} x internal streams in
 * {2, 4, 8} (streams only for plans of several problems; a single problem runs on the
 * caller's stream) -- with a plan per candidate,
 * one warm-up solve, one captured solve and two timed replays (CUDA events on
 * cuda_stream), device memory freed afterwards, and writes the fastest tuning to *out
 * (leaf and gemm_max_level 0 = library choice).  When the problems together exceed 2^28
 * unknowns the candidates are timed on a sample: problems taken evenly over the list sorted
 * by M*N, up to that many unknowns.  Blocks until done.  Errors: FTOEP_EINVAL (bad problems,
 * out NULL), FTOEP_ENOMEM, FTOEP_ECUDA; *out is left unchanged on error. */
ftoep_status ftoep_autotune(const ftoep_problem* probs, int nprob, void* cuda_stream, ftoep_tuning* out);

/* Wait for the plan's stream; returns FTOEP_ECUDA on an asynchronous CUDA error. */
ftoep_status ftoep_sync(ftoep_plan p);

/* Copy a NUL-terminated message for the last failure of p (or of plan creation if p is
 * NULL) into buf[n].  Returns FTOEP_EINVAL if buf is NULL or n == 0. */
ftoep_status ftoep_last_error(ftoep_plan p, char* buf, size_t n);

/* Release the plan and all device memory it owns (waits for its stream first). */
ftoep_status ftoep_destroy(ftoep_plan p);

#ifdef __cplusplus
}
#endif

#endif /* FTOEP_H */

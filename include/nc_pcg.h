/*
 * nc_pcg.h -- C ABI of the GB300 Newton-Chebyshev preconditioned CG library.
 *
 * Method: Bergamaschi & Martinez, "Parallel Newton-Chebyshev Polynomial
 * Preconditioners for the Conjugate Gradient method".  The library solves
 * A x = b (A symmetric positive definite, Sec. 1) by PCG whose preconditioner
 * is z = P_k(A) r, the degree-k Chebyshev polynomial of Sec. 3 applied with
 * k matrix-vector products by the three-term recurrence of Algorithm 2 (or,
 * for k = 2^nlev - 1, by the Newton recursion of Algorithm 1, Sec. 2: the
 * same polynomial by Theorem 3.1), with the modified parameter
 * theta' = s*theta of Sec. 4.  Entry points: matrices and bounds, one solver
 * per matrix (single or several right-hand sides), the batched engine for
 * many matrix-free systems, and an allocation-free apply.
 *
 * Conventions for every entry point
 *  - Pointers named *_dev are CUDA device pointers (for instance the storage
 *    of torch CUDA tensors) on the current device; pointers named *_host are
 *    host pointers.  Vectors are dense, contiguous, float64, length n.
 *  - Memory passed in is owned by the caller.  A matrix handle BORROWS the
 *    caller's arrays: they must stay alive and unchanged until the handle is
 *    destroyed.  Memory the library allocates (scaled copies, workspaces) is
 *    owned by the handle and released by its destroy call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; calls that return host values
 *    (results, bounds) synchronise that stream before returning.
 *  - Errors are reported only through nc_status; no call aborts the process.
 *    On error, output handles are set to NULL and nothing is leaked.
 *  - A handle may be used by one host thread and one stream at a time.
 */
#ifndef NC_PCG_H
#define NC_PCG_H

#include <stdint.h>

#if defined(__GNUC__)
#define NC_API __attribute__((visibility("default")))
#else
#define NC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nc_matrix_s* nc_matrix;
typedef struct nc_solver_s* nc_solver;
typedef struct nc_batch_s* nc_batch;

typedef enum {
    NC_OK = 0,
    NC_ERR_ARG = 1,          /* invalid argument (null pointer, size, bounds)        */
    NC_ERR_CUDA = 2,         /* a CUDA runtime call failed                            */
    NC_ERR_OOM = 3,          /* device allocation failed                              */
    NC_ERR_INDEFINITE = 4,   /* (p,Ap) <= 0 or (r,z) <= 0: A or P_k(A) not SPD       */
    NC_ERR_MAXIT = 5,        /* maxit reached before ||r|| <= tol ||b||               */
    NC_ERR_BREAKDOWN = 6,    /* NaN or Inf in a reduction                             */
    NC_ERR_UNSUPPORTED = 7,  /* option combination not implemented for this format    */
    NC_ERR_SCRATCH_LIMIT = 8, /* n above the fixed scratch of nc_apply_poly_csr_noalloc */
    NC_ERR_ADMISSION = 9,    /* batch engine: no free slot or not enough pooled memory */
    NC_ERR_TIMEOUT = 10      /* a staged step kernel's bounded wait for its own copies
                                ran out; the results of that call are not valid    */
} nc_status;

/* Value type of the matrix inside P_k(A) (the outer CG stays float64). */
typedef enum { NC_F64 = 0, NC_F32 = 1, NC_BF16 = 2 } nc_dtype;

/* Layout the solver's product kernels read (built once by pcg_setup).
 * SELL: slices of 32 rows (block rows for BSR3) stored slot-major, rows
 * padded to the slice's longest row (coalesced thread-per-row access); AUTO
 * picks SELL when the padding is at most 1.5x the nonzeros, else CSR (plain
 * block CSR for BSR3); TUNE builds SELL (padding up to 4x), times one fused
 * step in each layout on this matrix during pcg_setup and keeps the faster
 * (timings in nc_solver_info).  PSELL (scalar CSR matrices only): SELL
 * whose slices store no column indices; slice s holds the columns
 * row + o for the sorted set of offsets o = col - row of its 32 rows (rows
 * lacking an offset store a 0 there), and each distinct set is kept once.
 * It applies when every row's columns increase, a slice has at most 64
 * offsets, the padding is at most 1.5x, the distinct sets hold at most
 * 16384 offsets in all (regularly numbered grid matrices) and n <= 2^30;
 * otherwise the solver falls back to SELL.  AUTO tries PSELL first for CSR matrices,
 * except with use_graph = 2 (the cluster solve reads plain SELL).  Stencil
 * handles ignore the option. */
typedef enum {
    NC_FORMAT_AUTO = 0,
    NC_FORMAT_CSR = 1,
    NC_FORMAT_SELL = 2,
    NC_FORMAT_TUNE = 3,
    NC_FORMAT_PSELL = 4
} nc_format;

/* How the preconditioner is evaluated.  CHEBYSHEV: the three-term recurrence
 * of Algorithm 2 (Sec. 3, Eq. rhocheb), any degree k, one fused product step
 * per degree.  NEWTON: the recursion of Algorithm 1 (Sec. 2, Eqs. recursive
 * and zetaNewt), P_0 = zeta_0 I, P_{j+1} = zeta_{j+1} (2 P_j - P_j A P_j),
 * only for k = 2^nlev - 1 (NC_ERR_ARG otherwise) and a float64 apply
 * (NC_ERR_UNSUPPORTED otherwise); the same k products, evaluated depth
 * first, with 2 (nlev - 1) extra float64 work vectors.  By Theorem 3.1 both
 * give the same polynomial; the modified theta' (Sec. 4) enters both through
 * the interval [theta' - delta, theta' + delta].  The one-cluster solve
 * (use_graph = 2) runs the Chebyshev form only. */
typedef enum { NC_POLY_CHEBYSHEV = 0, NC_POLY_NEWTON = 1 } nc_poly_form;

/* Kernel variant of the fused product steps (Algorithm 2's loop body, and
 * q = A p with (p, q)) on the SELL-32 layouts.  DIRECT: one row per thread,
 * every operand loaded from global memory when it is needed.  STAGED
 * (offset-pattern layout, PSELL): persistent CTAs; each 256-row tile's
 * matrix slices and its rows of r and x_{k-2} are brought into shared memory
 * by bulk asynchronous copies a few tiles ahead of their use, so the HBM
 * stream does not wait on the gathers of x_{k-1}.  Both compute the same
 * fma chain in the same order (identical results for the same grid).  TUNE:
 * pcg_setup times a small set of candidates of both variants (stages in
 * flight, CTAs per SM, L2 prefetch distance, CTAs of the dot-product steps)
 * on the solver's own operator and keeps the fastest for the plain steps and
 * for the steps with a dot product; pcg_tune_candidate lists what was
 * measured.  SPLIT (steps with a dot product only; a tuner candidate, or
 * forced with direct plain steps): the step without its dot product, then a
 * separate deterministic dot product over the two finished vectors -- more
 * bytes, but the step kernel keeps the plain step's registers and
 * occupancy.  AUTO (default): TUNE for PSELL operators of at least 2^16 rows,
 * DIRECT otherwise.  For matrix-free stencils TUNE (AUTO: at least 2^20
 * points) times the z-chunk of the plain steps and, with a float apply, the
 * planes per z-march batch.  When the environment variable NC_TUNE_CACHE names a
 * file, the choices are looked up there by the operator's signature (rows,
 * stored entries, offset sets, apply precision, SM count, compute
 * capability) and measured and appended only when absent.  Layouts other than PSELL, and the stencil and block
 * kernels, always run their single variant. */
typedef enum {
    NC_STEP_AUTO = 0,
    NC_STEP_DIRECT = 1,
    NC_STEP_STAGED = 2,
    NC_STEP_TUNE = 3,
    NC_STEP_SPLIT = 4
} nc_step_kernel;

typedef struct {
    int apply_dtype;   /* nc_dtype: F64 = plain method; F32: float32 matrix and
                          vectors inside P_k; BF16: bfloat16 matrix values,
                          float32 vectors and accumulation.                     */
    int rr_period;     /* > 0: replace the recurrence residual by the true one,
                          r = b - A x in float64, after every rr_period-th
                          iteration that does not stop (mixed precision); the
                          search direction p is kept.  0 = never.              */
    int x0_is_zero;    /* 1: ignore x on input and start from x0 = 0 (saves the
                          initial product b - A x0).                            */
    int use_graph;     /* 1 (default): one CUDA graph per solve with the
                          stopping test evaluated on the device; 0: host loop
                          reading the residual every iteration; 2: the whole
                          solve in one kernel on one thread-block cluster of up
                          to 16 CTAs, operator and vectors held in the
                          cluster's shared memory (small systems, where
                          launches and L2 latency dominate).  Taken when the
                          solver is float64, SELL, without residual
                          replacement, and its slices fit (about 20k rows of a
                          7-point operator); else the graph.                    */
    int spmv_format;   /* nc_format of the solver's product kernels (AUTO).    */
    int poly_form;     /* nc_poly_form: how z = P(A) r is evaluated.           */
    int step_kernel;   /* nc_step_kernel (AUTO).  The six fields below fix a
                          STAGED or DIRECT choice; 0 = the library default.   */
    int step_stages;   /* STAGED: tiles in flight per CTA, 2..4 (default 2)    */
    int step_ctas_per_sm; /* STAGED: resident CTAs per SM (default 6, capped by
                          what the device holds)                               */
    int step_rows_per_thread; /* plain steps, either variant: 1 or 2 rows per
                          thread (default 1): tiles of 256 or 512 rows, the
                          loads of both rows in flight together               */
    int step_tile_order; /* STAGED: 0 (default) CTA b takes tiles b, b + grid,
                          ...; 1: a contiguous run of tiles per CTA            */
    int prefetch_tiles;/* DIRECT float kernels: L2 prefetch distance in 256-row
                          tiles (default 2 x the SM count; < 0: off)           */
    int red_ctas_per_sm; /* DIRECT steps with a dot product: persistent CTAs
                          per SM, 1..64 (default 8; 64 = one 256-row tile per
                          CTA on any device)                                   */
    int keep_diagonal; /* PSELL: 0 (default) leaves a constant diagonal (every
                          row's a_ii bitwise equal, as after nc_matrix_jacobi,
                          whose scaled diagonal is exactly 1) out of the
                          layout and applies it through the step's u
                          coefficient: one product and one value fewer per
                          row; 1 stores it like any entry                      */
} nc_options;

typedef struct {
    int64_t n;
    int32_t degree_k;
    int32_t spmv_format;  /* NC_FORMAT_CSR, _SELL or _PSELL (after AUTO)      */
    int32_t apply_dtype;
    int32_t persistent;   /* 1: solves run as one kernel on one cluster     */
    double padding;       /* stored entries / nonzeros of the chosen layout    */
    double theta, delta, sigma;   /* theta' = s(a+b)/2, delta, sigma (Sec. 3/4) */
    double shift;         /* the stored operator is A - shift*I (theta' with
                             SELL: the (1 - x/theta') factor of the p_k
                             recursion, Sec. 3), 0 = A itself               */
    double tune_us_plain; /* TUNE: measured step time, plain layout (us)   */
    double tune_us_sliced;/* TUNE: measured step time, sliced layout (us)  */
    int64_t patterns;     /* PSELL: distinct offset sets stored; else 0     */
    int32_t step_kernel;  /* NC_STEP_DIRECT or NC_STEP_STAGED: plain steps  */
    int32_t dot_step_kernel; /* the same for the steps with a dot product   */
    int32_t step_stages, step_ctas_per_sm;  /* STAGED shape, plain steps     */
    int32_t step_rows_per_thread, step_tile_order;
    int32_t dot_step_stages, dot_step_ctas_per_sm; /* and dot-product steps */
    int32_t dot_step_rows_per_thread, dot_step_tile_order;
    int32_t prefetch_tiles, red_ctas_per_sm; /* DIRECT configuration         */
    int32_t tune_candidates; /* TUNE: candidates measured (pcg_tune_candidate) */
    int32_t num_sms;      /* SM count of the device the solver was set up on */
    int32_t faults;       /* 1: a staged kernel's bounded wait ran out (the
                             results of that call are not valid)              */
    int32_t tune_from_cache; /* 1: the tuner's choices came from the file named
                             by NC_TUNE_CACHE (nothing measured)              */
    int32_t stencil_zchunk;  /* matrix-free stencil: z-chunk (planes per CTA)
                             of the plain steps; 0 for explicit matrices     */
    int32_t stencil_planes_per_batch; /* and planes per z-march batch (0:
                             the size policy, 2 or 4)                         */
    int32_t diag_folded;  /* PSELL: 1 when the constant diagonal is left out of
                             the layout (keep_diagonal 0)                     */
    int32_t reserved1;
    double diag_value;    /* and its value in the stored operator, a_ii - shift */
} nc_solver_info;

/* One configuration measured by the tuner (pcg_setup with step_kernel =
 * TUNE, or AUTO on a large PSELL operator). */
typedef struct {
    int32_t op;           /* 0: the operator inside P_k, plain step (DOT 0);
                             1: inside P_k, last step with (r, z);
                             2: the float64 operator, q = A p with (p, q)   */
    int32_t step_kernel;  /* NC_STEP_DIRECT or NC_STEP_STAGED              */
    int32_t stages, ctas_per_sm, rows_per_thread, tile_order; /* STAGED    */
    int32_t prefetch_tiles, red_ctas_per_sm;                   /* DIRECT    */
    int32_t zchunk, planes_per_batch; /* matrix-free stencil (else 0)      */
    double us;            /* mean duration of one launch (CUDA events)     */
    int32_t chosen;       /* 1: kept for that operator and step kind       */
    int32_t reserved0;
} nc_tune_candidate;

typedef struct {
    int32_t iters;        /* PCG iterations                                      */
    int32_t status;       /* nc_status of the solve                              */
    double relres;        /* ||r_i|| / ||b||, recurrence residual, scaled system */
    double true_relres;   /* ||b - A x|| / ||b|| recomputed at exit, same system */
    int64_t n_spmv;       /* products with A: (k+1) per iteration (Table 4), plus
                             one per residual replacement                        */
    int64_t n_dot;        /* dot products: 3 per iteration (Table 4)             */
    int64_t n_replace;    /* residual replacements performed                     */
} nc_result;

/* Fill `opt` with the defaults: F64, no residual replacement, x0 from x,
 * graph on, AUTO layout, Chebyshev form. */
NC_API void nc_options_default(nc_options* opt);
NC_API const char* nc_strerror(nc_status s);
NC_API const char* nc_version(void);
/* Text of the last CUDA runtime error seen by this thread (after NC_ERR_CUDA). */
NC_API const char* nc_last_cuda_error(void);

/* ---- Matrices ------------------------------------------------------------
 * The paper needs only v -> A v (Sec. 1, "matrix-free regime"); Sec. 5.2 keeps
 * complete consecutive rows together (block-row distribution).  Handles hold
 * the operator the polynomial is applied to.
 */

/* CSR, float64 values.  rowptr_dev: n+1 int32 (rowptr[0] = 0, nondecreasing,
 * rowptr[n] = nnz); col_dev: nnz int32 in [0, n); val_dev: nnz float64.
 * Borrowed.  n = 0 is accepted (an empty system).  NC_ERR_ARG on n < 0,
 * nnz < 0, nnz >= 2^31 or a null pointer with n > 0. */
NC_API nc_status nc_matrix_csr(int64_t n, int64_t nnz, const int32_t* rowptr_dev,
                        const int32_t* col_dev, const double* val_dev, nc_matrix* out);

/* 3x3-block CSR, float64 values (three dofs per node, as in the paper's
 * finite-element structural matrices, Sec. 5).  browptr_dev: nb+1 int32
 * block-row pointers; bcol_dev: nnzb int32 block columns in [0, nb); val_dev:
 * 9*nnzb float64, block p's entry (r, c) at val[9p + 3r + c].  Scalar
 * unknown 3*node + component; n = 3*nb.  Borrowed.  NC_ERR_ARG on negative
 * sizes, 3*nb or nnzb >= 2^31, or a null pointer with nb > 0. */
NC_API nc_status nc_matrix_bsr3(int64_t nb, int64_t nnzb, const int32_t* browptr_dev, const int32_t* bcol_dev,
                                const double* val_dev, nc_matrix* out);

/* Matrix-free constant-coefficient 7-point operator on an nx x ny x nz grid
 * (Sec. 1: only v -> A v is needed; Sec. 5.3: FD-3D Poisson), zero
 * Dirichlet halo, unknown (i, j, k) at index i + nx (j + ny k):
 *   (A u)_p = c0 u_p - cx (u_{p-ex} + u_{p+ex}) - cy (...) - cz (...).
 * No device memory is involved; the handle holds only the coefficients.
 * NC_ERR_ARG if a side is < 1, nx*ny*nz >= 2^31 or a coefficient is not
 * finite.  The operator is SPD when c0 > 2 sum_a |c_a| cos(pi/(n_a + 1))
 * (not checked). */
NC_API nc_status nc_matrix_stencil7(int nx, int ny, int nz, double c0, double cx, double cy, double cz,
                                    nc_matrix* out);

/* Symmetric diagonal (Jacobi) scaling A_s = D^{-1/2} A D^{-1/2}, D = diag(A)
 * (Sec. 2, end: "symmetrically scaled by the diagonal"; Sec. 5: all matrices
 * are scaled before solving).  Returns a new handle that OWNS the scaled
 * values and d^{-1/2}; it still borrows A's index arrays, so A's arrays must
 * outlive it.  pcg_solve on a solver built on this handle solves the
 * original system A x = b: it forms b_s = D^{-1/2} b, solves A_s y = b_s
 * (the stopping test is on this scaled system) and returns x = D^{-1/2} y.
 * For a stencil handle the scaled operator is again a stencil (c0 = 1,
 * c_a / c0) and D^{-1/2} = c0^{-1/2}; nothing is allocated.
 * NC_ERR_ARG if a diagonal entry is missing or not positive, or if A is
 * already a scaled handle. */
NC_API nc_status nc_matrix_jacobi(nc_matrix A, void* stream, nc_matrix* out);

/* Two-level variant (Sec. 6, conclusions: a first-level preconditioner in
 * factored form P_0 = W W^T, the Newton-Chebyshev polynomial applied to
 * W^T A W), with block Jacobi as the first level of a 3x3-block matrix:
 * W = blockdiag(L_i^{-T}), A_ii = L_i L_i^T the Cholesky factor of each
 * diagonal block, so W W^T = blockdiag(A_ii^{-1}) and W^T A W has identity
 * diagonal blocks.  Returns a new owning handle of W^T A W (same block
 * pattern, the parent's index arrays borrowed); a solver built on it takes
 * the original b and returns the original x (b_s = W^T b, x = W y), and the
 * bounds passed to pcg_setup refer to W^T A W.  NC_ERR_ARG for a handle that
 * is not an unscaled BSR3 matrix or has a block row without a positive
 * definite diagonal block. */
NC_API nc_status nc_matrix_block_jacobi(nc_matrix A, void* stream, nc_matrix* out);

/* y_dev = A x_dev for the handle's operator.  x_dev, y_dev: n float64,
 * distinct buffers. */
NC_API nc_status nc_matvec(nc_matrix A, const double* x_dev, double* y_dev, void* stream);

/* Estimate an interval [lmin, lmax] containing the spectrum (needed by
 * Algorithm 1 step 1 and by Algorithm 2; Sec. 5.1 uses the power method and
 * DACG, this library a `steps`-step Lanczos run without reorthogonalisation
 * from the start vector v0_dev, n float64, nonzero).  lmax is made safe:
 * max(ritz_max + |b_m s_m|, 1.01 ritz_max), capped by the Gershgorin bound
 * max_i sum_j |a_ij| when that lies in [ritz_max, lmax); lmin = ritz_min.
 * ritz_min / ritz_max (may be NULL) return the raw extreme Ritz values.
 * NC_ERR_ARG if steps < 1 or steps > 256. */
NC_API nc_status nc_bounds_lanczos(nc_matrix A, int steps, const double* v0_dev, void* stream,
                            double* lmin, double* lmax, double* ritz_min, double* ritz_max);

/* lambda_max estimate by the power method, as the paper obtains beta_0 from
 * a few power iterations (Sec. 5.1): v = v0/||v0||, then `iters` times
 * w = A v, lambda = (v, w), v = w/||w||; *lmax = the last Rayleigh quotient
 * (at or below lambda_max: a caller adds a safety margin, e.g. 1.01, since
 * an underestimate makes P_k(A) indefinite).  v0_dev: n float64 start
 * vector (not modified).  NC_ERR_ARG for iters < 1 or v0 = 0;
 * NC_ERR_BREAKDOWN if A v vanishes or the values are not finite.
 * Synchronises `stream` once per iteration. */
NC_API nc_status nc_bounds_power(nc_matrix A, int iters, const double* v0_dev, void* stream, double* lmax);

/* Gershgorin upper bound max_i sum_j |a_ij| of the handle's operator. */
NC_API nc_status nc_gershgorin(nc_matrix A, void* stream, double* bound);

NC_API nc_status nc_matrix_destroy(nc_matrix A);

/* ---- Solver -------------------------------------------------------------- */

/* Build a solver for the handle's operator with spectral interval
 * [lambda_min, lambda_max] (Sec. 3: I = [alpha, beta] containing the
 * spectrum), polynomial degree degree_k >= 0 (k matrix-vector products per
 * application; k = 0 is diagonal-scaled CG, P = 1/theta) and theta scale
 * theta_scale = s > 0 (Sec. 4: theta' = s theta, delta unchanged, sigma =
 * theta'/delta; s = 1 is the exact Chebyshev polynomial, the paper uses
 * 1.01 and 1.001).  The recurrence scalars rho_0..rho_k (Eq. rhocheb) are
 * computed here in float64.  opt may be NULL (defaults).  Allocates the
 * workspaces (about 8 float64 vectors) and, for F32/BF16 apply, a converted
 * copy of the matrix values.  The matrix handle must outlive the solver.
 * NC_ERR_ARG unless 0 < lambda_min < lambda_max, degree_k <= 4096. */
NC_API nc_status pcg_setup(nc_matrix A, double lambda_min, double lambda_max, int degree_k,
                    double theta_scale, const nc_options* opt, void* stream, nc_solver* out);

/* z_dev = P_k(A) v_dev (Algorithm 2 with the recurrence indices rho_k,
 * rho_{k-1} that its derivation requires), in the solver's apply precision
 * (inputs and outputs float64).  For parity checks and standalone use. */
NC_API nc_status pcg_apply_poly(nc_solver S, const double* v_dev, double* z_dev, void* stream);

/* Solve A x = b by PCG (three dot products and k+1 products with A per
 * iteration, Table 4), stopping when ||r_i|| <= tol ||b|| (Sec. 5) or after
 * maxit iterations.  b_dev: n float64 (read only); x_dev: n float64, the
 * initial guess on input (ignored if opt.x0_is_zero) and the solution on
 * output.  `res` (may be NULL) receives the counts and residuals; the
 * returned status equals res->status.  On NC_ERR_MAXIT, NC_ERR_INDEFINITE or
 * NC_ERR_BREAKDOWN x_dev holds the last iterate.  b = 0 returns x = 0 with
 * 0 iterations.  Synchronises `stream`. */
NC_API nc_status pcg_solve(nc_solver S, const double* b_dev, double* x_dev, double tol, int maxit,
                    void* stream, nc_result* res);

/* As pcg_solve with host buffers: copies b_host (n float64) to the device,
 * solves, and copies the solution back to x_host.  Pinned host memory gives
 * asynchronous copies; pageable memory works too. */
NC_API nc_status pcg_solve_host(nc_solver S, const double* b_host, double* x_host, double tol,
                         int maxit, void* stream, nc_result* res);

/* Solve A X = B for m right-hand sides at once, 1 <= m <= 8: m independent
 * PCG recurrences (each with its own alpha, beta, stopping test and Table 4
 * counts) whose products with A share the matrix -- every fused Chebyshev
 * step and every q = A p reads A once for all m columns (a sparse matrix
 * times a dense block).  A column that stops is frozen while the others go
 * on.  B_dev, X_dev: n x m float64 on the device, column-major (column c at
 * offset c*n); X_dev holds the initial guesses unless opt.x0_is_zero.  res:
 * host array of m results (required).  Returns NC_OK when every column
 * converged, else the first column's non-OK status.  Needs a sliced layout
 * (SELL or PSELL) and the Chebyshev form without residual replacement
 * (NC_ERR_UNSUPPORTED otherwise); allocates 9 m n-vectors of workspace on
 * first use for a given m (kept until pcg_destroy).  Synchronises `stream`.
 * Not in the paper: a throughput form of its solver for many right-hand
 * sides. */
NC_API nc_status pcg_solve_multi(nc_solver S, int m, const double* B_dev, double* X_dev, double tol, int maxit,
                                 void* stream, nc_result* res);

/* Layout and parameters the solver chose (info: caller-owned).  NC_ERR_ARG
 * for a null argument.  Reads the solver's fault flag from the device
 * (synchronises the device memory copy). */
NC_API nc_status pcg_get_info(nc_solver S, nc_solver_info* info);

/* Candidate i (0 <= i < info.tune_candidates) timed by the tuner during
 * pcg_setup, in the order measured; NC_ERR_ARG when i is out of range or an
 * argument is null.  Host only.  Not in the paper: launch parameters of the
 * product kernels chosen by measurement on the solver's own matrix. */
NC_API nc_status pcg_tune_candidate(nc_solver S, int i, nc_tune_candidate* out);

/* Frees the solver's workspaces and layouts (not the matrix handle); the
 * frees wait for work still running on the device.  NC_ERR_ARG for NULL. */
NC_API nc_status pcg_destroy(nc_solver S);

/* ---- Batched and continuous-batching engine --------------------------------
 * Many independent systems (matrix-free constant 7-point stencils of any
 * size, each with its own bounds, degree k and theta scale, and explicit
 * matrices through their solvers, pcg_batch_add_solver; one slot per
 * right-hand side) solved together: every PCG iteration of every slot is one
 * pass of a fixed sequence of persistent kernels over device-side work lists
 * (stencil tiles and vector chunks of all slots), captured once as a CUDA
 * graph with a device-evaluated WHILE loop.  Precision: float32 matrix-free
 * P_k(A) (Algorithm 2, theta' = s theta) inside a float64 PCG (residual,
 * dot products and stopping test in float64, Sec. 5: ||r|| <= tol ||b||).
 * Each slot is Jacobi scaled (c0 -> 1) and lambda_min/lambda_max refer to the
 * scaled operator; x0 = 0.  Every slot reduces its own dot products in a
 * fixed order, so its result does not depend on the other slots.
 *
 * pcg_batch_create: capacity of max_slots slots and max_unknowns pooled
 *   unknowns (6 float64 + 4 float32 vectors each: 64 bytes per unknown,
 *   allocated once -- the HBM budget); kmax = largest degree accepted;
 *   flags: 0, or NC_BATCH_HOST_LOOP to drive the same kernels from a host
 *   loop (one synchronisation per iteration; for profilers).
 * All calls on one engine are ordered on its `stream` (they enqueue work
 * there and only pcg_batch_run synchronises it); a caller that switches
 * streams orders them itself.
 * pcg_batch_add: admit one system with right-hand side b_dev (n float64,
 *   read by a kernel enqueued on `stream`).  NC_ERR_ADMISSION when no slot or
 *   pool space is free (retry after releasing finished slots).  The slot
 *   starts with the next pcg_batch_run.
 * pcg_batch_run: advance every admitted slot by up to iter_limit PCG
 *   iterations (<= 0: until all slots have stopped) in one graph launch;
 *   synchronises the stream; *active_left = slots not yet finished.
 * pcg_batch_status: done flag and result of a slot (as of the last run).
 * pcg_batch_collect: x_dev (n float64) = the slot's solution of the original
 *   (unscaled) system; only for finished slots.
 * pcg_batch_release: free a finished slot and its memory (collects already
 *   enqueued on `stream` still read it first).
 * pcg_batch_free_units: largest contiguous and total free pooled unknowns. */
#define NC_BATCH_HOST_LOOP 1
/* flags: NC_BATCH_F64_APPLY applies P_k in float64 (3 float64 work vectors
 * per unknown instead of 4 float32; 72 instead of 64 bytes per pooled
 * unknown) rather than the default float32 apply with float64 outer CG. */
#define NC_BATCH_F64_APPLY 2
NC_API nc_status pcg_batch_create(int max_slots, int64_t max_unknowns, int kmax, int flags, void* stream,
                                  nc_batch* out);
NC_API nc_status pcg_batch_add(nc_batch B, int nx, int ny, int nz, double c0, double cx, double cy, double cz,
                               double lambda_min, double lambda_max, int degree_k, double theta_scale,
                               const double* b_dev, void* stream, int* slot);
/* Admit one system given by a solver on an explicit matrix (pcg_setup of a
 * CSR handle, optionally Jacobi scaled, whose layout is SELL-32 or the
 * offset-pattern form; the Chebyshev form; no residual replacement) and one
 * right-hand side b_dev (n float64 on the device, the original system's).
 * The slot runs that solver's polynomial -- its degree (1..kmax), bounds,
 * theta scale, stored operator and step coefficients -- inside the engine's
 * persistent work lists: its tiles (8192 rows of the layout each) join the
 * other slots' tiles in every step kernel, its vectors come from the pools,
 * x0 = 0.  The solver's apply precision must be the engine's (float32 or bfloat16 values with a
 * float32 engine, float64 with NC_BATCH_F64_APPLY): NC_ERR_UNSUPPORTED
 * otherwise.  The solver (and its matrix) must stay alive until the slot is
 * released.  Not in the paper: many explicit systems in one launch. */
NC_API nc_status pcg_batch_add_solver(nc_batch B, nc_solver S, const double* b_dev, void* stream, int* slot);
/* Admit m (1..8) right-hand sides of one such solver in groups: column c
 * (n float64 at B_dev + c * ldb, ldb >= n when m > 1) becomes slot slots[c]
 * (host array of m ints), each with its own state, result, collect and
 * release like any slot, but the columns form groups of up to 4 (a last
 * single column stays a plain slot) whose step kernels load each row's
 * columns and values once and apply them to all the group's columns (a
 * sparse times dense-block product: the matrix is read once per step for up
 * to 4 right-hand sides).  A column's iterates are bit-for-bit those of the same
 * right-hand side in a slot of its own.  The group's vectors take m * n
 * contiguous pooled unknowns; NC_ERR_ADMISSION when m slots or that range
 * are not free.  m = 1 is pcg_batch_add_solver. */
NC_API nc_status pcg_batch_add_solver_multi(nc_batch B, nc_solver S, int m, const double* B_dev, int64_t ldb,
                                            void* stream, int* slots);

/* Solve nsys systems at once, system i (solver S[i], as in
 * pcg_batch_add_solver) with nrhs[i] right-hand sides B_dev[i] (n_i x nrhs[i]
 * float64 on the device, column-major) into X_dev[i] (same shape; x0 = 0):
 * every (system, right-hand side) pair is a slot of one engine, a system's
 * right-hand sides in groups of up to 8 (pcg_batch_add_solver_multi), and
 * all of them advance together in one graph launch.  res: host array of
 * sum(nrhs) results, system by system.  All solvers share one apply
 * precision (NC_ERR_UNSUPPORTED otherwise).  Returns NC_OK when every slot
 * converged, else the first non-OK status.  Allocates the engine's pools for
 * the call and frees them before returning; synchronises `stream`. */
NC_API nc_status pcg_solve_batched(int nsys, const nc_solver* S, const int* nrhs, const double* const* B_dev,
                                   double* const* X_dev, double tol, int maxit, void* stream, nc_result* res);
NC_API nc_status pcg_batch_run(nc_batch B, double tol, int maxit, int iter_limit, void* stream, int* active_left);
NC_API nc_status pcg_batch_status(nc_batch B, int slot, int* done, nc_result* res);
NC_API nc_status pcg_batch_collect(nc_batch B, int slot, double* x_dev, void* stream);
NC_API nc_status pcg_batch_release(nc_batch B, int slot, void* stream);
NC_API nc_status pcg_batch_free_units(nc_batch B, int64_t* largest, int64_t* total);
/* Engine iterations run and kernels launched (engine iterations x (kmax + 5),
 * plus one per admission and per collect) since pcg_batch_create.  Host only. */
NC_API nc_status pcg_batch_stats(nc_batch B, int64_t* iterations, int64_t* launches);
NC_API nc_status pcg_batch_destroy(nc_batch B);
NC_API const char* nc_batch_last_cuda_error(void);

/* ---- No-allocation apply ---------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory when they apply the preconditioner
 * (a solver that draws all device memory from its own fixed arena, a
 * real-time loop where cudaMalloc/cudaFree and the synchronisation they can
 * imply are not allowed, a plugin inside a framework that owns the device
 * heap).  It computes the same z_dev = P_k(A) v_dev as pcg_apply_poly for a
 * CSR matrix with float64 values (arguments as in nc_matrix_csr and
 * pcg_setup), but builds no handle and calls no allocator: the float64
 * recurrence keeps two of its three work vectors in one fixed device array
 * of 2 x nc_apply_poly_noalloc_max_n() doubles (16 MiB), and uses z_dev as
 * the third.  The array belongs to the library's module: under CUDA's
 * default lazy module loading its 16 MiB are taken on a device when the
 * module is first used there (possibly by the first call of this entry
 * point) and held until the process exits.  Every call looks up the array's
 * device address (cudaGetSymbolAddress) with the calling device current.
 * Callers that need the no-allocation guarantee make one warm-up call per
 * device at start-up, outside any stream capture; later calls then allocate
 * nothing.  n above nc_apply_poly_noalloc_max_n() (2^20) is rejected with
 * NC_ERR_SCRATCH_LIMIT before any work.  All calls share
 * the array: calls that overlap on the GPU (several streams or host threads
 * on one device) race and must be serialised by the caller.  Nothing in the
 * array needs to start at zero (every slot is written before it is read).
 * v_dev and z_dev: n float64, distinct; work is enqueued on `stream`. */
NC_API nc_status nc_apply_poly_csr_noalloc(int64_t n, const int32_t* rowptr_dev, const int32_t* col_dev,
                                           const double* val_dev, double lambda_min, double lambda_max,
                                           int degree_k, double theta_scale, const double* v_dev,
                                           double* z_dev, void* stream);
/* Largest n accepted by nc_apply_poly_csr_noalloc. */
NC_API int64_t nc_apply_poly_noalloc_max_n(void);

#ifdef __cplusplus
}
#endif
#endif /* NC_PCG_H */

/*
 * helm.h -- C ABI of a GB300 (sm_103a) fast direct solver for the FEM
 * discretised Helmholtz problem with first-order absorbing boundaries,
 * following Toivanen & Wolfmayr, "A fast Fourier transform based direct
 * solver for the Helmholtz problem" (arXiv 1809.03808).
 *
 * Problem (Section 2, eqs. helmholtz, 1st-order-abc, bf-1st-order-abc):
 *     -Lap u - w^2 u = f  in a box,   du/dn - i w u = 0  on every face,
 * discretised by bilinear (2D) / trilinear (3D) elements on a uniform tensor
 * mesh with n_j nodes and spacing h_j along axis j.  The linear system is
 * A u = f with A the Kronecker form of eq. A2D (2D) or eq. A3D (3D) built from
 * the 1D matrices of eqs. matrixK / matrixM; every node is an unknown.
 *
 * Method (Sections 3-5): the absorbing rows of one axis ("x1") are replaced by
 * periodic ones (auxiliary operator B, eqs. probB, B2D, B3D) so that axis is
 * diagonalised by a DFT; three steps -- Step 1 B v = f, Step 2 A w = (B - A) v,
 * Step 3 B u = f + (B - A)(v + w) (eqs. probStep2, probStep3) -- recover the
 * exact solution, touching the non-periodic eigenvectors only on the two
 * boundary rows (eqs. 2dBs1, step2-1..step2-3, step3term).  The remaining axis
 * is a batch of complex tridiagonal solves, one per mode (Section 4.1.2).  In
 * 3D each per-mode solve is itself the 2D solver (Section 5.1.2).
 *
 * Array layout (all entry points): interleaved complex (re, im), C order,
 * LAST axis fastest: index (ix, iy) -> ix*ny + iy in 2D and (ix, iy, iz) ->
 * (ix*ny + iy)*nz + iz in 3D.  In 2D x1 (the periodic/DFT axis) is y, the
 * last axis.  In 3D the outer x1 is y and the inner x2 (the DFT axis of the
 * per-mode 2D solves, Section 5.1.2) is z.  The tridiagonal axis is x in both.
 * The choice of x1 is free (Remark Rem:ABCx1).
 *
 * Element types by precision mode:
 *   HELM_C128         f, u complex128; all arithmetic FP64.
 *   HELM_C64_REFINED  f, u complex128; solves in FP32 (complex64), residual
 *                     r = f - A u in FP64 (or float-float, helm_set_residual),
 *                     iterative refinement until ||r|| / ||f|| <= tol
 *                     (default 1e-14) or max_iter.
 *   HELM_C64_RAW      f, u complex64; one FP32 solve, no refinement.
 *
 * Errors: every entry point returns a helm_status; no exception crosses the
 * ABI.  CUDA failures are reported as HELM_ECUDA and the plan keeps the CUDA
 * error string (helm_last_error).
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct helm_plan* helm_plan_t;

enum helm_dtype {
  HELM_C128 = 0,
  HELM_C64_REFINED = 1,
  HELM_C64_RAW = 2
};

/* Arithmetic of the refinement residual r = f - A u (HELM_C64_REFINED).
 *   HELM_RESID_FP64  u accumulated in complex128, residual in FP64.
 *   HELM_RESID_FF    f and u held as float-float pairs (hi + lo floats, about
 *                    48 significant bits), residual and accumulation on the
 *                    FP32 pipes; u converted to complex128 once at the end.
 *                    Residual floor about 1e-13 relative: use tol >= 1e-12. */
enum helm_residual {
  HELM_RESID_FP64 = 0,
  HELM_RESID_FF = 1
};

/* Boundary condition on both faces of one axis (Section 2): the first-order
 * absorbing condition du/dn - i w u = 0 (Gamma_A), or the natural condition
 * du/dn = 0 (Gamma_N: the corner entries of eq. matrixK become 1). */
enum helm_bc {
  HELM_BC_ABC = 0,
  HELM_BC_NEUMANN = 1
};

/* Elements (Section 1 names the modified ones as applicable to the solver).
 * HELM_ELEMENT_Q1: the bilinear / trilinear elements of Section 2 with every
 *   integral exact (eqs. matrixK, matrixM: M = (h/6) tridiag(1, 4, 1)).
 * HELM_ELEMENT_Q1_MODIFIED: every element integral (stiffness, mass and the
 *   absorbing boundary term) by the tensor-product 2-point rule at +-sqrt(2/3)
 *   of the reference half-width, the modified integration that cuts the
 *   dispersion error to fourth order: K unchanged, M = (h/12) tridiag(1, 10,
 *   1) with corners 5h/12 on every axis.  The operator keeps the Kronecker
 *   form of eqs. A2D / A3D, so Steps 1-3 apply unchanged. */
enum helm_element {
  HELM_ELEMENT_Q1 = 0,
  HELM_ELEMENT_Q1_MODIFIED = 1
};

/* Plan options of helm_plan_2d_ex / helm_plan_3d_ex. */
struct helm_plan_opts {
  int32_t axis_bc[3]; /* helm_bc of each axis (entries beyond the dimension ignored) */
  int32_t element;    /* helm_element */
};

enum helm_status {
  HELM_OK = 0,
  HELM_EINVAL = -1,        /* bad argument (sizes, spacings, w, null pointer) */
  HELM_ENOMEM = -2,        /* device or host allocation failed */
  HELM_ECUDA = -3,         /* a CUDA runtime call failed */
  HELM_ENOTCONV = -4,      /* refinement stopped above tol; u is still written */
  HELM_ETIMEOUT = -5,      /* a bounded device wait gave up (helm_get_info; sticky) */
  HELM_EUNSUPPORTED = -6,  /* size outside what the kernels support */
  HELM_ENUMERIC = -7       /* plan eigen-data failed to converge / degenerate */
};

/* Diagnostics of the most recent solve (valid after the solve's stream has
 * been synchronised; helm_get_info synchronises it). */
typedef struct helm_info {
  int32_t dim;
  int32_t dtype;
  int64_t n[3];            /* node counts (n[2] = 1 in 2D) */
  int32_t iterations;      /* refinement sweeps performed (0 for plain modes) */
  int32_t converged;       /* 1 if the last refinement residual met tol */
  double residual[16];     /* ||f - A u||_2 / ||f||_2 after each sweep (FP64) */
  double plan_seconds;     /* host time spent building the plan */
  double tol;              /* refinement tolerance */
  int32_t max_iter;        /* refinement sweep limit */
  int32_t n_dft_stages;    /* stages of the x1 transform */
  size_t device_bytes;     /* device memory owned by the plan */
  int32_t residual_kind;   /* helm_residual of the plan */
  int32_t aux_q;           /* auxiliary of the periodic axes: phase q ... */
  double aux_rho;          /* ... and damping rho (see helm_set_auxiliary) */
  double aux_trial_residual; /* plan-time trial residual of the chosen auxiliary
                                (-1 if set by helm_set_auxiliary) */
  int32_t axis_bc[3];      /* helm_bc of each axis (HELM_BC_ABC beyond dim) */
  int32_t fp64_lines;      /* inner lines solved in FP64 by precision routing
                              (3D complex64 plans; see helm_set_precision_routing) */
  int32_t element;         /* helm_element of the plan */
} helm_info;

/* --- Plan (the paper's "Initialization", Section 6) -----------------------
 * Builds the per-axis eigen-data: the periodic eigenvalues of eq.
 * eigvaluesPer, the absorbing-pencil eigenvalues Lam^A and boundary rows of
 * V (eqs. EVP1a, EVPcondA), the DFT twiddles and the per-plan pivot tables;
 * allocates all device scratch; chooses the auxiliary (see helm_set_auxiliary)
 * by trial solves, which is most of the plan time on large grids.
 * nx, ny (, nz): node counts, >= 3.  hx, hy (, hz): spacings > 0, finite.
 * omega: wave number > 0, finite.  dtype: helm_dtype.
 * On success *out owns device memory until helm_destroy; on failure *out is
 * set to NULL.  Limits: the x1 length must be <= 4096 (HELM_C128) or 8192
 * (complex64 modes) in 2D, and the 3D transform lengths <= 1024; otherwise
 * HELM_EUNSUPPORTED.  Requires a current CUDA device. */
int helm_plan_2d(helm_plan_t* out, int64_t nx, int64_t ny, double hx, double hy,
                 double omega, int dtype);
int helm_plan_3d(helm_plan_t* out, int64_t nx, int64_t ny, int64_t nz, double hx,
                 double hy, double hz, double omega, int dtype);

/* The same plans with a boundary condition per axis (Section 2's Gamma_A and
 * Gamma_N; eq. matrixK with corners 1 - i w h or 1): axis_bc[k] is the
 * helm_bc of both faces of axis k (2 entries in 2D, 3 in 3D; axis 0 = x).
 * At least one axis must be absorbing (HELM_EINVAL otherwise): that keeps A
 * non-singular for every w.  helm_plan_2d / helm_plan_3d are these with
 * HELM_BC_ABC everywhere.  A Neumann periodic axis takes the closed-form
 * cosine eigen-data in place of the absorbing pencil's, and C_bb's corner
 * becomes 1/h - w^2 h/3; a Neumann x axis changes the end entries of the
 * tridiagonal line matrices.  Everything else is unchanged. */
int helm_plan_2d_bc(helm_plan_t* out, int64_t nx, int64_t ny, double hx, double hy,
                    double omega, int dtype, const int32_t* axis_bc);
int helm_plan_3d_bc(helm_plan_t* out, int64_t nx, int64_t ny, int64_t nz, double hx,
                    double hy, double hz, double omega, int dtype, const int32_t* axis_bc);

/* The same plans with options: per-axis boundary conditions as for the _bc
 * calls, and the element (helm_element; HELM_EINVAL for another value).
 * opts = NULL: absorbing faces everywhere and HELM_ELEMENT_Q1. */
int helm_plan_2d_ex(helm_plan_t* out, int64_t nx, int64_t ny, double hx, double hy,
                    double omega, int dtype, const struct helm_plan_opts* opts);
int helm_plan_3d_ex(helm_plan_t* out, int64_t nx, int64_t ny, int64_t nz, double hx,
                    double hy, double hz, double omega, int dtype,
                    const struct helm_plan_opts* opts);

/* Auxiliary problem B.  The paper makes x1 periodic (eqs. matrixKper,
 * matrixMper).  Here the wrap-around entries of those circulant matrices are
 * multiplied by g (last row) and 1/g (first row), with g = e^{rho + i q pi/2}.
 * B - A is still supported on the x1 boundary rows, so Steps 1-3 are
 * unchanged.  B is diagonalised by F D^-1, D = diag(e^{t j}),
 * t = (rho + i q pi/2)/n1, with eigenvalues (2 - 2cosh(t + i theta_l))/h and
 * h (4 + 2cosh(t + i theta_l))/6.  rho = q = 0 is the paper's periodic
 * auxiliary.  Which (rho, q) keeps B's own problems well conditioned depends
 * on the grid, so a new plan tries five candidates, (rho, q) in {(1, 1),
 * (0.5, 0), (1, 0), (0.5, 1), (0, 0)}: one solve of a fixed pseudo-random
 * load each, in the plan's precision, keeping the smallest relative residual
 * (helm_info reports the choice).  This call overrides that choice.
 * Applies to every periodic axis of the plan.  rho must be in [0, 8]; any
 * integer q is taken mod 4.  Rebuilds the plan's auxiliary tables; call it
 * between solves, not while a solve is in flight on another stream. */
int helm_set_auxiliary(helm_plan_t p, double rho, int phase_quarters);

/* Precision routing of 3D complex64 plans: the inner tridiagonal lines
 * (Section 5.1.2's per-mode solves along x) whose matrix
 * K_x + (Lam_l + Lam_m - w^2) M_x is close to singular are solved with FP64
 * arithmetic (FP64 pivots, FP64 substitutions) by a separate kernel; all
 * other lines stay in complex64.  A line is routed when some eigenvalue
 * Lam^A_x,k of its own axis's pencil makes |Lam^A_x,k + Lam_l + Lam_m - w^2|
 * < tau w^2.  Off by default (tau = 0): the complex64 solve's error does sit
 * in those lines (on a 256^3 grid of the 512^3 workload's spacing and wave
 * number the closest 1 % of the lines carry 96 % of it), but it is the
 * complex64 rounding of their inputs, amplified by their conditioning, which
 * FP64 sweeps do not remove (measured: -0.6 %).  helm_info.fp64_lines counts
 * the routed lines (all line types).  Returns HELM_EUNSUPPORTED for 2D or
 * complex128 plans, HELM_EINVAL for tau outside [0, 1].  Call between
 * solves. */
int helm_set_precision_routing(helm_plan_t p, double tau);

/* Kernel variants (the autotuner's choices; the paper fixes none of them).
 * Every variant computes the same solution; they differ in speed by grid.
 *   HELM_VARIANT_INNER_CHUNK  3D: rows per chunk of the tiled inner sweeps
 *                             (8, 16 or 32; default 16, 32 for lines beyond
 *                             1024 rows, 512 in complex128).
 *   HELM_VARIANT_INNER_TILES  3D: tiles of 16 inner modes per CTA (1..8;
 *                             default 1..4 by grid size).
 *   HELM_VARIANT_TRI2D        2D complex64: 0 = bulk-copy fed passes where
 *                             the x1 length is even (default), 1 = register-
 *                             tile passes.
 *   HELM_VARIANT_DFT          complex64 plans whose contiguous transformed
 *                             axis (x1 in 2D, the inner axis in 3D) has at
 *                             most 128 nodes: 0 = FFT kernels (default), 1 =
 *                             that axis's transforms as dense products with
 *                             the scaled DFT matrix on the tensor cores
 *                             (TF32 with high/low splitting of both operands,
 *                             FP32 accumulation: 22-bit operands, so a raw
 *                             complex64 solve is up to ~15x less accurate
 *                             than with the FFT kernels at n = 128;
 *                             refinement removes the difference); the
 *                             matrix tables (2 x 8 (2n)^2 bytes at most) are
 *                             built when it is switched on.
 * helm_set_variant returns HELM_EUNSUPPORTED for a knob the plan does not
 * have, HELM_EINVAL for a value that does not fit.  Call between solves.
 * helm_time_solve: device milliseconds of one solve of the plan's compute
 * path (one complex64 or complex128 solve, no refinement), averaged over
 * `reps` solves of a fixed pseudo-random load after one warm-up, timed with
 * CUDA events on the plan's stream (allocates two vectors for the call). */
enum helm_variant {
  HELM_VARIANT_INNER_CHUNK = 0,
  HELM_VARIANT_INNER_TILES = 1,
  HELM_VARIANT_TRI2D = 2,
  HELM_VARIANT_DFT = 3
};
int helm_set_variant(helm_plan_t p, int knob, int value);
int helm_get_variant(helm_plan_t p, int knob, int* value);
int helm_time_solve(helm_plan_t p, int reps, double* ms_per_solve);

/* Stream on which helm_solve enqueues its kernels (a cudaStream_t passed as
 * void*; NULL = legacy default stream).  One plan serves one stream at a time. */
int helm_set_stream(helm_plan_t p, void* cuda_stream);

/* Refinement controls for HELM_C64_REFINED: stop when ||r||/||f|| <= tol or
 * after max_iter sweeps (tol >= 0, 1 <= max_iter <= 15). */
int helm_set_refinement(helm_plan_t p, double tol, int max_iter);

/* Residual arithmetic of HELM_C64_REFINED (helm_residual; default
 * HELM_RESID_FP64).  Iterative refinement is not part of the paper's method;
 * this selects how its residual is formed.  Selecting HELM_RESID_FF allocates
 * two more float-float vectors (32 bytes per unknown) here, once per plan
 * (HELM_ENOMEM if they do not fit; the plan keeps its previous kind), so
 * that no solve allocates.  Returns HELM_EINVAL for another kind or a plan of
 * another dtype.  Call between solves. */
int helm_set_residual(helm_plan_t p, int kind);

/* HELM_C64_REFINED: launch the first solve and the refinement loop as one
 * CUDA graph whose loop is a device-side conditional while node (default 1),
 * or kernel by kernel (0).  The graph is captured at the first solve and
 * reused; it is recaptured when f or u move (FP64 residual), the residual kind
 * or the auxiliary change.  Profiling (helm_set_profiling) and
 * helm_solve_debug always launch kernel by kernel.  Both give the same
 * result; the graph avoids the host launches of the sweeps after
 * convergence. */
int helm_set_graphs(helm_plan_t p, int enable);

/* --- Solve (Sections 4.2 and 5.2: Steps 1-3) ------------------------------
 * f, u: DEVICE pointers to N = nx*ny(*nz) complex values in the layout above
 * (complex128 or complex64 per dtype).  f is read only, u is overwritten.
 * The byte ranges [f, f + N*elem) and [u, u + N*elem) must be disjoint, and
 * f and u must be multiples of elem (16 B complex128, 8 B complex64): a
 * shared byte or a misaligned pointer returns HELM_EINVAL before the device
 * is touched.  (The same rules hold for every entry point below that takes
 * f and u.)
 * Asynchronous on the plan's stream: returns after enqueueing.  Allocates
 * nothing (all scratch belongs to the plan).  Convergence of refinement is
 * reported by helm_get_info. */
int helm_solve(helm_plan_t p, const void* f, void* u);

/* Many right-hand sides of one operator (the domain-decomposition sweeps of
 * Section 1 reuse one operator for many loads): f and u hold nrhs vectors of
 * N values each, one after another (the layout above for each); the byte
 * ranges of all of f and all of u must be disjoint.  Right-hand side i is
 * solved exactly as helm_solve(p, f_i, u_i) would solve it (same kernels on
 * the same operator data, so the same bits), but up to k of them at once
 * (helm_set_rhs_concurrency, default 4): the plan keeps k - 1 extra
 * workspaces (its scratch: about 24-56 bytes per unknown each, sharing the
 * eigen-data and pivot tables), made at the first call that needs them and
 * kept until helm_destroy, and k streams forked from and joined back to the
 * plan's stream.  Asynchronous like helm_solve.  helm_get_info then reports
 * the right-hand side whose refinement ended worst.  Workspaces are rebuilt
 * after any setting that changes the plan's solve. */
int helm_solve_many(helm_plan_t p, int64_t nrhs, const void* f, void* u);
int helm_set_rhs_concurrency(helm_plan_t p, int k);  /* 1 <= k <= 16 */

/* Same solve with HOST pointers: copies f to the device, solves, copies u
 * back and synchronises the stream before returning (for callers without
 * device buffers; the copies are part of the call).  Page-locked host memory
 * gives full copy bandwidth; pageable memory also works.  Unlike helm_solve,
 * the first call allocates two device staging vectors (N values each), kept
 * by the plan until helm_destroy.  For
 * HELM_C64_REFINED with HELM_RESID_FF and both buffers page-locked and
 * mapped, no copies are made: the kernels that convert f to float-float and
 * u back read and write the host buffers directly (same results).  For
 * HELM_C64_REFINED with HELM_RESID_FP64 the refinement runs sweep by sweep,
 * the call reading each convergence test's state before it enqueues the
 * next correction, and the copy of u back starts beside the test that the
 * last two residuals predict to converge (on a second stream of the plan,
 * made at the first call): the same kernels in the same order as the
 * kernel-by-kernel loop, so the same bits as helm_solve.  f and u must not
 * share a byte (HELM_EINVAL). */
int helm_solve_host(helm_plan_t p, const void* f_host, void* u_host);

/* Step-by-step variant for verification: runs the same kernels as helm_solve
 * and also copies out, to DEVICE buffers the caller owns (any may be NULL):
 *   fhat  : N values, the DFT of f along x1 (eq. step1FFTfcoeff) -- in the
 *           solve's compute precision (complex64 in the C64 modes);
 *   v_b   : the Step-1 boundary rows of v = B^-1 f (eq. 2dBs1 / 3dBs1), and
 *   w_b   : the Step-2 boundary rows of w = A^-1 (B - A) v (eq. step2-3 /
 *           step2-3-3d), each 2*N/n1 values: the x1 = first face, then the
 *           x1 = last face, each in the layout of the remaining axes,
 *           complex128 in HELM_C128 and complex64 otherwise.
 * Only the first (unrefined) solve's intermediates are reported. */
int helm_solve_debug(helm_plan_t p, const void* f, void* u, void* fhat, void* v_b,
                     void* w_b);

/* Synchronises the plan's stream and fills *info. */
int helm_get_info(helm_plan_t p, helm_info* info);

/* Per-kernel timing.  When enabled, every kernel launch of helm_solve is
 * bracketed by CUDA events recorded on the plan's stream.  helm_get_profile
 * synchronises the stream, writes up to max_entries aggregated entries (one
 * per kernel kind: launches and summed device milliseconds), clears the
 * record and returns the number of entries written (or a negative status). */
typedef struct helm_profile_entry {
  char name[32];
  int32_t launches;
  double total_ms;
} helm_profile_entry;

int helm_set_profiling(helm_plan_t p, int enable);
int helm_get_profile(helm_plan_t p, helm_profile_entry* out, int max_entries);

/* Frees everything the plan owns.  NULL is allowed. */
int helm_destroy(helm_plan_t p);

const char* helm_status_string(int status);

/* Last CUDA/diagnostic message recorded by the plan (never NULL). */
const char* helm_last_error(helm_plan_t p);

/* --- Batches of independent problems --------------------------------------
 * Many problems of different sizes, wave numbers and modes solved together
 * (the paper solves one problem at a time; it has no batch layer).  A batch
 * groups existing plans (2D or 3D, any dtype, any residual kind); it does not
 * own them, and they must outlive it.  helm_batch_solve runs every plan's
 * whole solve - for refined plans including the refinement loop - as ONE
 * CUDA graph launch in which each plan is an independent branch, so the GPU
 * overlaps the small problems and no host launches happen per problem.
 * Each plan's result is the same as its helm_solve (the same kernels on the
 * same data); helm_get_info(plan) reports its refinement afterwards.
 *
 * helm_batch_create: count >= 1 plans, none NULL.  Allocates the
 *   float-float vectors of refined plans with that residual kind.
 * helm_batch_solve: f[i], u[i] are device pointers of plan i, as for
 *   helm_solve (host arrays of count pointers).  Asynchronous on the batch
 *   stream.  The graph is captured at the first call and reused while the
 *   pointers and the plans' settings (refinement, residual kind, auxiliary)
 *   stay the same; otherwise it is captured again (the device is
 *   synchronised first).  Rejects plans with profiling on (HELM_EINVAL).
 *   Plans of one batch must not be solved concurrently by other calls.
 * helm_batch_set_stream: stream of the launches (NULL: legacy stream).
 * helm_batch_destroy: NULL is allowed; the plans are untouched. */
typedef struct helm_batch* helm_batch_t;
int helm_batch_create(helm_batch_t* out, int32_t count, const helm_plan_t* plans);
int helm_batch_set_stream(helm_batch_t b, void* cuda_stream);
int helm_batch_solve(helm_batch_t b, const void* const* f, void* const* u);
const char* helm_batch_last_error(helm_batch_t b);
int helm_batch_destroy(helm_batch_t b);

/* --- Allocation-free small solve (the paper has no counterpart) -------------
 * For callers that cannot allocate device memory when they need a solve:
 * code running under a larger framework's allocator lock, or in a process
 * whose device memory is reserved up front.  Such callers cannot build a
 * plan (helm_plan_2d allocates), so this entry point does the whole
 * complex128 2D solve (the HELM_C128 arithmetic of helm_solve, fixed
 * auxiliary rho = q = 1, no residual check) without a plan.  It
 * calls no cudaMalloc, cudaFree or allocating library routine.  Its device
 * scratch is one fixed 16 MiB array that the library reserves on every GPU
 * that loads it, held until the process exits.
 *   f, u: DEVICE pointers, complex128, [nx][ny] as for helm_solve; f read
 *         only, u overwritten; their byte ranges must be disjoint and
 *         both must be 16-byte aligned (HELM_EINVAL otherwise).
 *   cuda_stream: stream the work is enqueued on (NULL = legacy default
 *         stream); asynchronous like helm_solve.
 * Limits: ny <= 1024, and about 47 bytes per unknown plus O(nx + ny) must
 * fit the 16 MiB (about 350,000 unknowns; 512 x 512 fits); larger problems
 * return HELM_EUNSUPPORTED before touching the device.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  Every call shares the
 * one array: calls whose work overlaps on the GPU (different streams, or
 * threads calling at once) race and give wrong results, so serialise them.  Each call rebuilds its
 * eigen-data on the host (O(ny^2) work) and copies it into the array. */
int helm_solve_2d_static(int64_t nx, int64_t ny, double hx, double hy, double omega,
                         const void* f, void* u, void* cuda_stream);

/* --- Server: a stream of independent requests with plan reuse -------------
 * The paper's method has no serving layer; this one keeps plans and their
 * eigen-data on the device between requests (domain-decomposition sweeps
 * solve one operator for many right-hand sides), and overlaps independent
 * requests on the GPU.
 *
 * A server owns a scheduler thread, a builder thread, `nslots` CUDA streams
 * (1..16) and a cache of plans keyed by (dim, n, h, omega, dtype, residual,
 * tol, max_iter).  Requests enter a FIFO queue.  The scheduler starts the
 * oldest request that can start whenever a slot is free: its operator's plan
 * is taken from the cache, or handed to the builder thread if the device
 * memory in use (cached plans, counted by their helm_info.device_bytes, and
 * the estimates of plans being built) plus an estimate of the new plan stays
 * within `device_budget_bytes` after idle cached plans are evicted least
 * recently used first.  While a plan is built the scheduler goes on starting
 * other requests; requests for that operator wait for it, and the request it
 * was built for goes back to the front of the queue.  The estimate is 64 MiB plus, per unknown, 100 B (2D complex64
 * modes), 200 B (2D HELM_C128), 112 B (3D complex64) or 128 B (3D
 * HELM_C128).  A request whose plan is busy with another request waits while
 * later requests for other operators start (a plan serves one request at a
 * time).  Building a plan waits only for its own work (its kernels run on
 * the legacy stream, its memory comes from the stream-ordered allocator), not
 * for the requests in flight on the server's streams.  A request's
 * right-hand sides go through helm_solve_many on its slot's stream (several
 * at once on the plan's workspaces).  Server plans launch kernel by kernel,
 * never capturing CUDA graphs, so other threads may synchronise the device
 * at any time.  Every right-hand side is solved as the plan's helm_solve
 * would solve it: each result is the same as for that request alone.
 *
 * f and u are DEVICE pointers of the server's device, nrhs * N complex
 * values each (complex64 for HELM_C64_RAW, complex128 otherwise; N = nx ny
 * (nz)), right-hand side after right-hand side; they must stay valid and
 * untouched until the request is reported done, and f must not overlap u.
 * The server's streams do not wait on the caller's: the work that writes f
 * (or last touches u) must be complete when helm_server_submit is called
 * (e.g. its stream synchronised).  The caller owns them. */
typedef struct helm_server* helm_server_t;

typedef struct helm_request {
  int32_t dim;       /* 2 or 3 */
  int64_t n[3];      /* node counts, n[2] ignored in 2D */
  double h[3];       /* spacings, h[2] ignored in 2D */
  double omega;      /* wave number */
  int32_t dtype;     /* helm_dtype */
  int32_t residual;  /* helm_residual (HELM_C64_REFINED only, else ignored) */
  double tol;        /* refinement tolerance (HELM_C64_REFINED only) */
  int32_t max_iter;  /* refinement sweep limit 1..15 (HELM_C64_REFINED only) */
  int32_t nrhs;      /* right-hand sides, >= 1 */
  const void* f;     /* device, nrhs * N values */
  void* u;           /* device, nrhs * N values */
} helm_request;

typedef struct helm_request_result {
  int32_t done;        /* 1 once the request has finished (or failed) */
  int32_t status;      /* helm_status of the request (valid when done) */
  double queue_s;      /* submit -> start of its first launch (host clock) */
  double latency_s;    /* submit -> completion seen by the scheduler */
  int32_t plan_reused; /* 1 if its plan came from the cache */
  int32_t iterations;  /* refinement sweeps of its last right-hand side */
  int32_t converged;   /* 1 if its last right-hand side met tol (refined modes;
                          status HELM_ENOTCONV otherwise, u still written) */
  double residual;     /* final ||r||/||f|| of its last right-hand side */
} helm_request_result;

typedef struct helm_server_stats {
  int64_t submitted, completed, failed;
  int64_t plans_built, plans_reused, plans_evicted;
  double unknowns_solved;   /* sum of N * nrhs over completed requests */
  double elapsed_s;         /* first submit -> last completion */
  double latency_p50_s, latency_p99_s, latency_mean_s;  /* completed requests */
  size_t device_bytes_in_use, device_bytes_peak;        /* cached plans */
} helm_server_stats;

/* helm_server_create: nslots 1..16, device_budget_bytes > 0 (plans only; the
 * request buffers are the caller's).  Uses the CUDA device current in the
 * calling thread.  HELM_EINVAL on bad arguments, HELM_ECUDA if no device.
 * helm_server_submit: validates the request (HELM_EINVAL), copies it, and
 * returns at once with *ticket >= 1.  A request that cannot fit the budget
 * even with every idle plan evicted fails with HELM_ENOMEM; one the kernels
 * cannot run fails with that plan's status (e.g. HELM_EUNSUPPORTED).
 * helm_server_wait: waits up to timeout_s (< 0: no limit) for the request;
 * fills *res (may be NULL); returns HELM_ETIMEOUT if it is still running,
 * HELM_EINVAL for an unknown ticket, else HELM_OK (the request's own status
 * is res->status).  A finished request's result stays available until the
 * server is destroyed.
 * helm_server_drain: waits (bounded as above) until every submitted request
 * has finished.  helm_server_get_stats: counters and latency percentiles of
 * the completed requests.  helm_server_destroy: waits for the queued and
 * running requests, frees the plans, streams and thread; NULL is allowed.
 * Submit, wait, drain and get_stats may be called from any threads at once;
 * destroy must not overlap any other call on the same server.  Each
 * request's record (about 200 bytes) is kept until destroy. */
int helm_server_create(helm_server_t* out, int32_t nslots, size_t device_budget_bytes);
int helm_server_submit(helm_server_t s, const helm_request* req, int64_t* ticket);
int helm_server_wait(helm_server_t s, int64_t ticket, double timeout_s, helm_request_result* res);
int helm_server_drain(helm_server_t s, double timeout_s);
/* What failed for a request that finished with a status other than HELM_OK
 * or HELM_ENOTCONV: the step (plan build, solve, completion, helm_get_info),
 * its status and the plan's last error string; "" for a request that
 * completed, is still pending or is unknown.  The string belongs to the
 * server and stays valid until helm_server_destroy. */
const char* helm_server_error(helm_server_t s, int64_t ticket);
int helm_server_get_stats(helm_server_t s, helm_server_stats* st);
int helm_server_destroy(helm_server_t s);

/* --- Failure detection and allocation checks (for tests) -------------------
 * The paper has no counterpart; these exist so that the library's failure
 * paths can be exercised without faulting a GPU.
 *
 * helm_debug_fail_alloc: the k-th device allocation the library makes from
 *   now on (k >= 1) fails as if the device were out of memory; k = 0
 *   disarms.  Returns the number of failures injected so far in the process.
 *   Plans report such a failure as HELM_ENOMEM (with *out = NULL and nothing
 *   left allocated), except for optional memory (pivot tables, auxiliary
 *   trial buffers, tiled-sweep buffers) whose absence the plan works around.
 * helm_debug_live_allocations: number of the library's device allocations
 *   alive now (plans, float-float vectors, staging buffers); *bytes (may be
 *   NULL) receives their total size.
 * helm_debug_wait_timeout: enqueues on the plan's stream one kernel whose
 *   bounded mbarrier wait (the wait the bulk-copy kernels use) can never
 *   complete, with a limit of `tries` polls (1 .. 2^22).  The wait gives up,
 *   the kernel returns, and the plan's error word is set: helm_get_info then
 *   returns HELM_ETIMEOUT, as it would for a real copy that never arrived.
 *   The error word stays set for the life of the plan. */
int helm_debug_fail_alloc(int k);
int64_t helm_debug_live_allocations(size_t* bytes);
int helm_debug_wait_timeout(helm_plan_t p, int64_t tries);

/* --- Learned cost model of the autotuner ---------------------------------
 * The paper has no learned part (its direct solver is exact to rounding).
 * The autotuner's cost model is a small multilayer perceptron, trained on the
 * GPU by these kernels on measured solve times: x (n_in features) ->
 * tanh(W1 x + b1) -> tanh(W2 h1 + b2) -> y = w3 . h2 + b3 (both hidden
 * layers n_hidden wide); loss = mean squared error over the batch.
 * Parameters (FP32, contiguous): W1 [n_h][n_in], b1 [n_h], W2 [n_h][n_h],
 * b2 [n_h], w3 [n_h], b3 [1]; initialised from `seed` (uniform, scaled by
 * 1/sqrt(fan-in); biases 0).  x: DEVICE [batch][n_in] floats; t, y: DEVICE
 * [batch]; grad: DEVICE [num_params]; loss: DEVICE float (may be NULL).
 * Every reduction over the batch runs in a fixed order: results are
 * bit-reproducible.  helm_mlp_train runs `steps` full-batch Adam steps
 * (beta 0.9, 0.999, eps 1e-8, learning rate lr) and writes the final loss to
 * the HOST float *final_loss (may be NULL).  1 <= n_in, n_hidden <= 256.
 * Calls run on the legacy default stream and synchronise it. */
typedef struct helm_mlp* helm_mlp_t;
int helm_mlp_create(helm_mlp_t* out, int n_in, int n_hidden, uint64_t seed);
int helm_mlp_num_params(helm_mlp_t m);
int helm_mlp_get_params(helm_mlp_t m, float* host, int n);
int helm_mlp_set_params(helm_mlp_t m, const float* host, int n);
int helm_mlp_forward(helm_mlp_t m, const float* x, int64_t batch, float* y);
int helm_mlp_gradient(helm_mlp_t m, const float* x, const float* t, int64_t batch, float* grad, float* loss);
int helm_mlp_train(helm_mlp_t m, const float* x, const float* t, int64_t batch, int steps, float lr,
                   float* final_loss);
int helm_mlp_destroy(helm_mlp_t m);

/* --- Host-side plan helpers (no GPU needed) --------------------------------
 * Eigen-data of the 1D absorbing pencil K V = M V Lam (eq. EVP1a) with
 * V^T M V = I (eq. EVPcondA), K, M of eqs. matrixK / matrixM with n nodes,
 * spacing h and corner 1 - i w h; w = 0 gives the Neumann pencil (corner 1,
 * a Gamma_N axis), whose eigenpairs are the closed-form cosines.  Outputs,
 * caller-owned host arrays:
 *   lam    : 2n doubles, eigenvalues (re, im) interleaved;
 *   sigma  : 2n doubles, V[1,l]^2 (re, im) for the same eigenvector;
 *   parity : n int8, +1 if V[n,l] = V[1,l], -1 if V[n,l] = -V[1,l].
 * Order of the eigenpairs is unspecified.  Returns HELM_EINVAL for n < 2,
 * h <= 0 or w < 0, HELM_ENUMERIC if the eigenvalue iteration fails. */
int helm_abc_eigen(int64_t n, double h, double omega, double* lam, double* sigma,
                   int8_t* parity);

/* Mixed-radix factorisation the DFT kernels use for length n: writes up to
 * max_stages radices to `radices`, returns the number of stages (0 if n < 1).
 * Radices are 8, 4, 2 first, then odd primes. */
int helm_dft_factor(int64_t n, int32_t* radices, int32_t max_stages);

#ifdef __cplusplus
}
#endif

#endif /* HELM_H */

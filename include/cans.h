/*
 * cans.h -- C ABI of the B300 (sm_103a) pressure-Poisson library.
 *
 * The library solves the second-order, 7-point, staggered finite-difference Poisson equation
 *     L_h p = f                                                     (paper: Eq. poi)
 * by eigenfunction expansion: a forward real-to-real transform along x and along y chosen by the
 * boundary condition (periodic -> real DFT, Neumann-Neumann -> DCT-II, Dirichlet-Dirichlet ->
 * DST-II, the latter two through Makhoul's reordering around an FFT), one tridiagonal solve per
 * (x, y) mode along a possibly non-uniform z grid (Eq. poi_reduced, Gauss elimination), then the
 * inverse transforms (DFT^-1, DCT-III, DST-III).  Around it sit the fused divergence and projection
 * kernels of the fractional step (Eq. up / poi_ns and the correction that follows it).
 *
 * Conventions shared by every entry point
 *   - Fields are 3-D arrays of n[0] x n[1] x n[2] = Nx x Ny x Nz cells, x fastest:
 *     idx = i + Nx * (j + Ny * k).  No halos.  Values are IEEE double unless stated otherwise.
 *   - Device pointers are owned by the caller (any allocator, e.g. PyTorch).  The library never
 *     allocates device memory inside a solve; scratch comes from the caller's `workspace`, whose
 *     size cans_poisson_workspace_size() reports.  Plans own only small device tables.
 *   - Work is enqueued on the CUDA stream passed as `cuda_stream` (a cudaStream_t, NULL = legacy
 *     default stream) and is asynchronous unless stated otherwise.
 *   - Every function returns a cans_status; nothing is thrown across the ABI.  Argument errors are
 *     detected on the host before anything is enqueued.
 *   - Boundary conditions: the same type at both ends of a direction (CANS_BC_*).  x and y are
 *     uniform (spacing L/N); z is given by its cell widths dzf (Validation section: z may be
 *     non-uniform, x and y must be regular).  A periodic z must be uniform.
 *   - Singular problems (no Dirichlet direction) have solutions up to a constant: the library
 *     returns the one with zero cell-volume-weighted mean.
 */
#ifndef CANS_H
#define CANS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cans_plan_s* cans_plan_t;

/* Boundary conditions of a direction (cell-centred unknowns, walls half a cell beyond the first and
 * last cell): periodic, Neumann at both walls, Dirichlet at both walls, and the mixed pairs Neumann
 * at the low wall with Dirichlet at the high wall (ND) and the reverse (DN). */
enum cans_bc { CANS_BC_P = 0, CANS_BC_NN = 1, CANS_BC_DD = 2, CANS_BC_ND = 3, CANS_BC_DN = 4 };

/* CANS_FP64: every pass in IEEE double.
 * CANS_MIXED: transforms and most z-solves in float; the z-solves of the smallest-|mu| modes in
 * double; residual r = f - L_h p and the accumulated p in double-float (pairs of floats with
 * error-free sums and products, ~48 significant bits); max_sweeps refinement sweeps. */
enum cans_prec { CANS_FP64 = 0, CANS_MIXED = 1 };

enum cans_status {
  CANS_OK = 0,
  CANS_ERR_ARG = -1,           /* bad pointer, size, boundary condition, grid */
  CANS_ERR_UNSUPPORTED = -2,   /* valid problem this build does not handle (odd periodic N, ...) */
  CANS_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  CANS_ERR_WORKSPACE = -4,     /* workspace NULL or misaligned while one is required */
  CANS_ERR_INCOMPATIBLE = -5,  /* singular problem whose f has a non-zero weighted mean */
  CANS_ERR_NOT_CONVERGED = -6, /* refinement ended above opts.tol (only reported when synchronising) */
  CANS_ERR_TIMEOUT = -7        /* a bounded device-side wait gave up */
};

typedef struct {
  int prec;                  /* cans_prec */
  int max_sweeps;            /* CANS_MIXED: refinement sweeps after the first solve (0..8) */
  double tol;                /* CANS_MIXED: relative residual target checked when synchronising */
  double fp64_mode_fraction; /* CANS_MIXED: fraction of (x,y) modes solved in double along z */
  int autotune;              /* 1: time candidate tile shapes at plan time and keep the fastest (needs
                                temporary device scratch of about 12-16 bytes per point during planning;
                                results cached per device / shape / boundary conditions / precision,
                                and in the file named by CANS_AUTOTUNE_CACHE when set); 0: built-in */
  double shift;              /* Helmholtz shift sigma <= 0: the plan solves (L_h + sigma) p = f (the
                                implicit-diffusion equations of the Numerical method, Eq. up_id_2, are
                                of this form with sigma = -2 / (gamma_k nu dt)); 0 = Poisson.  Also the
                                default of cans_helmholtz_solve's per-call shift for the mixed path's
                                choice of double-precision modes. */
  int z_grid;                /* 0: unknowns at the cell centres of dzf (pressure, u, v).  1: unknowns on
                                the Nz - 1 interior z-faces of the dzf cells (a staggered w), with w = 0
                                on both walls (bc_z must be CANS_BC_DD); the solve then reads and writes
                                the first Nz - 1 planes of Nx*Ny*Nz arrays and leaves the top plane
                                (the wall face) alone. */
  int verify;                /* 1: every solve ends with ||f - L_h p||_2 / ||f||_2 evaluated on the
                                device (one more read of f and p, no host synchronisation) and a value
                                above tol recorded as CANS_ERR_NOT_CONVERGED in the plan's status word
                                (cans_plan_status); skipped for in-place FP64 solves (f == p), whose f is
                                gone.  0: only the checks that cost no extra pass (see cans_plan_status). */
} cans_opts;

/* Fill *opts with the defaults: FP64, 2 sweeps, tol 1e-12, fraction 0.01, autotune 0, shift 0,
 * z_grid 0, verify 0. */
void cans_opts_default(cans_opts* opts);

/*
 * Plan a solver for one grid and boundary-condition set (Eq. poi_reduced; host work only).
 *   n       : {Nx, Ny, Nz}, each >= 1.  x and y: N = 1, or N even with N/2 = 2^a 3^b, N <= 8192.
 *             z: Nz <= 512 for Neumann / Dirichlet z; a periodic z is uniform with Nz = 1 or
 *             Nz even, Nz/2 = 2^a 3^b, Nz <= 1024 (it is diagonalised by a real DFT as well).
 *   len_xy  : {Lx, Ly} > 0, domain lengths in x and y.
 *   bc      : {bc_x, bc_y, bc_z}, each a cans_bc.
 *   dzf     : host array of Nz positive cell widths along z, or NULL for Nz cells of width 1/Nz.
 *             Copied; the caller keeps ownership.
 *   opts    : NULL for the defaults.
 *   out     : receives the plan.  The plan uploads its coefficient tables to the current device.
 * Errors: CANS_ERR_ARG (bad n, bc, lengths, dzf non-positive or non-finite, periodic z not
 * uniform), CANS_ERR_UNSUPPORTED (sizes outside the list above), CANS_ERR_CUDA.
 * Along x and y the mixed pairs use the quarter-wave transforms (DCT-IV / DST-IV; output slot s =
 * mode s, eigenvalue -4 sin^2(pi (2s+1) / 4N)) of the shared-memory line engine.
 */
int cans_poisson_plan(const int n[3], const double len_xy[2], const int bc[3], const double* dzf,
                      const cans_opts* opts, cans_plan_t* out);

/* Bytes of device workspace one solve needs (0 for CANS_FP64, which works in p itself). */
int cans_poisson_workspace_size(cans_plan_t plan, size_t* bytes);

/*
 * Solve L_h p = f (Eq. poi) for one right-hand side ((L_h + opts.shift) p = f for a shifted plan).
 *   f, p       : device arrays of Nx*Ny*Nz doubles (z_grid 1: only the first Nz - 1 planes are used).  CANS_FP64 allows f == p (in place);
 *                CANS_MIXED needs f != p because f is re-read for the residual.
 *   workspace  : device buffer of at least cans_poisson_workspace_size() bytes, 256-byte aligned
 *                (may be NULL when that size is 0).  Contents on entry are ignored.
 *   cuda_stream: cudaStream_t to enqueue on.
 *   info       : NULL for a fully asynchronous call.  Otherwise a host array of max_sweeps+2
 *                doubles that receives ||f - L_h p_s||_2 / ||f||_2 after the first solve (s = 0)
 *                and after every sweep, and the call synchronises the stream; with info the call
 *                returns CANS_ERR_NOT_CONVERGED when the last value exceeds opts.tol (mixed only),
 *                and CANS_ERR_INCOMPATIBLE when a singular problem's f has a weighted mean above
 *                1e-10 of mean|f|; errors the device checks recorded in the plan's status word
 *                (cans_plan_status) are returned as well, and the word is cleared.  An in-place
 *                FP64 solve (f == p) has no f left to measure: its info values are NaN.
 * Singular problems always return the zero-mean solution of the compatible part of f.
 */
int cans_poisson_solve(cans_plan_t plan, const double* f, double* p, void* workspace, void* cuda_stream,
                       double* info);

/*
 * cans_helmholtz_solve -- (L_h + shift) p = f with this plan's grid, boundary conditions and precision
 * (Eq. up_id_2 written as a Helmholtz problem: the diagonal of every z system is shifted by `shift`
 * on top of the x-y eigenvalue term; the residual of the mixed path carries the shift).  shift <= 0
 * and finite, given per call (the plan's opts.shift is the default cans_poisson_solve uses).  A
 * nonzero shift makes every problem non-singular (no gauge).  Arguments, workspace, asynchrony and
 * errors as cans_poisson_solve; CANS_ERR_ARG for a positive or non-finite shift.
 */
int cans_helmholtz_solve(cans_plan_t plan, const double* f, double* p, double shift, void* workspace,
                         void* cuda_stream, double* info);

/*
 * cans_poisson_solve_divergence -- the pressure equation of the fractional step (Eq. poi_ns) with its
 * right-hand side formed inside the solve's first pass: f = scale / (gamma dt) D(u, v, w), D the
 * cell-centred divergence of a channel's face velocities (u on x-faces, v on y-faces, w on z-faces with
 * w = 0 on both walls: the layout of cans_rk3_step), dt read from dt_dev on the device (dt_dev NULL:
 * f = scale D(u, v, w)).  Channel plans only (x, y periodic, z Neumann, cell grid), otherwise
 * CANS_ERR_UNSUPPORTED.
 *   u, v, w : device, Nx*Ny*Nz doubles, read only.
 *   f       : device output that receives f, or NULL for FP64 plans and mixed plans with max_sweeps 0
 *             (the mixed refinement re-reads f, so it is required there: CANS_ERR_ARG).  Distinct from
 *             u, v, w and p.
 *   p, workspace, cuda_stream, info : as cans_poisson_solve (info needs f for the residual; with f
 *             NULL its values are NaN).
 * The result equals cans_poisson_solve applied to that f bit for bit (the divergence takes the same
 * roundings as the stand-alone divergence kernel of the RK3 step), without the separate pass that
 * would read u, v, w and write f and without the first x pass's read of f.  On B300 both forms are
 * bound by the divergence's FP64 operations, and cans_rk3_step keeps the separate kernel, which
 * measured faster.
 */
int cans_poisson_solve_divergence(cans_plan_t plan, const double* u, const double* v, const double* w, double scale,
                                  const double* dt_dev, double gamma, double* f, double* p, void* workspace,
                                  void* cuda_stream, double* info);

/* Release the plan and its device tables. */
/*
 * cans_poisson_solve_host -- the solve of cans_poisson_solve from and to host memory: the upload of f
 * (host -> f_dev) on copy_in_stream, the solve (f_dev -> p_dev, workspace as for cans_poisson_solve) on
 * compute_stream once the upload is done, and the download of p (p_dev -> p_host) on copy_out_stream
 * once the solve is done, ordered by two events the plan owns.  All asynchronous; p_host holds p when
 * copy_out_stream has passed the call.  Each stream waits only for what it consumes, so consecutive calls
 * with alternating device buffers (and separate host buffers) overlap one call's download and the next
 * call's upload with the solves; the solves themselves stay one at a time on compute_stream (a plan
 * serves one solve at a time).  The three streams may be the same stream.
 *   f_host, p_host : host arrays of Nx Ny Nz doubles (page-locked for the copies to be asynchronous).
 *   f_dev, p_dev   : caller-owned device arrays of Nx Ny Nz doubles, distinct (f_dev is overwritten by
 *                    the upload, p_dev by the solve); in place (f_dev == p_dev) is refused.
 * Errors: CANS_ERR_ARG for a NULL argument or f_dev == p_dev, CANS_ERR_WORKSPACE as cans_poisson_solve
 * (before anything is enqueued), CANS_ERR_CUDA when a copy, event or launch cannot be enqueued.
 */
int cans_poisson_solve_host(cans_plan_t plan, const double* f_host, double* p_host, double* f_dev, double* p_dev,
                            void* workspace, void* copy_in_stream, void* compute_stream, void* copy_out_stream);
int cans_plan_destroy(cans_plan_t plan);

/*
 * cans_plan_status -- the plan's device status word: the first error that any solve on this plan
 * (cans_poisson_solve, cans_helmholtz_solve, cans_poisson_solve_adjoint, the solves inside the RK3
 * steps and batches) detected on the device since the last call, written by the solve's last kernel
 * without a host synchronisation -- so it also covers solves replayed from a CUDA graph and solves
 * called without `info`.  The call synchronises the plan's device, stores the word in *status (or
 * CANS_OK) and clears it.  Checks, in this order:
 *   CANS_ERR_INCOMPATIBLE  singular problem whose f has a dzf-weighted mean above 1e-9 (FP64) or
 *                          1e-5 (mixed: the transforms round to float) of sqrt(Nx Ny sum_k dzf_k^2)
 *                          ||f||_2 -- the mean relative to the root-mean-square of f;
 *   CANS_ERR_NOT_CONVERGED a norm the solve accumulated (||f||^2, each sweep's residual) is not finite;
 *                          a refinement sweep (mixed, from the second on) that reduced the residual by
 *                          less than half while it was still above tol; with opts.verify = 1, a final
 *                          relative residual above tol;
 *   CANS_ERR_TIMEOUT       a bounded device-side wait of a persistent kernel gave up.
 * The return value is CANS_OK, or CANS_ERR_ARG / CANS_ERR_CUDA when the word could not be read.
 *
 * A plan serves one solve at a time: its device accumulators, its status word and (for
 * cans_helmholtz_solve, which sets the plan's shift for the duration of the call and restores it)
 * its shift are per plan, so solves that overlap on the GPU (several streams) or on the host
 * (several threads) must use separate plans.
 */
int cans_plan_status(cans_plan_t plan, int* status);

/*
 * cans_check_bounded_wait -- exercises the failure path of the bounded device-side waits (the
 * transaction-barrier waits of the TMA-fed z kernels) without a fault: one thread waits, with the same
 * bounded wait, on a shared-memory barrier whose phase either completes at once (complete != 0: the
 * thread's own arrival announces 0 bytes) or never completes (complete == 0: it announces 16 bytes that
 * no copy delivers; no copy is in flight).  A wait that runs out after `polls` polls (each a hardware
 * suspend of bounded length, later ones followed by a ~0.25 us sleep) records CANS_ERR_TIMEOUT in the
 * plan's status word, read with cans_plan_status.  polls: 1 .. 2^20.  Asynchronous on cuda_stream;
 * CANS_ERR_ARG for a NULL plan or polls out of range.
 */
int cans_check_bounded_wait(cans_plan_t plan, unsigned polls, int complete, void* cuda_stream);

/*
 * cans_fp64_fma_probe -- measures the GPU's FP64 fused multiply-add rate (the bound of the FP64 solve
 * path and of the RK3 momentum kernel): eight 256-thread blocks per SM, each thread running 8
 * independent FMA chains for `iters` steps and storing one double to out[thread].  Asynchronous on
 * cuda_stream; *flops receives the FP64 operations the launch performs (2 per FMA), to be divided by
 * the launch's CUDA-event time.  out: device, n_out >= SMs x 2048 doubles (else CANS_ERR_ARG).
 */
int cans_fp64_fma_probe(double* out, size_t n_out, unsigned iters, void* cuda_stream, size_t* flops);

/*
 * cans_poisson_solve_adjoint -- q = S^T g, the transpose (plain Euclidean inner product) of the solve
 * operator S: f -> p of cans_poisson_solve with this plan (the backward pass of a differentiable
 * solve; projection-adjoint reading R10).  With D = diag(dzf_k) along z, D A_z is symmetric, so S is
 * self-adjoint in the dzf-weighted inner product -- in the singular case S is the weighted
 * pseudo-inverse (compatible projection of f, zero weighted mean of p) -- and S^T = D S D^-1: the
 * library scales g by 1/dzf_k, solves with the plan's precision, and scales the result by dzf_k.
 *   g: device, Nx*Ny*Nz doubles, read only.  q: device output (may equal g).
 *   workspace: cans_poisson_adjoint_workspace_size() bytes, 256-byte aligned (the solve's workspace
 *   plus one FP64 field).
 * Asynchronous on cuda_stream, capturable; errors as cans_poisson_solve.
 */
int cans_poisson_adjoint_workspace_size(cans_plan_t plan, size_t* bytes);
int cans_poisson_solve_adjoint(cans_plan_t plan, const double* g, double* q, void* workspace, void* cuda_stream);

/* Static English text for a status code. */
const char* cans_status_string(int status);

/*
 * Single pass entry points (the steps of the solve, exposed for tests and for callers that want to
 * fuse their own work between them).  All operate on plan-shaped fields.
 *
 * cans_transform_xy: forward (dir = +1) or inverse (dir = -1) transforms along x then y (forward)
 * or y then x (inverse), in double, in place on `field`.  Forward output order per line: periodic
 * -> slot 0 = X_0, slot 1 = X_{N/2}, slots 2k, 2k+1 = Re X_k, Im X_k (1 <= k < N/2);
 * Neumann -> slot m = DCT-II_m; Dirichlet -> slot m = DST-II_m, all unnormalised (X_k = sum x_n
 * e^{-2 pi i k n/N}, DCT-II_m = 2 sum x_n cos(pi m (2n+1)/(2N)), DST-II_m = 2 sum x_n
 * sin(pi (m+1)(2n+1)/(2N))); Neumann-Dirichlet -> slot m = DCT-IV_m = 2 sum x_n
 * cos(pi (2m+1)(2n+1)/(4N)); Dirichlet-Neumann -> slot m = DST-IV_m (sin).  The inverse is the
 * exact inverse times Nx*Ny (so a forward-inverse round trip multiplies by Nx*Ny).
 */
int cans_transform_xy(cans_plan_t plan, double* field, int dir, void* cuda_stream);

/* cans_transform_xy_f32: the same transforms with the mixed-precision path's FP32 passes (mixed
 * plans only; CANS_ERR_ARG otherwise).  dir = +1: field (double, read only) -> work (float,
 * plan-shaped, same slot order as above).  dir = -1: work (float, overwritten) -> field (double),
 * unnormalised as above.  The FP32 rounding of every stage bounds the agreement with the double
 * transforms to a few float ulps times log2(Nx Ny). */
int cans_transform_xy_f32(cans_plan_t plan, double* field, float* work, int dir, void* cuda_stream);

/* cans_zsolve: in place on the transformed field, solve (A_z + mu_ij I) x = rhs along z for every
 * (i, j) slot, mu_ij = lam_x(i)/dx^2 + lam_y(j)/dy^2 (Eq. poi_reduced), in double. */
int cans_zsolve(cans_plan_t plan, double* field, void* cuda_stream);

/*
 * Per-pass timing with CUDA events on the solve's stream (the profiling hook a benchmark uses to
 * time one kernel inside the timed region).  enable = 1 clears earlier records and records a pair of
 * events around every pass launch of later solves on this plan; enable = 0 stops recording.
 * cans_plan_profile_read synchronises on the recorded events and returns, for pass kind `pass`
 * (a cans_pass), the summed milliseconds and the number of launches.
 */
enum cans_pass {
  CANS_PASS_XF = 0, /* forward x (FP64 -> working precision) */
  CANS_PASS_YF = 1, /* forward y */
  CANS_PASS_Z = 2,  /* tridiagonal z (all columns of the FP64 path; the float columns of the mixed path) */
  CANS_PASS_YI = 3, /* inverse y */
  CANS_PASS_XI = 4, /* inverse x of a first solve */
  CANS_PASS_XR = 5, /* forward x fused with the double-float residual (refinement sweep) */
  CANS_PASS_XU = 6, /* inverse x fused with the update of the iterate (refinement sweep) */
  CANS_PASS_RS = 7, /* residual stencil of a refinement sweep, when it runs as its own kernel (then
                       CANS_PASS_XR is the forward x transform of the residual alone) */
  CANS_PASS_ZD = 8, /* the mixed path's double-precision z columns (lowest |mu| and singular) */
  /* the fractional-step kernels around the solve (cans_rk3_step, cans_rk3_step_implicit,
   * cans_box_rk3_step, cans_project), recorded on the pressure plan */
  CANS_PASS_MOMENTUM = 9,    /* advection + diffusion + RK3 combination (Eq. up) */
  CANS_PASS_DIVERGENCE = 10, /* right-hand side of Eq. poi_ns */
  CANS_PASS_CORRECT = 11,    /* projection correction and pressure update (+ bulk-velocity sum) */
  CANS_PASS_CHKDT = 12,      /* stable time step: max reduction of the inverse time scale + dt */
  CANS_PASS_FORCING = 13,    /* constant-flow-rate shift of u */
  CANS_PASS_COUNT = 14
};
int cans_plan_profile(cans_plan_t plan, int enable);
int cans_plan_profile_read(cans_plan_t plan, int pass, double* total_ms, int* launches);

/*
 * Batched solves: many independent problems (each with its own plan: shapes, boundary conditions and
 * precisions may all differ) in one asynchronous call.  The batch fans the problems out over
 * `nstreams` internal streams (largest problems first, greedy balancing by point count; problems that
 * share a plan share a stream) that fork from and join back into the caller's stream with events, so
 * the call can be captured into one CUDA graph whose branches run concurrently.
 *   cans_batch_create : plans[count] stay owned by the caller and must outlive the batch.
 *   cans_batch_workspace_size : total workspace (sum of the problems' workspaces, 256-byte aligned).
 *   cans_batch_solve : f[i], p[i] device arrays of problem i (as in cans_poisson_solve); workspace of
 *                      the size above, 256-byte aligned; enqueued on cuda_stream.
 */
typedef struct cans_batch_s* cans_batch_t;
int cans_batch_create(int count, const cans_plan_t* plans, int nstreams, cans_batch_t* out);
int cans_batch_workspace_size(cans_batch_t batch, size_t* bytes);
int cans_batch_solve(cans_batch_t batch, const double* const* f, double* const* p, void* workspace,
                     void* cuda_stream);
int cans_batch_destroy(cans_batch_t batch);

/* cans_poisson_solve_batched -- the same in one call: count problems (plans[i], f[i], p[i] device
 * pointers as in cans_poisson_solve) solved concurrently on internal streams forked from cuda_stream.
 * workspace: cans_poisson_batched_workspace_size() bytes (the problems' workspaces, 256-byte aligned
 * each).  device_status (device, count ints, may be NULL) receives each problem's status, written
 * on the device after its solve: the checks of cans_plan_status for that problem alone --
 * CANS_ERR_INCOMPATIBLE (singular problem, f with a weighted mean), CANS_ERR_NOT_CONVERGED (a norm
 * the solve accumulated is not finite, a stalled refinement sweep, or, with the plan's opts.verify,
 * a final relative residual above its tol) -- else CANS_OK; when the call itself fails, every entry
 * receives the returned status.  The internal streams and events come from a per-device pool that the
 * first call on a device creates (make that first call outside any stream capture); later calls only
 * record events and enqueue work, so they can be captured into a CUDA graph.  Calls that overlap (two
 * host threads at once) share the pool's events and must be serialised by the caller. */
int cans_poisson_batched_workspace_size(int count, const cans_plan_t* plans, size_t* bytes);
int cans_poisson_solve_batched(int count, const cans_plan_t* plans, const double* const* f, double* const* p,
                               void* workspace, void* cuda_stream, int* device_status);

/*
 * Fractional-step pieces for a channel plan (bc = {CANS_BC_P, CANS_BC_P, CANS_BC_NN}: x and y
 * periodic, no-slip walls at z = 0 and z = Lz).  Velocities live on the faces of the staggered grid
 * (u on the x-face between cells i and i+1, v on the y-face between j and j+1, w on the z-face between
 * k and k+1, w[Nz-1] being the top wall, kept at 0), p at cell centres; all Nx*Ny*Nz doubles, x fastest.
 *
 * cans_rk3_step: one explicit low-storage RK3 step (Eq. up with alpha = {8/15, 5/12, 3/4},
 * beta = {0, -17/60, -5/12}, gamma = alpha + beta; Eq. poi_ns solved with the plan; correction
 * u = u* - gamma dt G Phi and p += Phi), in place on u, v, w, p.  Advection is the conservative
 * divergence of u (x) u with two-point averages, diffusion the 3-point Laplacian with no-slip ghosts.
 * dt = cfl * min(sqrt(3)/dti, 1.65 dl^2/nu) from the state at the start of the step (Eq. dt and the
 * chkdt listing, reduced on the device), or params->dt when > 0.  With params->forcing != 0, u is
 * shifted to bulk velocity params->ubulk after every substage (constant flow rate).  dt_dev: device
 * double that receives dt (NULL: kept in the workspace).  workspace: cans_rk3_workspace_size()
 * bytes, 256-byte aligned.  Asynchronous; no host synchronisation inside.
 */
typedef struct {
  double nu;    /* kinematic viscosity > 0 */
  double cfl;   /* Courant factor > 0 applied to the stability bound */
  double ubulk; /* bulk velocity kept by the forcing */
  double dt;    /* > 0: fixed time step; <= 0: computed */
  int forcing;  /* 1: constant-flow-rate forcing */
} cans_rk3_params;
int cans_rk3_workspace_size(cans_plan_t plan, size_t* bytes);
int cans_rk3_step(cans_plan_t plan, double* u, double* v, double* w, double* p, const cans_rk3_params* params,
                  double* dt_dev, void* workspace, void* cuda_stream);

/*
 * cans_rk3_step_implicit: one RK3 step with Crank-Nicolson viscous diffusion (the implicit variant of
 * the Numerical method): per substage u** of Eq. up_id (advection with alpha, beta; -G p and
 * nu L u^k with gamma), then Eq. up_id_2, u* - gamma nu dt/2 L u* = u** - gamma nu dt/2 L u^k, solved
 * per component as (L + sigma) u* = sigma (...), sigma = -2/(gamma nu dt), with the same direct
 * solver; then Eq. poi_ns_id, the correction, and p += Phi - gamma nu dt/2 L Phi.
 *   plan    : the pressure plan (x, y periodic, z Neumann), as for cans_rk3_step.
 *   uv_plan : x, y periodic, z Dirichlet, z_grid 0, same grid (the no-slip u and v).
 *   w_plan  : x, y periodic, z Dirichlet, z_grid 1 over the same dzf (w on the interior faces).
 *   params  : as cans_rk3_step, but params->dt must be > 0 (a fixed step: the shifts enter the
 *             solves as launch arguments).  Plans of either precision.
 *   workspace: cans_rk3_implicit_workspace_size() bytes, 256-byte aligned.
 * CANS_ERR_ARG for plans that do not describe the same grid or a non-positive dt.  Asynchronous.
 */
int cans_rk3_implicit_workspace_size(cans_plan_t plan, cans_plan_t uv_plan, cans_plan_t w_plan, size_t* bytes);
int cans_rk3_step_implicit(cans_plan_t plan, cans_plan_t uv_plan, cans_plan_t w_plan, double* u, double* v,
                           double* w, double* p, const cans_rk3_params* params, double* dt_dev, void* workspace,
                           void* cuda_stream);

/*
 * cans_box_rk3_step: the explicit RK3 step of cans_rk3_step in a box whose directions are periodic or
 * bounded by no-slip walls, read from the plan's boundary conditions: CANS_BC_P = periodic,
 * CANS_BC_NN = walls (the pressure is Neumann there).  It covers the flows the paper lists for its
 * solver: lid-driven cavity (NN, NN, NN with a lid), square duct (P, NN, NN with forcing), channel
 * (P, P, NN) and the periodic Taylor-Green box (P, P, P, uniform z).  A velocity component normal to
 * a walled direction lives on that direction's faces and stays 0 on its last stored face (the high
 * wall); tangential components take the no-slip ghost 2 U_wall - u, U_wall = lid for u at the top z
 * wall (lid != 0 needs z walls).  params as cans_rk3_step (forcing shifts u to ubulk).  Plans with
 * other boundary conditions, a shift or z_grid 1 return CANS_ERR_UNSUPPORTED.  workspace:
 * cans_box_rk3_workspace_size() bytes, 256-byte aligned.  Asynchronous.
 */
int cans_box_rk3_workspace_size(cans_plan_t plan, size_t* bytes);
int cans_box_rk3_step(cans_plan_t plan, double* u, double* v, double* w, double* p, const cans_rk3_params* params,
                      double lid, double* dt_dev, void* workspace, void* cuda_stream);

/*
 * cans_project: in place, u <- P u = u - G L^-1 D u, the discretely divergence-free part of a face field
 * (the correction of Eq. poi_ns with gamma dt cancelled).  cans_project_adjoint: u <- P^T u =
 * W_f P W_f^-1 u with W_f the face volumes (dzf for u and v faces, the centre distance for w faces),
 * which is the transpose because P is self-adjoint in the W_f inner product (D^T W_c = -W_f G).
 * Channel plans only.  workspace: cans_project_workspace_size() bytes, 256-byte aligned.
 */
int cans_project_workspace_size(cans_plan_t plan, size_t* bytes);
int cans_project(cans_plan_t plan, double* u, double* v, double* w, void* workspace, void* cuda_stream);
int cans_project_adjoint(cans_plan_t plan, double* u, double* v, double* w, void* workspace, void* cuda_stream);

/*
 * cans_poisson_solve_noalloc -- the solve for callers that cannot allocate device memory.
 * (An addition of this library; the paper has no counterpart.)
 *
 * Some callers cannot call cudaMalloc: a plugin inside a framework that owns the whole device
 * memory pool, code under a device-memory budget fixed at start-up, or a time-critical loop where
 * an allocation (which can wait for the device to go idle) is not acceptable.  Such a caller passes
 * f and p as for cans_poisson_solve but no workspace: the library uses a fixed scratch array of
 * cans_noalloc_scratch_bytes() bytes (48 MiB: mixed-precision problems up to 4,194,304 points) that
 * every GPU loading the library holds until the process exits.
 *   - Arguments and results are those of cans_poisson_solve (info as there).
 *   - A plan whose workspace exceeds the scratch size is rejected with CANS_ERR_WORKSPACE before any
 *     work is enqueued.  FP64 plans need no scratch and always fit.
 *   - The first call on each device looks up the scratch array's device address (with that device
 *     current); make that first call before any stream capture begins.  Under CUDA's lazy module
 *     loading (the default) that first call is also when the device commits the 48 MiB, so a caller
 *     whose memory pool will take the rest of the device makes it before the pool does.  A device
 *     reset in between is noticed and the address looked up again.
 *   - All calls share the one array: calls whose work overlaps on the GPU (several streams or threads
 *     at once) race on it and must be serialised by the caller.
 *   - Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.
 */
int cans_poisson_solve_noalloc(cans_plan_t plan, const double* f, double* p, void* cuda_stream, double* info);
size_t cans_noalloc_scratch_bytes(void);

/*
 * z-slab decomposition of one solve over several GPUs (the paper's Implementation section distributes
 * the grid over GPUs).  Rank r of P owns the z rows z0 .. z1-1 of the whole problem (all of x and y):
 * its x-y transforms are local (cans_transform_xy with a plan of the slab's shape), and only the
 * tridiagonal systems along z (Eq. poi_reduced) cross the slab boundaries:
 *   1. cans_zslab_eliminate: Thomas' forward sweep over the slab, each interior row expressed through
 *      the previous slab's last unknown and the slab's own last one; per (x, y) column 10 numbers go to
 *      `iface` (ncol x 10 doubles), and the slab's part of the singular (0,0) column to `col00` (nzs
 *      doubles, used when the problem is singular).
 *   2. the caller gathers every rank's `iface` (rank-major: P x ncol x 10 doubles) and `col00` (the
 *      slabs' parts in rank order: Nz doubles) on every rank (an all-gather; NCCL for GPUs).
 *   3. cans_zslab_finish: the reduced tridiagonal system of the P slabs' last rows (one per column, the
 *      system the warp-level partitioned solve forms across lanes), solved on every rank, then the
 *      slab's back substitution, the result times `scale` (1/(Nx Ny) undoes the transforms' factor);
 *      the singular column is solved whole from the gathered right-hand side, with the compatible
 *      projection and zero weighted mean of cans_poisson_solve.
 *   plan   : the whole problem's FP64 plan (Neumann, Dirichlet or mixed z walls; z_grid 0; a periodic
 *            or mixed-precision plan gives CANS_ERR_UNSUPPORTED).  Kept by the caller.
 *   field  : the slab's transformed field, Nx*Ny*(z1-z0) doubles, solved in place.
 *   workspace : cans_zslab_sizes() bytes, 256-byte aligned, kept between the two calls.
 * Asynchronous on cuda_stream.  All in FP64; P <= 64.
 */
typedef struct cans_zslab_s* cans_zslab_t;
int cans_zslab_create(cans_plan_t plan, int z0, int z1, cans_zslab_t* out);
int cans_zslab_sizes(cans_zslab_t slab, size_t* workspace_bytes, size_t* iface_doubles, size_t* col00_doubles);
int cans_zslab_eliminate(cans_zslab_t slab, double* field, double* iface, double* col00, void* workspace,
                         void* cuda_stream);
int cans_zslab_finish(cans_zslab_t slab, double* field, const double* iface_all, const double* col00_all, int nranks,
                      int rank, double scale, void* workspace, void* cuda_stream);
int cans_zslab_destroy(cans_zslab_t slab);

/* Host copies of the per-slot eigenvalue terms lam_x(i)/dx^2 (length Nx) and lam_y(j)/dy^2
 * (length Ny) the plan uses; either pointer may be NULL. */
int cans_plan_eigenvalues(cans_plan_t plan, double* mu_x, double* mu_y);

/*
 * cans_split_f64 -- the element-wise double/float conversions of the mixed-precision path, exposed
 * so that they can be checked on their own.  The mixed path represents extended-precision values as
 * pairs of floats (Section on the mixed-precision solve: FP32 transforms, residual and iterate in
 * higher precision); on this GPU the hardware double<->float conversions run at the FP64 rate, so
 * the library converts on the bit patterns instead.
 *   x     : device, n doubles (read only).
 *   rn    : device, n floats or NULL -- the nearest float to x[i], ties to even (bit-identical to
 *           a round-to-nearest hardware conversion, including zeros, subnormals, inf and NaN).
 *   hi,lo : device, n floats each or NULL -- x[i] = hi + lo with hi = rn and |x - hi - lo| <= 2^-46 |x|.
 *   back  : device, n doubles or NULL -- hi + lo evaluated in double (exact widening, one add).
 * Asynchronous on cuda_stream; CANS_ERR_ARG if x is NULL while n > 0.
 */
int cans_split_f64(const double* x, size_t n, float* rn, float* hi, float* lo, double* back, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* CANS_H */

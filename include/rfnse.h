/*
 * rfnse.h -- C ABI of the GB300 (sm_103a) tau-preconditioned GMRES time stepper for the Riesz
 * fractional nonlinear Schroedinger equation
 *
 *     i u_t + d^alpha u / d|x|^alpha + rho |u|^2 u = 0,   1 < alpha <= 2,  rho >= 0,
 *
 * on a box with homogeneous Dirichlet data (Chen, Yang, Zhang, "Sine-transform-based fast solvers
 * for Riesz fractional nonlinear Schroedinger equations with attractive nonlinearities",
 * arXiv 2410.03643; Sec. 2 for the discretisation, Sec. 3-4 for the solver).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Grid: axis a in {0 (x), 1 (y), 2 (z)} has n[a] interior points x_j = lo[a] + j h_a, j = 1..n[a],
 *   h_a = (hi[a] - lo[a]) / (n[a] + 1)  (Sec. 2.1).  n[a] + 1 must be a power of two in [4, 2048]:
 *   the fast sine transform (Sec. 4, "FST") is computed from a power-of-two FFT of length 2(n+1).
 * Layout: a grid function is N = n[0]*n[1]*n[2] complex numbers, interleaved FP64 (re, im), with
 *   x fastest: index = j_x + n[0]*(j_y + n[1]*j_z).  This is the column-stacking vec of Sec. 2.2.
 * Real block form: the paper's real vectors x = [z; y] (Sec. 3, u = y + i z) are stored as the
 *   complex vector y + i z; the real inner product of Sec. 3 is Re(a^H b).
 * Pointers: "device" arguments are CUDA device pointers of the current device; "host" arguments
 *   are ordinary host memory.  The caller owns every buffer it passes; the library owns only its
 *   context and workspace.  Buffers must not overlap unless stated.
 * Streams: all device work is issued on the stream given to rfnse_create (NULL = legacy default
 *   stream).  Entry points that return statistics to the host synchronise that stream.
 * Errors: every call returns an rfnse_status; no C++ exception crosses the ABI.  After an error,
 *   rfnse_last_error(ctx) describes it.  RFNSE_ENOCONV still writes the best iterate.
 * Debug mode: with the environment variable RFNSE_DEBUG=1 when rfnse_create runs, the context drives
 *   its loops from the host (as device_loop = 0) and checks every line pass after its launch: that its
 *   tiles cover the grid exactly, that it launched and ran without a CUDA error, and whether its
 *   outputs hold non-finite values.  The first pass that wrote one is named by rfnse_last_error when
 *   rfnse_run then returns RFNSE_ENUMERIC.  Every pass synchronises the stream, so this is slow.
 *   Profilers can group kernels by the NVTX ranges "rfnse step", "rfnse solve", "rfnse pass",
 *   "rfnse pass group", "rfnse autotune", "rfnse tape forward" and "rfnse reverse pass".
 */
#ifndef RFNSE_H
#define RFNSE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rfnse_ctx rfnse_ctx;

typedef enum {
  RFNSE_OK = 0,
  RFNSE_EINVAL = 1,   /* invalid argument (sizes, parameters, null pointers) */
  RFNSE_ENOMEM = 2,   /* device or pinned host allocation failed */
  RFNSE_ECUDA = 3,    /* a CUDA runtime call failed */
  RFNSE_ENOCONV = 4,  /* GMRES reached max_it before the tolerance (best iterate returned) */
  RFNSE_ENUMERIC = 5, /* a non-finite value appeared in a residual or Arnoldi norm */
  RFNSE_ETIMEOUT = 6  /* reserved: a bounded device-side wait gave up */
} rfnse_status;

typedef struct {
  int d;              /* space dimension, 1..3 */
  int n[3];           /* interior points per axis (n[a] + 1 a power of two, 4..2048); unused axes ignored */
  double lo[3], hi[3];/* box [lo, hi] per axis, hi > lo */
  double alpha;       /* Riesz order, 1 < alpha <= 2 */
  double rho;         /* nonlinearity strength, >= 0 */
  double dt;          /* time step, > 0 */
  double omega;       /* TBAN iteration parameter of the preconditioner, > 0 (the paper fixes 1) */
  int restart;        /* GMRES restart length m, 1..256 */
  int max_it;         /* maximum Arnoldi steps per linear solve (the paper uses 2000) */
  double tol;         /* stop when the relative residual ||f - R x|| / ||f|| < tol */
  int precision;      /* 0 = FP64 throughout; 1 = mixed: FP32 transforms inside an FGMRES inner
                         solve, FP64 Arnoldi/Givens, FP64 outer residual with iterative refinement */
  int first_step;     /* 0 = predictor only, 1 = predictor-corrector Crank-Nicolson first step */
  double inner_tol;   /* mixed form: relative tolerance of each inner solve (<= 0: 1e-6) */
  int max_outer;      /* mixed form: maximum refinement steps per solve (<= 0: 30) */
  int device_loop;    /* 1 = each solve is one CUDA graph whose conditional loops are decided on the
                         device (no host round trip per Arnoldi step); 0 = host-driven loop */
  int precond;        /* preconditioner of every GMRES solve:
                         0 = the sine-transform TBAN preconditioner F_tau (Sec. 4 eq. 'taupre');
                         1 = the circulant TBAN preconditioner F_C of Sec. 5 ("C-GMRES"): tau(T) replaced
                             by the Kronecker sum of Strang's circulant approximations of mu_a T_0;
                         2 = none (plain GMRES, the paper's "GMRES" column) */
} rfnse_params;

/* Fill p with defaults: d=1, n=255, box [-20,20], alpha=1.5, rho=2, dt=0.01, omega=1, restart=20,
   max_it=2000, tol=1e-10, precision=0, first_step=1, inner_tol=1e-6, max_outer=30, device_loop=1,
   precond=0. */
void rfnse_default_params(rfnse_params* p);

/* Create a solver context for the problem p (Sec. 2: grid, alpha, rho, dt) on the current CUDA
   device.  stream is a cudaStream_t (may be NULL).  Allocates the device workspace (Krylov basis
   of restart+1 vectors and about ten work vectors of N complex FP64 values; the mixed form adds
   restart+2 FP32 vectors) and computes, on the device, the coefficients c_k of eq. 'coefficients'
   (Sec. 2.1), the tau eigenvalues of eq. 'taudiagonal' (Sec. 4) per axis, and the circulant
   eigenvalues used for the Toeplitz products.  On success *out receives the context; on failure
   *out is NULL.  Errors: EINVAL, ENOMEM, ECUDA. */
int rfnse_create(const rfnse_params* p, void* stream, rfnse_ctx** out);

/* Release the context and its workspace (NULL is accepted). */
void rfnse_destroy(rfnse_ctx* ctx);

/* Text of the last error of ctx ("" if none); valid until the next call on ctx. */
const char* rfnse_last_error(const rfnse_ctx* ctx);

/* N = number of complex grid unknowns of the context. */
long long rfnse_size(const rfnse_ctx* ctx);

/* Load the time-stepping state.  step = 0: u_cur = u^0 (initial data on the grid, Sec. 2.1) and
   u_prev is ignored (may be NULL).  step >= 1: (u_prev, u_cur) = (u^{step-1}, u^{step}), e.g. to
   resume from rfnse_get_state.  on_device = 1: device pointers; 0: host pointers.  Each holds N
   complex FP64 values.  When the context has taken a step and step >= 1, the loaded vectors are
   compared bit by bit with the context's own (u^{n-1}, u^n): each one that comes back unchanged (a
   caller continuing its own run through host buffers) keeps what the context had computed for it
   (the mixed form's cached T u), so the next step costs no more than without the reload; the values
   used are the loaded ones in every case.  Synchronises the stream.  Errors: EINVAL, ECUDA. */
int rfnse_set_state(rfnse_ctx* ctx, const void* u_prev, const void* u_cur, int step, int on_device);

/* Read the state (u^{step-1}, u^{step}) and step.  u_prev is not written when step == 0.  Either
   pointer may be NULL.  Errors: EINVAL, ECUDA. */
int rfnse_get_state(rfnse_ctx* ctx, void* u_prev, void* u_cur, int* step, int on_device);

/* Advance nsteps time steps of the three-level linearly implicit scheme (Sec. 2.1 eq.
   'discretizedRFSE', Sec. 2.2 eq. 'discretizedRFSE2D'; the same Kronecker-sum form for d = 3).
   Step n >= 1 solves (D - T + iI) u^{n+1} = (T - D + iI) u^{n-1}, D = rho dt |u^n|^2, by GMRES
   with the sine-transform TBAN preconditioner (Sec. 4 eq. 'taupre'), zero initial guess (Sec. 5).
   The first step (step 0 -> 1) is the Crank-Nicolson step with mu -> mu/2, D -> rho (dt/2)|u~|^2,
   u~ = u^0 (predictor) and, if first_step = 1, u~ = (u^0 + u^1*)/2 (corrector).
   traj (may be NULL): nsteps * N complex FP64, receives u^{step+1} .. u^{step+nsteps}.
   iters (host, may be NULL): nsteps ints, Arnoldi steps per time step (inner steps for the mixed
   form; predictor + corrector for the first step).  relres (host, may be NULL): nsteps doubles,
   final relative residual estimate per step.  on_device refers to traj only.
   Errors: EINVAL, ECUDA, ENOCONV (the step is still taken), ENUMERIC. */
int rfnse_run(rfnse_ctx* ctx, int nsteps, void* traj, int* iters, double* relres, int on_device);

/* ---- batches of independent instances ----------------------------------------------------------- */

typedef struct rfnse_batch rfnse_batch;

/* Create `count` independent instances (params[i]: own grid, alpha, rho, dt, tolerance, precision),
   each a context with its own CUDA stream owned by the batch.  stream: the caller's cudaStream_t on
   which the batch step runs (may be NULL).  Errors: EINVAL, ENOMEM, ECUDA; on failure *out is NULL
   and rfnse_batch_last_error(NULL) describes the failure. */
int rfnse_batch_create(const rfnse_params* params, int count, void* stream, rfnse_batch** out);

/* Release the batch and its instances (NULL is accepted). */
void rfnse_batch_destroy(rfnse_batch* b);

/* Text of the last error of b (b = NULL: of the last failed rfnse_batch_create). */
const char* rfnse_batch_last_error(const rfnse_batch* b);

/* The context of instance i (owned by the batch: do not destroy it).  Use rfnse_set_state,
   rfnse_get_state and rfnse_get_coefficients on it to load and read each instance. */
rfnse_ctx* rfnse_batch_context(rfnse_batch* b, int i);

/* Advance every instance by nsteps time steps of the scheme (as rfnse_run).  While any instance is at
   its first step (or has a fresh state), the instances step one after another on their streams; once
   all are past it, one time step of the whole batch is a single CUDA graph launch: per instance its
   right-hand side, its solve with device-decided loops, the update of the mixed form's cached T u
   and the rotation of its history, then a gather of every instance's statistics.  iters, relres
   (host, may be NULL): nsteps * count values, step-major ([s * count + i]).  An instance that fails
   does not stop the others: every instance takes (or fails) the step, then the call returns the first
   failure, rfnse_batch_last_error naming its instance, without taking further steps.  Errors: EINVAL,
   ECUDA, ENOCONV (every step is still taken), ENUMERIC, ETIMEOUT. */
int rfnse_batch_run(rfnse_batch* b, int nsteps, int* iters, double* relres);

/* Lock-step mode of a batch (the paper has no counterpart: a scheduling choice).  The instances'
   solves advance together: one time step is one CUDA graph launch in which every Arnoldi step of all
   instances still iterating is one launch per line pass over a work list of every instance's
   (instance, tile) items, grouped by FFT length, plus one cooperative launch of modified Gram-Schmidt
   and Givens over all instances' vectors (blocks shared in proportion to their sizes, the grid-wide
   barrier after each sweep common to all); each refinement cycle's bookkeeping (back-substitution,
   solution update, residual product or recurrence, norm and refinement decision) is one launch for all
   instances.  Each instance keeps its own basis, Hessenberg matrix, rotations, tolerance and
   convergence; an instance that has finished its cycle or its solve skips its share of a launch, and
   the graph's loops run while any instance iterates.  Results equal those of the per-instance graphs
   up to the order of partial sums.  Available for batches of mixed-precision (precision 1) instances of
   one dimension with the sine-transform preconditioner (precond 0) and n[a] + 1 in 128..1024 on every
   axis, at most 1024 instances.  Such batches of at least 8 instances start in this mode (measured: 64
   uneven 2-D instances run faster lock-step, three 511^2 instances faster as concurrent per-instance
   graphs).  on = 0 switches to one CUDA graph branch per instance, on = 1 to lock-step.
   Errors: EINVAL (on = 1 for a batch that does not qualify). */
int rfnse_batch_set_lockstep(rfnse_batch* b, int on);

/* 1 when batch b runs its steady steps in lock-step mode, else 0. */
int rfnse_batch_lockstep(const rfnse_batch* b);

/* Autotune every instance (rfnse_autotune, reps timed launches per candidate; each distinct grid is
   timed once and its choices reused) and drop the batch's captured step graphs so that the next step
   captures them with the chosen geometries.  n_configs, n_changed (host, may be NULL): summed over the
   instances.  Errors: EINVAL, ECUDA. */
int rfnse_batch_autotune(rfnse_batch* b, int reps, int* n_configs, int* n_changed);

/* ---- reverse pass: gradients of a loss of u^N ---------------------------------------------------
 * The paper has no adjoint: these compute the exact derivative of its discrete scheme (eq.
 * 'discretizedCNLSMaxForm' of Sec. 2.1, eq. 'discretizedRFSE2DMaxForm' of Sec. 2.2, and the
 * first step as rfnse_run takes it).  For a real loss L the gradient of a complex grid function u is
 * g = dL/dRe(u) + i dL/dIm(u) (so dL = Re(g^H du)), stored like u.  Each step of the reverse pass is
 * one solve with the conjugate system matrix, M^{-H} g = conj(M^{-1} conj(g)) (M = D - T + iI is
 * complex symmetric), by the same tau-preconditioned GMRES, plus one Toeplitz product. */

/* Taped forward run: load u0 (step 0), take nsteps time steps exactly as rfnse_run, and keep u^0, the
   final pair and the pair (u^{kC-1}, u^{kC}) at every multiple kC < nsteps of C = every (library-owned
   device memory, about 2 nsteps / C + C + 8 grid vectors, kept until the context is destroyed and
   reused by the next taped run).  u0: N complex FP64; uN (may be NULL): receives u^nsteps; both host
   (on_device = 0) or device (1).  iters (host, may be NULL): nsteps counts.  On return the context
   holds the final state, as after rfnse_run.  Errors: EINVAL, ENOMEM, ECUDA, ENOCONV (the run and
   the tape are complete), ENUMERIC. */
int rfnse_tape_forward(rfnse_ctx* ctx, const void* u0, int nsteps, int every, void* uN, int* iters,
                       int on_device);

/* Reverse pass of the last taped run: from gN = dL/du^N, compute g0 = dL/du^0 and *grho = dL/drho
   (rho, dt, the grid and the first-step rule are the context's).  Each segment between checkpoints
   is recomputed once from its checkpoint, so the pass costs about one forward step and one
   conjugate solve per step.  gN, g0: N complex FP64, host (on_device = 0) or device (1), may not
   alias; grho, iters (host, may be NULL): iters receives the total Arnoldi steps of the conjugate
   solves.  On return the context holds the taped run's final state.  Errors: EINVAL (no taped run),
   ECUDA, ENOCONV (a solve stopped at max_it; the gradient is still written), ENUMERIC. */
int rfnse_tape_backward(rfnse_ctx* ctx, const void* gN, void* g0, double* grho, int* iters, int on_device);

/* lam = (D - T + iI)^{-H} g: one conjugate solve (mu_a / 2 when half = 1) with the context's
   tolerance and precision.  g, lam: N complex FP64 device values (may not alias); D: N FP64 device
   values; iters, relres: host, may be NULL.  Errors: EINVAL, ENOMEM, ECUDA, ENOCONV, ENUMERIC. */
int rfnse_adjoint_solve(rfnse_ctx* ctx, const double* D, const void* g, void* lam, int half, int* iters,
                        double* relres);

/* ---- building blocks (device pointers; used by the parity tests) ---------------------------- */

/* out = (D - T + iI) u, the system matrix of eq. 'equ3' (Sec. 2).  half = 1 uses mu_a/2 (first
   step).  u, out: N complex FP64 (may not alias); D: N FP64.  Errors: EINVAL, ECUDA. */
int rfnse_apply_A(rfnse_ctx* ctx, const void* u, void* out, const double* D, int half);

/* z = F~^{-1} v for F~ = (1/(2w)) [wI + tau(T_d)] (wI + D_d) of eq. 'taupre' (Sec. 4), in the
   complex storage of the real block vectors.  precision 0: FP64 transforms; 1: FP32 transforms
   (input and output still FP64).  v, z: N complex FP64 (may not alias); D: N FP64. */
int rfnse_apply_prec(rfnse_ctx* ctx, const void* v, void* z, const double* D, int half, int precision);

/* out = S in along one axis: the orthonormal DST-I [S]_{jk} = sqrt(2/(n+1)) sin(pi jk/(n+1))
   (Sec. 4, after eq. 'taudiagonal'), applied to every grid line of that axis.  precision 0/1 as
   above.  in, out: N complex FP64, may not alias. */
int rfnse_dst(rfnse_ctx* ctx, int axis, const void* in, void* out, int precision);

/* out = mu_a T_0 in along one axis: the symmetric Toeplitz matrix of eq. 'equ2' with first row
   c_0..c_{n-1} (Sec. 2.1), mu_a = dt / h_a^alpha (halved when half = 1), on every grid line of
   that axis.  FP64.  in, out: N complex FP64, may not alias. */
int rfnse_toeplitz(rfnse_ctx* ctx, int axis, const void* in, void* out, int half);

/* Solve (D - T + iI) u = b (eq. 'equ3') by right-preconditioned GMRES(restart) from u = 0 with the
   context's tolerance and precision (the real block form of Sec. 3, eq. 'positiveBlockForm').
   b, u: N complex FP64 (may not alias); D: N FP64; iters, relres: host, may be NULL.
   Errors: EINVAL, ECUDA, ENOCONV, ENUMERIC. */
int rfnse_solve(rfnse_ctx* ctx, const double* D, const void* b, void* u, int half, int* iters,
                double* relres);

/* Solve (D - T + iI) u = b like rfnse_solve, but by the TBAN iteration (Sec. 3, Method 3.1) in its
   stationary form F x^{k+1} = G x^k + f, i.e. x^{k+1} = x^k + F^{-1}(f - R x^k) from x^0 = 0, with the
   context's preconditioner as F: the sine-transform F~ (precond = 0; Method 3.1 with tau(T_d) in
   place of T_d inside F), the circulant F_C (1), or none (2, Richardson).  FP64 whatever the context's
   precision.  Stops when the relative residual < tol or after max_it iterations (*iters receives the
   count).  Arguments as rfnse_solve.  Errors: EINVAL, ECUDA, ENOCONV (u holds the last iterate),
   ENUMERIC. */
int rfnse_tban_solve(rfnse_ctx* ctx, const double* D, const void* b, void* u, int half, int* iters,
                     double* relres);

/* Copy the FCD coefficients c_0..c_{nmax-1} (nmax = largest n[a]) and the tau eigenvalues of T_0
   (not scaled by mu_a) of every axis, axis after axis (sum of n[a] values), to host memory.
   Either pointer may be NULL. */
int rfnse_get_coefficients(rfnse_ctx* ctx, double* c, double* lam);

/* z = F~^{-1} v exactly as rfnse_apply_prec with precision 0, but without a context and without
   allocating any device memory.  (The paper has no counterpart: this is a service for callers that
   cannot call cudaMalloc -- plug-ins whose host application owns the device-memory budget,
   real-time loops that must not allocate once running, programs whose memory comes from an
   allocator other than CUDA's.)  p describes the problem as for rfnse_create (restart, tolerance
   and precision are ignored); v, z: N complex FP64 device values (may not alias); D: N FP64 device
   values; stream: cudaStream_t (may be NULL).  Work is issued on stream and the call returns after
   synchronising it.
   Scratch: the coefficient, eigenvalue, twiddle and factor tables and the intermediate grid vectors live
   in one static device array of about 17 MB that every GPU loading this library holds until the
   process exits.  Limit: N = n[0]*n[1]*n[2] <= 262144 (e.g. 511 x 511), each n[a] + 1 a power of two
   in [4, 2048]; larger grids return RFNSE_EINVAL (use rfnse_create).  p is checked as rfnse_create
   checks it (d, grid, box, alpha, rho, dt, omega): what rfnse_create refuses is refused here.  Every
   call looks up the array's address on the current device (cudaGetSymbolAddress) and waits for the
   stream to finish (cudaStreamSynchronize) before returning.  All calls on a device share the array
   and each overwrites what it reads, so nothing needs clearing between calls, but calls whose work
   overlaps on the GPU race on it: serialise them.  A CUDA error already pending in the calling thread
   (from earlier work of the caller) is left in place for the caller to read, and the call then returns
   RFNSE_ECUDA without doing any work.  Errors: EINVAL, ECUDA. */
int rfnse_apply_prec_static(const rfnse_params* p, const void* v, void* z, const double* D, int half,
                            void* stream);

/* ---- autotuning of the line passes (the paper has no counterpart: a launch-geometry choice) ------ */

/* Choose the launch geometry of every line pass the context's solves run (the DST-I, tau-solve and
   Toeplitz passes of one axis each): the tile of B lines per block (a power of two; on strided axes B
   lines adjacent in x), the threads per line of the FFT (runtime-length FFT: one or two radix-4
   butterflies per thread; fixed-length FP32 FFT: L/8 threads, radix-8 butterflies) and the kernel
   variant (fixed-length FP32 passes: operands prefetched into registers or staged through shared
   memory), and the grid of the cooperative Arnoldi kernel (one to four blocks per SM, all co-resident;
   for N > 4096).  Each pass configuration runs once with its real operands (the context's work vectors,
   which it overwrites; the time-stepping state is untouched), then every candidate geometry is timed
   with CUDA events over `reps` launches (1..1000) on the context's stream and the fastest is kept in
   the context; later launches of that configuration use it, and the context's cached solve graphs are
   dropped so that the next solve captures them again.  Choices are shared between contexts of the same
   grid on the same device unless force = 1.  The arithmetic of a line does not depend on the
   geometry; only the order of the first MGS dot product's block partials does, so results agree with
   an untuned context to rounding (the Arnoldi kernel's grid changes the order of its partial sums).
   n_configs, n_changed (host, may be NULL): configurations tuned (passes, plus the Arnoldi grid) and
   how many got a geometry other than the default; est_speedup (host, may be NULL): summed default over
   summed chosen duration, one launch of each pass configuration.  Synchronises the stream.
   Errors: EINVAL, ECUDA. */
int rfnse_autotune(rfnse_ctx* ctx, int reps, int force, int* n_configs, int* n_changed, double* est_speedup);

/* Number of line-pass launches of ctx whose geometry came from rfnse_autotune's choices. */
long long rfnse_tuned_launches(const rfnse_ctx* ctx);

/* The launch of the Arnoldi kernel (modified Gram-Schmidt, Givens, convergence test; the paper's
   PGMRES orthogonalisation) used by ctx's solves: blocks > 0 runs the cooperative grid-wide kernel on
   that many blocks (all co-resident, a bounded grid-wide barrier after each sweep; 1 for N <= 4096);
   blocks = -8 or -16 runs it on one thread-block cluster of that many CTAs (hardware cluster barriers,
   reductions through distributed shared memory; for small grids, whose sweeps cost less than a
   grid-wide barrier); 0 restores the default.  rfnse_autotune sets it by timing.  The arithmetic is
   the same; only the order of the partial sums differs.  Errors: EINVAL (a grid that cannot be
   resident on this device). */
int rfnse_set_arnoldi_grid(rfnse_ctx* ctx, int blocks);

/* The current launch of ctx's Arnoldi kernel (as rfnse_set_arnoldi_grid takes it). */
int rfnse_arnoldi_grid(const rfnse_ctx* ctx);

/* ---- instrumentation -------------------------------------------------------------------------- */

/* Self-test of the bounded device-side waits (the grid-wide barrier of the cooperative Arnoldi kernel,
   which the paper does not have): one block waits at a barrier that nothing will release; the wait
   must give up after its poll limit, set its error flag and let the kernel finish, so the context
   stays usable.  *err (host) receives the flag (1 = the wait gave up, as it must); *ms (host, may be
   NULL) the kernel's duration.  stream: cudaStream_t (may be NULL); the call synchronises it.
   Allocates and frees a few bytes of device memory.  Errors: EINVAL, ENOMEM, ECUDA. */
int rfnse_selftest_bounded_wait(void* stream, int* err, double* ms);

/* Number of CUDA kernels this library has launched in the calling process (all contexts). */
long long rfnse_launch_count(void);

/* Test hook for the allocation-failure paths (the paper has no counterpart): after `after` more
   successful device or pinned-host allocations by contexts, batches and reverse-pass tapes of this
   process, every later one fails as if the GPU were out of memory, so the call that needed it returns
   RFNSE_ENOMEM (rfnse_create and rfnse_batch_create with *out = NULL and nothing leaked;
   rfnse_tape_forward with the context still usable).  after < 0 removes the limit (the default).  The
   limit is process-wide; no GPU memory is used up to provoke the failure.  Always RFNSE_OK. */
int rfnse_test_fail_allocations(long long after);

/* Measure the FMA throughput of the current device (flop/s, 2 flops per FMA) in FP64 (fp64 = 1) or
   FP32 (fp64 = 0) with independent FMA chains on 8 blocks of 256 threads per SM, timed with CUDA
   events on the legacy default stream.  Allocates and frees a small device buffer.  Used to confirm
   the FP64 arithmetic peak that bounds the FP64 line passes.  Errors: EINVAL, ENOMEM, ECUDA. */
int rfnse_probe_fma(int fp64, double* flops_per_s);

/* Time the cooperative Arnoldi kernel alone: one step of modified Gram-Schmidt against j + 1 basis
   vectors of n complex FP64 values, the Givens update and the convergence test (paper Sec. 5, the
   orthogonalisation inside PGMRES), on synthetic vectors, with the grid the solver uses for n.
   *us_per_step (host) receives the mean CUDA-event duration of `reps` launches after two untimed
   ones; *blocks_out (host, may be NULL) the grid size.  Allocates (j + 2) n complex values on the
   device and frees them before returning.  0 <= j <= 62, 1 <= n <= 2^28, 1 <= reps <= 1000.
   Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT (a bounded grid-barrier wait gave up). */
int rfnse_probe_arnoldi(long long n, int j, int reps, double* us_per_step, int* blocks_out);

/* Kernel classes of rfnse_profile: OR of the operations a line pass fuses, plus RFNSE_K_FP32 for
   passes computing in FP32 and RFNSE_K_DF for the Toeplitz passes of the mixed form's residual, which
   compute their FFTs in double-float (pairs of FP32 numbers, about 48 significant bits) when every
   axis has n + 1 in {128, 256, 512, 1024}.  RFNSE_K_INSCALE is ignored when matching.
   RFNSE_K_ARNOLDI alone selects the cooperative Arnoldi kernel (modified Gram-Schmidt against j + 1
   basis vectors, Givens, convergence test) as launched by the host-driven loops (device_loop = 0);
   its algorithmic figures per launch are 8 (j + 1) + 4 flops and 16 (j + 3) bytes per grid point. */
enum {
  RFNSE_K_INSCALE = 1,   /* Arnoldi normalisation v = w / h folded into the load */
  RFNSE_K_DST = 2,       /* DST-I along the axis */
  RFNSE_K_LAM = 4,       /* divide by (omega + i Lambda) and DST-I again (last axis) */
  RFNSE_K_DSCALE = 8,    /* (omega I + D) sub-solve of the preconditioner */
  RFNSE_K_TOEP_X = 16,   /* Toeplitz product along x with the diagonal and block coupling */
  RFNSE_K_TOEP_ACC = 32, /* Toeplitz product along y or z, accumulated */
  RFNSE_K_FP32 = 256,
  RFNSE_K_DF = 1024,
  RFNSE_K_ARNOLDI = 2048
};

/* Start timing every launch of kernel class `kind` (0 = off) issued by ctx: a CUDA event pair is
   recorded around each such launch on the context's stream.  Resets the accumulated figures. */
int rfnse_profile(rfnse_ctx* ctx, int kind);

/* Synchronise the context's stream and report, since rfnse_profile: the number of launches of the
   class, their summed device time in ms, and their summed algorithmic flops (5 L log2 L per complex
   FFT of length L per grid line) and bytes (each operand read once, each result written once).
   Any pointer may be NULL. */
int rfnse_profile_read(rfnse_ctx* ctx, int* launches, double* ms, double* flops, double* bytes);

#ifdef __cplusplus
}
#endif

#endif /* RFNSE_H */

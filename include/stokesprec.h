/*
 * stokesprec.h -- C ABI of the GB300 library for the hot path of
 * Stokes-preconditioned Newton (Tuckerman, Langham & Willis, arXiv:1804.05087).
 *
 * The method (Sec. 2) looks for roots of G(U) = B_dt(U) - U, where one
 * Backwards-Euler/Forwards-Euler step B_dt = (I - dt L)^-1 (I + dt N) is taken
 * with a very large dt (Eqs. befe, mycalc, Gstokes). Newton's method solves
 * G_U du = G(U) by matrix-free GMRES (Eqs. linear, biglin, Kspace), so the hot
 * path is the action of G_U: one linearised BEFE step (Eq. finitediff and the
 * linearisation N -> N_U that precedes it).
 *
 * Geometry: plane Couette flow, Fourier in x and z, Chebyshev in y (Sec. 3.2).
 * The state is the deviation u = U - y e_x from laminar flow (Sec. 3.1).
 *
 * ---------------------------------------------------------------------------
 * Conventions shared by every entry point
 *
 * State layout (device memory, owned by the caller): interleaved complex
 *   double [3][MX][MZ][NY] per state, component (u, v, w) slowest, then the
 *   x-wavenumber index in FFT order (0..Kx, -Kx..-1), then iz = 0..Kz, then
 *   the Chebyshev degree n = 0..N fastest. Kx = (Nx-1)/3, Kz = (Nz-1)/3 (2/3
 *   rule), MX = 2Kx+1, MZ = Kz+1, NY = Ny = N+1. A state holds
 *   sp_state_len() doubles (2 per complex coefficient). Batches of states are
 *   stored back to back.
 * Real fields: the kz = 0 plane is stored for both ix and -ix. Every map
 *   reads its input through the projection onto Hermitian-consistent states
 *   (mean of an entry and the conjugate of its mirror) and writes an exactly
 *   Hermitian-consistent output.
 * Inner product (norms, GMRES, adjoint): <a,b> = sum over stored coefficients
 *   of w(iz) Re(conj(a) b), with w(0) = 1 and w(iz>0) = 2.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream). Calls
 *   are asynchronous on it unless stated otherwise; pointers must stay valid
 *   until the work completes.
 * Errors: every call returns an sp_status; sp_last_error() gives a message.
 *   No call traps or aborts the process. Invalid arguments return SP_EINVAL
 *   before any work is enqueued.
 * Threads: a context may be used by one host thread at a time.
 */
#ifndef STOKESPREC_H
#define STOKESPREC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sp_ctx sp_ctx;

typedef enum {
  SP_OK = 0,
  SP_EINVAL = 1,    /* bad argument or unsupported size                      */
  SP_ENOMEM = 2,    /* device allocation at create time failed               */
  SP_ECUDA = 3,     /* a CUDA runtime call failed (message in last_error)    */
  SP_ENOTCONV = 4,  /* Newton stopped before |G| < tol                       */
  SP_ETIMEOUT = 5,  /* a bounded device wait expired                         */
  SP_ENAN = 6       /* non-finite value detected                             */
} sp_status;

typedef enum {
  SP_FP64 = 0,      /* every stage in double precision                       */
  SP_MIXED = 1      /* transforms and products in float, solve/residual in double */
} sp_prec;

typedef struct {
  int nx, ny, nz;   /* physical grid: Nx x Ny x Nz, Nx and Nz even, Ny odd    */
  double lx, lz;    /* box lengths in x and z (walls at y = -1, +1)          */
  double re;        /* Reynolds number, nu = 1/re                            */
  double dt;        /* the single BEFE step dt = T (Eq. Gstokes)             */
  int prec;         /* sp_prec: precision of the tangent (sp_jvp, sp_vjp)    */
  int max_batch;    /* largest n_dir a single internal pass handles (>= 1);
                       larger batches are processed in passes of this size   */
  int lam_adv;      /* 0: the Stokes step (Eq. befe). 1: laminar advection in L
                       (Sec. 3.6, the closing proposal): M u = y du/dx + v e_x
                       moves from N into the implicit operator, so one step solves
                       (1/dt - nu lap + M) u' + grad p = u/dt + N(u) + M u.
                       Same fixed points; per mode the solve becomes complex and
                       couples both Chebyshev parities. With 1, sp_vjp,
                       sp_vjp_euclid and the gradient hookstep return SP_EINVAL
                       (they are defined for the Stokes step); the members of a
                       group must all have the same value. */
} sp_config;

/* ---- lifetime ----------------------------------------------------------- */

/* Build a context: checks the sizes, precomputes the transform tables and the
 * per-mode Stokes solution operators (Sec. 3.2: exact direct inversions per
 * Fourier mode) and allocates the device workspaces. Uses the current CUDA
 * device. Synchronous. On failure *out is NULL. */
sp_status sp_create(const sp_config* cfg, sp_ctx** out);
sp_status sp_destroy(sp_ctx* ctx);
/* Message of the last failure on ctx; with ctx == NULL, the message of the last
 * failed sp_create on the calling thread. Never NULL. */
const char* sp_last_error(const sp_ctx* ctx);

/* Number of doubles in one state (2 * 3 * MX * MZ * NY). */
size_t sp_state_len(const sp_ctx* ctx);
/* Retained ranges: kx_max = Kx, kz_max = Kz, ny = N + 1. */
sp_status sp_dims(const sp_ctx* ctx, int* kx_max, int* kz_max, int* ny);

/* ---- pipe flow in a moving frame (Sec. 2 traveling waves, Sec. 3.1) --------
 *
 * Pipe of radius 1, deviation u = U - (1 - r^2) e_z from Hagen-Poiseuille flow
 * (centreline-velocity scale: Re = U_c R / nu, the paper's bulk x diameter number,
 * Sec. 3.1), frame moving with speed c along the axis: N_c(u) = U_tot x Omega_tot
 * + c du/dz (Sec. 2: C dU/dx added to N for traveling waves).
 * Fourier in theta (m = sym m', m' = 0..mt) and z (k = alpha kz, |kz| <= kz);
 * radial points r_j = cos(pi j / (2 nr - 1)), j = 0..nr-1 (the wall j = 0, the
 * axis excluded), 9-point finite differences with parity ghost points
 * (Sec. 3.2: Openpipeflow discretises r by finite differences). Per mode the
 * Stokes problem: momentum at interior points, no-slip, pressure Poisson at
 * interior points, continuity at the wall.
 * State layout: complex double [3][2kz+1][mt+1][nr] (u_r, u_theta, u_z; kz in
 * FFT order; m' = 0..mt; radial index), then ONE more complex value (c, 0)
 * holding the speed. sp_state_len() counts it. The inner product adds c_a c_b.
 * sp_step returns (B(u;c) - u, 0); sp_jvp and sp_jvp_fd return
 * (G_u du + G_c dc, <d/dz U, du>): the tangent plus the phase condition that
 * fixes the axial position of the wave. sp_vjp and sp_jvp_static are not
 * available for the pipe (SP_EINVAL). */
typedef struct {
  int nr;           /* radial points                                         */
  int mt, kz;       /* stored modes: 0 <= m' <= mt, |kz| <= kz               */
  int ntheta, nz;   /* physical grid over theta in [0, 2 pi/sym) and z      */
  int sym;          /* rotational symmetry (m = sym m')                      */
  double alpha;     /* axial wavenumber, box length 2 pi / alpha             */
  double re, dt;
  int prec, max_batch;
} sp_pipe_config;

sp_status sp_pipe_create(const sp_pipe_config* cfg, sp_ctx** out);

/* Seeded pipe state: u_z streaks a_m (1 - r^2) r^m (k = 0, m' = 1..3) scaled to
 * norm amp, plus a divergence-free k != 0 part from poloidal potentials
 * phi = (1 - r^2)^3 r^m sum_n pol_n r^(2n) (u = curl curl (phi e_z)) scaled to
 * norm frac * amp, and the speed c0. streak: host double [mt+1]; pol: host
 * complex double [2kz+1][mt+1][npoly], npoly <= 32. Synchronous. */
sp_status sp_pipe_seed_state(sp_ctx* ctx, const double* streak, const double* pol, int npoly,
                             double amp, double frac, double c0, double* U, void* stream);

/* ---- seeded initial states ---------------------------------------------- */

/* Build a divergence-free, no-slip perturbation from random shape series.
 * ra, rb, rc: device complex double [MX][MZ][NY] (the layout above without
 * the component axis): per mode v = (1-y^2)^2 sum ra_n T_n and wall-normal
 * vorticity eta = (1-y^2) sum rb_n T_n, then u = i(kx Dv - kz eta)/k^2,
 * w = i(kz Dv + kx eta)/k^2; mode (0,0): u = (1-y^2) sum rb_n T_n,
 * w = (1-y^2) sum rc_n T_n, v = 0. The result is scaled to norm `amp`.
 * ra must vanish for n > N-4 and rb, rc for n > N-2. Synchronous. */
sp_status sp_seed_state(sp_ctx* ctx, const double* ra, const double* rb,
                        const double* rc, double amp, double* U, void* stream);

/* ---- the BEFE step and its derivatives ---------------------------------- */

/* G = B_dt(U) - U, one BEFE step (Eqs. befe, Gstokes), always in FP64:
 * N(U) = (U + y e_x) x (curl U - e_z) pseudospectrally on the Nx x Ny x Nz grid
 * (2/3-dealiased in x and z), then per Fourier mode the Chebyshev-tau Stokes
 * problem (1/dt - nu lap) u_new + grad p = U/dt + N(U), div u_new = 0 for every
 * Chebyshev coefficient, u_new(+-1) = 0; G = u_new - U. U and G: one state
 * each (may not alias). */
sp_status sp_step(sp_ctx* ctx, const double* U, double* G, void* stream);

/* Set the linearisation point: stores U, the total fields (U + y e_x,
 * curl U - e_z) on the grid for sp_jvp/sp_vjp, and G(U) for sp_jvp_fd. */
sp_status sp_set_base(sp_ctx* ctx, const double* U, void* stream);

/* Jdu = G_U du for n_dir directions (batched, back to back): the linearised
 * step with N -> N_U = U_tot x omega(du) + du x Omega_tot and homogeneous
 * boundary data (Sec. 2). Precision: cfg.prec. Needs sp_set_base. */
sp_status sp_jvp(sp_ctx* ctx, const double* du, double* Jdu, int n_dir, void* stream);

/* sp_jvp for directions in HOST memory: du and Jdu are host arrays of n_dir
 * states (page-locked memory lets the copies overlap; pageable memory works
 * but serialises them). The directions are processed in chunks of `chunk`
 * (<= 0: n_dir/4 rounded up, at most cfg.max_batch): chunk i is copied in on
 * an internal stream while chunk i-1 is computed on `stream` and chunk i-2 is
 * copied out on another internal stream (two device slots held by the
 * context). Asynchronous: Jdu is complete once `stream` has reached this point
 * (for instance after cudaStreamSynchronize(stream)); du and Jdu must stay
 * valid until then. Same results as sp_jvp. */
sp_status sp_jvp_host(sp_ctx* ctx, const double* du, double* Jdu, int n_dir, int chunk, void* stream);

/* JTr = G_U^* r for n_dir vectors: the adjoint of sp_jvp in the inner product
 * above (the transpose of every stage, in reverse). Precision: cfg.prec. */
sp_status sp_vjp(sp_ctx* ctx, const double* r, double* JTr, int n_dir, void* stream);

/* The same adjoint in the plain Euclidean inner product of the stored real
 * and imaginary parts (sum Re(conj(a) b), no w(iz) weights): JTg = G_U^T g.
 * This is the vector-Jacobian product that reverse-mode automatic
 * differentiation of complex tensors expects (torch.autograd). */
sp_status sp_vjp_euclid(sp_ctx* ctx, const double* g, double* JTg, int n_dir, void* stream);

/* Finite-difference action [G(U + eps du) - G(U)]/eps (Eq. finitediff) for
 * n_dir directions, FP64, with eps = 1e-7 (1 + |U|)/|du| per direction.
 * Needs sp_set_base. Synchronous (reads the norms on the host). */
sp_status sp_jvp_fd(sp_ctx* ctx, const double* du, double* Jdu, int n_dir, void* stream);

/* ---- the multi-step operator G^int (Eq. Gint) ----------------------------
 *
 * G^int_T = (B_dt)^n - I with T = n dt: n BEFE steps of the context's dt, the
 * time-integration operator the paper compares Stokes preconditioning with
 * (Sec. 2, Sec. 3.3). n > 1 needs a plane Couette context; n = 1 is the
 * single step of any context. */

/* G = B^n(U) - U, FP64. U and G: one state each (may not alias). */
sp_status sp_step_n(sp_ctx* ctx, const double* U, double* G, int n, void* stream);
/* Linearisation point of G^int: stores the trajectory U_k = B^k(U), k < n (n
 * states of device memory held by the context), U, and G^int(U) for
 * sp_jvp_fd. n = 1 is sp_set_base. Calling sp_set_base afterwards returns to
 * the single step. */
sp_status sp_set_base_n(sp_ctx* ctx, const double* U, int n, void* stream);
/* Jdu = G^int_U du = (prod_k (I + G_{U_k})) du - du for n_dir directions: the
 * chain rule along the stored trajectory, one tangent step (as sp_jvp, in
 * cfg.prec) per k, the total fields of U_k recomputed from the stored state.
 * After sp_set_base_n; sp_jvp_fd then differentiates G^int as well. */
sp_status sp_jvp_n(sp_ctx* ctx, const double* du, double* Jdu, int n_dir, void* stream);

/* ---- tangent step without allocation ------------------------------------ */

/* Jdu = G_U du for ONE direction, exactly as sp_jvp computes it, but with the
 * intermediate fields kept in a fixed 8 MiB array that the library holds on
 * every device it runs on, so this call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine). The paper has no counterpart: it
 * is an interface for callers that cannot allocate device memory when they
 * need a Jacobian action, for instance a process whose GPU memory is already
 * committed to its own pool allocator, or a latency-critical loop where
 * cudaMalloc/cudaFree would synchronise the device.
 * Limit: 9 Ny MX MZ complex values of the transform type (16 bytes in FP64,
 * 8 in mixed) must fit in 8 MiB (48 x 65 x 48 FP64 needs 4.6 MB; larger grids
 * return SP_EINVAL). The context, its plan and the base (sp_set_base) are set
 * up as for sp_jvp.
 * The first call on each device looks up the array's device address; make
 * that first call before any stream capture. All calls share the one array:
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it and must be serialised by the caller. Every intermediate value
 * is written before it is read, so nothing has to be cleared between calls. */
sp_status sp_jvp_static(sp_ctx* ctx, const double* du, double* Jdu, void* stream);

/* ---- vector operations in the inner product above ---------------------- */

/* out[i] = <a_i, b_i> for i < n (states back to back), FP64. Synchronous. */
sp_status sp_inner(sp_ctx* ctx, const double* a, const double* b, int n,
                   double* out_host, void* stream);

/* ---- tracing ------------------------------------------------------------- */

/* Per-kernel timing. While enabled, every kernel the library launches is
 * bracketed by two CUDA events recorded on the call's stream, accumulated per
 * kernel family (the stage indices below). Enabling resets the totals. */
enum { SP_STAGE_YINV = 0,   /* k_yinv of the tangent / adjoint         */
       SP_STAGE_XZ = 1,     /* k_xz: x/z FFTs and the tangent product  */
       SP_STAGE_SOLVE = 2,  /* k_solve of the tangent / adjoint        */
       SP_STAGE_STEP = 3,   /* every kernel of sp_step and sp_set_base */
       SP_STAGE_VEC = 4,    /* vector kernels (norms, axpy, seeding)   */
       SP_STAGE_RHS = 5,    /* k_rhs of the batched tangent's O(N) solve
                               (Chebyshev coefficients + right-hand side;
                               k_chain counts as SP_STAGE_SOLVE)         */
       SP_NSTAGE = 6 };
sp_status sp_trace_enable(sp_ctx* ctx, int on);
/* Waits for the recorded events, then writes the accumulated milliseconds and
 * launch counts of the n (<= SP_NSTAGE) first stages. Host arrays. */
sp_status sp_trace_read(sp_ctx* ctx, double* ms, long long* launches, int n);

/* ---- FP64 rate probe -------------------------------------------------------- */

/* The paper has no counterpart: a measurement of the device's FP64 fused
 * multiply-add rate, the denominator of the roofline of the FP64-bound kernels
 * (the per-mode solve, the FP64 transforms). Launches blocks x 256 threads on
 * `stream`, each running 8 independent chains of `iters` FMAs: 4096 x blocks x
 * iters flops per launch. The caller times it with events on the same stream.
 * out: device buffer of blocks x 256 doubles (written, so the chains are not
 * optimised away). iters > 0, a multiple of 4. Asynchronous. SP_EINVAL on bad
 * arguments, SP_ECUDA if the launch fails. */
sp_status sp_probe_fp64_fma(double* out, int blocks, int iters, void* stream);

/* ---- tile autotuner -------------------------------------------------------- */

/* The per-mode solve kernel (the dominant kernel of the tangent) can run with
 * several tile shapes: solved modes per block x threads per block. Every shape
 * computes each mode with the same arithmetic, so results are identical bit for
 * bit; only the speed differs with the grid and the batch. sp_autotune times
 * every shape that fits in shared memory on this context's own workspaces
 * (zeroed scratch, so the context's data is untouched): n_dir directions in the
 * tangent's precision, and one direction in FP64 (the step of sp_step,
 * sp_set_base and the Newton residual). It keeps the fastest of each for every
 * later call on this context. Without it the context uses shape 0.
 * Synchronous; allocates and frees its scratch (2 n_dir states). */
#define SP_TUNE_MAX 8
typedef struct {
  int n_shapes;                  /* shapes in the table                             */
  int tile[SP_TUNE_MAX];         /* solved modes per block                          */
  int threads[SP_TUNE_MAX];      /* threads per block                               */
  double ms_tangent[SP_TUNE_MAX];/* mean launch time, n_dir directions (< 0: does not fit) */
  double ms_step[SP_TUNE_MAX];   /* mean launch time, one FP64 direction (< 0: does not fit) */
  int chosen_tangent, chosen_step;
} sp_tune_report;
sp_status sp_autotune(sp_ctx* ctx, int n_dir, sp_tune_report* report, void* stream);
/* Pin the tile shapes (indices into the report's table; -1 keeps the current
 * one), e.g. to reuse an earlier sp_autotune result without timing again.
 * SP_EINVAL for an index out of range; a shape that does not fit in shared
 * memory makes the later call fail with SP_ECUDA. */
sp_status sp_set_solve_shape(sp_ctx* ctx, int tangent_shape, int step_shape);

/* Choose the tensor-core forms of the mixed tangent's Chebyshev transforms
 * (Sec. 3.2; tcgen05 MMAs in split TF32, FP32 accumulation): inverse = 1 puts
 * the inverse transform and curl (values at the Gauss-Lobatto points) on the
 * tensor cores, forward = 1 the forward transform of the batched O(N) solve's
 * right-hand sides. They apply to plane Couette contexts in mixed precision
 * with 41 <= Ny <= 72 (elsewhere the CUDA-core kernels run regardless).
 * Defaults: inverse 1, forward 0 (the forward one measured slower than its
 * CUDA-core counterpart). The results agree with the CUDA-core kernels to
 * float accuracy, not bit for bit. SP_EINVAL for a null context. */
sp_status sp_set_tensor_cores(sp_ctx* ctx, int inverse, int forward);

/* ---- Newton-GMRES-hookstep ------------------------------------------------ */

typedef struct {
  int max_newton;     /* Newton iterations cap                               */
  int max_krylov;     /* GMRES dimension cap K (no restarts)                 */
  double tol;         /* stop when |G(U)| < tol                              */
  double eta;         /* GMRES stops at residual <= eta |G(U)| (Sec. 3.6)    */
  double delta0;      /* initial trust radius (<= 0: 0.1 max(|U|, 1))        */
  int use_fd;         /* 1: Jacobian actions by Eq. finitediff, 0: tangent   */
  int use_gradient;   /* 1: add the steepest-descent direction J^* G(U) (one
                         sp_vjp and one more action) to the Krylov space of the
                         hookstep, so the trust-region step also spans the
                         Cauchy (dogleg) direction                             */
  int int_steps;      /* <= 1: G = G^Stokes = B_dt - I (one step, Eq. Gstokes);
                         n > 1: G = G^int = (B_dt)^n - I (n steps of cfg.dt,
                         Eq. Gint; plane Couette, use_gradient = 0)            */
  int krylov;         /* 0: GMRES with hookstep (default); 1: BiCGSTAB(ell);
                         2: IDR(s) with biorthogonalised bases (Sec. 3.6: no
                         K^2 term; s seeded shadow vectors). 1 and 2: at most
                         max_krylov actions per Newton step, trust region along
                         the computed direction (one more action for its
                         predicted residual); need int_steps <= 1,
                         use_gradient = 0. Other values: SP_EINVAL.            */
  int ell;            /* BiCGSTAB(ell): ell (1..8, <= 0: 2); IDR(s): s (1..8,
                         <= 0: 4)                                              */
  int use_graphs;     /* 1: each Arnoldi step (action + orthogonalisation) is
                         captured once as a CUDA graph on a stream of the
                         context and replayed (tangent actions with int_steps
                         <= 1 and tracing off; otherwise plain launches). The
                         graphs stay with the context.                         */
} sp_newton_opts;

typedef struct {
  int newton_iters;   /* Newton steps taken                                   */
  int total_jvps;     /* Jacobian actions (GMRES iterations) over all steps  */
  int total_steps;    /* BEFE steps of G itself (residuals, hookstep trials) */
  double norm_F;      /* final |G(U)|                                        */
  double norm_F0;     /* initial |G(U)|                                      */
  double t_action_ms; /* time in Jacobian actions (first term of Eq. CPU)    */
  double t_orth_ms;   /* time in orthogonalisation (second term of Eq. CPU)  */
  double t_total_ms;
  int spec_jvps;      /* actions computed ahead of a GMRES stopping test that
                         then stopped, and discarded (not in total_jvps)      */
  int hook_trials;    /* hookstep trials (residual evaluations) over all steps */
  double delta;       /* trust-region radius at exit                         */
  double lin_rel;     /* relative residual |F - J X| / |F| of the last linear
                         solve (GMRES; -1 for the short recurrences)          */
  double newton_len;  /* length |X| of the last unconstrained Newton step
                         (before the trust region cuts it)                   */
} sp_newton_report;

/* Newton-GMRES with hookstep (Sec. 2, Sec. 3.2): U_inout holds the initial
 * guess and receives the result. Synchronous. Returns SP_ENOTCONV if the
 * iteration cap is reached with |G| >= tol (U_inout still holds the last
 * accepted iterate). */
sp_status sp_newton_gmres(sp_ctx* ctx, double* U_inout, const sp_newton_opts* opts,
                          sp_newton_report* report, void* stream);

/* One Newton linear system G_U X = F (Sec. 2, Eq. linear) solved by a
 * short-recurrence method (Sec. 3.6): krylov = 1 BiCGSTAB(l) (Sleijpen and
 * Fokkema), krylov = 2 IDR(s) with biorthogonalised bases (van Gijzen and
 * Sonneveld), param = l or s (1..8), from X = 0 until |r| <= eta |F| or
 * max_act Jacobian actions (tangent steps at the linearisation point of the
 * last sp_set_base, in the context's precision). The same solvers run inside
 * sp_newton_gmres with opts->krylov = 1, 2.
 * F, X: device states (layout and inner product as above), not aliased.
 * shadow: device pointer to the BiCGSTAB shadow residual (one state) or to
 * the s IDR shadow vectors (s consecutive states, used as given: the caller
 * makes them orthonormal), or NULL (F, resp. seeded vectors orthonormalised
 * by the library).
 * hist (host, max_hist entries): |r| at every residual update, |F| first
 * (BiCGSTAB(l): after each minimal-residual part; IDR(s): after every update
 * of r); *n_hist receives the full count (may exceed max_hist), *n_act the
 * actions used (both may be NULL). A recurrence that breaks down or diverges
 * hands back its smallest-residual iterate. The Krylov work vectors are
 * allocated on first use and kept with the context. Synchronous.
 * Errors: SP_EINVAL (bad arguments, no linearisation point), SP_ENOMEM,
 * SP_ECUDA. */
sp_status sp_krylov_solve(sp_ctx* ctx, const double* F, double* X, int krylov, int param, int max_act,
                          double eta, const double* shadow, double* hist, int max_hist, int* n_hist,
                          int* n_act, void* stream);

/* ---- many independent problems at once -------------------------------------
 *
 * A group holds n independent plane Couette problems, each with its own grid,
 * box, Reynolds number and dt (one precision for all), for instance the
 * members of a parameter continuation. The paper treats one problem at a time;
 * a group only batches independent problems so that many small ones fill the
 * GPU together. It changes no arithmetic: every member's results are those of
 * its own context.
 * Group vector: one state per member, member i at sp_group_offset(g, i)
 * doubles, sp_state_len(sp_group_member(g, i)) doubles long (layout and inner
 * product as above); the gaps between members (offsets are multiples of 32
 * doubles) are never read or written. A group vector has sp_group_state_len(g)
 * doubles. Every stage of sp_group_step and sp_group_jvp is one launch over the
 * blocks of all members (largest members first); the vector operations of
 * sp_group_newton_gmres are one launch over all members' slices. */
typedef struct sp_group sp_group;

/* cfgs: n (1..4096) plane Couette configurations with the same prec; their
 * max_batch is ignored (each member handles one direction). Uses the current
 * device. Synchronous. On failure *out is NULL and sp_group_last_error(NULL)
 * gives the reason. */
sp_status sp_group_create(const sp_config* cfgs, int n, sp_group** out);
sp_status sp_group_destroy(sp_group* g);
const char* sp_group_last_error(const sp_group* g);
int sp_group_size(const sp_group* g);
size_t sp_group_state_len(const sp_group* g);
/* Offset in doubles of member i in a group vector; (size_t)-1 if i is out of range. */
size_t sp_group_offset(const sp_group* g, int member);
/* The member's own context (owned by the group: do not destroy it). Every
 * single-problem call applies to it with pointers into the member's slice, e.g.
 * sp_seed_state(sp_group_member(g, i), ..., U + sp_group_offset(g, i), s). */
sp_ctx* sp_group_member(sp_group* g, int member);

/* G = B_dt(U) - U for every member (FP64, as sp_step). */
sp_status sp_group_step(sp_group* g, const double* U, double* G, void* stream);
/* Linearisation point of every member (as sp_set_base on each). */
sp_status sp_group_set_base(sp_group* g, const double* U, void* stream);
/* Jdu = G_U du for every member, one direction each (as sp_jvp with n_dir = 1,
 * in the group's precision). Needs sp_group_set_base. */
sp_status sp_group_jvp(sp_group* g, const double* du, double* Jdu, void* stream);
/* out_host[i] = <a_i, b_i> for every member (FP64). Synchronous. */
sp_status sp_group_inner(sp_group* g, const double* a, const double* b, double* out_host, void* stream);

/* Newton-GMRES-hookstep (as sp_newton_gmres) on every member in lock step:
 * Arnoldi step j of all members whose GMRES is still running is one sequence of
 * launches, and all hookstep trials of one round are one step of the group.
 * Each member has its own Krylov basis, trust radius and stopping tests, and
 * leaves the iteration when |G| < tol (or it fails). use_fd and use_gradient
 * must be 0 and int_steps <= 1. use_graphs = 1 captures the launches of each Arnoldi step j once as
 * a CUDA graph and replays it (graphs are kept with the group and rebuilt if
 * max_krylov grows). reports: n entries (or NULL); t_action_ms, t_orth_ms and
 * t_total_ms are the group's totals. Synchronous. Returns SP_OK when every
 * member converged, SP_ENAN if any member produced a non-finite value, else
 * SP_ENOTCONV. */
sp_status sp_group_newton_gmres(sp_group* g, double* U_inout, const sp_newton_opts* opts, int use_graphs,
                                sp_newton_report* reports, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* STOKESPREC_H */

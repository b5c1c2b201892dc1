/*
 * tdse.h -- C ABI of the GB300 (sm_103a) Volterra / spectral-recurrence solver
 * for the time-dependent Schroedinger equation with potential V(x,t) and a
 * uniform vector potential A(t):
 *
 *     i u_t = -Laplace(u) + V(x,t) u + i A(t).grad(u)              (eq. schrodfree)
 *
 * Method: Kaye, Barnett & Greengard, "A high-order integral equation-based
 * solver for the time-dependent Schroedinger equation", arXiv:2001.06113.
 * Each time step applies the history-dependent operator of Sec. 2: the mode
 * coefficients are advanced by the exact one-step phase
 *     exp(-i |k|^2 dt + i k.(phi(t) - phi(t-dt))),   phi(t) = int_0^t A    (eq. uhatkrecur)
 * plus an n-th order implicit Adams quadrature of the history of (Vu)^
 * (eq. uadamsk), the implicit step being diagonal in physical space.  The
 * first steps use iterated Richardson extrapolation of the trapezoidal rule
 * (eq. utrapkdisc, Sec. 2.2).
 *
 * Conventions (Sec. 2.1):
 *   periodic grid  x_j = -pi + 2 pi j / M, j = 0..M-1, per dimension;
 *   modes          k = -M/2 .. M/2-1 (stored in FFT order: index m holds k = m
 *                  for m < M/2 and k = m - M otherwise);
 *   forward DFT    f^_k = (1/M) sum_j e^{-2 pi i j k/M} f_j      (eq. ftperdisc)
 *   inverse DFT    f_j  = sum_k e^{+2 pi i j k/M} f^_k.
 *   2D arrays are row-major [n0][n1]; axis 0 is the first coordinate.
 *   Complex arrays are interleaved (re, im) doubles.
 *
 * Memory: the library never allocates device memory.  The caller queries
 * tdse_workspace_bytes() and passes one device buffer (e.g. a PyTorch uint8
 * tensor) to tdse_bind_workspace(); all state, history, tables and scratch
 * live in it.  The caller keeps that buffer alive until tdse_destroy().
 * Host pointers passed to calls are only read/written during the call (the
 * call synchronises the stream when it copies to or from host memory);
 * device pointers must stay valid until the stream reaches the call's work.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  All device work of a call is enqueued on that stream, in order.
 *
 * Errors: every call returns a tdse_status; nothing else crosses the ABI.
 * tdse_last_error() gives a message for the last failing call on a context.
 * A context is not thread-safe; distinct contexts are independent.
 */
#ifndef TDSE_H
#define TDSE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdse_ctx tdse_ctx;

typedef enum {
    TDSE_OK = 0,
    TDSE_EINVAL = -1,        /* bad argument or configuration                  */
    TDSE_ENOMEM = -2,        /* workspace too small / not bound                */
    TDSE_ECUDA = -3,         /* a CUDA runtime call or kernel launch failed    */
    TDSE_ETIMEOUT = -4,      /* a bounded device wait gave up                  */
    TDSE_ENONFINITE = -5,    /* NaN/Inf found in the state                     */
    TDSE_ESTATE = -6,        /* call out of order (e.g. step before inputs)    */
    TDSE_EUNSUPPORTED = -7   /* valid for the method, not built in this library */
} tdse_status;

enum { TDSE_PERIODIC = 0, TDSE_FREE = 1 };
enum { TDSE_FP64 = 0, TDSE_MIXED = 1 };
enum { TDSE_HOST = 0, TDSE_DEVICE = 1 };
enum { TDSE_V_SEPARABLE = 0, TDSE_V_TABLE = 1, TDSE_V_TABLE_SHARED = 2 };
enum { TDSE_BATCH_FUSED = 0, TDSE_BATCH_STREAMS = 1 };
enum { TDSE_PATH_AUTO = 0, TDSE_PATH_PASSES = 1, TDSE_PATH_CLUSTER = 2 };
enum { TDSE_CT_AUTO = 0, TDSE_CT_DIRECT = 1, TDSE_CT_CHEBYSHEV = 2 };
enum { TDSE_LAYOUT_AUTO = 0, TDSE_LAYOUT_CTA = 1, TDSE_LAYOUT_PASSES = 2 };

/*
 * Problem configuration.
 *   dim        1, 2 or 3 (grid n[0] x n[1] x n_z for 3, arrays row-major
 *              [n0][n1][n_z], axis 2 contiguous).  Periodic 3D: powers of
 *              two, axes 0 and 2 in 8..1024, axis 1 in 8..256, at most 2^24
 *              points, no FP64 residual check.  Free-space 3D: every axis as
 *              a free-space axis below (n_z, nu_z for axis 2); the modes are
 *              the tensor product of the three contour rules (Sec. 4.3).
 *   bc         TDSE_PERIODIC: domain [-pi,pi]^dim, Fourier modes (Sec. 2).
 *              TDSE_FREE: free space, data supported in [-1,1]^dim, modes on
 *              the deformed contour Gamma (Sec. 3-4).
 *   n[2]       grid points per dimension (powers of two; periodic 1D: 8..8192,
 *              and 16384 in TDSE_MIXED,
 *              periodic 2D: 8..1024 per dimension; free space: 32..512).
 *              n[1] is ignored for dim = 1.
 *   batch      number of independent instances that share n, dt, nsteps,
 *              order and precision; each has its own V, A and u0.  >= 1.
 *   dt         time step.
 *   nsteps     number of steps the precomputed tables cover (t_max = nsteps*dt).
 *   order      implicit Adams order n: even, 2..8 (Table 1 is n = 8).
 *   startup_steps  Richardson start-up steps; -1 selects order-1 (the paper's
 *              "seven" for n = 8).  Must be >= order-2 and <= nsteps.
 *   precision  TDSE_FP64: every stage in complex FP64.
 *              TDSE_MIXED: transforms, pointwise product and history sum in
 *              complex FP32; the mode state u^ and its phase recurrence, the
 *              phase tables and the Adams weights in FP64.  Free space: the
 *              transforms (with their tables), V u, the history ring, the 2D
 *              intermediate and the history sum in FP32; u^, the one-step
 *              phase p_0, W = p_0 (u^ - i h S_1), the update and u in FP64.
 *              The contour sums then carry FP32 rounding amplified by the
 *              growth of e^{i zeta x} off the real axis, so H must be chosen
 *              for FP32 (tdse_free_choose_H_prec).
 * Free space only (ignored for TDSE_PERIODIC), Sec. 3.4 and 4.1:
 *   nu[2]      length of the equispaced FFTs per dimension: nu = R n with
 *              R in {4, 8, 16} and nu <= 4096.  The equispaced blocks then
 *              have NE = nu/2 - 2 kappa + 1 nodes at spacing h = pi n / nu.
 *   alpert_p   order of Alpert's endpoint correction: 8 (kappa = 7) or 4
 *              (kappa = 4).
 *   gauss_q    Gauss-Legendre points per panel of Gamma_2, 1..32.
 *   n_r        dyadic refinement levels of the Gamma_2 panels toward 0, 0..4
 *              (0: a single panel on [-H, H]; else 2 n_r panels).
 *   H          contour offset, > 0 (tdse_free_choose_H gives the paper's
 *              choice); truncation K = H + pi n / 2.
 * Mode count per dimension N = 2 NE + 2 p + gauss_q * max(1, 2 n_r) (at most
 * 2 NE + 128 dense modes).
 * Both boundary conditions:
 *   potential  TDSE_V_SEPARABLE (0): V(x,t) = f(t) V0(x), tdse_set_potential.
 *              TDSE_V_TABLE (1): a general real V(x,t) (Sec. 1: any potential),
 *              given on the grid at the times the scheme evaluates it
 *              (tdse_potential_times) by tdse_set_potential_table; the
 *              workspace then holds 16 bytes per grid point and time.
 *              TDSE_V_TABLE_SHARED (2): as TDSE_V_TABLE with one table read
 *              by every instance (instances differ in u0 and A only).
 */
typedef struct {
    int dim;
    int bc;
    int n[2];
    int batch;
    double dt;
    int nsteps;
    int order;
    int startup_steps;
    int precision;
    /* free space only */
    int nu[2];
    int alpert_p;
    int gauss_q;
    int n_r;
    double H;
    /* potential form (both boundary conditions), appended last */
    int potential;
    /* dim = 3: grid points along axis 2; n[0], n[1] are axes 0 and 1.
     * Ignored for dim < 3.  Appended last. */
    int n_z;
    /* free space: how the C-type transforms (the Gauss modes on Gamma_2)
     * are evaluated (Sec. 4.1): TDSE_CT_DIRECT = direct sums, O(M N^C) per
     * line; TDSE_CT_CHEBYSHEV = the Chebyshev interpolant in tau of
     * e^{-+(1+i) tau x} (eqs. expintrpm, expintrpp), O(N_T (M + N^C)) with
     * N_T chosen so that the interpolant is exact to FP64 rounding at the
     * C nodes; TDSE_CT_AUTO (0) = Chebyshev when N_T < N^C.  Appended last. */
    int c_transform;
    /* free space, dim = 3: nu of axis 2 (as nu[2] above).  Appended last. */
    int nu_z;
    /* periodic dim = 1: how a step transforms an instance (the DFT pair of
     * Sec. 2.1, eq. ftperdisc; the step is the same).  TDSE_LAYOUT_CTA:
     * one CTA per instance, the whole n-point FFT in its shared memory (n up
     * to 8192 in TDSE_FP64, 16384 in TDSE_MIXED).  TDSE_LAYOUT_PASSES: the
     * four-step form of the same DFT (n = n0 n1, the 2D row and column pass
     * kernels with the twiddle between them, the grid stored transposed in
     * the workspace), so an instance spreads over many CTAs; n = 64..2^20.
     * TDSE_LAYOUT_AUTO (0): one CTA where it is built, the passes beyond.
     * Appended last. */
    int layout_1d;
} tdse_config;

/* Vector potential callback: writes A(t) (dim components) to A_out. */
typedef void (*tdse_field_fn)(double t, double* A_out, void* user);

/* Validate `cfg` and create a context (host only; no CUDA call).
 * Paper: the problem is the initial value problem eq. schrodfree (Sec. 1) on
 * [-pi,pi]^dim with periodic data (Sec. 2) or in free space with data
 * supported in [-1,1]^dim (Sec. 3); the grid, dt and the Adams order n are
 * the discretisation parameters of Sec. 2.1-2.2 (and Sec. 3.4 for the contour).
 * Errors: TDSE_EINVAL for an invalid configuration, TDSE_EUNSUPPORTED for a
 * size this build does not instantiate, TDSE_ENOMEM if host allocation fails. */
tdse_status tdse_create(const tdse_config* cfg, tdse_ctx** out);

/* Bytes of device workspace the context needs (0 if ctx is NULL).  The
 * paper has no counterpart (memory management of this library). */
size_t tdse_workspace_bytes(const tdse_ctx* ctx);

/* Bind caller-owned device memory of at least tdse_workspace_bytes() bytes,
 * 256-byte aligned (no paper counterpart), and build the device tables (twiddles, Adams weights,
 * kinetic phase tables) on `stream`.  Errors: TDSE_ENOMEM if too small,
 * TDSE_EINVAL if misaligned, TDSE_ECUDA on a CUDA failure. */
tdse_status tdse_bind_workspace(tdse_ctx* ctx, void* device_ptr, size_t bytes, void* stream);

/* V(x,t) = f(t) V0(x) for instance `instance` (0-based; -1 = every instance).
 * Paper: the potential V(x,t) of eq. schrodfree (Sec. 1); the scheme samples
 * it on the grid at the step times (eq. uadamsk) and at the trapezoid
 * sub-step times of the Richardson start-up (Sec. 2.2).
 *   V0           n0*n1 real values on the grid (host or device per `where`).
 *   time_factor  NULL for f = 1, else HOST array of 8*nsteps+1 values
 *                f(m dt/8), m = 0..8*nsteps (the step and Richardson sub-step
 *                times).  Copied during the call. */
tdse_status tdse_set_potential(tdse_ctx* ctx, int instance, const double* V0,
                               const double* time_factor, int where, void* stream);

/* TDSE_V_TABLE contexts: the times t_r at which the scheme evaluates V
 * (eq. uadamsk at t_n = n dt; the trapezoid sub-steps of the Richardson
 * start-up, Sec. 2.2, at every m dt/8 of the first startup_steps steps):
 * t_r = r dt/8 for r = 0..8 S, then t = n dt for n = S+1..nsteps
 * (S = min(startup_steps, nsteps)).  Returns the count R = 8 S + 1 +
 * nsteps - S and writes the times to t_out (host, R doubles) if not NULL;
 * -1 for a NULL or separable context. */
int tdse_potential_times(const tdse_ctx* ctx, double* t_out);

/* TDSE_V_TABLE contexts: V(x, t_r) for instance `instance` (-1 = every
 * instance): R x n0*n1 real values, row r = V on the grid at t_r
 * (tdse_potential_times), host or device per `where`; copied during the
 * call (a host source is synchronised before return).  TDSE_ESTATE for a
 * separable context (and tdse_set_potential for a table context);
 * TDSE_EINVAL for instance != -1 in a TDSE_V_TABLE_SHARED context. */
tdse_status tdse_set_potential_table(tdse_ctx* ctx, int instance, const double* V, int where, void* stream);

/* A(t) for an instance (-1 = all) from a callback (NULL = A == 0).  The library
 * computes phi(t) = int_0^t A (eq. phi) by 8-point Gauss-Legendre on each
 * sub-interval of length dt/8, then the per-interval phase tables on `stream`.
 * The callback is called only during this call. */
tdse_status tdse_set_vector_potential(tdse_ctx* ctx, int instance, tdse_field_fn A,
                                      void* user, void* stream);

/* Built-in pulse A(t) = A0 sin^2(pi t / T_pulse) sin(omega t) * direction
 * (direction: dim values).  phi(t) = int_0^t A (eq. phi) is evaluated in
 * closed form on the device, A0 / 2 [F(omega) - (F(omega + W) + F(omega - W)) / 2]
 * with W = 2 pi / T_pulse and F(a) = 2 sin^2(a t / 2) / a (0 for a = 0), then
 * the phase tables as for tdse_set_vector_potential; asynchronous on `stream`. */
tdse_status tdse_set_pulse(tdse_ctx* ctx, int instance, double A0, double omega,
                           double T_pulse, const double* direction, void* stream);

/* Initial wavefunction u0 (n0*n1 interleaved complex, host or device) for an
 * instance (-1 = all instances get the same u0): the initial data u(x,0) of
 * eq. schrodfree (Sec. 1), sampled on the grid of Sec. 2.1 (periodic) or
 * Sec. 3.4 (free space).  Resets the step counter of
 * the whole context to 0. */
tdse_status tdse_set_initial(tdse_ctx* ctx, int instance, const double* u0, int where,
                             void* stream);

/* Initial wavefunctions of every instance in one copy: u0 holds batch
 * consecutive arrays of n0*n1 interleaved complex values (instance b at
 * u0 + 2 b n0 n1), host or device per `where`; copied during the call.
 * Resets the step counter as tdse_set_initial. */
tdse_status tdse_set_initial_batch(tdse_ctx* ctx, const double* u0, int where, void* stream);

/* Advance every instance by `nsteps` steps of dt (asynchronous on `stream`):
 * the marching loop of Sec. 2.1-2.2 (periodic: eq. utrapkdisc for the
 * start-up chains, eq. uadamsk with Table 1's weights afterwards) and of
 * Sec. 3.4 with Remark highorderfs (free space: the same recurrence on the
 * contour modes, eqs. uhatzfd and fzdft/uciftdisc for the transforms).
 * The first call after tdse_set_initial transforms u0 and V(0)u0; the first
 * startup_steps steps use Richardson start-up, later ones the Adams scheme.
 * Errors: TDSE_ESTATE if an instance lacks V, A or u0 (A may be left unset:
 * then A == 0), TDSE_EINVAL if the tables' nsteps would be exceeded. */
tdse_status tdse_step(tdse_ctx* ctx, int nsteps, void* stream);

/* Step until t >= T (T rounded to the nearest multiple of dt): the marching
 * loop of Sec. 2.1-2.2 / Sec. 3.4 run to the final time, as tdse_step. */
tdse_status tdse_solve_to(tdse_ctx* ctx, double T, void* stream);

/* u(x, t_current) on the grid for one instance (or -1 = all, laid out
 * [batch][n0*n1]), into u_out (interleaved complex FP64, host or device).
 * Paper: the read-out is the inverse transform of the mode state (periodic:
 * the inverse DFT of Sec. 2.1 that eq. utrapkdisc applies; free space: the
 * grid values of eq. uciftdisc that the implicit solve produces, Sec. 3.4).
 * Periodic: the inverse DFT of u^ in FP64.  Free space: the grid values of the
 * last implicit solve (or the Richardson combination of the start-up, or u0
 * before the first step), which the scheme carries alongside u^ (u is not
 * the inverse transform of u^ outside [-1,1]^dim).
 * Host destinations are complete when the call returns. */
tdse_status tdse_read_u(tdse_ctx* ctx, int instance, double* u_out, int where, void* stream);

/* The mode state u^(t_current) of one instance (or -1 = all) into u_out
 * (interleaved complex FP64, host or device): periodic [n0][n1] in FFT order,
 * free space [N0][N1] in the node order of tdse_free_rule.  TDSE_FP64, and
 * free space in TDSE_MIXED (its mode state is FP64); TDSE_EUNSUPPORTED for the
 * periodic TDSE_MIXED state (double-float, interaction picture); TDSE_ESTATE
 * before the first step. */
tdse_status tdse_read_modes(tdse_ctx* ctx, int instance, double* u_out, int where, void* stream);

/* Free space: the contour rule of dimension `axis` (Sec. 3.4): *N receives
 * the mode count; if zeta and w are not NULL they receive the N nodes zeta_m
 * and weights w_m (interleaved complex, host) in the block order E1 (Gamma_1,
 * equispaced), A1 (Alpert), C (Gauss panels on Gamma_2), A3 (Alpert), E3
 * (Gamma_3, equispaced), each in ascending real part.  TDSE_EINVAL for a
 * periodic context or a bad axis. */
tdse_status tdse_free_rule(const tdse_ctx* ctx, int axis, int* N, double* zeta, double* w);

/* Free space: the number N_T of Chebyshev terms with which the C-type
 * transforms of dimension `axis` are evaluated (Sec. 4.1; see
 * tdse_config.c_transform), 0 if they are direct sums, -1 for a periodic
 * context, a bad axis or NULL. */
int tdse_free_cheb_terms(const tdse_ctx* ctx, int axis);

/* The contour offset of Remark Hchoice:
 *   H = log(eps / ((1 + vnorm) eps_m)) / (2 dim (1 + phimax)),  eps_m = 2^-52,
 * vnorm = max_t ||V(., t)||_2 on [-1,1]^dim, phimax = max_t |phi(t)|; dim 1..3.
 * TDSE_EINVAL if the result is not positive and finite. */
tdse_status tdse_free_choose_H(double eps, double vnorm, double phimax, int dim, double* H_out);

/* The same offset for the precision the contour sums are evaluated in:
 * eps_m = 2^-52 for TDSE_FP64 and 2^-23 (FP32 machine epsilon) for
 * TDSE_MIXED, whose free-space transforms run in FP32 (Remark Hchoice with
 * eps_m the machine epsilon of those sums).  TDSE_EINVAL for another
 * precision or a result that is not positive and finite. */
tdse_status tdse_free_choose_H_prec(double eps, double vnorm, double phimax, int dim, int precision, double* H_out);

/* FP64 residual check of the mixed-precision implicit step (TDSE_MIXED;
 * periodic 1D n <= 8192, 2D n <= 1024 per dimension; free space with the
 * contour forward / inverse transforms in place of DFT / IDFT, and u on the
 * grid replaced by the FP64 solve as well).  After every
 * `every`-th Adams step (0 = off) the library evaluates, in FP64 on the GPU,
 * with u^_n and R_n = (Vu)^_n as stored (taken back to the lab frame):
 *     W = u^_n + i mu_0 dt R_n,  R64 = DFT(V IDFT(W) / (1 + i mu_0 dt V)),
 *     rho = mu_0 dt ||R64 - R_n||_2 / ||u^_n||_2          (per instance)
 * i.e. the relative residual of the step's implicit equation (eq. uadamsk),
 * and where rho > tol (or is not finite) redoes the step in FP64:
 * u^_n <- W - i mu_0 dt R64, R_n <- R64.  The check and the redo stay on the
 * device (no host synchronisation).  Errors: TDSE_EUNSUPPORTED outside the
 * sizes above or for FP64 contexts (every > 0). */
tdse_status tdse_set_residual_check(tdse_ctx* ctx, int every, double tol);

/* Last checked residual rho per instance and the number of FP64 redos per
 * instance (host arrays of batch entries, either may be NULL), and the number
 * of checks run since tdse_set_initial.  Synchronises `stream`.
 * TDSE_ENONFINITE if a checked residual is not finite. */
tdse_status tdse_residual_report(tdse_ctx* ctx, double* rho, int* corrections, int* checks, void* stream);

/* Scan the mode state of every instance for NaN/Inf (synchronises `stream`).
 * Returns TDSE_ENONFINITE if any is found, TDSE_ETIMEOUT if a bounded wait
 * inside a step kernel gave up since the workspace was bound (the results
 * are then invalid). */
tdse_status tdse_check_finite(tdse_ctx* ctx, void* stream);

/* Checkpoint of the whole solve state: the context's workspace (mode state,
 * history ring, start-up buffers, V, A and phase tables) and its host step
 * counters, into a host blob.  blob == NULL: *size receives the bytes needed
 * (no workspace needed).  Otherwise *size is the blob's capacity and receives
 * the bytes written.  Synchronises `stream`.  The paper has no checkpoint; a
 * run resumed with tdse_load continues bit for bit like an uninterrupted one. */
tdse_status tdse_save(tdse_ctx* ctx, void* blob, size_t* size, void* stream);

/* Resume from a tdse_save blob into a bound context of the same
 * configuration (TDSE_EINVAL for another configuration or a short blob).
 * Synchronises `stream`. */
tdse_status tdse_load(tdse_ctx* ctx, const void* blob, size_t size, void* stream);

/* Kernels of the 2D periodic TDSE_MIXED Adams steps (the step operator of
 * eq. uadamsk, Sec. 2.2, in the interaction picture; no change to what is
 * computed):
 *   TDSE_PATH_PASSES   two launches per step: a row pass and a fused column
 *                      pass that exchange the transform intermediates
 *                      through global memory;
 *   TDSE_PATH_CLUSTER  512 x 512 grids: one launch per run of steps, each
 *                      instance on a cluster of 16 CTAs that keeps the
 *                      intermediates in (distributed) shared memory and
 *                      streams the state, history and V by TMA (measured
 *                      about 2x slower than the passes on a GB300: one CTA
 *                      per SM, 7 clusters resident, and only a 3-stage load
 *                      pipeline beside the 128 KB intermediate);
 *   TDSE_PATH_AUTO     (default) the pass kernels.
 * Both paths give the same bits.  TDSE_EUNSUPPORTED for TDSE_PATH_CLUSTER
 * where it is not available (another size or precision, 1D, free space, or a
 * device or driver that cannot run the cluster); TDSE_EINVAL for another
 * value.  May be called at any time between steps. */
tdse_status tdse_set_step_path(tdse_ctx* ctx, int path);

/* 2D periodic contexts, pass kernels: split the batch into `groups` (1..64,
 * at most the batch size is used) contiguous groups of instances whose Adams
 * step chains run on parallel streams that the library creates on first use
 * (forked from and joined to the caller's stream, so the call stays ordered
 * on it), so that the row pass of one group and the column pass of another
 * share the SMs.  Instances are independent: results are the same bits for
 * any number of groups.  Default 4.  The first steps after raising the count
 * create the streams; take them before any stream capture. */
tdse_status tdse_set_step_groups(tdse_ctx* ctx, int groups);

/* 1D periodic TDSE_MIXED contexts of n <= 16384 (one CTA per instance):
 * launch shape of the step kernel.  Shape 0 (default): n/8 threads per
 * instance (32..1024); shape 1: for n = 8192 1024 threads (8 points each),
 * for the other n >= 512 half the default threads, each thread taking twice
 * the points of every transform pass.  The transform's
 * butterflies and the step's arithmetic are the same in both (Sec. 2.1-2.2),
 * so the results are the same bits; tdse_batch_tune sets the faster shape
 * per member.  Errors: TDSE_EUNSUPPORTED for another context or where shape 1
 * is not built (the shape stays), TDSE_EINVAL for another value.
 * tdse_shape_1d returns the current shape (-1 for a null context). */
tdse_status tdse_set_shape_1d(tdse_ctx* ctx, int shape);
int tdse_shape_1d(const tdse_ctx* ctx);

/* The path the next 2D mixed Adams steps take (TDSE_PATH_PASSES or
 * TDSE_PATH_CLUSTER; TDSE_PATH_PASSES for every other context), or -1 for
 * NULL.  The cluster path needs the bound workspace (its plan is made at
 * tdse_bind_workspace). */
int tdse_step_path(const tdse_ctx* ctx);

/* The launch shape of the Adams steps as a JSON object into buf (len bytes,
 * NUL-terminated): "path" = "passes" (2D/3D pass kernels, 1D in the
 * four-step layout: "groups", and "four_step" = [n0, n1] for 1D), "cluster"
 * ("clusters" resident at once, "ctas_per_cluster", "threads",
 * "smem_bytes") or "cta" (1D, one CTA per instance: "shape", "threads").
 * TDSE_EINVAL for NULL arguments or a buffer too small. */
tdse_status tdse_describe_steps(const tdse_ctx* ctx, char* buf, size_t len);

/* Number of completed steps and the current time t = steps * dt. */
int tdse_step_index(const tdse_ctx* ctx);
double tdse_time(const tdse_ctx* ctx);

/* The implicit Adams weights mu_0..mu_{order-1} this library uses
 * (Sec. 2.2; Table 1 for order 8), written to mu_out. */
tdse_status tdse_adams_weights(int order, double* mu_out);

/*
 * Allocation-free read-out transform, for callers that cannot allocate device
 * memory at all (and so cannot provide a workspace): code where cudaMalloc is
 * forbidden or unavailable, e.g. a host application that owns every device
 * allocation itself or a plugin with a fixed device-memory budget.  The paper
 * has no counterpart; it is a packaging of this library's own read-out.
 *
 * Computes, for `batch` 2D arrays of n0 x n1 modes in FFT order (device
 * pointer `uhat`, interleaved complex FP64, [batch][n0][n1]), the grid values
 *     u_j = sum_k e^{+2 pi i j.k / n} uhat_k       (same as tdse_read_u)
 * into the device array `u` (same layout), in FP64, on `stream`.
 * n0, n1: powers of two in 8..1024.  batch*n0*n1 must not exceed
 * TDSE_NOALLOC_MAX_POINTS: larger requests return TDSE_ENOMEM and do nothing.
 * Its scratch is one fixed device array inside the library
 * (TDSE_NOALLOC_MAX_POINTS * 16 bytes plus tables) that every GPU loading the
 * library holds until the process exits.  All calls share that array: calls
 * whose work overlaps on the GPU (different streams or threads) race and give
 * wrong results, so serialise them.  The first call on a device looks up the
 * array's address with that device current; make it before any stream
 * capture.  Errors: TDSE_EINVAL (null pointer, bad size), TDSE_ENOMEM (too
 * large), TDSE_ECUDA (launch failure).
 */
#define TDSE_NOALLOC_MAX_POINTS 524288
tdse_status tdse_modes_to_grid_2d_noalloc(const double* uhat, double* u, int n0, int n1, int batch,
                                          void* stream);

/*
 * Uneven batches (1D periodic, TDSE_MIXED).  Several contexts, each with its
 * own n and its own batch of instances, but identical dt, nsteps,
 * order and startup_steps, are stepped together:
 *   - every Adams step of all of them is ONE persistent launch: a CTA of 512
 *     threads takes work items, an item being `count` instances of one
 *     context side by side, each transformed by a group of T threads (T and
 *     the CTA count are the launch shape); members created with
 *     TDSE_LAYOUT_PASSES (or beyond n = 16384) instead run their four-step
 *     pass chain on their own stream beside that launch;
 *   - the start (init, Richardson start-up, change of frame) of each member
 *     runs with the member's own kernels;
 *   - with a capturable stream (not the legacy NULL stream) the whole launch
 *     sequence of one tdse_batch_step call is captured into a CUDA graph the
 *     first time and replayed by later calls with the same start step and
 *     length (e.g. after tdse_set_initial reset the members).
 * The members stay owned by the caller and must outlive the batch; they must
 * not be stepped on their own while in a batch.
 */
typedef struct tdse_batch tdse_batch;

/* Group `count` (1..16) contexts.  Errors: TDSE_EINVAL (incompatible members,
 * unbound workspace, more than 1536 work items), TDSE_EUNSUPPORTED (not 1D
 * periodic mixed). */
tdse_status tdse_batch_create(tdse_ctx* const* members, int count, tdse_batch** out);

/* Execution of the Adams phase: TDSE_BATCH_FUSED (0, the default) = one
 * persistent launch per step for all members; TDSE_BATCH_STREAMS (1) = each
 * member's own single-size kernel on its own stream, forked from and joined
 * to the caller's stream (parallel branches of the captured graph).  Same
 * results either way.  Cached graphs are dropped.  TDSE_EINVAL otherwise. */
tdse_status tdse_batch_set_mode(tdse_batch* b, int mode);

/* Autotuner: choose, by timing `trial_steps` launches of each candidate on
 * `stream`, for the fused launch the launch shape of each member (threads per
 * instance among the variants built for its n: n/8, or half of that for
 * n = 2048, 4096, 8192), its instances per work item (all that fit the CTA, a
 * half or a quarter) and the CTA count; for the per-member streams each
 * member's kernel shape (tdse_set_shape_1d); then the faster of the two
 * modes (tdse_batch_set_mode).  The members must have V and u0 set; tuning runs their start
 * if needed and leaves their state undefined: call tdse_set_initial on every
 * member before the next tdse_batch_step.  Cached graphs are dropped. */
tdse_status tdse_batch_tune(tdse_batch* b, int trial_steps, void* stream);

/* Advance every member by nsteps (all members must be at the same step). */
tdse_status tdse_batch_step(tdse_batch* b, int nsteps, void* stream);

/* The launch shape as a JSON object (members' n, batch, T, instances per
 * item; items; CTAs; shared memory; graphs cached; tuned or default). */
tdse_status tdse_batch_describe(const tdse_batch* b, char* buf, size_t len);

const char* tdse_batch_last_error(const tdse_batch* b);
void tdse_batch_destroy(tdse_batch* b);

/* Message of the last failing call on `ctx` ("" if none; static string if
 * ctx is NULL). */
const char* tdse_last_error(const tdse_ctx* ctx);

/* Release the context (host memory only; the caller frees the workspace). */
void tdse_destroy(tdse_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* TDSE_H */

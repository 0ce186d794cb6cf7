/*
 * tdse.h - C ABI of the GB300 finite-difference TDSE propagation library.
 *
 * The library advances the partial-wave radial wavefunction of a one-electron
 * (hydrogen / single-active-electron) atom in a linearly polarised laser field,
 * in the length or the velocity gauge, with hand-written sm_103a CUDA kernels.
 * It follows arXiv 1308.1856 (CLTDSE):
 *
 *   state vector F, l-major  ............ Sec. 2, the vector F of Eq. (h_matrix)
 *   Hamiltonian H(t) ..................... Sec. 2, Eqs. (tdse-radial-field),
 *                                          (tdse-potential), (h_matrix)
 *   dF/dt = -i H(t) F .................... Eq. (tdse_matrix)
 *   Taylor / Runge-Kutta / Lanczos ....... Sec. 5 "TDSE": Eq. (Taylor),
 *                                          Eq. (RKDeriv), Appendix "Lanczos methods"
 *   embedded Runge-Kutta pairs ........... Appendix "Runge-Kutta"
 *   imaginary time ....................... Sec. 3
 *   pulse, vector potential .............. Sec. 3, Eqs. (EField), (VectorStep)
 *   absorber ............................. Sec. 2.1 (applied as a mask)
 *   observables .......................... Sec. 4: Eqs. (p_g), (p_b), (yield_1),
 *                                          (Norm), (Dipole)
 *   dipole velocity / acceleration ....... Sec. 4: Eqs. (DipoleVelocity), (DipoleAccel)
 *   radial flux, PAD, flux yield ......... Sec. 4: Eqs. (flux), (pad), (yield)
 *
 * Conventions
 *   - Atomic units.  Grid r_j = j*dr + offset, j = 1..N; partial waves
 *     l = 0..lmax with m = 0.  Finite-difference neighbours beyond the box are
 *     zero; the optional odd ghost sets f(-dr) = -f(dr).
 *   - Complex numbers are interleaved (re, im) doubles.  A state holds
 *     (lmax+1)*N complex values, l-major: element (l, j) sits at
 *     2*(l*N + (j-1)) (re) and the next double (im).
 *   - Ownership: the handle owns all device memory it allocates and one CUDA
 *     stream (or borrows the caller's through tdse_set_stream).  Every host
 *     pointer stays the caller's; inputs are copied before the call returns.
 *     Device pointers passed to tdse_apply_h / tdse_*_state_device are the
 *     caller's and must hold the stated number of bytes.
 *   - Asynchrony: tdse_propagate and tdse_apply_h only enqueue work on the
 *     handle's stream.  tdse_get_state, tdse_observables and tdse_sync wait
 *     for it.
 *   - Errors: every call returns a tdse_status; tdse_last_error() gives a
 *     message.  After TDSE_ERR_CUDA the handle is poisoned: later calls return
 *     TDSE_ERR_STATE.  Non-finite values found by a norm reduction are
 *     reported as TDSE_ERR_NONFINITE by the next synchronising call.
 */
#ifndef TDSE_H
#define TDSE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdse tdse_t;

typedef enum {
  TDSE_OK = 0,
  TDSE_ERR_ARG = -1,        /* invalid argument; nothing was changed         */
  TDSE_ERR_OOM = -2,        /* device or host allocation failed              */
  TDSE_ERR_CUDA = -3,       /* a CUDA call failed; the handle is poisoned     */
  TDSE_ERR_NONFINITE = -4,  /* the state holds Inf/NaN (e.g. unstable dt)     */
  TDSE_ERR_STATE = -7       /* handle poisoned by an earlier CUDA error       */
} tdse_status;

enum { TDSE_STENCIL_3 = 3, TDSE_STENCIL_5 = 5 };
enum { TDSE_TAYLOR = 0, TDSE_RK4 = 1, TDSE_LANCZOS = 2 };
enum { TDSE_GHOST_ZERO = 0, TDSE_GHOST_ODD = 1 };
enum { TDSE_FP64 = 0, TDSE_MIXED = 1 };
/*
 * Gauge of the laser coupling (Sec. 2).  Length: r E(t) kappa couplings.
 * Velocity: (A(t)/c) p_z, p_z = -i [(d/dr - l/r) kappa_l f_{l-1} +
 * (d/dr + (l+1)/r) kappa_{l+1} f_{l+1}] with the first derivative of the
 * chosen stencil (4th-order 5-point, or 3-point central); A(t) = -c int_0^t E
 * by composite 5-point Gauss quadrature on panels of at most 0.25 a.u. (the
 * paper prints the l/r terms with the opposite signs, which breaks
 * p_z = i[H_0, z] and gauge invariance).  The velocity gauge runs with the
 * zero ghost (TDSE_ERR_ARG otherwise), in FP64 or in mixed precision (the
 * coupling's first derivatives then FP32, formed part by part like the
 * Laplacian); observables are the same formulas.  In a batch it is FP64 only.
 */
enum { TDSE_GAUGE_LENGTH = 0, TDSE_GAUGE_VELOCITY = 1 };
/* largest Krylov dimension tdse_propagate accepts for TDSE_LANCZOS */
#define TDSE_MAX_KRYLOV 32

typedef struct {
  int ghost;            /* TDSE_GHOST_ZERO (default) or TDSE_GHOST_ODD          */
  double offset;        /* constant grid shift (default 0)                       */
  int absorber;         /* 1: multiply by the cos^(1/8) mask after every step    */
  double absorber_r;    /* mask is 1 for r <= absorber_r and falls to r_N        */
  double r_b;           /* yield radius: yield = 1 - sum_{r_j <= r_b} |f|^2 dr   */
  int precision;        /* TDSE_FP64 (default) or TDSE_MIXED (see tdse_propagate) */
  int gauge;            /* TDSE_GAUGE_LENGTH (default) or TDSE_GAUGE_VELOCITY     */
} tdse_opts;

/*
 * Create a handle for N radial points of spacing dr and partial waves
 * l = 0..lmax with a 3- or 5-point second derivative (Sec. 2).  The potential
 * is -Z/r, or v_table[j-1] = V(r_j) (length N, host, copied) when v_table is
 * not NULL.  The state starts as P(r) = 2 r exp(-r) in l = 0, scaled so that
 * dr * sum |P|^2 = 1; that wave is also the reference of p_ground.  Options
 * start at: zero ghost, offset 0, no absorber, r_b = 10.
 * Errors: TDSE_ERR_ARG (N < 1, lmax < 0, dr <= 0, stencil not 3/5),
 * TDSE_ERR_OOM, TDSE_ERR_CUDA.  *out is NULL on error.
 */
int tdse_create(int N, double dr, int lmax, int stencil, double Z, const double *v_table,
                tdse_t **out);

/* Release everything the handle owns (NULL is accepted). */
int tdse_destroy(tdse_t *h);

/* Message for the last error on this handle (static storage, never NULL). */
const char *tdse_last_error(const tdse_t *h);

/*
 * Replace the options (ghost, offset, absorber, r_b).  Changing ghost or
 * offset rebuilds the operator tables and the initial 1s state is NOT
 * recomputed.  Errors: TDSE_ERR_ARG (ghost not 0/1, absorber_r outside the
 * box while absorber is on).
 */
int tdse_set_options(tdse_t *h, const tdse_opts *opts);

/*
 * Use the caller's CUDA stream (a cudaStream_t; NULL restores the handle's own).
 * The kernels of a propagation step are launched on it with programmatic
 * stream serialization, so each may start while the kernel before it on the
 * stream finishes.  Each of them waits for that kernel to complete before it
 * touches memory, so work the caller enqueued earlier on the stream is
 * complete, as with ordinary launches.  A kernel the caller enqueues after a
 * call starts after the library's last kernel of that call has completed,
 * unless the caller gives it that attribute as well.
 */
int tdse_set_stream(tdse_t *h, void *cuda_stream);

/*
 * Length-gauge pulse E(t) = E0 sin^2(pi t / T) sin(omega t + cep) for
 * 0 <= t <= T = 2 pi ncycles / omega, zero elsewhere (Sec. 3, Eq. (EField)
 * with the Hann envelope).  E0 = 0 switches the field off.
 * Errors: TDSE_ERR_ARG (E0 != 0 with omega <= 0 or ncycles <= 0).
 */
int tdse_set_pulse(tdse_t *h, double E0, double omega, double ncycles, double cep);

/*
 * Envelope of the pulse (Sec. 3).  TDSE_PULSE_SIN2_E (default): the sin^2
 * envelope on E as above.  TDSE_PULSE_SIN2_A ("SineA", Eq. (VecSinSinCosE)):
 * the sin^2 envelope on the vector potential,
 *   A(t) = -(c E0/omega) sin^2(pi t/T) sin(omega t + cep),
 *   E(t) = -(1/c) dA/dt = (E0/omega) sin(W t) [omega sin(W t) cos(omega t + cep)
 *                                              + 2 W cos(W t) sin(omega t + cep)],
 * W = pi/T = omega/(2 ncycles), 0 <= t <= T, zero elsewhere; E0 is the peak
 * field of a many-cycle pulse in both shapes.  Errors: TDSE_ERR_ARG (unknown
 * shape).
 */
enum { TDSE_PULSE_SIN2_E = 0, TDSE_PULSE_SIN2_A = 1 };
int tdse_set_pulse_shape(tdse_t *h, int shape);

/* Evaluate the pulse set by tdse_set_pulse at time t (host arithmetic). */
double tdse_field(const tdse_t *h, double t);
/* A(t) = -c int_0^t E, by 5-point Gauss quadrature on equal panels of [0, T]
 * no wider than 0.25 a.u. (Sec. 3, Eq. (VectorStep)); constant after T. */
double tdse_vector_potential(const tdse_t *h, double t);

/* Current time of the state; tdse_propagate advances it by nsteps * dt. */
int tdse_set_time(tdse_t *h, double t);
double tdse_get_time(const tdse_t *h);

/* Copy a state in from / out to HOST memory ((lmax+1)*N interleaved complex). */
int tdse_set_state(tdse_t *h, const double *F_host);
int tdse_get_state(tdse_t *h, double *F_host);

/* The same from / to DEVICE memory of the caller (16*(lmax+1)*N bytes, 16-byte aligned). */
int tdse_set_state_device(tdse_t *h, const void *F_dev);
int tdse_get_state_device(tdse_t *h, void *F_dev);

/* Reference l = 0 wave of p_ground (N interleaved complex, host, copied). */
int tdse_set_reference(tdse_t *h, const double *f0_host);

/*
 * Advance the state by nsteps steps of size dt (asynchronous).
 *   TDSE_TAYLOR  - Taylor polynomial of exp(-i H dt) of degree `order`
 *                  (Eq. (Taylor); evaluated in Horner form), field at mid-step;
 *   TDSE_RK4     - classic fourth-order Runge-Kutta (Eq. (RKDeriv)), field at
 *                  the stage times; `order` is ignored;
 *   TDSE_LANCZOS - Lanczos with Krylov dimension `order` (Appendix "Lanczos
 *                  methods"), field at mid-step; the Krylov space is cut when
 *                  beta_j <= 1e-13 max(1, max|alpha|).
 * The absorber, if on, multiplies the state by the mask after every step.
 * Precision (tdse_opts.precision): TDSE_FP64 computes everything in FP64.
 * TDSE_MIXED keeps the state, every update of it, the Lanczos dot products,
 * norms and the tridiagonal exponential in FP64, and applies H in FP32 to the
 * FP32 hi/lo split of the state plus complex64 work vectors (Krylov vectors,
 * Taylor corrections, RK slopes; RK stage sums are compensated two-float
 * sums), with the radial Laplacian formed from differences.
 * Errors: TDSE_ERR_ARG (dt <= 0, nsteps < 0, order < 1 for Taylor/Lanczos,
 * order > TDSE_MAX_KRYLOV for Lanczos), TDSE_ERR_OOM, TDSE_ERR_CUDA.
 */
int tdse_propagate(tdse_t *h, int method, int order, double dt, long nsteps);

/*
 * Dipole moment, velocity and acceleration of the current state at the
 * handle's time t (Sec. 4, Eqs. (Dipole), (DipoleVelocity), (DipoleAccel)),
 * m = 0, dr-weighted sums over the grid:
 *   <z>     = 2 sum_l kappa_{l+1} sum_j r_j Re(f_l^* f_{l+1}) dr
 *   <zdot>  = 2 sum_l kappa_{l+1} sum_j Im(f_{l+1}^* (D1 f_l - (l+1)/r_j f_l)) dr
 *             [+ (A(t)/c) ||psi||^2 in the velocity gauge]
 *   <zddot> = -E(t) ||psi||^2 - 2 Z sum_l kappa_{l+1} sum_j Re(f_l^* f_{l+1}) / r_j^2 dr
 * D1 is the first-derivative formula of the velocity gauge (5- or 3-point,
 * with the grid's ghost).  <zdot> carries the factor 2 that Ehrenfest's
 * theorem d<z>/dt = <zdot> needs (the printed Eq. (DipoleVelocity) omits it)
 * and is the kinetic momentum.  The acceleration form needs dV/dr, so with a
 * tabulated potential *zddot is NaN.  Any output pointer may be NULL.
 * Synchronises the stream.  Errors: TDSE_ERR_OOM, TDSE_ERR_CUDA.
 */
int tdse_dipole_moments(tdse_t *h, double *z, double *zdot, double *zddot);

/*
 * Record <z>, <zdot> and <zddot> (as tdse_dipole_moments) after every
 * real-time step of tdse_propagate / tdse_propagate_rk into a device buffer
 * of `capacity` entries (one extra launch per step; recording stops when the
 * buffer is full).  capacity 0 turns recording off; every call discards what
 * was recorded.  TDSE_ERR_ARG for capacity < 0; TDSE_ERR_OOM.
 */
int tdse_dipole_series(tdse_t *h, long capacity);
/* Copy up to max_entries recorded entries to out as {t, <z>, <zdot>, <zddot>}
 * (4 doubles each, in step order); *count (may be NULL) receives the number
 * recorded so far.  out may be NULL to query the count.  Synchronises. */
int tdse_dipole_series_read(tdse_t *h, double *out, long max_entries, long *count);

/*
 * The per-step record (the paper's time-dependent output, Sec. 4): after every
 * `every`-th real-time step, one row of tdse_record_width(h) = lmax + 11
 * doubles is written on the device:
 *   t, norm, dipole, yield, p_ground, l_pop[0..lmax],   (as tdse_observables)
 *   <z>, <zdot>, <zddot>,                               (as tdse_dipole_moments)
 *   flux, flux yield                                    (as tdse_flux_read; NaN without a flux setup)
 * (p_e = (1 - yield) - p_ground.)  Two or three extra launches per recorded
 * step; recording stops when `capacity` rows are full; every call discards
 * what was recorded and restarts the step count.  capacity 0 turns it off.
 * tdse_record_read copies up to max_rows rows (out may be NULL to query the
 * count) and synchronises.  Errors: TDSE_ERR_ARG (every < 1, capacity < 0),
 * TDSE_ERR_OOM.
 */
int tdse_record_setup(tdse_t *h, long every, long capacity);
long tdse_record_width(const tdse_t *h);
int tdse_record_read(tdse_t *h, double *out, long max_rows, long *count);

/*
 * Flux through the sphere r = r_b (Sec. 4, Eqs. (flux), (pad), (yield)),
 * evaluated at the grid point nearest r_b (a tie goes to the inner point):
 *   flux       = sum_l Im(f_l^* D1 f_l) [+ 2 (A/c) sum_l kappa_{l+1} Re(f_l^* f_{l+1})]
 *              = r_b^2 times the radial current integrated over the sphere,
 *   density_k  = Im(S_k^* P_k) [+ (A/c) cos(theta_k) |S_k|^2]
 *              = r_b^2 j_r(r_b, theta_k),  S_k = sum_l Y_l0(theta_k) f_l,
 *                P_k = sum_l Y_l0(theta_k) D1 f_l,  Y_l0 = sqrt((2l+1)/(4 pi)) P_l,
 * outward positive (the paper prints -Im in Eq. (flux); the continuity
 * equation and Eq. (yield) fix the sign), the A terms in the velocity gauge
 * only.  After every real-time step the time integrals are advanced by the
 * trapezoid rule over the step: yield = int flux dt (Eq. (yield)), pad_k =
 * int density_k dt (Eq. (pad), dP/dOmega).  Setup evaluates the current state
 * and zeroes the integrals; r_b <= 0 turns the flux off.  cos_theta: ntheta
 * values in [-1, 1] (host, copied).  One extra single-block launch per step.
 * Errors: TDSE_ERR_ARG (r_b outside the box, bad angles, lmax > 1535),
 * TDSE_ERR_OOM, TDSE_ERR_CUDA.  Synchronises.
 */
int tdse_flux_setup(tdse_t *h, double r_b, int ntheta, const double *cos_theta);
/* The current flux and density (at the last step's end, or at setup) and their
 * time integrals; any pointer may be NULL (density and pad hold ntheta
 * values).  TDSE_ERR_ARG if the flux is not set up.  Synchronises. */
int tdse_flux_read(tdse_t *h, double *flux, double *yield, double *density, double *pad);

/*
 * Debug guard bands.  When the environment variable TDSE_GUARD_BYTES is a
 * positive number at tdse_create, every device buffer the handle allocates
 * sits between two bands of that many bytes (rounded up to 256) filled with
 * 0xff.  tdse_check_guards synchronises and checks every band: TDSE_OK if
 * all are intact (or guards are off), TDSE_ERR_STATE naming the buffer whose
 * band a kernel overwrote.  (A stand-in for a device memory checker: out-of-
 * bounds writes next to a buffer land in a band.)
 */
int tdse_check_guards(tdse_t *h);

/*
 * Checkpoint and resume.  A checkpoint holds the state, the time, the cached
 * norm the next Lanczos step starts from and, if the flux is set up, its
 * current values and time integrals: loading it into a handle of the same
 * grid, stencil, ghost, offset, gauge, precision and flux setup and
 * propagating gives bitwise the states of the uninterrupted run.  (Loading
 * into a handle of the other precision works but recomputes the norm.)
 * tdse_checkpoint_bytes: size of the host buffer.  save: synchronous copy to
 * host memory.  load: TDSE_ERR_ARG if the buffer is not a checkpoint, is too
 * small, or was taken on another grid, ghost, offset, gauge or flux setup.
 * The pulse, options and dipole series are the handle's, not the checkpoint's.
 */
size_t tdse_checkpoint_bytes(const tdse_t *h);
int tdse_checkpoint_save(tdse_t *h, void *buf, size_t bytes);
int tdse_checkpoint_load(tdse_t *h, const void *buf, size_t bytes);

/* Explicit Runge-Kutta methods of the appendix "Runge-Kutta". */
enum {
  TDSE_RK_EULER = 0,          /* forward Euler, no embedded pair */
  TDSE_RK_CLASSIC = 1,        /* classic RK4, no embedded pair */
  TDSE_RK_FEHLBERG = 2,       /* Runge-Kutta-Fehlberg 4(5), 6 stages */
  TDSE_RK_CASH_KARP = 3,      /* Cash-Karp 4(5), 6 stages */
  TDSE_RK_DORMAND_PRINCE = 4, /* Dormand-Prince 5(4), 7 stages */
  TDSE_RK_MERSON = 5          /* Merson 4("5"), 5 stages */
};

/*
 * nsteps steps of the explicit Runge-Kutta method `tableau` (TDSE_RK_*) with
 * the published Butcher tableau (appendix "Runge-Kutta"):
 *   k_i = -i H(t_n + c_i dt) (F_n + dt sum_{j<i} a_ij k_j),
 *   F_{n+1} = F_n + dt sum_i b_i k_i          (the higher-order solution),
 *   Delta = dt sum_i (b_i - bhat_i) k_i       (bhat: the embedded companion),
 *   sigma_n = sqrt(sum |Delta|^2 / S),  S = (L+1) N complex entries,
 * with the field (length gauge) or A/c (velocity gauge) at the stage times,
 * and the absorber mask, if on, after every step (sigma_n is taken before
 * the mask).  dt is fixed: the paper accumulates sigma = sum_n sigma_n as an
 * error measure and does not adapt the step.  *sigma (may be NULL) receives
 * the sum over these steps; synchronises the stream; advances t by
 * nsteps dt.  Methods without an embedded pair give sigma = 0.
 * One stage is one launch; slopes of earlier stages are stored, so the handle
 * keeps max(2, s + 1) state-sized work vectors (s stages).
 * FP64 only: TDSE_ERR_ARG with TDSE_MIXED, dt <= 0, nsteps < 0 or an
 * unknown tableau; TDSE_ERR_OOM; TDSE_ERR_CUDA; TDSE_ERR_NONFINITE if the
 * state became non-finite.
 */
int tdse_propagate_rk(tdse_t *h, int tableau, double dt, long nsteps, double *sigma);

/*
 * Imaginary-time propagation (Sec. 3, "Imaginary time"): nsteps steps of the
 * chosen propagator applied to exp(-H dtau) instead of exp(-i H dt), with no
 * field and no absorber; after every step the state is renormalised
 * (dr sum |f|^2 = 1) and the energy estimate
 *   E = -ln(||psi_new||^2 / ||psi||^2) / (2 dtau)
 * is formed (the paper prints -ln <psi|psi> / dt; the factor 1/2 makes an
 * eigenstate's estimate its eigenvalue).  *energy (may be NULL) receives the
 * last step's estimate; synchronises the stream.  The time t does not change.
 * FP64 only: TDSE_ERR_ARG with TDSE_MIXED, dtau <= 0, nsteps < 0 or a bad
 * method/order.
 */
int tdse_propagate_imag(tdse_t *h, int method, int order, double dtau, long nsteps, double *energy);

/*
 * Observables of the current state (synchronises the stream), Sec. 4, each
 * integral taken as dr * sum over grid points:
 *   norm     = dr sum_l sum_j |f_lj|^2
 *   l_pop[l] = dr sum_j |f_lj|^2                       (lmax+1 doubles)
 *   dipole   = 2 sum_{l<lmax} kappa_{l+1} dr sum_j r_j Re(conj(f_lj) f_{l+1,j})
 *   yield    = 1 - dr sum_l sum_{r_j <= r_b} |f_lj|^2
 *   p_ground = |dr sum_j conj(ref_j) f_0j|^2
 * Any output pointer may be NULL.  Returns TDSE_ERR_NONFINITE if the state
 * holds Inf/NaN.
 */
int tdse_observables(tdse_t *h, double *norm, double *l_pop, double *dipole, double *yield,
                     double *p_ground);

/*
 * y = H(E) x on caller-owned DEVICE buffers (asynchronous on the handle's
 * stream); x and y hold (lmax+1)*N interleaved complex doubles, 16-byte
 * aligned, and must not overlap.  This is the bare operator of Eq. (h_matrix),
 * in FP64, or in the mixed arithmetic when tdse_opts.precision is TDSE_MIXED.
 * In the velocity gauge E is the vector potential A.
 */
int tdse_apply_h(tdse_t *h, double E, const void *x_dev, void *y_dev);

/*
 * Small grids: a whole tdse_propagate call in one launch.  A grid of a few
 * thousand points is microseconds of arithmetic per step, so a step of one
 * launch per stage (Sec. 5: one kernel per Taylor term, per RK stage, per
 * Lanczos phase) is bound by launch and grid-reduction latency.  On the
 * small-grid path one thread-block cluster of at most 16 CTAs (one per SM)
 * runs every step of the call: CTA r holds radial columns [r W, (r+1) W) of
 * psi, of the diagonal table and of every work vector in its shared memory,
 * reads the stencil's halo columns from its neighbours' shared memory,
 * separates stages by cluster barriers and adds the Lanczos dot products and
 * norms in a fixed order (every CTA holds the same sums, and forms the small
 * exponential of each Lanczos step itself).  Taylor and RK4 give bitwise the
 * states of the multi-launch path; Lanczos differs only in the association
 * of its grid sums.  It applies to FP64 length-gauge propagation with no
 * per-step observables set up (dipole series, flux, record), when the state
 * and the method's work vectors (Taylor 3, RK4 4, Lanczos order + 1 vectors
 * of the state's size, plus the diagonal table) fit in the cluster's shared
 * memory (about 3 MB).
 *   TDSE_SMALL_GRID_AUTO (default): that path for grids of at most 16384
 *     points, the multi-launch path otherwise;
 *   TDSE_SMALL_GRID_OFF: always the multi-launch path;
 *   TDSE_SMALL_GRID_FORCE: that path whenever it applies, whatever the size.
 * tdse_small_grid_path_used returns 1 if the last tdse_propagate call ran on
 * it, else 0.  Errors: TDSE_ERR_ARG (unknown mode).
 */
enum { TDSE_SMALL_GRID_AUTO = 0, TDSE_SMALL_GRID_OFF = 1, TDSE_SMALL_GRID_FORCE = 2 };
int tdse_set_small_grid_path(tdse_t *h, int mode);
int tdse_small_grid_path_used(const tdse_t *h);

/*
 * Larger grids: every FP64 length-gauge Lanczos step of a tdse_propagate call
 * in one cooperative launch (Appendix "Lanczos methods"), when no per-step
 * observables are set up.  The multi-launch path issues 2 order + 1 launches
 * per step; here one grid of 2 blocks of 512 threads per SM stays resident,
 * separates the phases by grid-wide barriers (bounded waits) and has every
 * block add each reduction's block partials in the multi-launch path's fixed
 * order, so the results equal that path's bitwise.  The modes are those of
 * tdse_set_small_grid_path: FORCE takes this path at any size where the
 * device allows the cooperative launch (the small-grid path, if it applies,
 * still comes first); AUTO (default) and OFF keep the multi-launch path,
 * which is faster on the grids measured (its kernels read the Krylov vectors
 * through L1; here every read of data another block wrote goes to L2).
 * tdse_persistent_path_used returns 1 if the last tdse_propagate ran on it.
 * Errors: TDSE_ERR_ARG (unknown mode).
 */
int tdse_set_persistent_path(tdse_t *h, int mode);
int tdse_persistent_path_used(const tdse_t *h);

/* Wait for the handle's stream; reports pending TDSE_ERR_NONFINITE. */
int tdse_sync(tdse_t *h);

/*
 * Arithmetic-throughput probe (a measurement utility; the paper has no
 * counterpart): the fused multiply-add rate, in flop/s (an FMA counts 2), that
 * this GPU sustains on independent FP64 (fp64 = 1) or FP32 (fp64 = 0) chains:
 * 8 blocks of 256 threads per SM, 8 chains per thread, best of three timed
 * launches of about 20 ms after a warm-up, on cuda_stream (NULL: the legacy
 * default stream), synchronous.  The FP64 kernels of this library are bound
 * by this rate, so it measures the peak of their roofline.  Allocates
 * nothing.  Errors: TDSE_ERR_ARG (NULL output), TDSE_ERR_CUDA.
 */
int tdse_fma_throughput(int fp64, double *flops_per_s, void *cuda_stream);

/*
 * The small exponential of a Lanczos step on its own (Sec. 5 "Lanczos.c",
 * Appendix "Lanczos methods"): c = exp(-i T dt) e_1 (imag = 1: exp(-T dt) e_1)
 * for the real symmetric tridiagonal T with diagonal alpha[0..m-1] and
 * off-diagonal beta[0..m-2] (host arrays), on the GPU with the kernel body
 * every Lanczos step uses (FP32 Jacobi eigendecomposition, FP64 Ogita-Aishima
 * refinement, FP64 phases).  The Krylov space is cut at the first j with
 * beta_j <= 1e-13 max(1, max_{i<=j} |alpha_i|): *kdim (may be NULL) receives
 * the dimension kept and c_out (host, 2 m doubles, interleaved complex) the
 * coefficients, zero beyond it.  Synchronous on the legacy default stream;
 * allocates one small device buffer per call.  Errors: TDSE_ERR_ARG (m outside
 * 1..TDSE_MAX_KRYLOV, NULL arrays, dt <= 0), TDSE_ERR_OOM, TDSE_ERR_CUDA.
 */
int tdse_lanczos_expm(int m, const double *alpha, const double *beta, double dt, int imag, double *c_out,
                      int *kdim);

/* Number of kernel launches this handle has issued (for launch accounting). */
long long tdse_launch_count(const tdse_t *h);

/* Kernel kinds for per-kernel timing. */
enum {
  TDSE_K_APPLY_H = 0, TDSE_K_TAYLOR_STAGE, TDSE_K_RK_STAGE, TDSE_K_NORM, TDSE_K_LANCZOS_A,
  TDSE_K_LANCZOS_B, TDSE_K_LANCZOS_EXPM, TDSE_K_LANCZOS_COMBINE, TDSE_K_OBSERVABLES,
  TDSE_K_DIPOLE, TDSE_K_FLUX, TDSE_K_SMALL_GRID, TDSE_K_PERSISTENT, TDSE_K_COUNT
};

/*
 * Per-kernel timing: while enabled, every launch is bracketed by a pair of
 * CUDA events recorded on the handle's stream.  tdse_profile_read waits for
 * the stream and returns, for one kernel kind, the summed event time (ms) and
 * the number of launches since profiling was enabled; enable = 0 stops it,
 * enable = 1 (re)starts it with zeroed totals.  Timing adds small gaps between
 * launches, so time the throughput of a run with profiling off.
 */
int tdse_profile(tdse_t *h, int enable);
int tdse_profile_read(tdse_t *h, int kind, double *total_ms, long long *launches);

/*
 * Observables of a caller-held device state WITHOUT allocating anything.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (code running inside another component's graph
 * capture or real-time loop, where an allocation would synchronise the device
 * or break the capture, or an embedding that forbids the library from owning
 * device memory) and so cannot create a handle.
 *
 * Same quantities as tdse_observables, for the grid r_j = j*dr + offset
 * (each r_j rounded as a product, then a sum, like the handle's table):
 * out_dev (device, lmax+6 doubles, 8-byte aligned) receives
 * {norm, dipole, yield, p_ground, l_pop[0..lmax], nonfinite}, where
 * nonfinite is 1.0 when the state holds Inf or NaN (its norm sum is not
 * finite; the handle path reports this as TDSE_ERR_NONFINITE) and 0.0
 * otherwise: the call cannot return that status, since it does not wait for
 * the kernel.  psi_dev holds (lmax+1)*N
 * interleaved complex doubles (device, 16-byte aligned); ref0_dev holds the N
 * complex values of the p_ground reference (device) or is NULL (p_ground = 0).
 * The work is enqueued on cuda_stream (a cudaStream_t; NULL = legacy default
 * stream) and the call returns without waiting.
 *
 * Scratch: the block partial sums live in one fixed file-scope device array
 * (room for lmax <= TDSE_NOALLOC_MAX_LMAX, about 80 KB), which every GPU that
 * loads the library keeps until the process exits.  The first call on each
 * device looks up that array's device address; make that first call before
 * any stream capture.  All calls share the array: calls whose kernels can
 * overlap on the GPU (unordered streams) race; calls ordered on one stream
 * are safe.  Nothing is allocated or freed.
 * Errors: TDSE_ERR_ARG (N < 1, dr <= 0, r_1 <= 0, lmax < 0 or
 * lmax > TDSE_NOALLOC_MAX_LMAX, NULL or misaligned pointers), TDSE_ERR_CUDA.
 */
#define TDSE_NOALLOC_MAX_LMAX 255
int tdse_observables_noalloc(int N, double dr, int lmax, double offset, double r_b,
                             const void *psi_dev, const void *ref0_dev, double *out_dev,
                             void *cuda_stream);

/* ------------------------------------------------------------------------ */
/* Batched Lanczos propagation of many independent instances.               */
/* ------------------------------------------------------------------------ */
/*
 * One instance of a batch: its own grid, potential, pulse, absorber, Krylov
 * dimension and step.  Units and conventions as for a single handle; the
 * stencil (3 or 5) must be the same for every instance of a batch.
 */
typedef struct {
  int N;                /* radial points                                          */
  double dr;            /* grid spacing                                           */
  int lmax;             /* partial waves 0..lmax                                   */
  double Z;             /* nuclear charge of V(r) = -Z/r                           */
  double E0, omega, ncycles, cep;   /* sin^2 pulse as in tdse_set_pulse            */
  int krylov;           /* Lanczos dimension, 1..TDSE_MAX_KRYLOV                   */
  double dt;            /* step                                                   */
  double absorber_r;    /* cos^(1/8) mask for r > absorber_r; >= r_N switches it off */
  double r_b;           /* yield radius                                           */
  int gauge;            /* TDSE_GAUGE_LENGTH (0) or TDSE_GAUGE_VELOCITY (1)                   */
  int pulse_shape;      /* TDSE_PULSE_SIN2_E (0) or TDSE_PULSE_SIN2_A, as tdse_set_pulse_shape */
} tdse_instance_spec;

typedef struct tdse_batch tdse_batch_t;

/*
 * Create a batch of `count` instances advanced together by the Lanczos
 * propagator (Appendix "Lanczos methods"), in FP64 or mixed precision
 * (TDSE_FP64 / TDSE_MIXED, as for tdse_opts.precision).  Every instance starts
 * in the normalised 1s state of its grid at t = 0.  Each kernel launch covers
 * the Lanczos phase of all instances; every reduction is split into fixed
 * per-instance chunks, so an instance's results do not depend on which other
 * instances share the batch (bitwise).  All device memory is owned by the
 * batch.  In mixed precision the steps keep each state as two FP32 parts
 * (about 48 bits) and the FP64 state is formed from them, exactly, whenever
 * it is read (state and observables calls, the copies out, per-step
 * observables).  Errors: TDSE_ERR_ARG (count < 1, an invalid spec, mixed
 * stencils), TDSE_ERR_OOM, TDSE_ERR_CUDA.
 */
int tdse_batch_create(const tdse_instance_spec *specs, int count, int stencil, int precision,
                      tdse_batch_t **out);
int tdse_batch_destroy(tdse_batch_t *b);
const char *tdse_batch_last_error(const tdse_batch_t *b);
int tdse_batch_set_stream(tdse_batch_t *b, void *cuda_stream);

/* Per-instance state in / out of HOST memory ((lmax_i+1)*N_i interleaved complex). */
int tdse_batch_set_state(tdse_batch_t *b, int i, const double *F_host);
int tdse_batch_get_state(tdse_batch_t *b, int i, double *F_host);
double tdse_batch_get_time(const tdse_batch_t *b, int i);
/* Put instance i at time t (default 0): its next step starts at t, step n of
 * the following calls at t + n dt (the pulse is evaluated there).
 * Errors: TDSE_ERR_ARG (bad index, non-finite t). */
int tdse_batch_set_time(tdse_batch_t *b, int i, double t);

/* Every instance's state in / out of ONE host buffer: instance i's
 * (lmax_i+1)*N_i interleaved complex values follow instance i-1's, in
 * instance order (tdse_batch_points complex values in all).  The copies are
 * enqueued back to back and waited for once; pinned memory makes them
 * asynchronous DMA. */
int tdse_batch_set_states(tdse_batch_t *b, const double *F_all_host);
int tdse_batch_get_states(tdse_batch_t *b, double *F_all_host);

/*
 * Advance every instance by nsteps Lanczos steps of its own dt (asynchronous).
 * Errors: TDSE_ERR_ARG (nsteps < 0), TDSE_ERR_OOM, TDSE_ERR_CUDA.
 */
int tdse_batch_propagate(tdse_batch_t *b, long nsteps);

/*
 * Copy every state in, advance every instance by nsteps steps and copy every
 * state out, with the copies overlapping the compute (synchronous).  The
 * instances are cut into `groups` contiguous groups; group g is propagated
 * once its input copy is done, and its output copy runs while group g+1
 * computes, on two extra streams (one per copy direction).  Only the first
 * group's input copy and the last group's output copy are then exposed, so
 * the group sizes grow from the first group to the middle and shrink to the
 * last by a factor r, the compute time of the call over its input copy time
 * (r = 4 on a batch's first call; later calls take r from the previous call,
 * timed with events, times nsteps; r is kept within [1, 64]).  Where the
 * batch holds a wave per group, every group but a middle one is cut to a
 * whole number of waves of the stencil kernels' persistent grid (one chunk
 * of 64 row segments per warp), so that its launches end without a partial
 * last wave.
 * The input copies start once the work already queued on the batch's stream
 * is done.  F_in / F_out: host buffers laid out as tdse_batch_set_states
 * (page-locked for the copies to overlap); either may be NULL.  The
 * result equals tdse_batch_set_states + tdse_batch_propagate +
 * tdse_batch_get_states bitwise (an instance's arithmetic does not depend on
 * which instances run with it).  Errors: TDSE_ERR_ARG (nsteps < 0,
 * groups < 1), TDSE_ERR_OOM, TDSE_ERR_CUDA.
 */
int tdse_batch_propagate_io(tdse_batch_t *b, const double *F_in_host, double *F_out_host, long nsteps,
                            int groups);

/* Observables of instance i, as tdse_observables (synchronises the stream). */
int tdse_batch_observables(tdse_batch_t *b, int i, double *norm, double *l_pop, double *dipole,
                           double *yield, double *p_ground);

/*
 * Record <z>, <zdot> and <zddot> of every instance (as tdse_dipole_moments,
 * Sec. 4: Eqs. (Dipole), (DipoleVelocity), (DipoleAccel), with no ghost
 * point) after each of its steps, up to `capacity` entries per instance: one
 * extra launch per step covers the whole batch, and an instance's entries are
 * bitwise the same whatever else runs in the batch and however its steps are
 * split into calls.  Recording stops for an instance whose record is full.
 * capacity 0 turns recording off; every call discards what was recorded.
 * The record takes 32 * capacity * count bytes of device memory.
 * Errors: TDSE_ERR_ARG (capacity < 0 or too large), TDSE_ERR_OOM, TDSE_ERR_CUDA.
 */
int tdse_batch_dipole_series(tdse_batch_t *b, long capacity);
/* Instance i's entries as {t, <z>, <zdot>, <zddot>} (4 doubles each, in step
 * order): at most max_entries of them into out (may be NULL); *count (may be
 * NULL) receives the number recorded.  Synchronises the stream.
 * Errors: TDSE_ERR_ARG (bad index), TDSE_ERR_CUDA. */
int tdse_batch_dipole_series_read(tdse_batch_t *b, int i, double *out, long max_entries, long *count);

/*
 * Imaginary time (Sec. 3) for every instance of an FP64 batch: nsteps
 * Lanczos steps of dtau = the instance's dt with exp(-T dtau) in place of
 * exp(-i T dt), no field, and the state renormalised to dr sum |f|^2 = 1
 * after each step, as tdse_propagate_imag with TDSE_LANCZOS (ground states of
 * many grids at once).  The instances' times do not change.  energies (count
 * doubles, may be NULL): each instance's energy estimate of the last step,
 * -ln(||psi_new|| / ||psi_old||) / dtau (NaN before the first step); the call
 * is synchronous when it is given.  Errors: TDSE_ERR_ARG (a mixed-precision
 * batch, nsteps < 0), TDSE_ERR_CUDA.
 */
int tdse_batch_propagate_imag(tdse_batch_t *b, long nsteps, double *energies);

/*
 * Integrate the flux through the sphere r = r_b of every instance (its
 * spec's r_b; Sec. 4, Eqs. (flux), (pad), (yield)) at the same ntheta angles
 * cos_theta[k] in [-1, 1], as tdse_flux_setup: the current states open the
 * integrals at zero, and after every step one launch over the batch forms
 * each instance's flux and densities at the new state and advances their
 * trapezoid-rule time integrals.  The first derivative at r_b is the velocity
 * gauge's, with zero beyond the box.  ntheta < 0 turns it off (cos_theta
 * unused); ntheta = 0 integrates the total only.  Synchronous.
 * Errors: TDSE_ERR_ARG (an r_b outside its instance's box, a cos_theta outside
 * [-1, 1], a largest lmax above 1535), TDSE_ERR_OOM, TDSE_ERR_CUDA.
 */
int tdse_batch_flux_setup(tdse_batch_t *b, int ntheta, const double *cos_theta);
/* Instance i's flux now, its time integral (the yield through r_b), and the
 * densities now and integrated (ntheta each; any pointer may be NULL).
 * Synchronises the stream.  TDSE_ERR_ARG if the flux is not set up. */
int tdse_batch_flux_read(tdse_batch_t *b, int i, double *flux, double *yield, double *density, double *pad);

/* Total grid points of the batch and kernel launches issued (accounting).
 * tdse_batch_graph_steps: steps (of all instances together) that ran as a
 * replay of a captured step graph rather than as separate launches. */
long long tdse_batch_points(const tdse_batch_t *b);
long long tdse_batch_launch_count(const tdse_batch_t *b);
long long tdse_batch_graph_steps(const tdse_batch_t *b);

/* Per-kernel timing of a batch, as tdse_profile / tdse_profile_read (TDSE_K_* kinds). */
int tdse_batch_profile(tdse_batch_t *b, int enable);
int tdse_batch_profile_read(tdse_batch_t *b, int kind, double *total_ms, long long *launches);

/*
 * Launch schedule of the batched kernels.
 *   prefetch_rows: the rows the FP64 stencil kernel prefetches ahead into L2
 *     (0, 3, 6 or 10);
 *   ring_rows: the mixed-precision stencil kernel walks tiles of 256 radial
 *     columns x 32 partial waves, its rows brought into a ring of shared-memory
 *     slots by bulk asynchronous copies; 0, 3 or 5 selects a ring of 4, 8 or
 *     12 slots (1, 5 or 9 rows in flight beyond the three it reads);
 *   stencil_blocks_per_sm: blocks per SM of the stencil kernels (1 or 2; 3 is
 *     accepted and used by the mixed tile kernel, whose blocks are smaller);
 *   elem_blocks_per_sm: blocks per SM of the elementwise kernels (1 or 2, of
 *     512 threads).
 * Results do not depend on the schedule (bitwise): every reduction is split
 * into fixed per-instance chunks (tiles) whatever the grid.  A run is cut into segments
 * where its set of active instances changes; a segment of three or more
 * steps, or one that repeats the previous call's segment (a caller that
 * advances one step per call), runs as a captured CUDA graph of one step,
 * replayed once per step.  The batch keeps up to eight such graphs across
 * calls and replays a cached one whenever a segment's launches are the same.
 *
 * tdse_batch_autotune times every schedule on Lanczos phase 0 of the batch's
 * instances (launches whose outputs the next step recomputes, so the state is
 * untouched), keeps the fastest and returns it in *chosen (may be NULL);
 * synchronous.  tdse_batch_set_schedule installs one (TDSE_ERR_ARG outside
 * the choices above); tdse_batch_get_schedule reads the current one.
 */
typedef struct {
  int prefetch_rows;
  int ring_rows;              /* mixed precision: 0, or 3 or 5 rows staged in shared memory */
  int stencil_blocks_per_sm;
  int elem_blocks_per_sm;
} tdse_schedule;
int tdse_batch_autotune(tdse_batch_t *b, tdse_schedule *chosen);
int tdse_batch_set_schedule(tdse_batch_t *b, const tdse_schedule *s);
int tdse_batch_get_schedule(const tdse_batch_t *b, tdse_schedule *s);

/* ------------------------------------------------------------------------ */
/* Served instances: continuous batching under a device-memory budget.       */
/* ------------------------------------------------------------------------ */
/*
 * A request is one tdse_instance_spec plus a number of Lanczos steps from
 * t = 0 (the normalised 1s state of its grid), propagated as in the batch.
 * The paper has no serving layer; the server schedules many such requests
 * on one GPU:
 *   - tdse_server_create takes the whole budget at once (one device
 *     allocation of hbm_budget bytes, the arena) and at most max_resident
 *     requests resident (admitted and not yet released) at a time;
 *   - submitted requests wait in a FIFO queue; tdse_server_step first admits
 *     the head of the queue while a slot is free and the arena has a
 *     contiguous range for it (nothing overtakes the head), then advances
 *     every running request by min(k, steps left) steps, one launch per
 *     Lanczos phase over all of them (asynchronous on the server's stream);
 *   - a finished request keeps its state resident for readout until
 *     tdse_server_release, which also cancels a queued or running request.
 * A request's results are bitwise the same whatever else runs beside it and
 * however its steps are split into step batches.
 * Errors: TDSE_ERR_ARG (bad arguments, an invalid spec, a spec larger than the
 * budget, an unknown or non-resident id), TDSE_ERR_OOM, TDSE_ERR_CUDA.
 */
typedef struct tdse_server tdse_server_t;

/* Device bytes one request of this spec occupies in the arena (0 if invalid). */
unsigned long long tdse_server_instance_bytes(const tdse_instance_spec *spec, int precision);

int tdse_server_create(unsigned long long hbm_budget, int max_resident, int stencil, int precision,
                       tdse_server_t **out);
int tdse_server_destroy(tdse_server_t *s);
const char *tdse_server_last_error(const tdse_server_t *s);
int tdse_server_set_stream(tdse_server_t *s, void *cuda_stream);

/* Queue a request of nsteps >= 1 steps; *id receives its id (> 0). */
int tdse_server_submit(tdse_server_t *s, const tdse_instance_spec *spec, long nsteps, long long *id);

/* Admit what fits, then advance all running requests by up to k >= 1 steps
 * (asynchronous); *finished (may be NULL) = requests that took their last
 * step in this call. */
int tdse_server_step(tdse_server_t *s, long k, int *finished);

/* Wait for every step enqueued so far. */
int tdse_server_sync(tdse_server_t *s);

/* Ids of finished requests not reported before, oldest first: at most cap of
 * them into ids[], their number into *n; the rest are reported next time. */
int tdse_server_poll(tdse_server_t *s, long long *ids, int cap, int *n);

/* State of a request: 0 queued, 1 running, 2 finished; steps enqueued / asked. */
int tdse_server_status(const tdse_server_t *s, long long id, int *state, long *steps_done,
                       long *steps_total);

/* Observables / state of a resident request, as tdse_batch_* (synchronise). */
int tdse_server_observables(tdse_server_t *s, long long id, double *norm, double *l_pop,
                            double *dipole, double *yield, double *p_ground);
int tdse_server_get_state(tdse_server_t *s, long long id, double *F_host);

/* Drop a request (queued, running or finished) and free its slot and memory. */
int tdse_server_release(tdse_server_t *s, long long id);

typedef struct {
  long long queued, running, resident, finished_total;
  unsigned long long bytes_budget, bytes_in_use, largest_free;
  long long gp_steps;   /* grid-point steps enqueued since creation */
  long long launches;   /* kernel launches issued since creation */
} tdse_server_stats_t;
int tdse_server_stats(const tdse_server_t *s, tdse_server_stats_t *st);

/* Schedule of the server's launches, as tdse_batch_*_schedule; autotune times
 * the schedules on the requests running now (none running: nothing changes). */
int tdse_server_autotune(tdse_server_t *s, tdse_schedule *chosen);
int tdse_server_set_schedule(tdse_server_t *s, const tdse_schedule *sch);

/* Per-kernel timing, as tdse_profile / tdse_profile_read. */
int tdse_server_profile(tdse_server_t *s, int enable);
int tdse_server_profile_read(tdse_server_t *s, int kind, double *total_ms, long long *launches);

#ifdef __cplusplus
}
#endif
#endif /* TDSE_H */

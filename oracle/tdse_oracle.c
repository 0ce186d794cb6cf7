/*
 * Serial CPU oracle for the finite-difference TDSE propagation path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header or
 * table generator with the CUDA library: it builds its own grid, Hamiltonian
 * coefficients, pulse and absorber from the paper's formulas.
 *
 * Precision: REAL is `double` by default.  Compiling with -DORC_LONG_DOUBLE
 * makes every state vector, Hamiltonian coefficient and reduction `long
 * double`; that build measures the rounding floor of the double build.  The
 * pulse E(t) and the absorber mask are evaluated in double in both builds
 * (the paper evaluates them in double on the host, Sec. 5 "Pulse").
 * Build with -ffp-contract=off so x86 and Arm give bit-identical results.
 *
 * Paper map (arXiv 1308.1856):
 *   grid, stencils, block-tridiagonal H ... Sec. 2, Eqs. (tdse-radial-field),
 *                                            (tdse-potential), the 4th-order
 *                                            difference formulas, (h_matrix)
 *   box boundary (zero beyond the box) ..... Sec. 2.1 first paragraph
 *   absorber (applied as a per-step mask) .. Sec. 2.1
 *   sin^2 pulse (on E, or on A "SineA") .... Sec. 3, Eqs. (EField), (VecSinSinCosE)
 *   Taylor propagator ...................... Sec. 5 "Taylor.c", Eq. (Taylor)
 *   Runge-Kutta (classic RK4) .............. Sec. 5 "RungeKutta.c", Eq. (RKDeriv)
 *   Lanczos propagator ..................... Sec. 5 "Lanczos.c", Appendix
 *                                            "Lanczos methods"
 *   explicit RK and embedded pairs ......... Sec. "Runge-Kutta" (method list
 *                                            and the error estimate sigma)
 *   imaginary-time propagation ............. Sec. 3 (dt -> -i dtau)
 *   velocity gauge ......................... Sec. 2, Eq. (tdse-potential) (G = V)
 *                                            and Sec. 3, Eq. (VectorStep)
 *   observables ............................ Sec. 4, Eqs. (p_g), (p_b),
 *                                            (yield_1), (Norm), (Dipole)
 *   dipole velocity and acceleration ....... Sec. 4, Eqs. (DipoleVelocity),
 *                                            (DipoleAccel)
 *   radial flux, PAD and flux yield ........ Sec. 4, Eqs. (flux), (pad), (yield)
 *
 * Readings where the paper is silent or garbled (each is also listed in the
 * design notes):
 *   - grid r_j = j*h + offset, j = 1..N (the "Start = 1" setting); finite
 *     difference neighbours outside 1..N are zero ("zero ghost"), optionally
 *     the odd reflection f_{-1} = -f_{1} at the origin ("odd ghost");
 *   - the 3-point stencil is the standard (f_{j+1} - 2 f_j + f_{j-1})/h^2;
 *   - Eq. (Taylor) prints the factor -i dt/p; the Taylor series of
 *     exp(-i H dt) needs -i dt/(p+1), which is what is computed here;
 *   - Taylor and Lanczos take the field at mid-step t_n + dt/2;
 *   - the envelope of Eq. (EField) is read as sin^2(pi t / T), T = 2 pi n_c /
 *     omega, with carrier sin(omega t + phi), and E = 0 outside [0, T];
 *   - the Lanczos listing of the appendix is garbled; the standard three-term
 *     recurrence is used, without re-orthogonalisation; the Krylov space is
 *     truncated when beta_j <= 1e-13 * max(1, max|alpha|);
 *   - the small exponential exp(-i T dt) e_1 is formed from a Jacobi
 *     eigendecomposition of the real symmetric tridiagonal T;
 *   - the absorber is the mask M(r) = cos^{1/8}(pi/2 (r - r_a)/(R - r_a)) for
 *     r > r_a (R = r_N), applied once after every full step;
 *   - integrals are h * sum over grid points; p_g is |<psi_0|psi>|^2;
 *   - an embedded RK pair propagates its higher-order solution, and the S of
 *     sigma_n = sqrt(|Delta|^2 / S) counts complex entries of psi; Euler and
 *     classic RK4 have no embedded pair (sigma = 0).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORC_LONG_DOUBLE
typedef long double REAL;
#define RSQRT sqrtl
#define RFABS fabsl
#define RCOS cosl
#define RSIN sinl
#define REXP expl
#define RLOG logl
#else
typedef double REAL;
#define RSQRT sqrt
#define RFABS fabs
#define RCOS cos
#define RSIN sin
#define REXP exp
#define RLOG log
#endif

/* ------------------------------------------------------------------------ */
/* Complex numbers as a plain pair of REALs.                                 */
/* ------------------------------------------------------------------------ */
typedef struct { REAL re, im; } cplx;

static cplx c_make(REAL re, REAL im) { cplx z; z.re = re; z.im = im; return z; }
static cplx c_add(cplx a, cplx b) { return c_make(a.re + b.re, a.im + b.im); }
static cplx c_sub(cplx a, cplx b) { return c_make(a.re - b.re, a.im - b.im); }
static cplx c_scale(REAL s, cplx a) { return c_make(s * a.re, s * a.im); }
static cplx c_mul(cplx a, cplx b) {
  return c_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
/* multiplication by -i: (-i)(x + i y) = y - i x */
static cplx c_mul_minus_i(cplx a) { return c_make(a.im, -a.re); }

/* ------------------------------------------------------------------------ */
/* Public parameter structs (mirrored by the Python ctypes wrapper).         */
/* ------------------------------------------------------------------------ */
typedef struct {
  int N;               /* radial points per partial wave                      */
  int L;               /* lmax; partial waves l = 0..L                        */
  int stencil;         /* 3 or 5                                              */
  int ghost;           /* 0 = zero beyond the box, 1 = odd reflection at r=0  */
  double h;            /* grid spacing dr                                     */
  double offset;       /* constant shift of every grid point                  */
  double Z;            /* nuclear charge for V(r) = -Z/r                      */
  const double *vtable;/* optional V(r_j), length N; NULL selects -Z/r        */
  int gauge;           /* 0 = length gauge (field E), 1 = velocity gauge (A)  */
} orc_grid;

typedef struct {
  double E0;           /* peak field (a.u.); 0 = field-free                   */
  double omega;        /* carrier frequency (a.u.)                            */
  double ncycles;      /* number of carrier cycles under the envelope         */
  double cep;          /* carrier phase                                       */
  int shape;           /* 0: sin^2 envelope on E; 1: sin^2 envelope on A      */
} orc_pulse;

typedef struct {
  int on;              /* 0 = no absorber                                     */
  double r_a;          /* mask is 1 for r <= r_a, decays to r_N               */
} orc_mask;

enum { ORC_TAYLOR = 0, ORC_RK4 = 1, ORC_LANCZOS = 2 };
#define ORC_MAX_KRYLOV 64
enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_OOM = -2 };

/* ------------------------------------------------------------------------ */
/* Grid and operator coefficients, Sec. 2.                                   */
/* ------------------------------------------------------------------------ */
static REAL grid_r(const orc_grid *g, int j /* 1-based */) {
  return (REAL)j * (REAL)g->h + (REAL)g->offset;
}

static REAL potential(const orc_grid *g, int j /* 1-based */) {
  if (g->vtable) return (REAL)g->vtable[j - 1];
  return -(REAL)g->Z / grid_r(g, j);
}

/* kappa_l = k_{l,l-1}(m=0) = sqrt(l^2 / (4 l^2 - 1)), Eq. (tdse-potential). */
static REAL kappa(int l) {
  REAL ll = (REAL)l * (REAL)l;
  return RSQRT(ll / (4 * ll - 1));
}

/* Value of partial wave l at radial index j (1-based), honouring the box:
 * zero outside 1..N except the optional odd reflection f_{-1} = -f_1. */
static cplx f_at(const orc_grid *g, const cplx *F, int l, int j) {
  if (j >= 1 && j <= g->N) return F[(size_t)l * g->N + (j - 1)];
  if (g->ghost == 1 && j == -1) return c_scale(-1, F[(size_t)l * g->N + 0]);
  return c_make(0, 0);
}

/* First derivative at index j: the 4th-order formula of Sec. 2 (printed as
 * 1/(12 h^2)[...] with a garbled f_{j-1} term; read as the standard
 * [-f_{j+2} + 8 f_{j+1} - 8 f_{j-1} + f_{j-2}] / (12 h)) for the 5-point
 * stencil, [f_{j+1} - f_{j-1}] / (2 h) for the 3-point one.                 */
static cplx d1_at(const orc_grid *g, const cplx *x, int l, int j) {
  const REAL h = (REAL)g->h;
  if (g->stencil == 5) {
    cplx s = c_scale(-1, f_at(g, x, l, j + 2));
    s = c_add(s, c_scale(8, f_at(g, x, l, j + 1)));
    s = c_add(s, c_scale(-8, f_at(g, x, l, j - 1)));
    s = c_add(s, f_at(g, x, l, j - 2));
    return c_scale(1 / (12 * h), s);
  }
  return c_scale(1 / (2 * h), c_sub(f_at(g, x, l, j + 1), f_at(g, x, l, j - 1)));
}

/* Speed of light in atomic units. */
#define ORC_C_AU 137.035999084

/*
 * y = H(E) x for the length-gauge Hamiltonian of Eq. (h_matrix):
 *   diagonal blocks h_l = -1/2 d^2/dr^2 + l(l+1)/(2 r^2) + V(r)
 *   off-diagonal blocks d_{l,l+-1} = r E kappa, Eq. (tdse-radial-field) and
 *   the length-gauge coupled equation of Sec. 2.
 * The second derivative is the 5-point formula of Sec. 2 or the standard
 * 3-point formula.
 */
static void apply_H(const orc_grid *g, REAL E, const cplx *x, cplx *y) {
  const int N = g->N, L = g->L;
  const REAL h = (REAL)g->h;
  for (int l = 0; l <= L; ++l) {
    for (int j = 1; j <= N; ++j) {
      const REAL r = grid_r(g, j);
      cplx d2;
      if (g->stencil == 5) {
        /* d2f/dr2 = [-f_{j+2} + 16 f_{j+1} - 30 f_j + 16 f_{j-1} - f_{j-2}] / (12 h^2) */
        cplx s = c_scale(-1, f_at(g, x, l, j + 2));
        s = c_add(s, c_scale(16, f_at(g, x, l, j + 1)));
        s = c_add(s, c_scale(-30, f_at(g, x, l, j)));
        s = c_add(s, c_scale(16, f_at(g, x, l, j - 1)));
        s = c_add(s, c_scale(-1, f_at(g, x, l, j - 2)));
        d2 = c_scale(1 / (12 * h * h), s);
      } else {
        /* d2f/dr2 = [f_{j+1} - 2 f_j + f_{j-1}] / h^2 */
        cplx s = f_at(g, x, l, j + 1);
        s = c_add(s, c_scale(-2, f_at(g, x, l, j)));
        s = c_add(s, f_at(g, x, l, j - 1));
        d2 = c_scale(1 / (h * h), s);
      }
      const REAL centrifugal = (REAL)l * (REAL)(l + 1) / (2 * r * r);
      cplx v = c_scale(-0.5, d2);
      v = c_add(v, c_scale(centrifugal + potential(g, j), f_at(g, x, l, j)));
      if (g->gauge == 0) {
        if (l >= 1) v = c_add(v, c_scale(r * E * kappa(l), f_at(g, x, l - 1, j)));
        if (l < L) v = c_add(v, c_scale(r * E * kappa(l + 1), f_at(g, x, l + 1, j)));
      } else {
        /* velocity gauge (Sec. 2, E holds A(t)): (A/c) p_z with p_z = -i d/dz in the
         * partial-wave basis of psi = sum_l f_l(r)/r Y_l0,
         *   -i (A/c) [ (d/dr - l/r) kappa_l f_{l-1} + (d/dr + (l+1)/r) kappa_{l+1} f_{l+1} ].
         * Reading: the paper prints the l/r terms with the opposite signs; those
         * fail p_z = i[H_0, z] and gauge invariance (see the design notes). */
        cplx w = c_make(0, 0);
        if (l >= 1)
          w = c_add(w, c_scale(kappa(l), c_sub(d1_at(g, x, l - 1, j),
                                               c_scale((REAL)l / r, f_at(g, x, l - 1, j)))));
        if (l < L)
          w = c_add(w, c_scale(kappa(l + 1), c_add(d1_at(g, x, l + 1, j),
                                                   c_scale((REAL)(l + 1) / r, f_at(g, x, l + 1, j)))));
        v = c_add(v, c_mul_minus_i(c_scale(E / (REAL)ORC_C_AU, w)));
      }
      y[(size_t)l * N + (j - 1)] = v;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Pulse, Sec. 3.  Shape 0: Eq. (EField) with the Hann (sin^2) envelope on E. */
/* Shape 1 ("SineA"): the Hann envelope on A, Eq. (VecSinSinCosE):            */
/*   A(t) = -(c E0 / omega) sin^2(W t) sin(omega t + cep),  W = omega/(2 n_c), */
/*   E(t) = -(1/c) dA/dt                                                      */
/*        = (E0/omega) sin(W t) [omega sin(W t) cos(omega t + cep)            */
/*                               + 2 W cos(W t) sin(omega t + cep)].          */
/* Reading: E0 is the peak field in both shapes (the printed Eq.              */
/* (VecSinSinCosE) multiplies the bracket by E0, which makes omega E0 the     */
/* peak); A then follows from A = -c int E, the convention of Eq. (VectorStep).*/
/* ------------------------------------------------------------------------ */
double orc_field(const orc_pulse *p, double t) {
  if (p->E0 == 0.0 || p->omega <= 0.0) return 0.0;
  const double T = 2.0 * M_PI * p->ncycles / p->omega;
  if (t < 0.0 || t > T) return 0.0;
  const double env = sin(M_PI * t / T);
  if (p->shape == 1) {
    const double W = M_PI / T, ph = p->omega * t + p->cep;
    return p->E0 / p->omega * env * (p->omega * env * cos(ph) + 2.0 * W * cos(M_PI * t / T) * sin(ph));
  }
  return p->E0 * env * env * sin(p->omega * t + p->cep);
}

/*
 * Vector potential of the pulse, A(t) = -c int_0^t E(t') dt' (Sec. 3: A is
 * obtained from E by 5-point Gauss quadrature).  Reading: the integral runs
 * over fixed panels of [0, T] (the smallest number of equal panels no wider
 * than 0.25 a.u.), each by 5-point Gauss-Legendre, plus the part of the
 * panel that holds t; A(t) = A(T) for t > T and 0 for t < 0.
 */
static double gauss5(const orc_pulse *p, double a, double b) {
  static const double x[5] = {-0.9061798459386640, -0.5384693101056831, 0.0,
                              0.5384693101056831, 0.9061798459386640};
  static const double w[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889,
                              0.4786286704993665, 0.2369268850561891};
  const double m = 0.5 * (a + b), hw = 0.5 * (b - a);
  double s = 0.0;
  for (int k = 0; k < 5; ++k) s += w[k] * orc_field(p, m + hw * x[k]);
  return hw * s;
}

double orc_vecpot(const orc_pulse *p, double t) {
  if (p->E0 == 0.0 || p->omega <= 0.0 || t <= 0.0) return 0.0;
  const double T = 2.0 * M_PI * p->ncycles / p->omega;
  const double tt = t < T ? t : T;
  const long panels = (long)ceil(T / 0.25);
  const double w = T / (double)panels;
  const long full = (long)floor(tt / w);
  double s = 0.0;
  for (long k = 0; k < full && k < panels; ++k) s += gauss5(p, (double)k * w, (double)(k + 1) * w);
  if (full < panels && tt > (double)full * w) s += gauss5(p, (double)full * w, tt);
  return -ORC_C_AU * s;
}

/* Absorbing mask value at radius r (Sec. 2.1, applied as a mask). */
double orc_mask_value(const orc_mask *m, double r, double R) {
  if (!m->on || r <= m->r_a) return 1.0;
  const double x = 0.5 * M_PI * (r - m->r_a) / (R - m->r_a);
  return pow(cos(x), 0.125);
}

/* ------------------------------------------------------------------------ */
/* Helpers on whole vectors.                                                 */
/* ------------------------------------------------------------------------ */
static size_t dim(const orc_grid *g) { return (size_t)(g->L + 1) * g->N; }

static REAL vec_norm(const cplx *x, size_t n) {
  REAL s = 0;
  for (size_t i = 0; i < n; ++i) s += x[i].re * x[i].re + x[i].im * x[i].im;
  return RSQRT(s);
}

static void load_state(const double *in, cplx *out, size_t n) {
  for (size_t i = 0; i < n; ++i) out[i] = c_make((REAL)in[2 * i], (REAL)in[2 * i + 1]);
}

static void store_state(const cplx *in, double *out, size_t n) {
  for (size_t i = 0; i < n; ++i) { out[2 * i] = (double)in[i].re; out[2 * i + 1] = (double)in[i].im; }
}

/* ------------------------------------------------------------------------ */
/* Taylor propagator, Eq. (Taylor):                                          */
/*   F_{n+1} = sum_{p=0}^{P} F^{(p)},  F^{(0)} = F_n,                        */
/*   F^{(p)} = (-i dt / p) H F^{(p-1)}     (factor read as 1/p, see header)  */
/* ------------------------------------------------------------------------ */
/* imag != 0: imaginary time (Sec. 3), F^{(p)} = (-dt / p) H F^{(p-1)}.      */
static void taylor_step(const orc_grid *g, REAL E, int P, REAL dt, cplx *psi,
                        cplx *term, cplx *tmp, int imag) {
  const size_t n = dim(g);
  memcpy(term, psi, n * sizeof(cplx));
  for (int p = 1; p <= P; ++p) {
    apply_H(g, E, term, tmp);
    const REAL s = dt / (REAL)p;
    for (size_t i = 0; i < n; ++i) {
      term[i] = imag ? c_scale(-s, tmp[i]) : c_scale(s, c_mul_minus_i(tmp[i]));
      psi[i] = c_add(psi[i], term[i]);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Classic RK4, Eq. (RKDeriv) with dF/dt = -i H(t) F (Eq. (tdse_matrix)):    */
/* c = (0, 1/2, 1/2, 1), a_{21} = a_{32} = 1/2, a_{43} = 1, b = (1,2,2,1)/6. */
/* ------------------------------------------------------------------------ */
/* imag != 0: imaginary time, dF/dt = -H F.                                  */
static void rk4_step(const orc_grid *g, const REAL Ec[4], REAL dt, cplx *psi,
                     cplx *k, cplx *g_arg, cplx *acc, int imag) {
  static const REAL a_prev[4] = {0, 0.5, 0.5, 1.0};   /* a_{i,i-1}          */
  static const REAL b[4] = {1, 2, 2, 1};              /* times 1/6          */
  const size_t n = dim(g);
  for (size_t i = 0; i < n; ++i) acc[i] = c_make(0, 0);
  for (int s = 0; s < 4; ++s) {
    /* g = F_n + dt * a_{s,s-1} k_{s-1}; the classic tableau has one nonzero a per row */
    for (size_t i = 0; i < n; ++i)
      g_arg[i] = (s == 0) ? psi[i] : c_add(psi[i], c_scale(dt * a_prev[s], k[i]));
    apply_H(g, Ec[s], g_arg, k);
    for (size_t i = 0; i < n; ++i) {
      k[i] = imag ? c_scale(-1, k[i])      /* k_s = -H g (imaginary time) */
                  : c_mul_minus_i(k[i]);   /* k_s = -i H(t_n + c_s dt) g */
      acc[i] = c_add(acc[i], c_scale(b[s], k[i]));
    }
  }
  for (size_t i = 0; i < n; ++i) psi[i] = c_add(psi[i], c_scale(dt / 6, acc[i]));
}

/* ------------------------------------------------------------------------ */
/* Jacobi eigendecomposition of a small real symmetric matrix (cyclic        */
/* Jacobi rotations).  A (n x n, row major) is overwritten; eigenvalues go   */
/* to w, eigenvectors to the columns of V.                                   */
/* ------------------------------------------------------------------------ */
static void jacobi_eig(int n, REAL *A, REAL *w, REAL *V) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1 : 0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    REAL off = 0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (off == 0) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const REAL apq = A[p * n + q];
        if (apq == 0) continue;
        const REAL app = A[p * n + p], aqq = A[q * n + q];
        /* rotation angle that annihilates A[p][q] */
        const REAL theta = (aqq - app) / (2 * apq);
        const REAL t = (theta >= 0 ? 1 : -1) / (RFABS(theta) + RSQRT(theta * theta + 1));
        const REAL c = 1 / RSQRT(t * t + 1), s = t * c;
        for (int k = 0; k < n; ++k) {       /* A <- A J  (columns p, q) */
          const REAL akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {       /* A <- J^T A (rows p, q) */
          const REAL apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {       /* V <- V J */
          const REAL vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
}

/* ------------------------------------------------------------------------ */
/* Lanczos propagator, Sec. 5 "Lanczos.c" and Appendix "Lanczos methods":     */
/*   q_1 = F/||F||, beta_0 = 0, q_0 = 0                                      */
/*   for j = 1..m: w = H q_j - beta_{j-1} q_{j-1}; alpha_j = Re<q_j, w>;     */
/*                 w -= alpha_j q_j; beta_j = ||w||; q_{j+1} = w / beta_j    */
/*   F_{n+1} = ||F|| Q exp(-i T dt) e_1,  T = tridiag(beta, alpha, beta).    */
/* Returns the Krylov dimension actually used.                               */
/* ------------------------------------------------------------------------ */
/* imag != 0: F_{n+1} = ||F|| Q exp(-T dt) e_1 (imaginary time).             */
static int lanczos_step(const orc_grid *g, REAL E, int m, REAL dt, cplx *psi,
                        cplx *Q /* (m+1) * n */, cplx *w, REAL *alpha, REAL *beta, int imag) {
  const size_t n = dim(g);
  const REAL nrm = vec_norm(psi, n);
  if (nrm == 0) return 0;
  for (size_t i = 0; i < n; ++i) Q[i] = c_scale(1 / nrm, psi[i]);
  int k = m;                                   /* dimension of the space */
  REAL amax = 0;
  for (int j = 0; j < m; ++j) {
    cplx *qj = Q + (size_t)j * n;
    apply_H(g, E, qj, w);
    if (j > 0) {
      const cplx *qprev = Q + (size_t)(j - 1) * n;
      for (size_t i = 0; i < n; ++i) w[i] = c_sub(w[i], c_scale(beta[j - 1], qprev[i]));
    }
    REAL a = 0;                                /* Re <q_j, w> */
    for (size_t i = 0; i < n; ++i) a += qj[i].re * w[i].re + qj[i].im * w[i].im;
    alpha[j] = a;
    if (RFABS(a) > amax) amax = RFABS(a);
    for (size_t i = 0; i < n; ++i) w[i] = c_sub(w[i], c_scale(a, qj[i]));
    if (j == m - 1) break;                     /* beta_m is not needed */
    const REAL b = vec_norm(w, n);
    beta[j] = b;
    if (b <= (REAL)1e-13 * (amax > 1 ? amax : 1)) { k = j + 1; break; }
    cplx *qnext = Q + (size_t)(j + 1) * n;
    for (size_t i = 0; i < n; ++i) qnext[i] = c_scale(1 / b, w[i]);
  }

  /* c = exp(-i T dt) e_1 through T = V diag(lambda) V^T */
  /* k <= m <= ORC_MAX_KRYLOV, checked by the callers */
  REAL A[ORC_MAX_KRYLOV * ORC_MAX_KRYLOV], V[ORC_MAX_KRYLOV * ORC_MAX_KRYLOV];
  REAL lam[ORC_MAX_KRYLOV];
  cplx c[ORC_MAX_KRYLOV];
  memset(A, 0, sizeof(A));
  for (int i = 0; i < k; ++i) {
    A[i * k + i] = alpha[i];
    if (i + 1 < k) { A[i * k + i + 1] = beta[i]; A[(i + 1) * k + i] = beta[i]; }
  }
  jacobi_eig(k, A, lam, V);
  for (int i = 0; i < k; ++i) {
    cplx s = c_make(0, 0);
    for (int e = 0; e < k; ++e) {
      const REAL ph = -lam[e] * dt;            /* exp(-i lambda dt), or exp(-lambda dt) */
      const cplx f = imag ? c_make(REXP(ph), 0) : c_make(RCOS(ph), RSIN(ph));
      s = c_add(s, c_scale(V[i * k + e] * V[0 * k + e], f));
    }
    c[i] = s;
  }
  /* F_{n+1} = ||F|| sum_j c_j q_j */
  for (size_t i = 0; i < n; ++i) {
    cplx s = c_make(0, 0);
    for (int j = 0; j < k; ++j) s = c_add(s, c_mul(c[j], Q[(size_t)j * n + i]));
    psi[i] = c_scale(nrm, s);
  }
  return k;
}

static void apply_mask(const orc_grid *g, const orc_mask *m, cplx *psi) {
  if (!m || !m->on) return;
  const double R = (double)grid_r(g, g->N);
  for (int j = 1; j <= g->N; ++j) {
    const REAL mv = (REAL)orc_mask_value(m, (double)grid_r(g, j), R);
    if (mv == 1) continue;
    for (int l = 0; l <= g->L; ++l) {
      cplx *z = &psi[(size_t)l * g->N + (j - 1)];
      *z = c_scale(mv, *z);
    }
  }
}

static int check_grid(const orc_grid *g) {
  if (!g || g->N < 1 || g->L < 0 || g->h <= 0) return 0;
  if (g->stencil != 3 && g->stencil != 5) return 0;
  if (g->ghost != 0 && g->ghost != 1) return 0;
  if (g->gauge != 0 && g->gauge != 1) return 0;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points (double in / double out).                           */
/* ------------------------------------------------------------------------ */

/* y = H(E) x; x, y interleaved complex, length 2 (L+1) N doubles, l-major. */
int orc_apply_H(const orc_grid *g, double E, const double *x, double *y) {
  if (!check_grid(g)) return ORC_ERR_ARG;
  const size_t n = dim(g);
  cplx *X = (cplx *)malloc(n * sizeof(cplx)), *Y = (cplx *)malloc(n * sizeof(cplx));
  if (!X || !Y) { free(X); free(Y); return ORC_ERR_OOM; }
  load_state(x, X, n);
  apply_H(g, (REAL)E, X, Y);
  store_state(Y, y, n);
  free(X); free(Y);
  return ORC_OK;
}

/*
 * Advance psi (in place, interleaved complex) by nsteps steps of size dt
 * starting at time t0.  method: 0 Taylor (order = P), 1 RK4 (order ignored),
 * 2 Lanczos (order = Krylov dimension m).  The mask (if on) is applied after
 * every full step.  min_krylov (may be NULL) receives the smallest Krylov
 * dimension used by any step.
 */
int orc_propagate(const orc_grid *g, const orc_pulse *pulse, const orc_mask *mask,
                  int method, int order, double dt, double t0, long nsteps,
                  double *psi_io, int *min_krylov) {
  if (!check_grid(g) || !pulse || nsteps < 0 || !(dt > 0)) return ORC_ERR_ARG;
  if (method == ORC_TAYLOR && order < 1) return ORC_ERR_ARG;
  if (method == ORC_LANCZOS && order < 1) return ORC_ERR_ARG;
  if (method < 0 || method > 2) return ORC_ERR_ARG;
  const size_t n = dim(g);
  const int nvec = (method == ORC_LANCZOS) ? order + 3 : 4;
  cplx *buf = (cplx *)malloc((size_t)nvec * n * sizeof(cplx));
  if (!buf) return ORC_ERR_OOM;
  cplx *psi = buf, *w1 = buf + n, *w2 = buf + 2 * n, *w3 = buf + 3 * n;
  REAL alpha[ORC_MAX_KRYLOV], beta[ORC_MAX_KRYLOV];
  if (method == ORC_LANCZOS && order > ORC_MAX_KRYLOV) { free(buf); return ORC_ERR_ARG; }
  load_state(psi_io, psi, n);
  int kmin = order;
  /* the coupling's time-dependent factor: E(t) in the length gauge, A(t) in the velocity gauge */
  double (*coupling)(const orc_pulse *, double) = g->gauge ? orc_vecpot : orc_field;
  for (long s = 0; s < nsteps; ++s) {
    const double tn = t0 + (double)s * dt;
    if (method == ORC_TAYLOR) {
      taylor_step(g, (REAL)coupling(pulse, tn + 0.5 * dt), order, (REAL)dt, psi, w1, w2, 0);
    } else if (method == ORC_RK4) {
      const REAL Ec[4] = {(REAL)coupling(pulse, tn), (REAL)coupling(pulse, tn + 0.5 * dt),
                          (REAL)coupling(pulse, tn + 0.5 * dt), (REAL)coupling(pulse, tn + dt)};
      rk4_step(g, Ec, (REAL)dt, psi, w1, w2, w3, 0);
    } else {
      const int k = lanczos_step(g, (REAL)coupling(pulse, tn + 0.5 * dt), order, (REAL)dt,
                                 psi, w2 /* Q: order+1 vectors */, w1, alpha, beta, 0);
      if (k < kmin) kmin = k;
    }
    apply_mask(g, mask, psi);
  }
  store_state(psi, psi_io, n);
  if (min_krylov) *min_krylov = kmin;
  free(buf);
  return ORC_OK;
}

/*
 * Imaginary-time propagation (Sec. 3, "Imaginary time"): the same propagators
 * with -i replaced by -1 (no field, no mask).  Each step:
 *   n0 = dr sum |F|^2;  F <- P(-H dt) F;  n1 = dr sum |F|^2;
 *   E = -ln(n1 / n0) / (2 dt);  F <- F / sqrt(n1).
 * For an eigenstate of eigenvalue lambda, E is lambda (Lanczos, exactly up to
 * rounding) or -ln(T_P(-lambda dt)^2) / (2 dt) (Taylor-P; RK4 = Taylor-4).
 * energy (may be NULL) receives the last step's E.
 */
int orc_propagate_imag(const orc_grid *g, int method, int order, double dt, long nsteps,
                       double *psi_io, double *energy) {
  if (!check_grid(g) || nsteps < 0 || !(dt > 0)) return ORC_ERR_ARG;
  if (method < 0 || method > 2) return ORC_ERR_ARG;
  if (method != ORC_RK4 && order < 1) return ORC_ERR_ARG;
  if (method == ORC_LANCZOS && order > ORC_MAX_KRYLOV) return ORC_ERR_ARG;
  const size_t n = dim(g);
  const int nvec = (method == ORC_LANCZOS) ? order + 3 : 4;
  cplx *buf = (cplx *)malloc((size_t)nvec * n * sizeof(cplx));
  if (!buf) return ORC_ERR_OOM;
  cplx *psi = buf, *w1 = buf + n, *w2 = buf + 2 * n, *w3 = buf + 3 * n;
  REAL alpha[ORC_MAX_KRYLOV], beta[ORC_MAX_KRYLOV];
  const REAL zero4[4] = {0, 0, 0, 0};
  load_state(psi_io, psi, n);
  REAL e = 0;
  for (long s = 0; s < nsteps; ++s) {
    const REAL n0 = (REAL)g->h * vec_norm(psi, n) * vec_norm(psi, n);
    if (method == ORC_TAYLOR) taylor_step(g, 0, order, (REAL)dt, psi, w1, w2, 1);
    else if (method == ORC_RK4) rk4_step(g, zero4, (REAL)dt, psi, w1, w2, w3, 1);
    else lanczos_step(g, 0, order, (REAL)dt, psi, w2, w1, alpha, beta, 1);
    const REAL n1 = (REAL)g->h * vec_norm(psi, n) * vec_norm(psi, n);
    e = -RLOG(n1 / n0) / (2 * (REAL)dt);
    const REAL sc = 1 / RSQRT(n1);
    for (size_t i = 0; i < n; ++i) psi[i] = c_scale(sc, psi[i]);
  }
  store_state(psi, psi_io, n);
  if (energy) *energy = (double)e;
  free(buf);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Explicit Runge-Kutta methods of Sec. "Runge-Kutta" (Euler, classic RK4,   */
/* and the embedded pairs RKF 4(5), Cash-Karp, Dormand-Prince, Merson):      */
/*   k_i = f(t_n + c_i h, F_n + h sum_{j<i} a_ij k_j),  f = -i H(t) F,       */
/*   F^(2) = F_n + h sum b2_i k_i (higher order), F^(1) with b1 (lower),     */
/*   Delta = F^(2) - F^(1),  sigma_n = sqrt(|Delta|^2 / S),  sigma = sum.     */
/* Reading: the step keeps the higher-order solution F^(2); S is the number  */
/* of complex components of F.  Coefficients: the published tableaus         */
/* (Fehlberg 1969; Cash & Karp 1990; Dormand & Prince 1980; Merson 1957).    */
/* ------------------------------------------------------------------------ */
typedef struct {
  int s;                      /* stages */
  double c[7];
  double a[7][7];             /* a[i][j], j < i */
  double b2[7], b1[7];        /* higher and lower order weights */
} orc_tableau;

static const orc_tableau ORC_TABLEAUS[6] = {
  /* 0: Euler (no embedded pair) */
  {1, {0}, {{0}}, {1}, {1}},
  /* 1: classic RK4 (no embedded pair) */
  {4, {0, 0.5, 0.5, 1},
   {{0}, {0.5}, {0, 0.5}, {0, 0, 1}},
   {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6}},
  /* 2: Runge-Kutta-Fehlberg 4(5) */
  {6, {0, 1.0 / 4, 3.0 / 8, 12.0 / 13, 1, 1.0 / 2},
   {{0},
    {1.0 / 4},
    {3.0 / 32, 9.0 / 32},
    {1932.0 / 2197, -7200.0 / 2197, 7296.0 / 2197},
    {439.0 / 216, -8, 3680.0 / 513, -845.0 / 4104},
    {-8.0 / 27, 2, -3544.0 / 2565, 1859.0 / 4104, -11.0 / 40}},
   {16.0 / 135, 0, 6656.0 / 12825, 28561.0 / 56430, -9.0 / 50, 2.0 / 55},
   {25.0 / 216, 0, 1408.0 / 2565, 2197.0 / 4104, -1.0 / 5, 0}},
  /* 3: Cash-Karp 4(5) */
  {6, {0, 1.0 / 5, 3.0 / 10, 3.0 / 5, 1, 7.0 / 8},
   {{0},
    {1.0 / 5},
    {3.0 / 40, 9.0 / 40},
    {3.0 / 10, -9.0 / 10, 6.0 / 5},
    {-11.0 / 54, 5.0 / 2, -70.0 / 27, 35.0 / 27},
    {1631.0 / 55296, 175.0 / 512, 575.0 / 13824, 44275.0 / 110592, 253.0 / 4096}},
   {37.0 / 378, 0, 250.0 / 621, 125.0 / 594, 0, 512.0 / 1771},
   {2825.0 / 27648, 0, 18575.0 / 48384, 13525.0 / 55296, 277.0 / 14336, 1.0 / 4}},
  /* 4: Dormand-Prince 5(4) */
  {7, {0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1, 1},
   {{0},
    {1.0 / 5},
    {3.0 / 40, 9.0 / 40},
    {44.0 / 45, -56.0 / 15, 32.0 / 9},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}},
   {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0},
   {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200, 187.0 / 2100, 1.0 / 40}},
  /* 5: Merson 4("5"): fourth-order solution, third-order companion */
  {5, {0, 1.0 / 3, 1.0 / 3, 1.0 / 2, 1},
   {{0},
    {1.0 / 3},
    {1.0 / 6, 1.0 / 6},
    {1.0 / 8, 0, 3.0 / 8},
    {1.0 / 2, 0, -3.0 / 2, 2}},
   {1.0 / 6, 0, 0, 2.0 / 3, 1.0 / 6},
   {1.0 / 10, 0, 3.0 / 10, 2.0 / 5, 1.0 / 5}},
};

/*
 * Advance psi by nsteps steps of the explicit RK method `tableau` (0..5 as
 * above); the mask (if on) after every step.  sigma (may be NULL) receives
 * sum_n sigma_n over these steps.
 */
int orc_propagate_rk(const orc_grid *g, const orc_pulse *pulse, const orc_mask *mask, int tableau,
                     double dt, double t0, long nsteps, double *psi_io, double *sigma) {
  if (!check_grid(g) || !pulse || nsteps < 0 || !(dt > 0)) return ORC_ERR_ARG;
  if (tableau < 0 || tableau > 5) return ORC_ERR_ARG;
  const orc_tableau *tb = &ORC_TABLEAUS[tableau];
  const size_t n = dim(g);
  cplx *buf = (cplx *)malloc((size_t)(tb->s + 2) * n * sizeof(cplx));
  if (!buf) return ORC_ERR_OOM;
  cplx *psi = buf, *arg = buf + n, *k = buf + 2 * n;   /* k_i at k + i n */
  double (*coupling)(const orc_pulse *, double) = g->gauge ? orc_vecpot : orc_field;
  load_state(psi_io, psi, n);
  REAL sig = 0;
  for (long st = 0; st < nsteps; ++st) {
    const double tn = t0 + (double)st * dt;
    for (int i = 0; i < tb->s; ++i) {
      for (size_t q = 0; q < n; ++q) {
        cplx v = psi[q];
        for (int j = 0; j < i; ++j)
          v = c_add(v, c_scale((REAL)dt * (REAL)tb->a[i][j], k[(size_t)j * n + q]));
        arg[q] = v;
      }
      cplx *ki = k + (size_t)i * n;
      apply_H(g, (REAL)coupling(pulse, tn + tb->c[i] * dt), arg, ki);
      for (size_t q = 0; q < n; ++q) ki[q] = c_mul_minus_i(ki[q]);   /* k_i = -i H g */
    }
    REAL d2 = 0;
    for (size_t q = 0; q < n; ++q) {
      cplx hi = psi[q], delta = c_make(0, 0);
      for (int i = 0; i < tb->s; ++i) {
        const cplx ki = k[(size_t)i * n + q];
        hi = c_add(hi, c_scale((REAL)dt * (REAL)tb->b2[i], ki));
        delta = c_add(delta, c_scale((REAL)dt * ((REAL)tb->b2[i] - (REAL)tb->b1[i]), ki));
      }
      psi[q] = hi;
      d2 += delta.re * delta.re + delta.im * delta.im;
    }
    sig += RSQRT(d2 / (REAL)n);
    apply_mask(g, mask, psi);
  }
  store_state(psi, psi_io, n);
  if (sigma) *sigma = (double)sig;
  free(buf);
  return ORC_OK;
}

/*
 * Lanczos coefficients for one step from psi: alpha[0..k-1], beta[0..k-2];
 * returns k (the Krylov dimension kept), or a negative status.
 */
int orc_lanczos_coefficients(const orc_grid *g, double E, int m, const double *psi_in,
                             double *alpha_out, double *beta_out) {
  if (!check_grid(g) || m < 1 || m > ORC_MAX_KRYLOV) return ORC_ERR_ARG;
  const size_t n = dim(g);
  cplx *buf = (cplx *)malloc((size_t)(m + 3) * n * sizeof(cplx));
  if (!buf) return ORC_ERR_OOM;
  REAL alpha[ORC_MAX_KRYLOV], beta[ORC_MAX_KRYLOV];
  cplx *psi = buf, *w = buf + n, *Q = buf + 2 * n;
  load_state(psi_in, psi, n);
  const int k = lanczos_step(g, (REAL)E, m, (REAL)1e-300, psi, Q, w, alpha, beta, 0);
  for (int i = 0; i < k; ++i) alpha_out[i] = (double)alpha[i];
  for (int i = 0; i + 1 < k; ++i) beta_out[i] = (double)beta[i];
  free(buf);
  return k;
}

/*
 * Observables of Sec. 4, every integral as h * sum over grid points:
 *   out[0] norm      = h sum_l sum_j |f_{l,j}|^2
 *   out[1] dipole    = 2 sum_{l<L} kappa_{l+1} h sum_j r_j Re(conj(f_{l,j}) f_{l+1,j})  Eq. (Dipole)
 *   out[2] yield     = 1 - h sum_l sum_{r_j <= r_b} |f_{l,j}|^2                         Eq. (yield_1)
 *   out[3] p_ground  = |h sum_j conj(ref0_j) f_{0,j}|^2                                 Eq. (p_g)
 *   out[4 + l] P_l   = h sum_j |f_{l,j}|^2
 * ref0 is the l = 0 reference wave (N interleaved complex values) or NULL.
 */
int orc_observables(const orc_grid *g, const double *psi_in, const double *ref0,
                    double r_b, double *out) {
  if (!check_grid(g) || !out) return ORC_ERR_ARG;
  const size_t n = dim(g);
  cplx *F = (cplx *)malloc(n * sizeof(cplx));
  if (!F) return ORC_ERR_OOM;
  load_state(psi_in, F, n);
  const REAL h = (REAL)g->h;
  const int N = g->N, L = g->L;
  REAL norm = 0, inside = 0, dip = 0;
  for (int l = 0; l <= L; ++l) {
    REAL pl = 0;
    for (int j = 1; j <= N; ++j) {
      const cplx z = F[(size_t)l * N + (j - 1)];
      const REAL a = z.re * z.re + z.im * z.im;
      pl += a;
      if (grid_r(g, j) <= (REAL)r_b) inside += a;
    }
    out[4 + l] = (double)(h * pl);
    norm += pl;
  }
  for (int l = 0; l < L; ++l) {
    REAL s = 0;
    for (int j = 1; j <= N; ++j) {
      const cplx a = F[(size_t)l * N + (j - 1)], b = F[(size_t)(l + 1) * N + (j - 1)];
      s += grid_r(g, j) * (a.re * b.re + a.im * b.im);   /* r Re(conj(a) b) */
    }
    dip += 2 * kappa(l + 1) * h * s;
  }
  REAL pg = 0;
  if (ref0) {
    cplx ov = c_make(0, 0);
    for (int j = 1; j <= N; ++j) {
      const cplx r0 = c_make((REAL)ref0[2 * (j - 1)], -(REAL)ref0[2 * (j - 1) + 1]);
      ov = c_add(ov, c_mul(r0, F[j - 1]));
    }
    ov = c_scale(h, ov);
    pg = ov.re * ov.re + ov.im * ov.im;
  }
  out[0] = (double)(h * norm);
  out[1] = (double)dip;
  out[2] = (double)(1 - h * inside);
  out[3] = (double)pg;
  free(F);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Dipole moment, velocity and acceleration (Sec. 4, Eqs. (Dipole),          */
/* (DipoleVelocity), (DipoleAccel)) of psi at time t, m = 0:                 */
/*   <z>    = 2 sum_l kappa_{l+1} h sum_j r_j Re(f_l^* f_{l+1})              */
/*   <zdot> = 2 sum_l kappa_{l+1} h sum_j Im(f_{l+1}^* (D1 f_l - (l+1)/r f_l))*/
/*            [+ (A(t)/c) norm in the velocity gauge]                         */
/*   <zddot> = -E(t) norm - 2 Z sum_l kappa_{l+1} h sum_j Re(f_l^* f_{l+1})/r^2 */
/* D1 is the first-derivative formula of the velocity gauge (d1_at).          */
/* Readings: Eq. (DipoleVelocity) is printed without the factor 2 that        */
/* Eq. (Dipole) carries; d<z>/dt = <zdot> (Ehrenfest) needs it.  <zdot> is    */
/* the kinetic momentum, so the velocity gauge adds (A/c) norm; the paper's   */
/* -E(t) is -E(t) norm (the two agree for a normalised state).  The           */
/* acceleration form needs dV/dr: with a tabulated potential out[2] is NaN.   */
/* ------------------------------------------------------------------------ */
int orc_dipole_moments(const orc_grid *g, const orc_pulse *pulse, double t, const double *psi_in,
                       double *out) {
  if (!check_grid(g) || !pulse || !psi_in || !out) return ORC_ERR_ARG;
  const size_t n = dim(g);
  cplx *F = (cplx *)malloc(n * sizeof(cplx));
  if (!F) return ORC_ERR_OOM;
  load_state(psi_in, F, n);
  const REAL h = (REAL)g->h;
  const int N = g->N, L = g->L;
  REAL norm = 0, z = 0, pz = 0, fz = 0;
  for (int l = 0; l <= L; ++l)
    for (int j = 1; j <= N; ++j) {
      const cplx a = F[(size_t)l * N + (j - 1)];
      norm += a.re * a.re + a.im * a.im;
    }
  for (int l = 0; l < L; ++l) {
    REAL sz = 0, sp = 0, sf = 0;
    for (int j = 1; j <= N; ++j) {
      const REAL r = grid_r(g, j);
      const cplx a = F[(size_t)l * N + (j - 1)], b = F[(size_t)(l + 1) * N + (j - 1)];
      const REAL re = a.re * b.re + a.im * b.im;                 /* Re(conj(a) b) */
      const cplx w = c_sub(d1_at(g, F, l, j), c_scale((REAL)(l + 1) / r, a));
      sz += r * re;
      sp += b.re * w.im - b.im * w.re;                           /* Im(conj(b) w) */
      sf += re / (r * r);
    }
    z += 2 * kappa(l + 1) * h * sz;
    pz += 2 * kappa(l + 1) * h * sp;
    fz += 2 * kappa(l + 1) * h * sf;
  }
  norm *= h;
  out[0] = (double)z;
  out[1] = (double)(pz + (g->gauge ? (REAL)orc_vecpot(pulse, t) / (REAL)ORC_C_AU * norm : 0));
  out[2] = g->vtable ? NAN : (double)(-(REAL)orc_field(pulse, t) * norm - (REAL)g->Z * fz);
  free(F);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Flux through the sphere r = r_b (Sec. 4, Eqs. (flux), (pad), (yield)),     */
/* m = 0, psi = sum_l f_l(r)/r Y_l0:                                          */
/*   total:  r_b^2 int dOmega j_r = sum_l Im(f_l^* D1 f_l)                    */
/*                                  [+ 2 (A/c) sum_l kappa_{l+1} Re(f_l^* f_{l+1})] */
/*   angle:  r_b^2 j_r(theta) = Im(S^* P) [+ (A/c) cos(theta) |S|^2],         */
/*           S = sum_l f_l Y_l0(theta),  P = sum_l (D1 f_l) Y_l0(theta),      */
/*           Y_l0 = sqrt((2l+1)/(4 pi)) P_l(cos theta)                        */
/* at the grid point nearest r_b (the A terms in the velocity gauge only).    */
/* Readings: Eq. (flux) prints -Im; the continuity equation (outward flux     */
/* empties the inside) and Eq. (yield) need +Im.  The A term of Eq. (yield)   */
/* is complex as printed; the flux is its real part.                          */
/* ------------------------------------------------------------------------ */
static int nearest_index(const orc_grid *g, double r_b) {
  int best = 1;
  for (int j = 2; j <= g->N; ++j)
    if (RFABS(grid_r(g, j) - (REAL)r_b) < RFABS(grid_r(g, best) - (REAL)r_b)) best = j;
  return best;
}

int orc_flux(const orc_grid *g, const orc_pulse *pulse, double t, const double *psi_in, double r_b,
             int ntheta, const double *cos_theta, double *total, double *per_angle) {
  if (!check_grid(g) || !pulse || !psi_in || !total || ntheta < 0) return ORC_ERR_ARG;
  if (ntheta > 0 && (!cos_theta || !per_angle)) return ORC_ERR_ARG;
  const size_t n = dim(g);
  const int N = g->N, L = g->L;
  cplx *F = (cplx *)malloc((n + 2 * (size_t)(L + 1)) * sizeof(cplx));
  if (!F) return ORC_ERR_OOM;
  load_state(psi_in, F, n);
  cplx *fb = F + n, *db = fb + (L + 1);     /* f_l(r_b) and (D1 f_l)(r_b) */
  const int jb = nearest_index(g, r_b);
  for (int l = 0; l <= L; ++l) {
    fb[l] = F[(size_t)l * N + (jb - 1)];
    db[l] = d1_at(g, F, l, jb);
  }
  const REAL ac = g->gauge ? (REAL)orc_vecpot(pulse, t) / (REAL)ORC_C_AU : 0;
  REAL tot = 0;
  for (int l = 0; l <= L; ++l) tot += fb[l].re * db[l].im - fb[l].im * db[l].re;
  for (int l = 0; l < L; ++l)
    tot += 2 * ac * kappa(l + 1) * (fb[l].re * fb[l + 1].re + fb[l].im * fb[l + 1].im);
  *total = (double)tot;
  for (int k = 0; k < ntheta; ++k) {
    const REAL x = (REAL)cos_theta[k];
    cplx S = c_make(0, 0), P = c_make(0, 0);
    REAL pm = 0, pl = 1;                      /* P_{l-1}(x), P_l(x) */
    for (int l = 0; l <= L; ++l) {
      const REAL y = RSQRT((REAL)(2 * l + 1) / (4 * (REAL)M_PI)) * pl;
      S = c_add(S, c_scale(y, fb[l]));
      P = c_add(P, c_scale(y, db[l]));
      const REAL next = ((REAL)(2 * l + 1) * x * pl - (REAL)l * pm) / (REAL)(l + 1);   /* Bonnet */
      pm = pl;
      pl = next;
    }
    per_angle[k] = (double)(S.re * P.im - S.im * P.re + ac * x * (S.re * S.re + S.im * S.im));
  }
  free(F);
  return ORC_OK;
}

/* Precision of REAL in this build, in bytes (8 or the platform's long double). */
int orc_real_bytes(void) { return (int)sizeof(REAL); }

/*
 * pc_oracle.c -- plain, slow FP64 CPU restatement of the augmented
 * Picard-Chebyshev (PC) orbit propagator of Masat, Colombo & Boutonnet,
 * "GPU-based high-precision orbital propagation of large sets of initial
 * conditions through Picard-Chebyshev augmentation" (arXiv 2301.03989).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the oracle the CUDA library is checked
 * against.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header, table or constant
 * generator with the CUDA library, and the library never calls it.
 *
 * Precision: every state, force and error quantity is IEEE FP64, compiled
 * without fast-math and with floating-point contraction off (-ffp-contract=off),
 * so the same binary arithmetic runs on x86-64 and aarch64.  The PC operator
 * is built in long double and rounded to double once.
 *
 * Parity status per function (what pins each one, see tests/test_oracle_*.py):
 *   ora_cgl_nodes        pinned: closed form, symmetry, endpoints
 *   ora_pc_operator      pinned: exact on polynomials, Clenshaw-Curtis weights
 *   ora_ephem_eval       pinned: numpy chebval, interpolation at fit nodes,
 *                                 the later granule on a boundary
 *   ora_stop_rule        pinned: hand-derived outcomes of written-out
 *                                change sequences (tol, stall, cap, blow-up)
 *   ora_propagate_log    pinned: hand-derived attempt sequences (halve,
 *                                accept, grow back, clip at tf, backward)
 *   ora_accel            pinned: finite-difference gradient of the potential,
 *                                collinear closed form, Kepler conservation
 *   ora_kepler           pinned: Kepler's-equation residual, energy/momentum,
 *                                return after one period, scipy DOP853
 *   ora_pc_segment       pinned: constant acceleration exact, harmonic
 *                                oscillator closed form, two-body vs Kepler
 *   ora_propagate        pinned: Gauss-Legendre collocation integrator,
 *                                forward/backward, batch invariance
 *   ora_gl_*             pinned: Legendre quadrature exactness, order check
 *   ora_ephem_vel        pinned: numpy chebder/chebval, circular-orbit speed
 *   ora_tidal            pinned: finite differences of ora_accel, zero trace
 *   ora_stm_propagate    pinned: finite differences of analytic Kepler and of
 *                                ora_propagate, symplecticity, Gauss-Legendre
 *                                variational integration, composition
 *   ora_gl_stm_propagate pinned: finite differences of ora_gl_propagate
 *   ora_bplane           pinned: straight-line limit, hyperbola built from a
 *                                chosen asymptote and aim point
 *   ora_pc2_segment      pinned: constant acceleration exact, harmonic
 *                                oscillator closed form, same fixed point as
 *                                ora_pc_segment on a flyby-free segment
 *   ora_eih_terms        pinned: Schwarzschild closed form (one body at rest),
 *                                a body and a particle in uniform common motion
 *                                (the boosted rest-frame field), perihelion
 *                                advance 6 pi mu / (c^2 a (1 - e^2)), and every
 *                                term (those of the bodies' accelerations and
 *                                potentials included) against the geodesic of
 *                                the harmonic-gauge 1PN metric of the bodies
 *   order 2 of ora_pc_segment / ora_propagate
 *                        pinned: bitwise ora_pc2_segment on a segment; same
 *                                fixed point as order 1 end to end; Gauss-
 *                                Legendre; fewer sweeps
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Public structures (mirrored by oracle/oracle.py with ctypes).       */
/* ------------------------------------------------------------------ */

/* Force model: Newtonian heliocentric point masses.  Positions of the B
 * perturbing bodies come from a Chebyshev table: granule g covers
 * [t_begin + g*L, t_begin + (g+1)*L); inside it sigma = 2(t - t_g)/L - 1 and
 * r_b = sum_k c[b][g][axis][k] T_k(sigma). */
typedef struct {
  int n_bodies;
  double mu_central;      /* GM of the central body, km^3/s^2 */
  const double *mu;       /* [n_bodies] */
  int indirect;           /* 1: add the frame (indirect) term mu_b r_b/|r_b|^3 */
  double t_begin;         /* table start epoch, s */
  double granule;         /* granule length L, s */
  int degree;             /* Chebyshev degree of the table */
  int n_granules;
  const double *coef;     /* [n_bodies][n_granules][3][degree+1] */
  double c_light;         /* speed of light, km/s: > 0 adds the EIH (1PN) terms; 0 Newtonian */
} ora_model;

/* Dynamics selector (the N-body model is the method's; the other two are the
 * analytic test problems used to pin the PC machinery). */
enum { ORA_DYN_NBODY = 0, ORA_DYN_CONST_ACCEL = 1, ORA_DYN_HARMONIC = 2 };

/* Segment-attempt outcomes. */
enum { ORA_SEG_OK = 0, ORA_SEG_STALLED = 1, ORA_SEG_FAIL_CAP = 2, ORA_SEG_FAIL_DIV = 3, ORA_SEG_FAIL_TRUNC = 4 };

/* Per-trajectory status bits (0 = OK). */
enum { ORA_IC_OK = 0, ORA_IC_STALLED = 1, ORA_IC_UNRESOLVED = 2, ORA_IC_NOT_CONVERGED = 4, ORA_IC_NONFINITE = 8 };

typedef struct {
  int N;               /* Chebyshev degree; n = N + 1 CGL nodes */
  int truncated;       /* 1: drop the degree-(N+1) coefficient of the integral */
  double tol;          /* stopping tolerance on the sweep-to-sweep change */
  int relative;        /* 1: relative to |r|, |v| of the new iterate; 0: absolute */
  int max_iters;       /* sweeps per segment attempt */
  int max_depth;       /* how many times a segment may be halved */
  int warm_start;      /* 1: Kepler two-body guess; 0: every node = x0 */
  int seg_mode;        /* 0: `segments` equal segments per arc;
                          1: `segments` segments per osculating period of x0 */
  int segments;
  int stall_sweeps;    /* accept when e has not improved for this many sweeps ... */
  double stall_factor; /* ... and the best e so far is below stall_factor * tol */
  double div_limit;    /* a sweep change above this (or non-finite) fails the attempt */
  double trunc_tol;    /* resolution test on the Chebyshev tail (<= 0 disables) */
  int dyn;             /* ORA_DYN_* */
  double dyn_param[3]; /* constant acceleration vector, or omega^2 in [0] */
  int order;           /* 1: the paper's sweep; 2: the second-order form (ora_pc2_segment) */
} ora_opts;

/* ------------------------------------------------------------------ */
/* Chebyshev-Gauss-Lobatto nodes, Eq. (chnodes2) with n = N + 1 nodes:  */
/* tau_j = -cos(j pi / N), j = 0..N, so tau_0 = -1 is the segment start.*/
/* Evaluated as sin(pi (2j - N) / (2N)), the same value, so that the    */
/* nodes are exactly antisymmetric and the middle node is exactly 0.    */
/* ------------------------------------------------------------------ */
static long double ora_tau_ld(int j, int N) {
  const long double pi = 3.141592653589793238462643383279502884L;
  return sinl(pi * (long double)(2 * j - N) / (long double)(2 * N));
}

void ora_cgl_nodes(int N, double *tau) {
  for (int j = 0; j <= N; j++) tau[j] = (double)ora_tau_ld(j, N);
}

/* ------------------------------------------------------------------ */
/* PC operator.  The paper's B = [S A F + 2 y0; A F] and y = C B (Section */
/* "Matrix form for vectorized and parallel computation") fit a Chebyshev */
/* series to the node forces, integrate it once from tau = -1, and      */
/* evaluate at the nodes.  The matrices are not printed in the paper, so */
/* they are built here from their definition:                           */
/*   Fit:  a_k = (2/N) sum''_j g_j T_k(tau_j), then a_0 /= 2, a_N /= 2   */
/*         (sum'' halves the j = 0 and j = N terms) -- the interpolant.  */
/*   Int:  beta_1 = a_0 - a_2/2, beta_k = (a_{k-1} - a_{k+1})/(2k)       */
/*         for k >= 2 (a_{N+1} = a_{N+2} = 0), beta_0 = -sum_{k>=1}      */
/*         (-1)^k beta_k so the integral vanishes at tau = -1.           */
/*   Eval: y_j = sum_k beta_k T_k(tau_j).                                */
/* K = Eval * Int * Fit, so that y_j = x0 + omega2 * sum_k K_jk f_k.     */
/* truncated = 1 drops beta_{N+1} (the paper's B has only N+1 rows).     */
/* ------------------------------------------------------------------ */
void ora_pc_operator(int N, int truncated, double *K) {
  const int n = N + 1;
  const int nb = N + 2; /* beta_0 .. beta_{N+1} */
  long double *T = (long double *)malloc(sizeof(long double) * (size_t)(N + 2) * n);   /* T[k][j] */
  long double *Fit = (long double *)malloc(sizeof(long double) * (size_t)n * n);       /* a = Fit g */
  long double *Int = (long double *)calloc((size_t)nb * n, sizeof(long double));       /* beta = Int a */
  long double *IF = (long double *)calloc((size_t)nb * n, sizeof(long double));        /* Int * Fit */
  long double *tau = (long double *)malloc(sizeof(long double) * n);
  for (int j = 0; j < n; j++) tau[j] = ora_tau_ld(j, N);
  /* T_k(tau_j) by the three-term recurrence, k = 0..N+1 */
  for (int j = 0; j < n; j++) {
    T[0 * n + j] = 1.0L;
    T[1 * n + j] = tau[j];
    for (int k = 2; k <= N + 1; k++) T[k * n + j] = 2.0L * tau[j] * T[(k - 1) * n + j] - T[(k - 2) * n + j];
  }
  /* Fit */
  for (int k = 0; k < n; k++) {
    for (int j = 0; j < n; j++) {
      long double w = (j == 0 || j == N) ? 0.5L : 1.0L;
      long double v = (2.0L / (long double)N) * w * T[k * n + j];
      if (k == 0 || k == N) v *= 0.5L;
      Fit[k * n + j] = v;
    }
  }
  /* Int: rows beta_0..beta_{N+1}, columns a_0..a_N */
  /* beta_1 = a_0 - a_2 / 2 */
  Int[1 * n + 0] += 1.0L;
  if (2 <= N) Int[1 * n + 2] -= 0.5L;
  for (int k = 2; k <= N + 1; k++) {
    if (k - 1 <= N) Int[k * n + (k - 1)] += 1.0L / (2.0L * (long double)k);
    if (k + 1 <= N) Int[k * n + (k + 1)] -= 1.0L / (2.0L * (long double)k);
  }
  if (truncated)
    for (int c = 0; c < n; c++) Int[(N + 1) * n + c] = 0.0L;
  /* beta_0 = -sum_{k>=1} (-1)^k beta_k */
  for (int c = 0; c < n; c++) {
    long double s = 0.0L;
    for (int k = 1; k <= N + 1; k++) s += ((k & 1) ? -1.0L : 1.0L) * Int[k * n + c];
    Int[0 * n + c] = -s;
  }
  /* IF = Int * Fit */
  for (int r = 0; r < nb; r++)
    for (int c = 0; c < n; c++) {
      long double s = 0.0L;
      for (int m = 0; m < n; m++) s += Int[r * n + m] * Fit[m * n + c];
      IF[r * n + c] = s;
    }
  /* K = Eval * IF, Eval[j][k] = T_k(tau_j), k = 0..N+1 */
  for (int j = 0; j < n; j++)
    for (int c = 0; c < n; c++) {
      long double s = 0.0L;
      for (int k = 0; k < nb; k++) s += T[k * n + j] * IF[k * n + c];
      K[j * n + c] = (double)s;
    }
  free(T); free(Fit); free(Int); free(IF); free(tau);
}

/* ------------------------------------------------------------------ */
/* Ephemeris: Clenshaw evaluation of the table's Chebyshev series      */
/*   r_b = sum_{k=0}^{deg} c_k T_k(sigma)                                */
/* by the backward recurrence b_k = c_k + 2 sigma b_{k+1} - b_{k+2},     */
/* r_b = c_0 + sigma b_1 - b_2 (Clenshaw 1955), each operation rounded  */
/* on its own.  The paper evaluates planetary states once at the fixed  */
/* node times before the iterations (Section "Dynamics model, array     */
/* sorting, and CUDA kernel") and does not fix how the tables are       */
/* summed; Clenshaw's recurrence is the textbook evaluation of a        */
/* Chebyshev series.  A time exactly on a granule boundary uses the     */
/* later granule; times outside the table use the nearest granule.      */
/* ------------------------------------------------------------------ */
void ora_ephem_eval(const ora_model *m, double t, double *rb /* [n_bodies][3] */) {
  const int nc = m->degree + 1;
  int g = (int)floor((t - m->t_begin) / m->granule);
  if (g < 0) g = 0;
  if (g > m->n_granules - 1) g = m->n_granules - 1;
  const double tg = m->t_begin + (double)g * m->granule;
  const double sigma = 2.0 * (t - tg) / m->granule - 1.0;
  for (int b = 0; b < m->n_bodies; b++) {
    for (int ax = 0; ax < 3; ax++) {
      const double *c = m->coef + (((size_t)b * m->n_granules + g) * 3 + ax) * nc;
      double b1 = 0.0, b2 = 0.0;
      for (int k = nc - 1; k >= 1; k--) {
        double b0 = c[k] + 2.0 * sigma * b1 - b2;
        b2 = b1;
        b1 = b0;
      }
      rb[b * 3 + ax] = c[0] + sigma * b1 - b2;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Newtonian heliocentric acceleration of a massless particle:          */
/*  a = -mu_S r/|r|^3 - sum_b mu_b [ (r - r_b)/|r - r_b|^3 + r_b/|r_b|^3 ]*/
/* The second term in the bracket (the indirect term, the Sun's own     */
/* acceleration towards body b) is included when m->indirect is set.    */
/* The paper's own model is the relativistic EIH one; the Newtonian     */
/* point-mass model is the one this build propagates.                   */
/* ------------------------------------------------------------------ */
void ora_accel(const ora_model *m, const double *rb, const double r[3], double a[3]) {
  double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  double r3 = r2 * sqrt(r2);
  double k = m->mu_central / r3;
  a[0] = -k * r[0];
  a[1] = -k * r[1];
  a[2] = -k * r[2];
  for (int b = 0; b < m->n_bodies; b++) {
    const double *p = rb + 3 * b;
    double d0 = r[0] - p[0], d1 = r[1] - p[1], d2 = r[2] - p[2];
    double dd = d0 * d0 + d1 * d1 + d2 * d2;
    double kd = m->mu[b] / (dd * sqrt(dd));
    a[0] -= kd * d0;
    a[1] -= kd * d1;
    a[2] -= kd * d2;
    if (m->indirect) {
      double pp = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
      double kp = m->mu[b] / (pp * sqrt(pp));
      a[0] -= kp * p[0];
      a[1] -= kp * p[1];
      a[2] -= kp * p[2];
    }
  }
}

/* ------------------------------------------------------------------ */
/* Einstein-Infeld-Hoffmann (1PN, beta = gamma = 1) terms of the         */
/* acceleration of a massless particle at X with velocity W among nb    */
/* point masses mu_j at P_j with velocities V_j, Newtonian accelerations */
/* A_j and Newtonian potentials Phi_j = sum_{k != j} mu_k/|P_k - P_j|   */
/* (the paper's force model, Section "Dynamics model", after the        */
/* Explanatory Supplement).  With d_j = P_j - X, r_j = |d_j|, n_j =      */
/* -d_j/r_j and phi = sum_j mu_j / r_j, the 1/c^2 part is               */
/*   sum_j mu_j d_j/r_j^3 [ -4 phi - Phi_j + W.W + 2 V_j.V_j - 4 W.V_j   */
/*                          - 3/2 (n_j.V_j)^2 + 1/2 d_j.A_j ] / c^2      */
/* + sum_j mu_j/r_j^3 [ (-d_j).(4 W - 3 V_j) ] (W - V_j) / c^2           */
/* + 7/2 sum_j mu_j A_j / r_j / c^2;                                     */
/* the Newtonian part sum_j mu_j d_j/r_j^3 is not included.  Positions  */
/* enter only as differences, velocities in the barycentric frame.     */
/* ------------------------------------------------------------------ */
void ora_eih_terms(int nb, const double *mu, const double *P, const double *V, const double *A, const double *Phi,
                   const double X[3], const double W[3], double c, double out[3]) {
  const double c2 = c * c;
  double phi = 0.0;
  for (int j = 0; j < nb; j++) {
    const double d0 = P[3 * j] - X[0], d1 = P[3 * j + 1] - X[1], d2 = P[3 * j + 2] - X[2];
    phi += mu[j] / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  }
  const double ww = W[0] * W[0] + W[1] * W[1] + W[2] * W[2];
  out[0] = out[1] = out[2] = 0.0;
  for (int j = 0; j < nb; j++) {
    const double *Pj = P + 3 * j, *Vj = V + 3 * j, *Aj = A + 3 * j;
    const double d[3] = {Pj[0] - X[0], Pj[1] - X[1], Pj[2] - X[2]};
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r = sqrt(r2), r3 = r2 * r;
    const double vv = Vj[0] * Vj[0] + Vj[1] * Vj[1] + Vj[2] * Vj[2];
    const double wv = W[0] * Vj[0] + W[1] * Vj[1] + W[2] * Vj[2];
    const double nv = -(d[0] * Vj[0] + d[1] * Vj[1] + d[2] * Vj[2]) / r;
    const double da = d[0] * Aj[0] + d[1] * Aj[1] + d[2] * Aj[2];
    const double br = -4.0 * phi - Phi[j] + ww + 2.0 * vv - 4.0 * wv - 1.5 * nv * nv + 0.5 * da;
    double sdot = 0.0;
    for (int q = 0; q < 3; q++) sdot += -d[q] * (4.0 * W[q] - 3.0 * Vj[q]);
    for (int q = 0; q < 3; q++)
      out[q] += (mu[j] * d[q] / r3 * br + mu[j] / r3 * sdot * (W[q] - Vj[q]) + 3.5 * mu[j] * Aj[q] / r) / c2;
  }
}

void ora_ephem_vel(const ora_model *m, double t, double *vb);

/* EIH terms of the model at time t for the heliocentric state y: the Sun
 * (body 0, at the heliocentric origin) and the table's bodies, velocities
 * shifted to the barycentre by V_S = -sum_b mu_b v_b / (mu_S + sum_b mu_b),
 * Newtonian accelerations and potentials of every body from the others.
 * Added to the Newtonian heliocentric acceleration (which already carries the
 * Sun's Newtonian acceleration as the indirect term) this is the barycentric
 * EIH acceleration minus the Sun's Newtonian barycentric acceleration. */
static void ora_eih_model(const ora_model *m, double t, const double *rb, const double y[6], double out[3]) {
  const int B = m->n_bodies, nb = B + 1;
  double mu[33], P[99], V[99], A[99], Phi[33], vb[96];
  if (B > 0) ora_ephem_vel(m, t, vb);
  double msum = m->mu_central, vs[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < B; b++) {
    msum += m->mu[b];
    for (int q = 0; q < 3; q++) vs[q] -= m->mu[b] * vb[3 * b + q];
  }
  for (int q = 0; q < 3; q++) vs[q] /= msum;
  mu[0] = m->mu_central;
  for (int q = 0; q < 3; q++) {
    P[q] = 0.0;
    V[q] = vs[q];
  }
  for (int b = 0; b < B; b++) {
    mu[b + 1] = m->mu[b];
    for (int q = 0; q < 3; q++) {
      P[3 * (b + 1) + q] = rb[3 * b + q];
      V[3 * (b + 1) + q] = vb[3 * b + q] + vs[q];
    }
  }
  for (int j = 0; j < nb; j++) {
    Phi[j] = 0.0;
    for (int q = 0; q < 3; q++) A[3 * j + q] = 0.0;
    for (int k = 0; k < nb; k++) {
      if (k == j) continue;
      const double d[3] = {P[3 * k] - P[3 * j], P[3 * k + 1] - P[3 * j + 1], P[3 * k + 2] - P[3 * j + 2]};
      const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r = sqrt(r2);
      Phi[j] += mu[k] / r;
      for (int q = 0; q < 3; q++) A[3 * j + q] += mu[k] * d[q] / (r2 * r);
    }
  }
  const double W[3] = {y[3] + vs[0], y[4] + vs[1], y[5] + vs[2]};
  ora_eih_terms(nb, mu, P, V, A, Phi, y, W, m->c_light, out);
}

/* Public: the model's EIH terms at t (tests). */
void ora_eih_at(const ora_model *m, double t, const double y[6], double out[3]) {
  double rb[96];
  if (m->n_bodies > 0) ora_ephem_eval(m, t, rb);
  ora_eih_model(m, t, rb, y, out);
}

/* First-order dynamics f(y, t) = (v, a) of Eq. (ibvp); rb holds the bodies'
 * positions at t. */
static void ora_f(const ora_model *m, const ora_opts *o, double t, const double *rb, const double y[6],
                  double f[6]) {
  f[0] = y[3];
  f[1] = y[4];
  f[2] = y[5];
  if (o->dyn == ORA_DYN_NBODY) {
    ora_accel(m, rb, y, f + 3);
    if (m->c_light > 0.0) {
      double e[3];
      ora_eih_model(m, t, rb, y, e);
      for (int q = 0; q < 3; q++) f[3 + q] += e[q];
    }
  } else if (o->dyn == ORA_DYN_CONST_ACCEL) {
    f[3] = o->dyn_param[0];
    f[4] = o->dyn_param[1];
    f[5] = o->dyn_param[2];
  } else { /* harmonic oscillator x'' = -w^2 x */
    f[3] = -o->dyn_param[0] * y[0];
    f[4] = -o->dyn_param[0] * y[1];
    f[5] = -o->dyn_param[0] * y[2];
  }
}

/* Public wrapper of f for tests. */
void ora_dynamics(const ora_model *m, const ora_opts *o, double t, const double y[6], double f[6]) {
  double *rb = NULL;
  if (o->dyn == ORA_DYN_NBODY && m->n_bodies > 0) {
    rb = (double *)malloc(sizeof(double) * 3 * m->n_bodies);
    ora_ephem_eval(m, t, rb);
  }
  ora_f(m, o, t, rb, y, f);
  free(rb);
}

/* ------------------------------------------------------------------ */
/* Keplerian two-body propagation, used as the warm start ("Keplerian   */
/* initial guess", Sections "Integration concept" and "Matrix form").   */
/* Kepler's equation is written for the change of eccentric anomaly x   */
/* over dt (Battin's form), which has no singularity at e = 0 or i = 0:  */
/*   n dt = x - (1 - r0/a) sin x + (sigma0/sqrt(a)) (1 - cos x),        */
/*   sigma0 = r0.v0/sqrt(mu),                                            */
/* and solved by Newton's method safeguarded by bisection on the        */
/* bracket [n dt - 2, n dt + 2] that always holds the root.  The state  */
/* follows from the Lagrange f and g functions.                          */
/* Returns 0 on success, 1 for a non-elliptic orbit, 2 if Newton failed. */
/* ------------------------------------------------------------------ */
int ora_kepler(double mu, const double x0[6], double dt, double x[6]) {
  const double *r = x0, *v = x0 + 3;
  double r0 = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double rv = r[0] * v[0] + r[1] * v[1] + r[2] * v[2];
  double alpha = 2.0 / r0 - v2 / mu; /* 1/a */
  if (!(alpha > 0.0)) return 1;
  double a = 1.0 / alpha;
  double sa = sqrt(a);
  double sigma0 = rv / sqrt(mu);
  double ec = 1.0 - r0 / a;   /* e cos E0 */
  double es = sigma0 / sa;    /* e sin E0 */
  double nmean = sqrt(mu / (a * a * a));
  double M = nmean * dt;
  double lo = M - 2.0, hi = M + 2.0, xk = M;
  int ok = 0;
  for (int it = 0; it < 100; it++) {
    double s = sin(xk), c = cos(xk);
    double F = xk - ec * s + es * (1.0 - c) - M;
    if (F > 0.0) hi = xk; else lo = xk;
    double dF = 1.0 - ec * c + es * s;
    double xn = xk - F / dF;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    double step = fabs(xn - xk);
    xk = xn;
    if (step <= 1e-15 * (1.0 + fabs(xk))) { ok = 1; break; }
  }
  if (!ok) return 2;
  double c = cos(xk), s = sin(xk);
  double rr = a + (r0 - a) * c + sigma0 * sa * s;
  double f = 1.0 - a / r0 * (1.0 - c);
  double g = a * sigma0 / sqrt(mu) * (1.0 - c) + r0 * sqrt(a / mu) * s;
  double fd = -sqrt(mu * a) / (rr * r0) * s;
  double gd = 1.0 - a / rr * (1.0 - c);
  for (int i = 0; i < 3; i++) {
    x[i] = f * r[i] + g * v[i];
    x[3 + i] = fd * r[i] + gd * v[i];
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Resolution test.  The paper stops on the sweep-to-sweep change only,  */
/* which a segment too long for its degree also passes (the iteration   */
/* converges to the fixed point of an under-resolved interpolant).  The  */
/* last two Chebyshev coefficients of the force fit estimate the         */
/* interpolation error; with T_N(tau_j) = (-1)^(N+j) and                 */
/* T_{N-1}(tau_j) = (-1)^(N+j) tau_j on the CGL nodes they are           */
/*   a_N     = (1/N) sum''_j (-1)^(N+j) g_j,                              */
/*   a_{N-1} = (2/N) sum''_j (-1)^(N+j) tau_j g_j.                        */
/* The integral's error is then about 2|omega2| (|a_{N-1}| + |a_N|); it  */
/* is measured against max_j |r_j| for the position components (whose   */
/* derivatives are g_0..g_2) and max_j |v_j| for the velocity ones       */
/* (relative mode; raw values in absolute mode).  Returns the larger.    */
/* ------------------------------------------------------------------ */
static double ora_tail(const ora_opts *o, const double *G, const double *Y, int N, const double *tau, double w2) {
  const int n = N + 1;
  double tailc[6];
  for (int c = 0; c < 6; c++) {
    double sN = 0.0, sN1 = 0.0;
    for (int j = 0; j < n; j++) {
      double w = (j == 0 || j == N) ? 0.5 : 1.0;
      double sg = ((N + j) & 1) ? -1.0 : 1.0;
      sN += w * sg * G[6 * j + c];
      sN1 += w * sg * tau[j] * G[6 * j + c];
    }
    double aN = sN / (double)N, aN1 = 2.0 * sN1 / (double)N;
    tailc[c] = 2.0 * fabs(w2) * (fabs(aN1) + fabs(aN));
  }
  double er = 0.0, ev = 0.0, rmax = 0.0, vmax = 0.0;
  for (int c = 0; c < 3; c++) {
    if (!(tailc[c] <= er)) er = tailc[c];
    if (!(tailc[3 + c] <= ev)) ev = tailc[3 + c];
  }
  if (o->relative) {
    for (int j = 0; j < n; j++) {
      const double *y = Y + 6 * j;
      double nr = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
      double nv = sqrt(y[3] * y[3] + y[4] * y[4] + y[5] * y[5]);
      if (nr > rmax) rmax = nr;
      if (nv > vmax) vmax = nv;
    }
    if (rmax > 0.0) er /= rmax;
    if (vmax > 0.0) ev /= vmax;
  }
  return er > ev ? er : ev;
}

/* Public: tail estimate of a force table G [n][6] (tests). */
double ora_tail_estimate(const ora_opts *o, const double *G, const double *Y, double w2) {
  double *tau = (double *)malloc(sizeof(double) * (o->N + 1));
  ora_cgl_nodes(o->N, tau);
  double r = ora_tail(o, G, Y, o->N, tau, w2);
  free(tau);
  return r;
}

/* ------------------------------------------------------------------ */
/* Stop rule of a segment attempt, applied after sweep `sweep` (1-based) */
/* with change e.  The paper stops when the change drops below the      */
/* tolerance (Section "Matrix form", stopping criterion); it leaves the */
/* cap and stagnation unstated, so this restatement adds, in this order:*/
/*   e non-finite or above div_limit   -> ORA_SEG_FAIL_DIV              */
/*   e < tol (strict)                  -> ORA_SEG_OK                    */
/*   e not below the best change so far for stall_sweeps sweeps in a    */
/*   row while that best is below stall_factor * tol -> ORA_SEG_STALLED */
/*   sweep == max_iters                -> ORA_SEG_FAIL_CAP              */
/*   otherwise -1 (sweep again).                                        */
/* A change equal to the best counts as no improvement.  st carries the */
/* best change and the count between calls; start it at {INFINITY, 0}.  */
/* ------------------------------------------------------------------ */
typedef struct {
  double e_best;
  int nstall;
} ora_stop_state;

int ora_stop_rule(const ora_opts *o, ora_stop_state *st, double e, int sweep) {
  if (!(e <= o->div_limit)) return ORA_SEG_FAIL_DIV;
  if (e < o->tol) return ORA_SEG_OK;
  if (e < st->e_best) {
    st->e_best = e;
    st->nstall = 0;
  } else {
    st->nstall++;
  }
  if (st->nstall >= o->stall_sweeps && st->e_best < o->stall_factor * o->tol) return ORA_SEG_STALLED;
  if (sweep >= o->max_iters) return ORA_SEG_FAIL_CAP;
  return -1;
}

/* ------------------------------------------------------------------ */
/* One PC segment for one trajectory: the Picard iteration of Eq. (2) in */
/* the matrix form of the paper (order 1), or its second-order form       */
/* (order 2: V' = v0 + omega2 K A(Y), R' = r0 + omega2 K V'; the stop,    */
/* stall and resolution rules are the same, the resolution test on the   */
/* force table of the iterate the sweep started from).                   */
/* Order 1: */
/* the matrix form of the paper with the operator K built above.        */
/*   t_j = omega1 + omega2 tau_j, omega1 = (tb+ta)/2, omega2 = (tb-ta)/2 */
/*   y^(0)_j: warm (Kepler) or cold (x0) start                           */
/*   sweep i: g_j = f(y^(i-1)_j, t_j);  y^(i)_j = x0 + omega2 sum_k K_jk g_k */
/*   e_i = max_j max(|dr_j|/|r_j|, |dv_j|/|v_j|)   (relative mode,       */
/*         norms of the new iterate; per-state maximum of the position   */
/*         and velocity errors as in Section "CPU-GPU cooperated         */
/*         iteration error computation"), or without the denominators  */
/*         in absolute mode.  A zero norm falls back to the absolute one.*/
/* Stops on e_i < tol (OK), on a stall (no improvement for stall_sweeps  */
/* sweeps while the best e is below stall_factor*tol: accepted), on a   */
/* non-finite or huge e (FAIL_DIV) or at max_iters (FAIL_CAP).  An       */
/* accepted segment whose Chebyshev tail exceeds trunc_tol is reported  */
/* as FAIL_TRUNC (under-resolved).                                       */
/* Y holds the last iterate, [n][6].  ephem: [n][n_bodies][3] or NULL.   */
/* ------------------------------------------------------------------ */
static int ora_pc_segment_core(const ora_model *m, const ora_opts *o, const double *K, const double *tau,
                               double ta, double tb, const double x0[6], double *Y, double *G, double *Ynew,
                               double *tj, double *ephem, int *iters_out, double *err_out) {
  const int N = o->N, n = N + 1, B = (o->dyn == ORA_DYN_NBODY) ? m->n_bodies : 0;
  const double w1 = 0.5 * (tb + ta), w2 = 0.5 * (tb - ta);
  for (int j = 0; j < n; j++) tj[j] = w1 + w2 * tau[j];
  if (B > 0)
    for (int j = 0; j < n; j++) ora_ephem_eval(m, tj[j], ephem + (size_t)j * B * 3);
  /* initial guess */
  for (int j = 0; j < n; j++) {
    int bad = 1;
    if (o->warm_start && o->dyn == ORA_DYN_NBODY) bad = ora_kepler(m->mu_central, x0, tj[j] - ta, Y + 6 * j);
    if (bad)
      for (int c = 0; c < 6; c++) Y[6 * j + c] = x0[c];
  }
  for (int c = 0; c < 6; c++) Y[c] = x0[c];
  double e = INFINITY;
  ora_stop_state st = {INFINITY, 0};
  int outcome = ORA_SEG_FAIL_CAP, i;
  for (i = 1; i <= o->max_iters; i++) {
    for (int j = 0; j < n; j++) ora_f(m, o, tj[j], B ? ephem + (size_t)j * B * 3 : NULL, Y + 6 * j, G + 6 * j);
    if (o->order == 2) {
      /* second-order form: velocities from the integrated accelerations, then
         positions from the integrated new velocities (as ora_pc2_segment) */
      for (int j = 0; j < n; j++)
        for (int c = 3; c < 6; c++) {
          double s = 0.0;
          for (int k = 0; k < n; k++) s += K[j * n + k] * G[6 * k + c];
          Ynew[6 * j + c] = x0[c] + w2 * s;
        }
      for (int j = 0; j < n; j++)
        for (int c = 0; c < 3; c++) {
          double s = 0.0;
          for (int k = 0; k < n; k++) s += K[j * n + k] * Ynew[6 * k + 3 + c];
          Ynew[6 * j + c] = x0[c] + w2 * s;
        }
    } else {
      for (int j = 0; j < n; j++) {
        for (int c = 0; c < 6; c++) {
          double s = 0.0;
          for (int k = 0; k < n; k++) s += K[j * n + k] * G[6 * k + c];
          Ynew[6 * j + c] = x0[c] + w2 * s;
        }
      }
    }
    e = 0.0;
    for (int j = 0; j < n; j++) {
      const double *yn = Ynew + 6 * j, *yo = Y + 6 * j;
      double dr = sqrt((yn[0] - yo[0]) * (yn[0] - yo[0]) + (yn[1] - yo[1]) * (yn[1] - yo[1]) +
                       (yn[2] - yo[2]) * (yn[2] - yo[2]));
      double dv = sqrt((yn[3] - yo[3]) * (yn[3] - yo[3]) + (yn[4] - yo[4]) * (yn[4] - yo[4]) +
                       (yn[5] - yo[5]) * (yn[5] - yo[5]));
      if (o->relative) {
        double nr = sqrt(yn[0] * yn[0] + yn[1] * yn[1] + yn[2] * yn[2]);
        double nv = sqrt(yn[3] * yn[3] + yn[4] * yn[4] + yn[5] * yn[5]);
        if (nr > 0.0) dr = dr / nr;
        if (nv > 0.0) dv = dv / nv;
      }
      double ej = dr > dv ? dr : dv;
      if (!(ej <= e)) e = ej; /* propagates NaN */
    }
    int out = ora_stop_rule(o, &st, e, i);
    /* resolution test on an accepted segment: the force table of this sweep
       against the norms of the iterate it was evaluated on (Y, not yet updated) */
    if ((out == ORA_SEG_OK || out == ORA_SEG_STALLED) && o->trunc_tol > 0.0 &&
        !(ora_tail(o, G, Y, N, tau, w2) <= o->trunc_tol))
      out = ORA_SEG_FAIL_TRUNC;
    memcpy(Y, Ynew, sizeof(double) * 6 * n);
    if (out >= 0) { outcome = out; break; }
  }
  if (i > o->max_iters) i = o->max_iters;
  if (iters_out) *iters_out = i;
  if (err_out) *err_out = e;
  return outcome;
}

/* Public single-segment entry (tests): Y [n][6] out. */
int ora_pc_segment(const ora_model *m, const ora_opts *o, double ta, double tb, const double x0[6], double *Y,
                   int *iters, double *err) {
  const int n = o->N + 1, B = (o->dyn == ORA_DYN_NBODY) ? m->n_bodies : 0;
  double *K = (double *)malloc(sizeof(double) * n * n);
  double *tau = (double *)malloc(sizeof(double) * n);
  double *G = (double *)malloc(sizeof(double) * 6 * n);
  double *Yn = (double *)malloc(sizeof(double) * 6 * n);
  double *tj = (double *)malloc(sizeof(double) * n);
  double *eph = (double *)malloc(sizeof(double) * (size_t)n * (B > 0 ? B : 1) * 3);
  ora_pc_operator(o->N, o->truncated, K);
  ora_cgl_nodes(o->N, tau);
  int r = ora_pc_segment_core(m, o, K, tau, ta, tb, x0, Y, G, Yn, tj, eph, iters, err);
  free(K); free(tau); free(G); free(Yn); free(tj); free(eph);
  return r;
}

/* ------------------------------------------------------------------ */
/* Whole arc for one trajectory: piecewise PC "orbit by orbit in        */
/* sequence" (Section "Matrix form", footnote: forward or backward).    */
/* Segment schedule: base length h = |tf - t0| / segments (seg_mode 0)  */
/* or T_osc / segments with T_osc the osculating two-body period of x0   */
/* (seg_mode 1; uniform fallback if x0 is not elliptic).  Positions are */
/* counted in units u = h / 2^max_depth: a segment at depth d starting  */
/* at integer position p spans [t0 + s p u, t0 + s (p + 2^(D-d)) u],    */
/* s = sign(tf - t0), clipped to end exactly at tf.  A failed attempt   */
/* halves the segment (d + 1); an accepted one advances p and lets the  */
/* next segment grow one level (d - 1, not below 0).                    */
/* ------------------------------------------------------------------ */
typedef struct {
  const ora_model *m;
  const ora_opts *o;
  const double *K, *tau;
  double t0, tf;
  const double *x0;
  double *xf;
  int *status, *iters, *nseg;
  int max_ckpt;
  double *ckpt;
  int max_log;         /* attempt log of one trajectory (tests), or 0 */
  double *log;         /* [max_log][5] = (ta, tb, outcome, sweeps, depth) */
  int *n_log;          /* attempts made (may exceed max_log) */
  long begin, end;
} ora_job;

static void ora_one_ic(const ora_job *J, long ic) {
  const ora_model *m = J->m;
  const ora_opts *o = J->o;
  const int n = o->N + 1, B = (o->dyn == ORA_DYN_NBODY) ? m->n_bodies : 0;
  double *Y = (double *)malloc(sizeof(double) * 6 * n);
  double *G = (double *)malloc(sizeof(double) * 6 * n);
  double *Yn = (double *)malloc(sizeof(double) * 6 * n);
  double *tj = (double *)malloc(sizeof(double) * n);
  double *eph = (double *)malloc(sizeof(double) * (size_t)n * (B > 0 ? B : 1) * 3);
  double x[6];
  for (int c = 0; c < 6; c++) x[c] = J->x0[ic * 6 + c];
  const double t0 = J->t0, tf = J->tf;
  const double total = fabs(tf - t0);
  const double sgn = (tf >= t0) ? 1.0 : -1.0;
  double h = total / (double)o->segments;
  if (o->seg_mode == 1 && o->dyn == ORA_DYN_NBODY) {
    double r0 = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    double v2 = x[3] * x[3] + x[4] * x[4] + x[5] * x[5];
    double alpha = 2.0 / r0 - v2 / m->mu_central;
    if (alpha > 0.0) {
      double a = 1.0 / alpha;
      h = 2.0 * M_PI * sqrt(a * a * a / m->mu_central) / (double)o->segments;
    }
  }
  const int D = o->max_depth;
  const double u = ldexp(h, -D);
  long long p = 0;
  int depth = 0, status = ORA_IC_OK, sweeps = 0, nseg = 0;
  int finite_in = 1;
  for (int c = 0; c < 6; c++) if (!isfinite(x[c])) finite_in = 0;
  if (!finite_in) status |= ORA_IC_NONFINITE;
  while (finite_in && total > 0.0) {
    long long L = 1LL << (D - depth);
    double ta = t0 + sgn * ((double)p * u);
    double tb;
    int last = 0;
    if ((double)(p + L) * u >= total) { tb = tf; last = 1; }
    else tb = t0 + sgn * ((double)(p + L) * u);
    if (J->ckpt && nseg < J->max_ckpt) {
      double *ck = J->ckpt + ((size_t)ic * J->max_ckpt + nseg) * 7;
      ck[0] = ta;
      for (int c = 0; c < 6; c++) ck[1 + c] = x[c];
    }
    int it = 0;
    double err = 0.0;
    int r = ora_pc_segment_core(m, o, J->K, J->tau, ta, tb, x, Y, G, Yn, tj, eph, &it, &err);
    sweeps += it;
    if (J->n_log) {
      if (*J->n_log < J->max_log) {
        double *lg = J->log + (size_t)(*J->n_log) * 5;
        lg[0] = ta; lg[1] = tb; lg[2] = (double)r; lg[3] = (double)it; lg[4] = (double)depth;
      }
      (*J->n_log)++;
    }
    int accept = (r == ORA_SEG_OK || r == ORA_SEG_STALLED);
    if (r == ORA_SEG_FAIL_TRUNC && depth >= D) { accept = 1; status |= ORA_IC_UNRESOLVED; }
    if (accept) {
      if (r == ORA_SEG_STALLED) status |= ORA_IC_STALLED;
      for (int c = 0; c < 6; c++) x[c] = Y[6 * (n - 1) + c];
      nseg++;
      p += L;
      if (depth > 0) depth--;
      if (last) break;
    } else {
      depth++;
      if (depth > D) { status |= (r == ORA_SEG_FAIL_DIV) ? ORA_IC_NONFINITE : ORA_IC_NOT_CONVERGED; break; }
    }
  }
  for (int c = 0; c < 6; c++) J->xf[ic * 6 + c] = x[c];
  if (J->status) J->status[ic] = status;
  if (J->iters) J->iters[ic] = sweeps;
  if (J->nseg) J->nseg[ic] = nseg;
  free(Y); free(G); free(Yn); free(tj); free(eph);
}

static void *ora_worker(void *arg) {
  ora_job *J = (ora_job *)arg;
  for (long ic = J->begin; ic < J->end; ic++) ora_one_ic(J, ic);
  return NULL;
}

/* Propagates n_ic independent trajectories x0 [n_ic][6] from t0 to tf.
 * The augmented system of the paper stacks trajectories as columns; its
 * columns never interact, so the oracle runs them one by one (optionally on
 * n_threads host threads over contiguous chunks).  ckpt, if not NULL, gets
 * [n_ic][max_ckpt][7] = (t_a, x_a) at the start of every accepted segment. */
void ora_propagate(const ora_model *m, const ora_opts *o, long n_ic, const double *x0, double t0, double tf,
                   double *xf, int *status, int *iters, int *nseg, int max_ckpt, double *ckpt, int n_threads) {
  const int n = o->N + 1;
  double *K = (double *)malloc(sizeof(double) * n * n);
  double *tau = (double *)malloc(sizeof(double) * n);
  ora_pc_operator(o->N, o->truncated, K);
  ora_cgl_nodes(o->N, tau);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n_ic) n_threads = (int)(n_ic > 0 ? n_ic : 1);
  ora_job *jobs = (ora_job *)calloc((size_t)n_threads, sizeof(ora_job));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  for (int w = 0; w < n_threads; w++) {
    ora_job *J = &jobs[w];
    J->m = m; J->o = o; J->K = K; J->tau = tau; J->t0 = t0; J->tf = tf; J->x0 = x0; J->xf = xf;
    J->status = status; J->iters = iters; J->nseg = nseg; J->max_ckpt = max_ckpt; J->ckpt = ckpt;
    J->begin = n_ic * w / n_threads;
    J->end = n_ic * (w + 1) / n_threads;
  }
  if (n_threads == 1) {
    ora_worker(&jobs[0]);
  } else {
    for (int w = 0; w < n_threads; w++) pthread_create(&th[w], NULL, ora_worker, &jobs[w]);
    for (int w = 0; w < n_threads; w++) pthread_join(th[w], NULL);
  }
  free(jobs); free(th); free(K); free(tau);
}

/* One trajectory with its attempt log (tests of the segment schedule): */
/* log[k] = (t_a, t_b, outcome ORA_SEG_*, sweeps, depth) of the k-th     */
/* segment attempt, for k < max_log; *n_log = attempts made.  Same       */
/* schedule and results as ora_propagate.                                */
void ora_propagate_log(const ora_model *m, const ora_opts *o, const double x0[6], double t0, double tf, double xf[6],
                       int *status, int *iters, int *nseg, int max_log, double *log, int *n_log) {
  const int n = o->N + 1;
  double *K = (double *)malloc(sizeof(double) * n * n);
  double *tau = (double *)malloc(sizeof(double) * n);
  ora_pc_operator(o->N, o->truncated, K);
  ora_cgl_nodes(o->N, tau);
  ora_job J;
  memset(&J, 0, sizeof(J));
  J.m = m; J.o = o; J.K = K; J.tau = tau; J.t0 = t0; J.tf = tf; J.x0 = x0; J.xf = xf;
  J.status = status; J.iters = iters; J.nseg = nseg;
  J.max_log = max_log; J.log = log; J.n_log = n_log;
  *n_log = 0;
  ora_one_ic(&J, 0);
  free(K); free(tau);
}

/* ------------------------------------------------------------------ */
/* Independent check integrator: s-stage Gauss-Legendre collocation     */
/* Runge-Kutta (order 2s).  Not part of the paper's method; it exists   */
/* to pin the PC oracle on small cases.  Its coefficients are computed  */
/* here: the nodes c_i = (1 + x_i)/2 from the roots x_i of the Legendre */
/* polynomial P_s (Newton iteration on the three-term recurrence), the  */
/* stage weights a_ij = int_0^{c_i} L_j and b_j = int_0^1 L_j of the    */
/* Lagrange basis L_j on the nodes (exact polynomial integration).      */
/* ------------------------------------------------------------------ */
void ora_gl_coeffs(int s, double *c_out, double *A_out, double *b_out) {
  const long double pi = 3.141592653589793238462643383279502884L;
  long double x[16], c[16];
  for (int i = 0; i < s; i++) {
    long double z = cosl(pi * ((long double)i + 0.75L) / ((long double)s + 0.5L));
    for (int it = 0; it < 100; it++) {
      long double p0 = 1.0L, p1 = z;
      for (int k = 2; k <= s; k++) {
        long double p2 = ((2.0L * k - 1.0L) * z * p1 - (k - 1.0L) * p0) / (long double)k;
        p0 = p1;
        p1 = p2;
      }
      /* p1 = P_s(z), p0 = P_{s-1}(z); P_s' = s (z P_s - P_{s-1}) / (z^2 - 1) */
      long double dp = (long double)s * (z * p1 - p0) / (z * z - 1.0L);
      long double dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    x[i] = z;
  }
  for (int i = 0; i < s; i++) c[s - 1 - i] = (1.0L + x[i]) / 2.0L; /* ascending */
  for (int j = 0; j < s; j++) {
    /* coefficients of L_j(t) = prod_{m != j} (t - c_m)/(c_j - c_m), power basis */
    long double poly[17] = {0};
    poly[0] = 1.0L;
    int deg = 0;
    for (int mm = 0; mm < s; mm++) {
      if (mm == j) continue;
      long double den = c[j] - c[mm];
      long double np[17] = {0};
      for (int q = 0; q <= deg; q++) {
        np[q + 1] += poly[q] / den;
        np[q] += -c[mm] * poly[q] / den;
      }
      deg++;
      for (int q = 0; q <= deg; q++) poly[q] = np[q];
    }
    /* b_j = int_0^1 L_j, a_ij = int_0^{c_i} L_j */
    long double bj = 0.0L;
    for (int q = 0; q <= deg; q++) bj += poly[q] / (long double)(q + 1);
    b_out[j] = (double)bj;
    for (int i = 0; i < s; i++) {
      long double acc = 0.0L, pw = c[i];
      for (int q = 0; q <= deg; q++) {
        acc += poly[q] * pw / (long double)(q + 1);
        pw *= c[i];
      }
      A_out[i * s + j] = (double)acc;
    }
  }
  for (int i = 0; i < s; i++) c_out[i] = (double)c[i];
}

/* Fixed-step Gauss-Legendre propagation of one state over [t0, tf] in
 * nsteps steps; implicit stages solved by fixed-point iteration until the
 * stage derivatives stop changing (or 200 iterations).  Returns the number
 * of steps whose stage iteration hit the cap. */
int ora_gl_propagate(const ora_model *m, const ora_opts *o, int s, const double x0[6], double t0, double tf,
                     long nsteps, double xf[6]) {
  double c[16], A[256], b[16];
  ora_gl_coeffs(s, c, A, b);
  const int B = (o->dyn == ORA_DYN_NBODY) ? m->n_bodies : 0;
  double *rb = (double *)malloc(sizeof(double) * 3 * (B > 0 ? B : 1));
  double Kst[16][6], Kn[16][6], y[6], ys[6];
  for (int q = 0; q < 6; q++) y[q] = x0[q];
  const double h = (tf - t0) / (double)nsteps;
  int capped = 0;
  for (long st = 0; st < nsteps; st++) {
    const double tn = t0 + (double)st * h;
    if (B) ora_ephem_eval(m, tn, rb);
    double f0[6];
    ora_f(m, o, tn, rb, y, f0);
    for (int i = 0; i < s; i++)
      for (int q = 0; q < 6; q++) Kst[i][q] = f0[q];
    int it;
    for (it = 0; it < 200; it++) {
      double chg = 0.0, scl = 0.0;
      for (int i = 0; i < s; i++) {
        for (int q = 0; q < 6; q++) {
          double acc = 0.0;
          for (int j = 0; j < s; j++) acc += A[i * s + j] * Kst[j][q];
          ys[q] = y[q] + h * acc;
        }
        if (B) ora_ephem_eval(m, tn + c[i] * h, rb);
        ora_f(m, o, tn + c[i] * h, rb, ys, Kn[i]);
      }
      for (int i = 0; i < s; i++)
        for (int q = 0; q < 6; q++) {
          double d = fabs(Kn[i][q] - Kst[i][q]);
          if (d > chg) chg = d;
          if (fabs(Kn[i][q]) > scl) scl = fabs(Kn[i][q]);
          Kst[i][q] = Kn[i][q];
        }
      if (chg <= 1e-17 * scl) break;
    }
    if (it == 200) capped++;
    for (int q = 0; q < 6; q++) {
      double acc = 0.0;
      for (int j = 0; j < s; j++) acc += b[j] * Kst[j][q];
      y[q] = y[q] + h * acc;
    }
  }
  for (int q = 0; q < 6; q++) xf[q] = y[q];
  free(rb);
  return capped;
}

/* ================================================================== */
/* Differentiation (reverse-mode checks).  None of this is in the paper */
/* (its Conclusions name gradient-based trajectory optimisation as the  */
/* use of a fast propagator); these routines give the derivatives the   */
/* adjoint sweep of the CUDA library is checked against.                */
/* ================================================================== */

/* ------------------------------------------------------------------ */
/* Body velocities from the ephemeris table: the time derivative of the */
/* Chebyshev series of ora_ephem_eval,                                  */
/*   dr_b/dt = (2/L) sum_{k>=1} c_k T_k'(sigma),  T_k' = k U_{k-1},     */
/* U the Chebyshev polynomials of the second kind (U_0 = 1, U_1 = 2s,   */
/* U_{k+1} = 2s U_k - U_{k-1}).  The b-plane needs the planet-relative  */
/* velocity; the force itself needs positions only.  Same granule rule  */
/* as ora_ephem_eval.  Degrees above 63 are not supported (zeros).      */
/* ------------------------------------------------------------------ */
void ora_ephem_vel(const ora_model *m, double t, double *vb /* [n_bodies][3] */) {
  const int nc = m->degree + 1;
  int g = (int)floor((t - m->t_begin) / m->granule);
  if (g < 0) g = 0;
  if (g > m->n_granules - 1) g = m->n_granules - 1;
  const double tg = m->t_begin + (double)g * m->granule;
  const double sigma = 2.0 * (t - tg) / m->granule - 1.0;
  double U[64];
  for (int b = 0; b < m->n_bodies; b++)
    for (int ax = 0; ax < 3; ax++) vb[b * 3 + ax] = 0.0;
  if (nc > 64) return;
  U[0] = 1.0;
  if (nc > 1) U[1] = 2.0 * sigma;
  for (int k = 2; k < nc; k++) U[k] = 2.0 * sigma * U[k - 1] - U[k - 2];
  for (int b = 0; b < m->n_bodies; b++) {
    for (int ax = 0; ax < 3; ax++) {
      const double *c = m->coef + (((size_t)b * m->n_granules + g) * 3 + ax) * nc;
      double s = 0.0;
      for (int k = 1; k < nc; k++) s += c[k] * (double)k * U[k - 1];
      vb[b * 3 + ax] = s * 2.0 / m->granule;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Gravity gradient A = da/dr of ora_accel (row-major 3x3; the indirect */
/* term does not depend on r):                                          */
/*   A = -mu_S (I/|r|^3 - 3 r r^T/|r|^5)                                 */
/*       - sum_b mu_b (I/|d|^3 - 3 d d^T/|d|^5),   d = r - r_b.          */
/* ------------------------------------------------------------------ */
static void ora_add_point_gradient(double mu, const double d[3], double A[9]) {
  double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double dn = sqrt(d2);
  double i3 = 1.0 / (d2 * dn);
  double i5 = i3 / d2;
  for (int p = 0; p < 3; p++)
    for (int q = 0; q < 3; q++) A[3 * p + q] -= mu * ((p == q ? i3 : 0.0) - 3.0 * d[p] * d[q] * i5);
}

void ora_tidal(const ora_model *m, const double *rb, const double r[3], double A[9]) {
  for (int i = 0; i < 9; i++) A[i] = 0.0;
  ora_add_point_gradient(m->mu_central, r, A);
  for (int b = 0; b < m->n_bodies; b++) {
    const double d[3] = {r[0] - rb[3 * b], r[1] - rb[3 * b + 1], r[2] - rb[3 * b + 2]};
    ora_add_point_gradient(m->mu[b], d, A);
  }
}

/* Variational equations of the N-body dynamics: z = (y, Phi), Phi the   */
/* 6x6 state transition matrix (row-major), dPhi/dt = F(y) Phi with      */
/* F = [[0, I], [A(r), 0]].                                               */
static void ora_f_var(const ora_model *m, const double *rb, const double z[42], double fz[42]) {
  fz[0] = z[3];
  fz[1] = z[4];
  fz[2] = z[5];
  ora_accel(m, rb, z, fz + 3);
  double A[9];
  ora_tidal(m, rb, z, A);
  const double *P = z + 6;
  double *dP = fz + 6;
  for (int col = 0; col < 6; col++) {
    for (int q = 0; q < 3; q++) dP[q * 6 + col] = P[(3 + q) * 6 + col];
    for (int q = 0; q < 3; q++) {
      double s = 0.0;
      for (int p = 0; p < 3; p++) s += A[3 * q + p] * P[p * 6 + col];
      dP[(3 + q) * 6 + col] = s;
    }
  }
}

/* ------------------------------------------------------------------ */
/* The PC iteration of Eq. 2 on the variational equations, over a given */
/* segment schedule tb[0] < tb[1] < ... < tb[nseg] (or decreasing), with */
/* no halving: on segment k the 42 components z = (y, Phi) start from    */
/* (x_k, Phi_k) and every sweep is z_j = z_0 + omega2 sum_k K_jk f(z_k).  */
/* Node times, operator and the Kepler warm start of y are those of      */
/* ora_pc_segment_core; Phi starts as Phi_k at every node.  A segment    */
/* stops when the state change (the measure of ora_pc_segment_core) is  */
/* below tol and the STM change max_j |dPhi_j|_F / |Phi_j|_F is too; or  */
/* when the larger of the two has not improved for stall_sweeps sweeps   */
/* while its best is below stall_factor*tol; or at max_iters.  Since the */
/* y part is the state iteration and the Phi part is its linearisation   */
/* at the same nodes, Phi is the derivative of the converged discrete    */
/* map x0 -> xf.  Returns the number of segments that hit max_iters.    */
/* ------------------------------------------------------------------ */
int ora_stm_propagate(const ora_model *m, const ora_opts *o, const double x0[6], int nseg, const double *tb,
                      double xf[6], double Phi[36], int *sweeps_out) {
  const int N = o->N, n = N + 1, B = m->n_bodies;
  double *K = (double *)malloc(sizeof(double) * n * n);
  double *tau = (double *)malloc(sizeof(double) * n);
  double *Z = (double *)malloc(sizeof(double) * 42 * n);
  double *Zn = (double *)malloc(sizeof(double) * 42 * n);
  double *G = (double *)malloc(sizeof(double) * 42 * n);
  double *eph = (double *)malloc(sizeof(double) * (size_t)n * (B > 0 ? B : 1) * 3);
  ora_pc_operator(N, o->truncated, K);
  ora_cgl_nodes(N, tau);
  double z0[42];
  for (int c = 0; c < 6; c++) z0[c] = x0[c];
  for (int i = 0; i < 36; i++) z0[6 + i] = (i % 7 == 0) ? 1.0 : 0.0;
  int capped = 0, sweeps = 0;
  for (int k = 0; k < nseg; k++) {
    const double ta = tb[k], tbb = tb[k + 1];
    const double w1 = 0.5 * (tbb + ta), w2 = 0.5 * (tbb - ta);
    for (int j = 0; j < n; j++) {
      const double t = w1 + w2 * tau[j];
      if (B > 0) ora_ephem_eval(m, t, eph + (size_t)j * B * 3);
      double *z = Z + 42 * j;
      for (int c = 0; c < 42; c++) z[c] = z0[c];
      if (j > 0 && o->warm_start) {
        double y[6];
        if (ora_kepler(m->mu_central, z0, t - ta, y) == 0)
          for (int c = 0; c < 6; c++) z[c] = y[c];
      }
    }
    double best = INFINITY;
    int nstall = 0, done = 0, it;
    for (it = 1; it <= o->max_iters && !done; it++) {
      for (int j = 0; j < n; j++) ora_f_var(m, B ? eph + (size_t)j * B * 3 : NULL, Z + 42 * j, G + 42 * j);
      for (int j = 0; j < n; j++)
        for (int c = 0; c < 42; c++) {
          double s = 0.0;
          for (int q = 0; q < n; q++) s += K[j * n + q] * G[42 * q + c];
          Zn[42 * j + c] = z0[c] + w2 * s;
        }
      double ey = 0.0, ep = 0.0;
      for (int j = 0; j < n; j++) {
        const double *a = Zn + 42 * j, *b = Z + 42 * j;
        double dr = 0.0, dv = 0.0, nr = 0.0, nv = 0.0, dp = 0.0, np = 0.0;
        for (int c = 0; c < 3; c++) {
          dr += (a[c] - b[c]) * (a[c] - b[c]);
          nr += a[c] * a[c];
          dv += (a[3 + c] - b[3 + c]) * (a[3 + c] - b[3 + c]);
          nv += a[3 + c] * a[3 + c];
        }
        for (int c = 6; c < 42; c++) {
          dp += (a[c] - b[c]) * (a[c] - b[c]);
          np += a[c] * a[c];
        }
        dr = sqrt(dr); dv = sqrt(dv); dp = sqrt(dp);
        if (o->relative) {
          if (nr > 0.0) dr /= sqrt(nr);
          if (nv > 0.0) dv /= sqrt(nv);
        }
        if (np > 0.0) dp /= sqrt(np);
        double e = dr > dv ? dr : dv;
        if (!(e <= ey)) ey = e;
        if (!(dp <= ep)) ep = dp;
      }
      memcpy(Z, Zn, sizeof(double) * 42 * n);
      double e = ey > ep ? ey : ep;
      if (ey < o->tol && ep < o->tol) {
        done = 1;
      } else {
        if (e < best) { best = e; nstall = 0; } else { nstall++; }
        if (nstall >= o->stall_sweeps && best < o->stall_factor * o->tol) done = 1;
      }
    }
    sweeps += it - 1;
    if (!done) capped++;
    for (int c = 0; c < 42; c++) z0[c] = Z[42 * (n - 1) + c];
  }
  for (int c = 0; c < 6; c++) xf[c] = z0[c];
  for (int i = 0; i < 36; i++) Phi[i] = z0[6 + i];
  if (sweeps_out) *sweeps_out = sweeps;
  free(K); free(tau); free(Z); free(Zn); free(G); free(eph);
  return capped;
}

/* Gauss-Legendre collocation (the integrator of ora_gl_propagate) on the */
/* variational equations: an independent check of ora_stm_propagate.      */
int ora_gl_stm_propagate(const ora_model *m, int s, const double x0[6], double t0, double tf, long nsteps,
                         double xf[6], double Phi[36]) {
  double c[16], A[256], b[16];
  ora_gl_coeffs(s, c, A, b);
  const int B = m->n_bodies;
  double *rb = (double *)malloc(sizeof(double) * 3 * (B > 0 ? B : 1));
  double (*Kst)[42] = malloc(sizeof(double) * 16 * 42);
  double (*Kn)[42] = malloc(sizeof(double) * 16 * 42);
  double y[42], ys[42];
  for (int q = 0; q < 6; q++) y[q] = x0[q];
  for (int i = 0; i < 36; i++) y[6 + i] = (i % 7 == 0) ? 1.0 : 0.0;
  const double h = (tf - t0) / (double)nsteps;
  int capped = 0;
  for (long st = 0; st < nsteps; st++) {
    const double tn = t0 + (double)st * h;
    if (B) ora_ephem_eval(m, tn, rb);
    double f0[42];
    ora_f_var(m, rb, y, f0);
    for (int i = 0; i < s; i++)
      for (int q = 0; q < 42; q++) Kst[i][q] = f0[q];
    int it;
    for (it = 0; it < 200; it++) {
      double chg = 0.0, scl = 0.0;
      for (int i = 0; i < s; i++) {
        for (int q = 0; q < 42; q++) {
          double acc = 0.0;
          for (int j = 0; j < s; j++) acc += A[i * s + j] * Kst[j][q];
          ys[q] = y[q] + h * acc;
        }
        if (B) ora_ephem_eval(m, tn + c[i] * h, rb);
        ora_f_var(m, rb, ys, Kn[i]);
      }
      for (int i = 0; i < s; i++)
        for (int q = 0; q < 42; q++) {
          double d = fabs(Kn[i][q] - Kst[i][q]);
          if (d > chg) chg = d;
          if (fabs(Kn[i][q]) > scl) scl = fabs(Kn[i][q]);
          Kst[i][q] = Kn[i][q];
        }
      if (chg <= 1e-17 * scl) break;
    }
    if (it == 200) capped++;
    for (int q = 0; q < 42; q++) {
      double acc = 0.0;
      for (int j = 0; j < s; j++) acc += b[j] * Kst[j][q];
      y[q] = y[q] + h * acc;
    }
  }
  for (int q = 0; q < 6; q++) xf[q] = y[q];
  for (int i = 0; i < 36; i++) Phi[i] = y[6 + i];
  free(rb); free(Kst); free(Kn);
  return capped;
}

/* ------------------------------------------------------------------ */
/* b-plane coordinates of a flyby (the paper cites Valsecchi's b-plane   */
/* for close approaches and prints no formula).  From the planet-relative */
/* state rel = (r, v) and the planet's GM mu:                            */
/*   h = r x v,  e_vec = ((v^2 - mu/|r|) r - (r.v) v)/mu,  e = |e_vec|,  */
/*   P = e_vec/e,  Q = (h/|h|) x P,                                       */
/*   S = P/e + sqrt(e^2 - 1)/e Q   (direction of the incoming asymptote), */
/*   T = S x z / |S x z|  (z = (0, 0, 1), the pole of the reference plane),*/
/*   R = S x T,  B = S x h / v_inf,  v_inf = sqrt(v^2 - 2 mu/|r|),         */
/* and out = (B.T, B.R).  Returns 1 (out = 0) if the orbit is not         */
/* hyperbolic.                                                            */
/* ------------------------------------------------------------------ */
static void ora_cross(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

int ora_bplane(double mu, const double rel[6], double out[2]) {
  const double *r = rel, *v = rel + 3;
  out[0] = out[1] = 0.0;
  double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double rv = r[0] * v[0] + r[1] * v[1] + r[2] * v[2];
  double vinf2 = v2 - 2.0 * mu / rn;
  if (!(vinf2 > 0.0)) return 1;
  double vinf = sqrt(vinf2);
  double h[3], ev[3], P[3], Q[3], S[3], T[3], R[3], Bv[3], hh[3];
  ora_cross(r, v, h);
  double hn = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
  for (int i = 0; i < 3; i++) ev[i] = ((v2 - mu / rn) * r[i] - rv * v[i]) / mu;
  double e = sqrt(ev[0] * ev[0] + ev[1] * ev[1] + ev[2] * ev[2]);
  if (!(e > 1.0)) return 1;
  for (int i = 0; i < 3; i++) { P[i] = ev[i] / e; hh[i] = h[i] / hn; }
  ora_cross(hh, P, Q);
  double se = sqrt(e * e - 1.0) / e;
  for (int i = 0; i < 3; i++) S[i] = P[i] / e + se * Q[i];
  const double z[3] = {0.0, 0.0, 1.0};
  ora_cross(S, z, T);
  double tn = sqrt(T[0] * T[0] + T[1] * T[1] + T[2] * T[2]);
  for (int i = 0; i < 3; i++) T[i] /= tn;
  ora_cross(S, T, R);
  ora_cross(S, h, Bv);
  for (int i = 0; i < 3; i++) Bv[i] /= vinf;
  out[0] = Bv[0] * T[0] + Bv[1] * T[1] + Bv[2] * T[2];
  out[1] = Bv[0] * R[0] + Bv[1] * R[1] + Bv[2] * R[2];
  return 0;
}

/* ------------------------------------------------------------------ */
/* Second-order form of the Picard iteration (groundwork for the        */
/* second-order PC the paper names as a further gain, after Junkins et   */
/* al. 2013; not used by the CUDA library).  For r'' = a(r, v, t) the    */
/* velocity nodes come from the integral of the acceleration interpolant */
/* and the position nodes from the integral of the interpolant of those  */
/* new velocities, with the same operator K:                             */
/*   V' = v0 + omega2 K A(R, V),   R' = r0 + omega2 K V'.                 */
/* Same node times, warm start, stopping rule (the state change of       */
/* ora_pc_segment_core), stall rule and cap; no resolution test.         */
/* Returns the outcome (ORA_SEG_*); Y [n][6] holds the last iterate.     */
/* ------------------------------------------------------------------ */
int ora_pc2_segment(const ora_model *m, const ora_opts *o, double ta, double tb, const double x0[6], double *Y,
                    int *iters, double *err) {
  const int N = o->N, n = N + 1, B = (o->dyn == ORA_DYN_NBODY) ? m->n_bodies : 0;
  double *K = (double *)malloc(sizeof(double) * n * n);
  double *tau = (double *)malloc(sizeof(double) * n);
  double *A = (double *)malloc(sizeof(double) * 3 * n);
  double *Yn = (double *)malloc(sizeof(double) * 6 * n);
  double *eph = (double *)malloc(sizeof(double) * (size_t)n * (B > 0 ? B : 1) * 3);
  ora_pc_operator(N, o->truncated, K);
  ora_cgl_nodes(N, tau);
  const double w1 = 0.5 * (tb + ta), w2 = 0.5 * (tb - ta);
  for (int j = 0; j < n; j++) {
    const double t = w1 + w2 * tau[j];
    if (B > 0) ora_ephem_eval(m, t, eph + (size_t)j * B * 3);
    int bad = 1;
    if (o->warm_start && o->dyn == ORA_DYN_NBODY) bad = ora_kepler(m->mu_central, x0, t - ta, Y + 6 * j);
    if (bad)
      for (int c = 0; c < 6; c++) Y[6 * j + c] = x0[c];
  }
  for (int c = 0; c < 6; c++) Y[c] = x0[c];
  double e = INFINITY;
  ora_stop_state st = {INFINITY, 0};
  int outcome = ORA_SEG_FAIL_CAP, i;
  for (i = 1; i <= o->max_iters; i++) {
    for (int j = 0; j < n; j++) {
      double f[6];
      ora_f(m, o, w1 + w2 * tau[j], B ? eph + (size_t)j * B * 3 : NULL, Y + 6 * j, f);
      for (int c = 0; c < 3; c++) A[3 * j + c] = f[3 + c];
    }
    for (int j = 0; j < n; j++)      /* velocities from the accelerations */
      for (int c = 0; c < 3; c++) {
        double s = 0.0;
        for (int k = 0; k < n; k++) s += K[j * n + k] * A[3 * k + c];
        Yn[6 * j + 3 + c] = x0[3 + c] + w2 * s;
      }
    for (int j = 0; j < n; j++)      /* positions from the new velocities */
      for (int c = 0; c < 3; c++) {
        double s = 0.0;
        for (int k = 0; k < n; k++) s += K[j * n + k] * Yn[6 * k + 3 + c];
        Yn[6 * j + c] = x0[c] + w2 * s;
      }
    e = 0.0;
    for (int j = 0; j < n; j++) {
      const double *yn = Yn + 6 * j, *yo = Y + 6 * j;
      double dr = sqrt((yn[0] - yo[0]) * (yn[0] - yo[0]) + (yn[1] - yo[1]) * (yn[1] - yo[1]) +
                       (yn[2] - yo[2]) * (yn[2] - yo[2]));
      double dv = sqrt((yn[3] - yo[3]) * (yn[3] - yo[3]) + (yn[4] - yo[4]) * (yn[4] - yo[4]) +
                       (yn[5] - yo[5]) * (yn[5] - yo[5]));
      if (o->relative) {
        double nr = sqrt(yn[0] * yn[0] + yn[1] * yn[1] + yn[2] * yn[2]);
        double nv = sqrt(yn[3] * yn[3] + yn[4] * yn[4] + yn[5] * yn[5]);
        if (nr > 0.0) dr = dr / nr;
        if (nv > 0.0) dv = dv / nv;
      }
      double ej = dr > dv ? dr : dv;
      if (!(ej <= e)) e = ej;
    }
    memcpy(Y, Yn, sizeof(double) * 6 * n);
    int out = ora_stop_rule(o, &st, e, i);
    if (out >= 0) { outcome = out; break; }
  }
  if (i > o->max_iters) i = o->max_iters;
  if (iters) *iters = i;
  if (err) *err = e;
  free(K); free(tau); free(A); free(Yn); free(eph);
  return outcome;
}

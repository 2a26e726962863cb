/*
 * Plain, slow, FP64 CPU oracle of the fractional Adams-Bashforth-Moulton
 * (ABM) predictor-corrector of Diethelm, Ford and Freed, as stated in
 * "Parallel simulations for Fractional-Order Systems" (arXiv 1611.08678),
 * Section 2 (eq. (1) problem, eq. (2) predictor, the unnumbered corrector and
 * the weight definitions that follow it).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  The product path (the
 * CUDA library and its Python binding) never calls it and shares no code,
 * header, table or helper with it.
 *
 * What it computes, step by step, in the paper's order and notation:
 *   h_hat = h^alpha, g = 1/Gamma(alpha+2)
 *   b_m   = ((m+1)^alpha - m^alpha) / Gamma(alpha+1)              (Sec. 2)
 *   a_m   = ((m+2)^(alpha+1) - 2(m+1)^(alpha+1) + m^(alpha+1)) / Gamma(alpha+2)
 *   c_m   = (m^(alpha+1) - (m-alpha)(m+1)^alpha) / Gamma(alpha+2)
 *   F_0   = f(0, y_0)
 *   for n = 0..N-1:
 *     y^P_{n+1} = y_0 + h_hat * sum_{k=0..n} b_{n-k} F_k                (eq. 2)
 *     y_{n+1}   = y_0 + h_hat * (c_n F_0 + sum_{k=1..n} a_{n-k} F_k
 *                                + g * f(t_{n+1}, y^P_{n+1}))         (corrector)
 *     F_{n+1}   = f(t_{n+1}, y_{n+1}),  t_n = n h
 * Readings of the paper where it is garbled or silent:
 *   - the printed b_n has a '+' between the two powers; it is read as '-',
 *     the product-rectangle weight (the '+' version does not reduce to the
 *     rectangle rule at alpha = 1 and is not the integral of the kernel);
 *   - oracle_solve and oracle_solve_pecm take alpha in (0, 1], where the
 *     Taylor sum of eq. (2) is y_0 alone; oracle_solve_ext takes the general
 *     problem of eq. (1): alpha in (0, 2] with the initial derivative y'(0)
 *     in the Taylor sum where ceil(alpha) = 2, and one order per component;
 *   - one corrector pass per step (PECE), F_k evaluated at the corrected y_k.
 * The weights are evaluated from the plain definitions in binary128
 * (__float128 on x86-64, long double on AArch64 Linux, both IEEE quad) and
 * rounded once to FP64, so large-lag cancellation does not reach FP64.
 * All sums run in FP64 in index order.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#if defined(__x86_64__) || defined(__i386__)
#include <quadmath.h>
typedef __float128 qreal;
#define QPOW powq
#define QGAMMA tgammaq
#else
typedef long double qreal;
#define QPOW powl
#define QGAMMA tgammal
_Static_assert(LDBL_MANT_DIG == 113, "oracle needs IEEE binary128 long double on this platform");
#endif

/* ---- system catalogue (right-hand sides f, Jacobians, parameter derivatives) ----
 * Ids are local to the oracle; the Python wrapper maps system names to them. */
enum { OR_LINEAR = 0, OR_MANUFACTURED = 1, OR_LORENZ = 2, OR_CHEN = 3,
       OR_ROSSLER = 4, OR_FINANCIAL = 5, OR_HINDMARSH_ROSE = 6, OR_NSYS = 7 };

int oracle_dim(int sys) {
  switch (sys) {
    case OR_LINEAR: case OR_MANUFACTURED: return 1;
    case OR_LORENZ: case OR_CHEN: case OR_ROSSLER: case OR_FINANCIAL: case OR_HINDMARSH_ROSE: return 3;
  }
  return -1;
}

int oracle_nparams(int sys) {
  switch (sys) {
    case OR_LINEAR: return 3;
    case OR_MANUFACTURED: return 9;
    case OR_LORENZ: case OR_CHEN: case OR_ROSSLER: case OR_FINANCIAL: return 3;
    case OR_HINDMARSH_ROSE: return 8;
  }
  return -1;
}

/* Manufactured reference curve Y(t) = e0 + c1 t^a + c2 t^(1+a) + c3 t^(2+a). */
static double manu_curve(double alpha, const double* p, double t) {
  double ta = (t > 0.0) ? pow(t, alpha) : 0.0;
  return p[5] + p[6] * ta + p[7] * ta * t + p[8] * ta * t * t;
}

/* f(t, y).  Parameter layouts:
 *  linear       : (lam, q0, q1)             f = lam*y + q0 + q1*t
 *  manufactured : (q0,q1,q2,beta,gam,e0,c1,c2,c3)
 *                 f = q0 + q1 t + q2 t^2 + beta*r + gam*r^3,  r = y - Y(t)
 *  lorenz       : (sigma, rho, beta)
 *  chen         : (a, b, c)   x'=a(y-x), y'=(c-a)x-xz+cy, z'=xy-bz
 *  rossler      : (a, b, c)   x'=-y-z, y'=x+a y, z'=b+z(x-c)
 *  financial    : (a, b, c)   x'=z+(y-a)x, y'=1-b y-x^2, z'=-x-c z
 *  hindmarsh_rose: (a, b, c, d, r, s, xR, I)
 *                 x'=y-a x^3+b x^2-z+I, y'=c-d x^2-y, z'=r(s(x-xR)-z)        */
void oracle_rhs(int sys, double alpha, const double* p, double t, const double* y, double* f) {
  switch (sys) {
    case OR_LINEAR:
      f[0] = p[0] * y[0] + p[1] + p[2] * t;
      break;
    case OR_MANUFACTURED: {
      double r = y[0] - manu_curve(alpha, p, t);
      f[0] = p[0] + p[1] * t + p[2] * t * t + p[3] * r + p[4] * r * r * r;
      break;
    }
    case OR_LORENZ:
      f[0] = p[0] * (y[1] - y[0]);
      f[1] = y[0] * (p[1] - y[2]) - y[1];
      f[2] = y[0] * y[1] - p[2] * y[2];
      break;
    case OR_CHEN:
      f[0] = p[0] * (y[1] - y[0]);
      f[1] = (p[2] - p[0]) * y[0] - y[0] * y[2] + p[2] * y[1];
      f[2] = y[0] * y[1] - p[1] * y[2];
      break;
    case OR_ROSSLER:
      f[0] = -y[1] - y[2];
      f[1] = y[0] + p[0] * y[1];
      f[2] = p[1] + y[2] * (y[0] - p[2]);
      break;
    case OR_FINANCIAL:
      f[0] = y[2] + (y[1] - p[0]) * y[0];
      f[1] = 1.0 - p[1] * y[1] - y[0] * y[0];
      f[2] = -y[0] - p[2] * y[2];
      break;
    case OR_HINDMARSH_ROSE:
      f[0] = y[1] - p[0] * y[0] * y[0] * y[0] + p[1] * y[0] * y[0] - y[2] + p[7];
      f[1] = p[2] - p[3] * y[0] * y[0] - y[1];
      f[2] = p[4] * (p[5] * (y[0] - p[6]) - y[2]);
      break;
  }
}

/* J = df/dy (d x d, row-major) and Q = df/dp (d x np, row-major) at (t, y). */
void oracle_jac(int sys, double alpha, const double* p, double t, const double* y, double* J, double* Q) {
  switch (sys) {
    case OR_LINEAR:
      J[0] = p[0];
      Q[0] = y[0]; Q[1] = 1.0; Q[2] = t;
      break;
    case OR_MANUFACTURED: {
      double ta = (t > 0.0) ? pow(t, alpha) : 0.0;
      double r = y[0] - manu_curve(alpha, p, t);
      double dfdr = p[3] + 3.0 * p[4] * r * r;
      J[0] = dfdr;
      Q[0] = 1.0; Q[1] = t; Q[2] = t * t; Q[3] = r; Q[4] = r * r * r;
      Q[5] = -dfdr; Q[6] = -dfdr * ta; Q[7] = -dfdr * ta * t; Q[8] = -dfdr * ta * t * t;
      break;
    }
    case OR_LORENZ:
      J[0] = -p[0];        J[1] = p[0];  J[2] = 0.0;
      J[3] = p[1] - y[2];  J[4] = -1.0;  J[5] = -y[0];
      J[6] = y[1];         J[7] = y[0];  J[8] = -p[2];
      Q[0] = y[1] - y[0];  Q[1] = 0.0;   Q[2] = 0.0;
      Q[3] = 0.0;          Q[4] = y[0];  Q[5] = 0.0;
      Q[6] = 0.0;          Q[7] = 0.0;   Q[8] = -y[2];
      break;
    case OR_CHEN:
      J[0] = -p[0];               J[1] = p[0];  J[2] = 0.0;
      J[3] = p[2] - p[0] - y[2];  J[4] = p[2];  J[5] = -y[0];
      J[6] = y[1];                J[7] = y[0];  J[8] = -p[1];
      Q[0] = y[1] - y[0];  Q[1] = 0.0;    Q[2] = 0.0;
      Q[3] = -y[0];        Q[4] = 0.0;    Q[5] = y[0] + y[1];
      Q[6] = 0.0;          Q[7] = -y[2];  Q[8] = 0.0;
      break;
    case OR_ROSSLER:
      J[0] = 0.0;   J[1] = -1.0;  J[2] = -1.0;
      J[3] = 1.0;   J[4] = p[0];  J[5] = 0.0;
      J[6] = y[2];  J[7] = 0.0;   J[8] = y[0] - p[2];
      Q[0] = 0.0;   Q[1] = 0.0;   Q[2] = 0.0;
      Q[3] = y[1];  Q[4] = 0.0;   Q[5] = 0.0;
      Q[6] = 0.0;   Q[7] = 1.0;   Q[8] = -y[2];
      break;
    case OR_FINANCIAL:
      J[0] = y[1] - p[0];  J[1] = y[0];   J[2] = 1.0;
      J[3] = -2.0 * y[0];  J[4] = -p[1];  J[5] = 0.0;
      J[6] = -1.0;         J[7] = 0.0;    J[8] = -p[2];
      Q[0] = -y[0];  Q[1] = 0.0;    Q[2] = 0.0;
      Q[3] = 0.0;    Q[4] = -y[1];  Q[5] = 0.0;
      Q[6] = 0.0;    Q[7] = 0.0;    Q[8] = -y[2];
      break;
    case OR_HINDMARSH_ROSE: {
      double x = y[0];
      J[0] = -3.0 * p[0] * x * x + 2.0 * p[1] * x;  J[1] = 1.0;   J[2] = -1.0;
      J[3] = -2.0 * p[3] * x;                       J[4] = -1.0;  J[5] = 0.0;
      J[6] = p[4] * p[5];                           J[7] = 0.0;   J[8] = -p[4];
      for (int k = 0; k < 24; ++k) Q[k] = 0.0;
      Q[0] = -x * x * x;  Q[1] = x * x;  Q[7] = 1.0;            /* row 0: a, b, I */
      Q[8 + 2] = 1.0;     Q[8 + 3] = -x * x;                    /* row 1: c, d */
      Q[16 + 4] = p[5] * (x - p[6]) - y[2];                     /* row 2: r, s, xR */
      Q[16 + 5] = p[4] * (x - p[6]);
      Q[16 + 6] = -p[4] * p[5];
      break;
    }
  }
}

/* ---- weights (Sec. 2), binary128 from the plain definitions, rounded to FP64 ----
 * Fills b[m], a[m], c[m] for m = 0..M and *g = 1/Gamma(alpha+2). */
int oracle_weights(double alpha, long M, double* b, double* a, double* c, double* g) {
  if (!(alpha > 0.0 && alpha <= 2.0) || M < 0) return 1;
  qreal al = (qreal)alpha, one = 1;
  qreal ga1 = QGAMMA(al + one);      /* Gamma(alpha+1) */
  qreal ga2 = QGAMMA(al + 2 * one);  /* Gamma(alpha+2) */
  for (long m = 0; m <= M; ++m) {
    qreal q = (qreal)m;
    qreal pm_a = (m == 0) ? 0 : QPOW(q, al);           /* m^alpha       */
    qreal pm1_a = QPOW(q + one, al);                    /* (m+1)^alpha   */
    qreal pm_a1 = (m == 0) ? 0 : QPOW(q, al + one);    /* m^(alpha+1)   */
    qreal pm1_a1 = QPOW(q + one, al + one);             /* (m+1)^(a+1)   */
    qreal pm2_a1 = QPOW(q + 2 * one, al + one);         /* (m+2)^(a+1)   */
    b[m] = (double)((pm1_a - pm_a) / ga1);
    a[m] = (double)((pm2_a1 - 2 * pm1_a1 + pm_a1) / ga2);
    c[m] = (double)((pm_a1 - (q - al) * pm1_a) / ga2);
  }
  *g = (double)(one / ga2);
  return 0;
}

/* ---- history sums of one target step (the quantity the GPU far/near kernels split) ----
 * For target step n (producing y_{n+1}) and history rows k in [k_lo, k_hi):
 *   P[col] = sum_k b_{n-k} F[k][col]
 *   C[col] = sum_k w_k F[k][col],  w_0 = c_n, w_k = a_{n-k} for k >= 1
 * F is row-major (rows x cols).  Weights must cover lags 0..n. */
void oracle_history(const double* b, const double* a, const double* c, long cols,
                    const double* F, long n, long k_lo, long k_hi, double* P, double* C) {
  for (long col = 0; col < cols; ++col) {
    double sp = 0.0, sc = 0.0;
    for (long k = k_lo; k < k_hi; ++k) {
      double fk = F[k * cols + col];
      sp += b[n - k] * fk;
      sc += ((k == 0) ? c[n] : a[n - k]) * fk;
    }
    P[col] = sp;
    C[col] = sc;
  }
}

/* ---- the general problem of eq. (1): orders above one, one order per component ----
 * Component i of D_*^{alpha_i} y_i = f_i(t, y) has its own order alpha_i in
 * (0, 2] (a non-commensurate system when they differ), its own weights
 * b^(i), a^(i), c^(i) (Sec. 2 definitions at alpha_i), h^{alpha_i} and
 * 1/Gamma(alpha_i+2), and the Taylor sum of eq. (2) and of the corrector,
 *   T_i(t) = sum_{k=0..ceil(alpha_i)-1} t^k / k! y_i^{(k)}(0),
 * which for alpha_i in (1, 2] adds t y_i'(0) to y_i(0).  y0d holds the d
 * initial derivatives y_i'(0) (NULL: all zero); they enter only components
 * with alpha_i > 1.  m corrector passes per step (m = 1: PECE):
 *   y^P_{n+1,i} = T_i(t_{n+1}) + h^{alpha_i} sum_{k=0..n} b^(i)_{n-k} F_{k,i}
 *   y^(j)_i     = T_i(t_{n+1}) + h^{alpha_i} (c^(i)_n F_{0,i} + sum_{k=1..n} a^(i)_{n-k} F_{k,i}
 *                                             + g_i f_i(t_{n+1}, y^(j-1))),  y^(0) = y^P
 *   y_{n+1} = y^(m),  F_{n+1} = f(t_{n+1}, y_{n+1}).
 * With every alpha_i equal and in (0, 1] this is oracle_solve (m = 1) or
 * oracle_solve_pecm, operation for operation.  The system's own use of alpha
 * (the manufactured right-hand side) takes alpha_0. */
int oracle_solve_ext(int sys, const double* alpha, const double* y0d, double h, long N, const double* p,
                     const double* y0, int m, double* Y, double* YP, double* Fout) {
  int d = oracle_dim(sys);
  if (d < 1 || !(h > 0.0) || N < 1 || m < 1) return 1;
  for (int i = 0; i < d; ++i)
    if (!(alpha[i] > 0.0 && alpha[i] <= 2.0)) return 1;
  double *wb[3] = {0}, *wa[3] = {0}, *wc[3] = {0};
  double g[3], hat[3];
  int ceil_a[3];
  double* F = Fout ? Fout : malloc(sizeof(double) * (N + 1) * d);
  int bad = !F;
  for (int i = 0; i < d && !bad; ++i) {
    wb[i] = malloc(sizeof(double) * (N + 1));
    wa[i] = malloc(sizeof(double) * (N + 1));
    wc[i] = malloc(sizeof(double) * (N + 1));
    bad = !wb[i] || !wa[i] || !wc[i];
    if (!bad) oracle_weights(alpha[i], N, wb[i], wa[i], wc[i], &g[i]);
    hat[i] = pow(h, alpha[i]);
    ceil_a[i] = alpha[i] > 1.0 ? 2 : 1;
  }
  if (bad) {
    for (int i = 0; i < d; ++i) { free(wb[i]); free(wa[i]); free(wc[i]); }
    if (!Fout) free(F);
    return 2;
  }
  double yp[3], yj[3], fj[3], sc[3], taylor[3];
  for (int i = 0; i < d; ++i) { Y[i] = y0[i]; YP[i] = y0[i]; }
  oracle_rhs(sys, alpha[0], p, 0.0, y0, F);
  for (long n = 0; n < N; ++n) {
    double tn1 = (double)(n + 1) * h;
    for (int i = 0; i < d; ++i) {             /* Taylor sum of the initial values */
      double term = y0[i], tk = 1.0;
      taylor[i] = 0.0;
      for (int k = 0; k < ceil_a[i]; ++k) {
        taylor[i] += term;
        tk *= tn1;
        term = (y0d ? y0d[i] : 0.0) * tk;     /* k = 1: t y'(0) (1! = 1) */
      }
    }
    for (int i = 0; i < d; ++i) {             /* predictor, eq. (2), component i's weights */
      double sum = 0.0;
      for (long k = 0; k <= n; ++k) sum += wb[i][n - k] * F[k * d + i];
      yp[i] = taylor[i] + hat[i] * sum;
      yj[i] = yp[i];
    }
    for (int i = 0; i < d; ++i) {             /* corrector history part */
      double sum = wc[i][n] * F[i];
      for (long k = 1; k <= n; ++k) sum += wa[i][n - k] * F[k * d + i];
      sc[i] = sum;
    }
    for (int pass = 1; pass <= m; ++pass) {   /* m corrector passes */
      oracle_rhs(sys, alpha[0], p, tn1, yj, fj);
      for (int i = 0; i < d; ++i) yj[i] = taylor[i] + hat[i] * (sc[i] + g[i] * fj[i]);
    }
    for (int i = 0; i < d; ++i) {
      Y[(n + 1) * d + i] = yj[i];
      YP[(n + 1) * d + i] = yp[i];
    }
    oracle_rhs(sys, alpha[0], p, tn1, Y + (n + 1) * d, F + (n + 1) * d);
  }
  for (int i = 0; i < d; ++i) { free(wb[i]); free(wa[i]); free(wc[i]); }
  if (!Fout) free(F);
  return 0;
}

/* ---- the ABM PECE solve (Sec. 2) ----
 * Y and YP hold (N+1) x d values; Y[0] = YP[0] = y0.  F (optional, may be NULL)
 * receives the history f_k.  Returns 0 on success, 1 on bad arguments, 2 on
 * allocation failure. */
int oracle_solve(int sys, double alpha, double h, long N, const double* p, const double* y0,
                 double* Y, double* YP, double* Fout) {
  int d = oracle_dim(sys);
  if (d < 1 || !(alpha > 0.0 && alpha <= 1.0) || !(h > 0.0) || N < 1) return 1;
  double *b = malloc(sizeof(double) * (N + 1)), *a = malloc(sizeof(double) * (N + 1));
  double *c = malloc(sizeof(double) * (N + 1));
  double* F = Fout ? Fout : malloc(sizeof(double) * (N + 1) * d);
  if (!b || !a || !c || !F) { free(b); free(a); free(c); if (!Fout) free(F); return 2; }
  double g;
  oracle_weights(alpha, N, b, a, c, &g);
  double hh = pow(h, alpha);
  double yp[3], fp[3];
  for (int i = 0; i < d; ++i) { Y[i] = y0[i]; YP[i] = y0[i]; }
  oracle_rhs(sys, alpha, p, 0.0, y0, F);
  for (long n = 0; n < N; ++n) {
    double t1 = (double)(n + 1) * h;
    for (int i = 0; i < d; ++i) {             /* predictor, eq. (2) */
      double s = 0.0;
      for (long k = 0; k <= n; ++k) s += b[n - k] * F[k * d + i];
      yp[i] = y0[i] + hh * s;
    }
    oracle_rhs(sys, alpha, p, t1, yp, fp);
    for (int i = 0; i < d; ++i) {             /* corrector */
      double s = c[n] * F[i];
      for (long k = 1; k <= n; ++k) s += a[n - k] * F[k * d + i];
      Y[(n + 1) * d + i] = y0[i] + hh * (s + g * fp[i]);
      YP[(n + 1) * d + i] = yp[i];
    }
    oracle_rhs(sys, alpha, p, t1, Y + (n + 1) * d, F + (n + 1) * d);
  }
  free(b); free(a); free(c);
  if (!Fout) free(F);
  return 0;
}

/* ---- P(EC)^m E: the same scheme with m corrector passes per step ----
 * The corrector is an implicit equation for y_{n+1} (its last term is
 * g f(t_{n+1}, y_{n+1})); PECE evaluates that term once, at the predictor.
 * P(EC)^m E repeats the corrector m times, each pass evaluating f at the
 * previous pass's value, then evaluates F_{n+1} once at the last one:
 *   y^(0) = y^P_{n+1}
 *   y^(j) = y_0 + h_hat * (c_n F_0 + sum_{k=1..n} a_{n-k} F_k + g f(t_{n+1}, y^(j-1))),
 *           j = 1..m
 *   y_{n+1} = y^(m),  F_{n+1} = f(t_{n+1}, y_{n+1}).
 * m = 1 is the PECE of oracle_solve.  Not in the paper: a common variant of
 * the Adams predictor-corrector, whose passes move y_{n+1} toward the
 * solution of the implicit corrector.  YP holds y^P as in oracle_solve. */
int oracle_solve_pecm(int sys, double alpha, double h, long N, const double* p, const double* y0,
                      int m, double* Y, double* YP, double* Fout) {
  int d = oracle_dim(sys);
  if (d < 1 || !(alpha > 0.0 && alpha <= 1.0) || !(h > 0.0) || N < 1 || m < 1) return 1;
  double *b = malloc(sizeof(double) * (N + 1)), *a = malloc(sizeof(double) * (N + 1));
  double *c = malloc(sizeof(double) * (N + 1));
  double* F = Fout ? Fout : malloc(sizeof(double) * (N + 1) * d);
  if (!b || !a || !c || !F) { free(b); free(a); free(c); if (!Fout) free(F); return 2; }
  double g;
  oracle_weights(alpha, N, b, a, c, &g);
  double hat = pow(h, alpha);
  double yp[3], yj[3], fj[3], sc[3];
  for (int i = 0; i < d; ++i) { Y[i] = y0[i]; YP[i] = y0[i]; }
  oracle_rhs(sys, alpha, p, 0.0, y0, F);
  for (long n = 0; n < N; ++n) {
    double tn1 = (double)(n + 1) * h;
    for (int i = 0; i < d; ++i) {             /* predictor, eq. (2) */
      double sum = 0.0;
      for (long k = 0; k <= n; ++k) sum += b[n - k] * F[k * d + i];
      yp[i] = y0[i] + hat * sum;
      yj[i] = yp[i];
    }
    for (int i = 0; i < d; ++i) {             /* corrector history part, fixed over the passes */
      double sum = c[n] * F[i];
      for (long k = 1; k <= n; ++k) sum += a[n - k] * F[k * d + i];
      sc[i] = sum;
    }
    for (int j = 1; j <= m; ++j) {            /* m corrector passes */
      oracle_rhs(sys, alpha, p, tn1, yj, fj);
      for (int i = 0; i < d; ++i) yj[i] = y0[i] + hat * (sc[i] + g * fj[i]);
    }
    for (int i = 0; i < d; ++i) {
      Y[(n + 1) * d + i] = yj[i];
      YP[(n + 1) * d + i] = yp[i];
    }
    oracle_rhs(sys, alpha, p, tn1, Y + (n + 1) * d, F + (n + 1) * d);
  }
  free(b); free(a); free(c);
  if (!Fout) free(F);
  return 0;
}

/* ---- tangent-linear gradient of a trajectory loss ----
 * Sensitivities S_n = d y_n / d theta, theta = (p[0..np-1], y0[0..d-1]), are
 * carried through exactly the same discrete scheme (differentiate every line
 * of oracle_solve).  Given dLdY ((N+1) x d, the partial derivatives of the
 * loss with respect to each y_n), returns dL/dp = sum_n S_n^T dLdY_n
 * restricted to p and dL/dy0 likewise. */
int oracle_tangent(int sys, double alpha, double h, long N, const double* p, const double* y0,
                   const double* dLdY, double* dLdp, double* dLdy0) {
  int d = oracle_dim(sys), np = oracle_nparams(sys);
  if (d < 1 || !(alpha > 0.0 && alpha <= 1.0) || !(h > 0.0) || N < 1) return 1;
  int P = np + d;
  long SZ = (long)d * P;
  double* Y = malloc(sizeof(double) * (N + 1) * d);
  double* YP = malloc(sizeof(double) * (N + 1) * d);
  double* SF = malloc(sizeof(double) * (N + 1) * SZ);  /* d F_k / d theta */
  double *b = malloc(sizeof(double) * (N + 1)), *a = malloc(sizeof(double) * (N + 1));
  double *c = malloc(sizeof(double) * (N + 1));
  if (!Y || !YP || !SF || !b || !a || !c) {
    free(Y); free(YP); free(SF); free(b); free(a); free(c);
    return 2;
  }
  int rc = oracle_solve(sys, alpha, h, N, p, y0, Y, YP, NULL);
  if (rc) { free(Y); free(YP); free(SF); free(b); free(a); free(c); return rc; }
  double g;
  oracle_weights(alpha, N, b, a, c, &g);
  double hh = pow(h, alpha);
  double J[9], Q[27], S0[3 * 12], S[3 * 12], SP[3 * 12], SfP[3 * 12];
  double grad[12];
  /* S_0 = d y0 / d theta = [0 | I] */
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < P; ++j) S0[i * P + j] = (j == np + i) ? 1.0 : 0.0;
  for (int j = 0; j < P; ++j) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += dLdY[i] * S0[i * P + j];
    grad[j] = s;
  }
  /* SF_k = J(t_k, y_k) S_k + [Q(t_k, y_k) | 0] */
  oracle_jac(sys, alpha, p, 0.0, y0, J, Q);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < P; ++j) {
      double s = (j < np) ? Q[i * np + j] : 0.0;
      for (int l = 0; l < d; ++l) s += J[i * d + l] * S0[l * P + j];
      SF[i * P + j] = s;
    }
  for (long n = 0; n < N; ++n) {
    double t1 = (double)(n + 1) * h;
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < P; ++j) {
        double s = 0.0;
        for (long k = 0; k <= n; ++k) s += b[n - k] * SF[k * SZ + i * P + j];
        SP[i * P + j] = S0[i * P + j] + hh * s;
      }
    oracle_jac(sys, alpha, p, t1, YP + (n + 1) * d, J, Q);
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < P; ++j) {
        double s = (j < np) ? Q[i * np + j] : 0.0;
        for (int l = 0; l < d; ++l) s += J[i * d + l] * SP[l * P + j];
        SfP[i * P + j] = s;
      }
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < P; ++j) {
        double s = c[n] * SF[i * P + j];
        for (long k = 1; k <= n; ++k) s += a[n - k] * SF[k * SZ + i * P + j];
        S[i * P + j] = S0[i * P + j] + hh * (s + g * SfP[i * P + j]);
      }
    oracle_jac(sys, alpha, p, t1, Y + (n + 1) * d, J, Q);
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < P; ++j) {
        double s = (j < np) ? Q[i * np + j] : 0.0;
        for (int l = 0; l < d; ++l) s += J[i * d + l] * S[l * P + j];
        SF[(n + 1) * SZ + i * P + j] = s;
      }
    for (int j = 0; j < P; ++j) {
      double s = 0.0;
      for (int i = 0; i < d; ++i) s += dLdY[(n + 1) * d + i] * S[i * P + j];
      grad[j] += s;
    }
  }
  for (int j = 0; j < np; ++j) dLdp[j] = grad[j];
  for (int i = 0; i < d; ++i) dLdy0[i] = grad[np + i];
  free(Y); free(YP); free(SF); free(b); free(a); free(c);
  return 0;
}

/*
 * Oracle (test infrastructure only): line constants, the Hjerting-Voigt
 * function and the core/wing crossover, in FP64.
 *
 *   Sec. 2          : v_th, a, sigma_0, tau_x = n sigma_0 l H(a,x)
 *   Sec. 2 / 3.2.1  : H(a,x) = (a/pi) int exp(-y^2) / (a^2 + (y-x)^2) dy
 *   App. A1         : H_approx(a, z = x^2), Eq. AB with Table AB
 *   Sec. 3.2.2      : x_cw = sqrt(-W_{-1}(-a/sqrt(pi))) and its rational fit
 *   Sec. 3.2.4      : x_crit(a tau_0), Eq. xcrit
 */
#include "oracle.h"
#include <math.h>

#define O_PI 3.14159265358979323846
#define O_SQRTPI 1.77245385090551602730

/* Sec. 2: all line constants scale with T4 = T / 1e4 K. */
double o_vth_kms(double T)   { return 12.85 * sqrt(T / 1.0e4); }
double o_damping_a(double T) { return 4.702e-4 / sqrt(T / 1.0e4); }
double o_sigma0(double T)    { return 5.898e-14 / sqrt(T / 1.0e4); }
double o_recoil_g(double T)  { return 2.536e-4 / sqrt(T / 1.0e4); }

/* ------------------------------------------------------------------------ */
/* Exact H(a,x) by adaptive Gauss-Kronrod quadrature.
 *
 * For |x| <= 9 the substitution y = x + a tan(t) in the Sec. 2 integral removes
 * the Lorentzian denominator exactly:
 *   H = (1/pi) int_{-pi/2}^{pi/2} exp(-(x + a tan t)^2) dt.
 * For |x| > 9 the Lorentzian pole lies outside the Gaussian's support and the
 * integral is taken directly in y.  In both forms |y| > 8 is dropped: the
 * integrand there is below exp(-64) (relative loss < 1e-20 of any H here).
 * Intervals are pre-split so that every feature is bracketed.              */
typedef struct { double a, x; int yspace; } hq;

static double h_integrand(const hq* q, double v) {
  if (q->yspace) {
    double d = v - q->x;
    return (q->a / O_PI) * exp(-v * v) / (q->a * q->a + d * d);
  }
  double y = q->x + q->a * tan(v);
  return exp(-y * y) / O_PI;
}

/* 15-point Kronrod / 7-point Gauss nodes and weights on [-1,1]
 * (standard published values of the Gauss-Kronrod (7,15) rule). */
static const double gk_xk[8] = {
  0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
  0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
  0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
  0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double gk_wk[8] = {
  0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
  0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
  0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
  0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double gk_wg[4] = {
  0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
  0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

static double gk15(const hq* q, double lo, double hi, double* err) {
  double c = 0.5 * (lo + hi), h = 0.5 * (hi - lo);
  double fc = h_integrand(q, c);
  double rk = fc * gk_wk[7], rg = fc * gk_wg[3];
  for (int j = 0; j < 7; ++j) {
    double dx = h * gk_xk[j];
    double f1 = h_integrand(q, c - dx), f2 = h_integrand(q, c + dx);
    rk += gk_wk[j] * (f1 + f2);
    if (j % 2 == 1) rg += gk_wg[j / 2] * (f1 + f2);
  }
  *err = fabs((rk - rg) * h);
  return rk * h;
}

static double adapt(const hq* q, double lo, double hi, double tol, int depth) {
  double err;
  double v = gk15(q, lo, hi, &err);
  if (depth >= 40 || err <= tol) return v;
  double m = 0.5 * (lo + hi);
  return adapt(q, lo, m, 0.5 * tol, depth + 1) + adapt(q, m, hi, 0.5 * tol, depth + 1);
}

static int cmp_d(const void* p, const void* q) {
  double u = *(const double*)p, v = *(const double*)q;
  return (u > v) - (u < v);
}

#include <stdlib.h>
double o_H_exact(double a, double x) {
  const double ymax = 8.0;
  hq q = {a, x, fabs(x) > 9.0};
  double pts[64];
  int n = 0;
  double v_lo, v_hi;
  if (q.yspace) {
    v_lo = -ymax; v_hi = ymax;
    for (int i = -8; i <= 8; ++i) pts[n++] = (double)i;
  } else {
    v_lo = atan((-ymax - x) / a); v_hi = atan((ymax - x) / a);
    pts[n++] = v_lo;
    pts[n++] = v_hi;
    static const double ys[] = {-6, -4, -3, -2, -1.5, -1, -0.5, 0, 0.5, 1, 1.5, 2, 3, 4, 6};
    for (size_t i = 0; i < sizeof(ys) / sizeof(ys[0]); ++i) pts[n++] = atan((ys[i] - x) / a);
    static const double ka[] = {-100, -10, -1, 1, 10, 100};
    for (size_t i = 0; i < sizeof(ka) / sizeof(ka[0]); ++i) pts[n++] = atan(ka[i]);
    pts[n++] = 0.0;
  }
  qsort(pts, (size_t)n, sizeof(double), cmp_d);
  double est = 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    double lo = pts[i] < v_lo ? v_lo : pts[i];
    double hi = pts[i + 1] > v_hi ? v_hi : pts[i + 1];
    if (hi > lo) { double e; est += gk15(&q, lo, hi, &e); }
  }
  double tol = fabs(est) * 1e-13 + 1e-300;
  double sum = 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    double lo = pts[i] < v_lo ? v_lo : pts[i];
    double hi = pts[i + 1] > v_hi ? v_hi : pts[i + 1];
    if (hi > lo) sum += adapt(&q, lo, hi, tol / n, 0);
  }
  return sum;
}

void o_H_exact_many(const double* a, const double* x, double* H, size_t n) {
  for (size_t i = 0; i < n; ++i) H[i] = o_H_exact(a[i], x[i]);
}

/* ------------------------------------------------------------------------ */
/* App. A1, Eq. AB: three-region approximation in z = x^2, first order in a.
 * Coefficients are Table AB.  The regions are z <= 3 (core), 3 < z < 25
 * (intermediate) and z >= 25 (wing asymptotic series).                     */
static const double TA[7] = {15.75328153963877, 286.9341762324778, 19.05706700907019,
                             28.22644017233441, 9.526399802414186, 35.29217026286130,
                             0.8681020834678775};
static const double TB[9] = {0.0003300469163682737, 0.5403095364583999, 2.676724102580895,
                             12.82026082606220,    3.21166435627278,   32.032981933420,
                             9.0328158696,         23.7489999060,      1.82106170570};

double o_H_approx(double a, double x) {
  double z = x * x;
  if (z <= 3.0) {
    double cf = TA[1] / (z - TA[2] + TA[3] / (z - TA[4] + TA[5] / (z - TA[6])));
    return exp(-z) * (1.0 - a * (TA[0] + cf));
  } else if (z < 25.0) {
    double cf = TB[1] / (z - TB[2] + TB[3] / (z + TB[4] + TB[5] / (z - TB[6] + TB[7] / (z - TB[8]))));
    return exp(-z) + a * (TB[0] + cf);
  } else {
    return (a / O_SQRTPI) / (z - 1.5 - 1.5 / (z - 3.5 - 5.0 / (z - 5.5)));
  }
}

void o_H_approx_many(const double* a, const double* x, double* H, size_t n) {
  for (size_t i = 0; i < n; ++i) H[i] = o_H_approx(a[i], x[i]);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2.2, Eq. xcw.  The crossover solves exp(-x^2) = a / (sqrt(pi) x^2)
 * (the x^2 form is the one the Lambert-W expression and the fit solve), so
 * x_cw = sqrt(-W_{-1}(-a/sqrt(pi))).  The fit uses the natural logarithm.   */
double o_x_cw_fit(double a) {
  return 6.9184721 + 81.766279 / (log(a) - 14.651253);
}

/* W_{-1}(zarg) for zarg in (-1/e, 0) by Halley iteration on w e^w = zarg,
 * started from the asymptotic series L1 - L2 + L2/L1 (L1 = ln(-zarg),
 * L2 = ln(-L1)) that Sec. 3.2.2 quotes.                                   */
static double lambert_wm1(double zarg) {
  double L1 = log(-zarg), L2 = log(-L1);
  double w = L1 - L2 + L2 / L1;
  for (int it = 0; it < 100; ++it) {
    double ew = exp(w);
    double f = w * ew - zarg;
    double fp = ew * (w + 1.0);
    double fpp = ew * (w + 2.0);
    double dw = f / (fp - 0.5 * fpp * f / fp);
    w -= dw;
    if (fabs(dw) <= 1e-16 * fabs(w)) break;
  }
  return w;
}

double o_x_cw_lambert(double a) {
  return sqrt(-lambert_wm1(-a / O_SQRTPI));
}

/* Sec. 3.2.4, Eq. atau0J: the local a tau_0 of a uniform region one Jeans
 * length across (primordial gas, mu = 1.23 m_H, X = 0.75). */
double o_atau_jeans(double T, double n_HI) {
  return 6.428e4 / sqrt(T / 1.0e4) * sqrt(n_HI);
}

/* Sec. 3.2.4, Eq. xcrit. */
double o_x_crit(double atau0) {
  if (atau0 < 1.0) return 0.0;
  return 0.2 * cbrt(atau0);
}

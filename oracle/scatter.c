/*
 * Oracle (test infrastructure only): one resonant scattering, in FP64.
 *
 *   Sec. 3.1.3, Eq. x_f, Eq. recoil : x_f = x_i + (k_f - k_i).u_atom + g (k_i.k_f - 1)
 *   Sec. 3.1.3, Eq. uparf           : f(u_par) = a exp(-u^2) / (pi H (a^2 + (x-u)^2))
 *   Sec. 3.2.3                      : the u_par rejection sampler in four regimes
 *   Sec. 3.2.4                      : core-skipping, truncated Box-Muller u_perp
 *   Sec. 3.1.3, Eq. phaseW          : W ~ 1 + (R/Q) cos^2(theta)
 *
 * Random draws (a reading of this implementation; the paper only says "a
 * univariate R"): an interaction with event index e uses Philox blocks
 * (pid, e, b) with
 *   block 0 : [interaction type, dust albedo, next tau_event, core R/Q choice]
 *   block 1 : [u_perp R1, u_perp R2, phase mu, phase phi]
 *   block 2+t : u_par rejection trial t
 * Readings of the paper that this file takes:
 *   - every u_par regime test uses |x|; the draw is made for |x| and the sign
 *     of u_par is flipped when x < 0, since f(-x,u) = f(x,-u) (Sec. 3.2.3);
 *   - x >= 9 draws a Gaussian of mean 1/|x| and variance 1/2 (the width of
 *     exp(-u^2)); no rejection step there.  In the exact-physics mode (used
 *     to measure the approximations' bias) it is instead the numeric
 *     inversion of Eq. uparf itself;
 *   - the piecewise proposal picks theta in [theta0, pi/2] when p < R and in
 *     [-pi/2, theta0] otherwise; acceptance is exp(-u^2) on the lower piece
 *     and exp(u0^2 - u^2) on the upper one, accepted when R' < acceptance;
 *   - core-skipping is used only when |x| < x_crit ("already in the wing"
 *     otherwise), with x_crit from Eq. xcrit;
 *   - core vs wing for the phase function compares the incoming |x| with
 *     x_cw; core R/Q is 0 with probability 1/3 and 3/7 otherwise; wing 1;
 *   - mu is drawn by inverting the CDF of 1 + (R/Q) mu^2 with Cardano's
 *     formula; the perpendicular basis is the branchless construction of
 *     Duff et al. 2017 ("Building an Orthonormal Basis, Revisited").
 */
#include "oracle.h"
#include <math.h>

#define O_PI 3.14159265358979323846
#define O_MAX_TRIALS 1000000

static void draw_block(const uint32_t key[2], uint64_t pid, uint32_t event, uint32_t blk, double u[4]) {
  uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), event, blk};
  uint32_t r[4];
  o_philox4x32_10(ctr, key, r);
  for (int i = 0; i < 4; ++i) u[i] = o_uniform(r[i]);
}

/* Exact-physics mode, |x| >= 9: u_par from the distribution of Eq. uparf,
 * f(u) ~ exp(-u^2) / ((|x| - u)^2 + a^2), by inverting its CDF numerically:
 * the CDF by the trapezoid rule on O_EXACT_N intervals of [-8, 8] (beyond,
 * exp(-u^2) < 2e-28 and |x| - u >= 1), inverted at R by linear interpolation
 * inside the interval that holds R (error O(h^2), h = 16 / O_EXACT_N). */
#define O_EXACT_N 16384
static double sample_upar_inverse(double xa, double a, double R) {
  double cdf[O_EXACT_N + 1];
  const double L = 8.0, h = 2.0 * L / O_EXACT_N;
  double u = -L, fprev = exp(-u * u) / ((xa - u) * (xa - u) + a * a);
  cdf[0] = 0.0;
  for (int i = 1; i <= O_EXACT_N; ++i) {
    u = -L + i * h;
    double f = exp(-u * u) / ((xa - u) * (xa - u) + a * a);
    cdf[i] = cdf[i - 1] + 0.5 * h * (fprev + f);
    fprev = f;
  }
  double target = R * cdf[O_EXACT_N];
  int lo = 1, hi = O_EXACT_N;             /* first i with cdf[i] >= target */
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    if (cdf[mid] >= target) hi = mid; else lo = mid + 1;
  }
  double w = cdf[lo] - cdf[lo - 1];
  double frac = w > 0.0 ? (target - cdf[lo - 1]) / w : 0.5;
  return -L + (lo - 1 + frac) * h;
}

/* Sec. 3.2.3.  Returns u_par for frequency x; *n_trials gets the number of
 * proposals drawn (O_MAX_TRIALS + 1 when the cap was hit). */
static double sample_upar(double x, double a, double x_cw, const uint32_t key[2],
                          uint64_t pid, uint32_t event, int* n_trials, int exact) {
  double xa = fabs(x);
  double u = 0.0;
  double R[4];
  if (xa >= 9.0) {
    draw_block(key, pid, event, 2, R);
    if (exact) {
      u = sample_upar_inverse(xa, a, R[0]);
    } else {
      /* far wing: Gaussian with its peak shifted to 1/x */
      u = 1.0 / xa + sqrt(-log(R[0])) * cos(2.0 * O_PI * R[1]);
    }
    *n_trials = 1;
  } else if (xa <= 1.0) {
    /* small |x|: Lorentzian comparison function g ~ 1/(a^2 + (x-u)^2),
     * accepted with probability f/g = exp(-u^2) */
    int t = 0;
    for (;;) {
      if (t >= O_MAX_TRIALS) { *n_trials = O_MAX_TRIALS + 1; break; }
      draw_block(key, pid, event, 2u + (uint32_t)t, R);
      ++t;
      double theta = O_PI * (R[0] - 0.5);
      u = a * tan(theta) + xa;
      if (R[1] < exp(-u * u)) { *n_trials = t; break; }
    }
  } else {
    /* intermediate frequencies: piecewise comparison function with
     * separation u0 (core form below x_cw, linear wing form above) */
    double u0 = (xa < x_cw) ? xa - 1.0 / (xa + exp(1.0 - xa * xa) / a)
                            : x_cw - 1.0 / x_cw + 0.15 * (xa - x_cw);
    double theta0 = atan((u0 - xa) / a);
    double e0 = exp(-u0 * u0);
    double p = (theta0 + 0.5 * O_PI) / ((1.0 - e0) * theta0 + (1.0 + e0) * 0.5 * O_PI);
    int t = 0;
    for (;;) {
      if (t >= O_MAX_TRIALS) { *n_trials = O_MAX_TRIALS + 1; break; }
      draw_block(key, pid, event, 2u + (uint32_t)t, R);
      ++t;
      int upper = (p < R[0]);
      double theta = upper ? theta0 + (0.5 * O_PI - theta0) * R[1]
                           : -0.5 * O_PI + (theta0 + 0.5 * O_PI) * R[1];
      u = a * tan(theta) + xa;
      double acc = upper ? exp(u0 * u0 - u * u) : exp(-u * u);
      if (R[2] < acc) { *n_trials = t; break; }
    }
  }
  return (x < 0.0) ? -u : u;
}

double o_sample_upar(double x, double a, uint64_t pid, uint32_t event,
                     const uint32_t key[2], int* n_trials) {
  return sample_upar(x, a, o_x_cw_fit(a), key, pid, event, n_trials, 0);
}

/* Eq. phaseW: CDF of W(mu) ~ 1 + RQ mu^2 on [-1,1] is
 * F(mu) = (mu + RQ mu^3/3 + 1 + RQ/3) / (2 (1 + RQ/3)); solve F(mu) = u. */
double o_sample_mu(double RQ, double u) {
  if (RQ == 0.0) return 2.0 * u - 1.0;
  double c = (2.0 * u - 1.0) * (1.0 + RQ / 3.0);
  /* (RQ/3) mu^3 + mu - c = 0  ->  mu^3 + p mu + q = 0 */
  double p = 3.0 / RQ, q = -3.0 * c / RQ;
  double disc = sqrt(0.25 * q * q + p * p * p / 27.0);
  return cbrt(-0.5 * q + disc) + cbrt(-0.5 * q - disc);
}

/* Duff et al. 2017 orthonormal basis perpendicular to the unit vector n. */
static void onb(const double n[3], double e1[3], double e2[3]) {
  double s = copysign(1.0, n[2]);
  double aa = -1.0 / (s + n[2]);
  double bb = n[0] * n[1] * aa;
  e1[0] = 1.0 + s * n[0] * n[0] * aa; e1[1] = s * bb; e1[2] = -s * n[0];
  e2[0] = bb; e2[1] = s + n[1] * n[1] * aa; e2[2] = -n[1];
}

static double dot3(const double p[3], const double q[3]) {
  return p[0] * q[0] + p[1] * q[1] + p[2] * q[2];
}

void o_scatter_hi(o_scatter_io* s, const uint32_t key[2]) {
  double B0[4], B1[4];
  draw_block(key, s->pid, s->event, 0, B0);
  draw_block(key, s->pid, s->event, 1, B1);
  double x = s->x, a = s->a;
  double x_cw = o_x_cw_fit(a);

  /* Sec. 3.2.4: critical frequency; no cutoff once |x| >= x_crit */
  double x_crit = (s->atau0 >= 0.0) ? o_x_crit(s->atau0) : 0.0;
  if (fabs(x) >= x_crit) x_crit = 0.0;
  s->x_crit = x_crit;

  /* perpendicular velocity: truncated Box-Muller (Sec. 3.2.4);
   * with x_crit = 0 it is the untruncated Gaussian of Sec. 3.1.3 */
  double rho = sqrt(x_crit * x_crit - log(B1[0]));
  double up1 = rho * cos(2.0 * O_PI * B1[1]);
  double up2 = rho * sin(2.0 * O_PI * B1[1]);

  /* parallel velocity (Sec. 3.2.3) */
  int ntr = 0;
  double upar = sample_upar(x, a, x_cw, key, s->pid, s->event, &ntr, s->exact);
  s->n_trials = ntr;
  s->u_par = upar;

  /* phase function (Eq. phaseW) */
  double RQ;
  if (s->phase == 1) RQ = 0.0;
  else if (fabs(x) < x_cw) RQ = (B0[3] < 1.0 / 3.0) ? 0.0 : 3.0 / 7.0;
  else RQ = 1.0;
  s->RQ = RQ;
  double mu = o_sample_mu(RQ, B1[2]);
  double phi = 2.0 * O_PI * B1[3];
  s->mu = mu;

  double e1[3], e2[3];
  onb(s->k, e1, e2);
  double st = sqrt(fmax(0.0, 1.0 - mu * mu));
  double cp = cos(phi), sp = sin(phi);
  for (int i = 0; i < 3; ++i) {
    s->k_f[i] = mu * s->k[i] + st * (cp * e1[i] + sp * e2[i]);
    s->u_atom[i] = upar * s->k[i] + up1 * e1[i] + up2 * e2[i];
  }
  /* Eq. x_f */
  double dk[3] = {s->k_f[0] - s->k[0], s->k_f[1] - s->k[1], s->k_f[2] - s->k[2]};
  s->x_f = x + dot3(dk, s->u_atom) + s->g * (dot3(s->k, s->k_f) - 1.0);
}

void o_scatter_many(o_scatter_io* s, size_t n, const uint32_t key[2]) {
  for (size_t i = 0; i < n; ++i) o_scatter_hi(&s[i], key);
}

/* Batched draws for distribution pins: sample i uses packet id pid0 + i,
 * event index `event`. */
void o_sample_upar_many_ex(double x, double a, uint64_t pid0, uint32_t event, const uint32_t key[2],
                           double* out, int32_t* ntr, size_t n, int exact) {
  double x_cw = o_x_cw_fit(a);
  for (size_t i = 0; i < n; ++i) {
    int t = 0;
    out[i] = sample_upar(x, a, x_cw, key, pid0 + i, event, &t, exact);
    if (ntr) ntr[i] = t;
  }
}

void o_sample_upar_many(double x, double a, uint64_t pid0, uint32_t event,
                        const uint32_t key[2], double* out, int32_t* ntr, size_t n) {
  o_sample_upar_many_ex(x, a, pid0, event, key, out, ntr, n, 0);
}

void o_sample_mu_many(double RQ, const double* u, double* mu, size_t n) {
  for (size_t i = 0; i < n; ++i) mu[i] = o_sample_mu(RQ, u[i]);
}

// Device building blocks of the packet loop (sm_103a).  Every kernel of the
// library -- the persistent transport and the parity entry points -- uses
// these same functions, templated on the arithmetic type R of the
// frequency/direction/sampling math (float in the mixed-precision path,
// double in the plain FP64 path).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace colt {

constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.77245385090551602730;
constexpr int kMaxTrials = 1000000;   // u_par proposals before a packet is capped

// ------------------------------------------------------------ math shims --
__device__ __forceinline__ float m_exp(float v) { return expf(v); }
__device__ __forceinline__ double m_exp(double v) { return exp(v); }
__device__ __forceinline__ float m_log(float v) { return logf(v); }
__device__ __forceinline__ double m_log(double v) { return log(v); }
__device__ __forceinline__ float m_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double m_sqrt(double v) { return sqrt(v); }
__device__ __forceinline__ void m_sincospi(float v, float* s, float* c) { sincospif(v, s, c); }
__device__ __forceinline__ void m_sincospi(double v, double* s, double* c) { sincospi(v, s, c); }
__device__ __forceinline__ void m_sincos(float v, float* s, float* c) { sincosf(v, s, c); }
__device__ __forceinline__ void m_sincos(double v, double* s, double* c) { sincos(v, s, c); }
__device__ __forceinline__ float m_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double m_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float m_asinh(float v) { return asinhf(v); }
__device__ __forceinline__ double m_asinh(double v) { return asinh(v); }
__device__ __forceinline__ float m_sinh(float v) { return sinhf(v); }
__device__ __forceinline__ double m_sinh(double v) { return sinh(v); }
__device__ __forceinline__ float m_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double m_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float m_copysign1(float v) { return copysignf(1.0f, v); }
__device__ __forceinline__ double m_copysign1(double v) { return copysign(1.0, v); }
// Division on the latency-critical path: in FP32 the hardware reciprocal
// form (within 2 ulp for divisors of normal magnitude, which is all this code
// divides by); in FP64 the correctly rounded quotient.
__device__ __forceinline__ float m_div(float x, float y) { return __fdividef(x, y); }
__device__ __forceinline__ double m_div(double x, double y) { return x / y; }

// ---------------------------------------------------------------- Philox --
// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11).
struct u4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u4 philox10(u4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = u4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Uniform on the odd multiples of 2^-24: strictly inside (0,1), exact in FP32
// and FP64, symmetric under u -> 1 - u.
template <typename R>
__device__ __forceinline__ R uni(uint32_t r) {
  return R((r >> 8) | 1u) * R(5.9604644775390625e-8);  // 2^-24
}

struct Rng {
  uint32_t k0, k1;
  __device__ __forceinline__ u4 block(uint64_t pid, uint32_t event, uint32_t blk) const {
    return philox10(u4{uint32_t(pid), uint32_t(pid >> 32), event, blk}, k0, k1);
  }
};

template <typename R>
struct U4 { R v[4]; };

template <typename R>
__device__ __forceinline__ U4<R> uniforms(const Rng& g, uint64_t pid, uint32_t event, uint32_t blk) {
  u4 r = g.block(pid, event, blk);
  return U4<R>{{uni<R>(r.x), uni<R>(r.y), uni<R>(r.z), uni<R>(r.w)}};
}

// ----------------------------------------------------------------- Voigt --
// App. A1, Eq. AB, Table AB.  The three continued fractions are evaluated as
// single rational functions (one division each); z = x^2 is formed exactly as
// z_hi + z_lo and the region is chosen from the exact z, and
// exp(-z) = exp(-z_hi) (1 - z_lo).  Not inlined: the march and three peel-off
// phases call it, and one copy keeps the kernel's instruction footprint small.
struct VoigtCoef {
  static constexpr double A0 = 15.75328153963877, A1 = 286.9341762324778, A2 = 19.05706700907019,
                          A3 = 28.22644017233441, A4 = 9.526399802414186, A5 = 35.29217026286130,
                          A6 = 0.8681020834678775;
  static constexpr double B0 = 0.0003300469163682737, B1 = 0.5403095364583999, B2 = 2.676724102580895,
                          B3 = 12.82026082606220, B4 = 3.21166435627278, B5 = 32.032981933420,
                          B6 = 9.0328158696, B7 = 23.7489999060, B8 = 1.82106170570;
};

template <typename R>
__device__ __noinline__ R voigt(R a, R x) {
  using C = VoigtCoef;
  const R zh = x * x;
  const R zl = m_fma(x, x, -zh);
  const bool core = (zh < R(3)) || (zh == R(3) && zl <= R(0));
  const bool mid = !core && ((zh < R(25)) || (zh == R(25) && zl < R(0)));
  const R z = zh;
  if (core) {
    const R d3 = z - R(C::A6);
    const R d2 = m_fma(z - R(C::A4), d3, R(C::A5));
    const R d1 = m_fma(z - R(C::A2), d2, R(C::A3) * d3);
    const R cf = m_div(R(C::A1) * d2, d1);
    const R ez = m_exp(-zh) * (R(1) - zl);
    return ez * (R(1) - a * (R(C::A0) + cf));
  } else if (mid) {
    const R e4 = z - R(C::B8);
    const R e3 = m_fma(z - R(C::B6), e4, R(C::B7));
    const R e2 = m_fma(z + R(C::B4), e3, R(C::B5) * e4);
    const R e1 = m_fma(z - R(C::B2), e2, R(C::B3) * e3);
    const R cf = m_div(R(C::B1) * e2, e1);
    const R ez = m_exp(-zh) * (R(1) - zl);
    return ez + a * (R(C::B0) + cf);
  } else if (z < R(1e10)) {
    const R f3 = z - R(5.5);
    const R f2 = m_fma(z - R(3.5), f3, R(-5));
    const R f1 = m_fma(z - R(1.5), f2, R(-1.5) * f3);
    return m_div((a * R(1.0 / kSqrtPi)) * f2, f1);
  } else {
    return m_div(a * R(1.0 / kSqrtPi), z - R(1.5));
  }
}

// Sec. 3.2.2, Eq. xcw: rational fit in the natural log of a.
template <typename R>
__device__ __forceinline__ R x_cw_fit(R a) {
  return R(6.9184721) + m_div(R(81.766279), m_log(a) - R(14.651253));
}

// Sec. 3.2.4, Eq. xcrit.
template <typename R>
__device__ __forceinline__ R x_crit_of(R atau0) {
  return atau0 < R(1) ? R(0) : R(0.2) * cbrt(atau0);
}

// ---------------------------------------------------------------- u_par --
// Sec. 3.2.3.  Draws for |x|, sign restored at the end.  Trial t uses Philox
// block 2 + t of the event; the caller passes block 2 (computed alongside the
// event's other blocks).  The proposal angle is carried in units of pi as
// w = (theta + pi/2) / pi in (0, 1), so that tan(theta) = -cos(pi w)/sin(pi w)
// is well conditioned near theta = +-pi/2 in FP32 (sincospi is exact in its
// argument's scaling):
//   |x| <= 1        : w = R1                               (accept R2 < e^{-u^2})
//   lower piece     : w = alpha' R2                        (accept R3 < e^{-u^2})
//   upper piece     : w = alpha' + (1 - alpha') R2         (accept R3 < e^{u0^2-u^2})
// with alpha' = atan2(a, |x| - u0) / pi and p = alpha' / ((1 - e0) alpha' + e0),
// algebraically the paper's theta0 and p.  The |x| <= 1 regime is the lower
// piece with alpha' = 1, its draws taken from the slots the paper's order
// gives it (angle R1, acceptance R2), so both regimes share one trial loop.
template <typename R>
__device__ __forceinline__ R sample_upar(R x, R a, R xcw, const Rng& rng, uint64_t pid, uint32_t event,
                                         const U4<R>& first, int* n_trials) {
  const R xa = fabs(x);
  R u = R(0);
  if (xa >= R(9)) {
    R s, c;
    m_sincospi(R(2) * first.v[1], &s, &c);
    u = m_div(R(1), xa) + m_sqrt(-m_log(first.v[0])) * c;
    *n_trials = 1;
  } else {
    const bool small = xa <= R(1);
    R d = R(0), ap = R(1), p = R(2);   // |x| <= 1: never the upper piece
    if (!small) {
      // d = |x| - u0 taken straight from the two u0 forms (u0_core = x - 1/(x +
      // e^{1-x^2}/a), u0_wing = x_cw - 1/x_cw + 0.15 (x - x_cw)): forming it as
      // |x| - u0 would cancel (d ~ a near |x| = 1) and cost FP32 its accuracy
      d = (xa < xcw) ? m_div(R(1), xa + m_div(m_exp(R(1) - xa * xa), a))
                     : R(0.85) * (xa - xcw) + m_div(R(1), xcw);
      const R u0 = xa - d;
      ap = m_atan2(a, d) * R(1.0 / kPi);
      const R e0 = m_exp(-u0 * u0);
      p = m_div(ap, (R(1) - e0) * ap + e0);
    }
    int t = 0;
    U4<R> q = first;
    for (;;) {
      if (t >= kMaxTrials) { *n_trials = kMaxTrials + 1; break; }
      if (t > 0) q = uniforms<R>(rng, pid, event, 2u + uint32_t(t));
      ++t;
      const R ra = small ? q.v[0] : q.v[1];     // angle draw
      const R rc = small ? q.v[1] : q.v[2];     // acceptance draw
      const bool upper = p < q.v[0];
      // upper piece past w = 1/2: the exact complement 1 - w = (1 - alpha')(1 - R)
      // keeps sin(pi w) well conditioned
      const R w = upper ? m_fma(R(1) - ap, ra, ap) : ap * ra;
      const bool flip = upper && w > R(0.5);
      R s, c;
      m_sincospi(flip ? (R(1) - ap) * (R(1) - ra) : w, &s, &c);
      const R tt = flip ? -m_div(a * c, s) : m_div(a * c, s);   // |x| - u
      u = xa - tt;
      // upper piece: exp(u0^2 - u^2) with u0 - u = tt - d, u0 + u = 2|x| - d - tt
      const R acc = upper ? m_exp((tt - d) * (R(2) * xa - d - tt)) : m_exp(-u * u);
      if (rc < acc) { *n_trials = t; break; }
    }
  }
  return x < R(0) ? -u : u;
}

// Eq. phaseW: invert F(mu) = u for W ~ 1 + RQ mu^2.  (RQ/3) mu^3 + mu - c = 0,
// c = (2u - 1)(1 + RQ/3); one real root, hyperbolic form of Cardano's formula.
template <typename R>
__device__ __forceinline__ R sample_mu(R RQ, R u) {
  if (RQ == R(0)) return R(2) * u - R(1);
  const R c = (R(2) * u - R(1)) * (R(1) + RQ * R(1.0 / 3.0));
  // sqrt(p/3) = sqrt(1/RQ), p = 3/RQ; mu^3 + p mu - p c = 0.  The two values
  // R/Q takes (3/7 in the core, 1 in the wing) use constants.
  R sp3, isp3;
  if (RQ == R(1)) {
    sp3 = R(1);
    isp3 = R(1);
  } else if (RQ == R(3.0 / 7.0)) {
    sp3 = R(1.5275252316519468);     // sqrt(7/3)
    isp3 = R(0.65465367070797714);   // sqrt(3/7)
  } else {
    sp3 = m_sqrt(m_div(R(1), RQ));
    isp3 = m_div(R(1), sp3);
  }
  // root = -2 sqrt(p/3) sinh( asinh( (3q/(2p)) sqrt(3/p) ) / 3 ),  3q/(2p) = -1.5 c
  return R(2) * sp3 * m_sinh(m_asinh(R(1.5) * c * isp3) * R(1.0 / 3.0));
}

// Duff, Burgess, Christensen, Hery, Kensler, Liani, Villemin (2017),
// "Building an Orthonormal Basis, Revisited": e1, e2 perpendicular to n.
template <typename R>
__device__ __forceinline__ void onb(const R n[3], R e1[3], R e2[3]) {
  const R s = m_copysign1(n[2]);
  const R aa = m_div(R(-1), s + n[2]);
  const R bb = n[0] * n[1] * aa;
  e1[0] = R(1) + s * n[0] * n[0] * aa; e1[1] = s * bb; e1[2] = -s * n[0];
  e2[0] = bb; e2[1] = s + n[1] * n[1] * aa; e2[2] = -n[1];
}

// One resonant scattering (Sec. 3.1.3 with Sec. 3.2.3-3.2.4).  The caller
// passes x_cw of the cell's damping parameter (Eq. xcw, x_cw_fit) and the
// event's draw blocks 0 (word 3: core R/Q choice), 1 (u_perp R1, R2, mu, phi)
// and 2 (first u_par trial); later trials draw blocks 3, 4, ...
// Returns outgoing direction, atom velocity and x_f.
template <typename R>
struct ScatterOut {
  R x_f, k_f[3], u_atom[3], u_par, x_crit, RQ, mu;
  int n_trials;
};

template <typename R>
__device__ __forceinline__ ScatterOut<R> scatter_hi(R x, const R k[3], R a, R g, R atau0, int phase,
                                                    const Rng& rng, uint64_t pid, uint32_t event,
                                                    R core_choice, const U4<R>& b1, const U4<R>& b2, R xcw) {
  ScatterOut<R> o;
  R xc = atau0 >= R(0) ? x_crit_of<R>(atau0) : R(0);
  if (fabs(x) >= xc) xc = R(0);
  o.x_crit = xc;
  // u_perp: truncated Box-Muller (Sec. 3.2.4)
  const R rho = m_sqrt(m_fma(xc, xc, -m_log(b1.v[0])));
  R s1, c1;
  m_sincospi(R(2) * b1.v[1], &s1, &c1);
  const R up1 = rho * c1, up2 = rho * s1;
  int nt = 0;
  const R upar = sample_upar<R>(x, a, xcw, rng, pid, event, b2, &nt);
  o.n_trials = nt;
  o.u_par = upar;
  R RQ;
  if (phase == 1) RQ = R(0);
  else if (fabs(x) < xcw) RQ = core_choice < R(1.0 / 3.0) ? R(0) : R(3.0 / 7.0);
  else RQ = R(1);
  o.RQ = RQ;
  const R mu = sample_mu<R>(RQ, b1.v[2]);
  o.mu = mu;
  R sp, cp;
  m_sincospi(R(2) * b1.v[3], &sp, &cp);
  R e1[3], e2[3];
  onb<R>(k, e1, e2);
  const R st = m_sqrt(fmax(R(0), R(1) - mu * mu));
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    o.k_f[i] = mu * k[i] + st * (cp * e1[i] + sp * e2[i]);
    o.u_atom[i] = upar * k[i] + up1 * e1[i] + up2 * e2[i];
  }
  // Eq. x_f with k_i.u_atom = u_par and k_f.u_atom = mu u_par + st (cp up1 + sp up2)
  o.x_f = x + (mu - R(1)) * (upar + g) + st * (cp * up1 + sp * up2);
  return o;
}

}  // namespace colt

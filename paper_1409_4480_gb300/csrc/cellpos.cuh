// Packet position inside its cell, one coordinate per axis in units of the
// cell size (0 = lower face, 1 = upper face).
//
// The FP64 path keeps it in FP64.  The FP32 path keeps an unevaluated float
// pair hi + lo, advanced with Knuth's two-sum: in a very optically thick cell a
// flight is many orders of magnitude shorter than the cell, and a single FP32
// coordinate (resolution 2^-24 of the cell) would lose such steps entirely.
// The pair resolves ~2^-48 of the cell, finer than an FP64 coordinate of the
// whole box for any cell deeper than ~5 levels, and stays on the FP32 pipe
// (GB300's FP64 pipe runs at 1/64 of the FP32 rate).
#pragma once
#include <cuda_runtime.h>

namespace colt {

template <typename R>
struct CellPos {
  R v;
  __device__ __forceinline__ void set(R t) { v = t; }
  __device__ __forceinline__ void set_d(double t) { v = R(t); }
  __device__ __forceinline__ void add(R d) { v += d; }
  __device__ __forceinline__ R val() const { return v; }
  __device__ __forceinline__ R from_top() const { return R(1) - v; }   // 1 - position
  // (n + position) * 2^-e as a new position (n, e small integers, exact scale)
  __device__ __forceinline__ void shift_scale(int n, R scale) { v = (R(n) + v) * scale; }
  // child step of a descent: doubles the coordinate and returns the child bit
  // (upper half when above 1/2, or at 1/2 with a direction component >= 0)
  __device__ __forceinline__ int descend(bool k_nonneg) {
    const R f2 = v + v;
    const int up = (f2 > R(1)) || (f2 == R(1) && k_nonneg);
    v = f2 - R(up);
    return up;
  }
};

template <>
struct CellPos<float> {
  float hi, lo;
  __device__ __forceinline__ void set(float t) { hi = t; lo = 0.f; }
  __device__ __forceinline__ void set_d(double t) {
    hi = (float)t;
    lo = (float)(t - (double)hi);
  }
  __device__ __forceinline__ void add(float d) {
    const float s = __fadd_rn(hi, d);           // two-sum: s + e == hi + d exactly
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(d, bb));
    const float t = __fadd_rn(lo, e);
    hi = __fadd_rn(s, t);                       // renormalise (fast two-sum)
    lo = __fsub_rn(t, __fsub_rn(hi, s));
  }
  __device__ __forceinline__ float val() const { return __fadd_rn(hi, lo); }
  // 1 - hi is exact for hi in [0.5, 2] (Sterbenz) and accurate to 2^-24 of
  // the small result otherwise
  __device__ __forceinline__ float from_top() const { return __fsub_rn(__fsub_rn(1.f, hi), lo); }
  __device__ __forceinline__ void shift_scale(int n, float scale) {
    // (n + hi + lo) * scale with n + hi as an exact pair; scale is a power of two
    const float nf = (float)n;
    const float s = __fadd_rn(nf, hi);
    const float bb = __fsub_rn(s, nf);
    const float e = __fadd_rn(__fsub_rn(nf, __fsub_rn(s, bb)), __fsub_rn(hi, bb));
    const float t = __fadd_rn(lo, e);
    const float h2 = __fadd_rn(s, t);
    lo = __fmul_rn(__fsub_rn(t, __fsub_rn(h2, s)), scale);
    hi = __fmul_rn(h2, scale);
  }
  __device__ __forceinline__ int descend(bool k_nonneg) {
    const float h2 = __fadd_rn(hi, hi), l2 = __fadd_rn(lo, lo);   // exact
    const int up = (h2 > 1.f) || (h2 == 1.f && (l2 > 0.f || (l2 == 0.f && k_nonneg)));
    hi = __fsub_rn(h2, (float)up);             // exact: h2 in [1, 2) when up
    lo = l2;
    return up;
  }
};

}  // namespace colt

// scalar.cuh -- scalar types of the device code: double, and forward-mode dual numbers (value plus one
// or K directional derivatives) used by the discrete adjoint for exact Hessian-vector and mixed
// parameter-state terms.  The helpers below reduce to the plain double operations for double, so the
// forward integrator's arithmetic is unchanged by the templating.
#pragma once

#include "elementary_tables.h"

namespace chemgb {

// e^x by table-driven reduction (Tang, ACM TOMS 15(2), 1989), in a variant with 256 table entries:
//   k = nearest integer to 256 x / ln2, read from the low word of x * 256/ln2 + 1.5 * 2^52;
//   r = x - k ln2/256 in two fused steps (the first is exact because k * kExpCHi is), |r| <= ln2/512;
//   e^r - 1 = r (1 + r/2 + r^2/6 + r^3/24), truncation below r^5/120 < 4e-17 relative;
//   e^x = 2^m * T[j] * e^r with k = 256 m + j, the power of two added to the exponent field.
// Nine FP64 operations; error about one ulp.  |x| >= 704 (results near overflow or in the subnormal
// range) and NaN take the library exp.
__device__ __forceinline__ double fast_exp(double x) {
  if ((__double2hiint(x) & 0x7fffffff) >= 0x40860000) return exp(x);
  constexpr double kShift = 0x1.8p52;
  const double t = fma(x, kExpInvC, kShift);
  const int k = __double2loint(t);
  const double kd = t - kShift;
  double r = fma(kd, -kExpCHi, x);
  r = fma(kd, -kExpCLo, r);
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  q = fma(r, q, 1.0);
  const double tj = __ldg(kExpTab + (k & 255));
  const double e = fma(tj, r * q, tj);
  return __hiloint2double(__double2hiint(e) + (k >> 8) * (1 << 20), __double2loint(e));
}

struct Dual {
  double v, d;
  __device__ __forceinline__ Dual() = default;
  __device__ __forceinline__ constexpr Dual(double x) : v(x), d(0.0) {}
  __device__ __forceinline__ constexpr Dual(double x, double dx) : v(x), d(dx) {}
};

__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, fma(a.v, b.d, a.d * b.v)); }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
__device__ __forceinline__ Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
__device__ __forceinline__ Dual operator/(double a, Dual b) {
  const double q = a / b.v;
  return Dual(q, -q * b.d / b.v);
}
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
__device__ __forceinline__ Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
__device__ __forceinline__ Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
__device__ __forceinline__ Dual& operator*=(Dual& a, double b) { a = a * b; return a; }

// ---- several directional derivatives at once: value and K tangents.  The discrete adjoint needs the
// Jacobian's derivative along the four stage vectors of a step at the same point; one evaluation with
// K = 4 tangents shares the value arithmetic (and every exp, log and division) among the four.
template <int K>
struct DualN {
  double v, d[K];
  __device__ __forceinline__ DualN() = default;
  __device__ __forceinline__ DualN(double x) : v(x) {
#pragma unroll
    for (int i = 0; i < K; ++i) d[i] = 0.0;
  }
};
using Dual4 = DualN<4>;

template <int K>
__device__ __forceinline__ DualN<K> operator+(const DualN<K>& a, const DualN<K>& b) {
  DualN<K> r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int K>
__device__ __forceinline__ DualN<K> operator-(const DualN<K>& a, const DualN<K>& b) {
  DualN<K> r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int K>
__device__ __forceinline__ DualN<K> operator-(const DualN<K>& a) {
  DualN<K> r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int K>
__device__ __forceinline__ DualN<K> operator*(const DualN<K>& a, const DualN<K>& b) {
  DualN<K> r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = fma(a.v, b.d[i], a.d[i] * b.v);
  return r;
}
template <int K>
__device__ __forceinline__ DualN<K> operator*(const DualN<K>& a, double b) {
  DualN<K> r; r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int K>
__device__ __forceinline__ DualN<K> operator*(double a, const DualN<K>& b) { return b * a; }
template <int K>
__device__ __forceinline__ DualN<K> operator+(const DualN<K>& a, double b) { DualN<K> r = a; r.v += b; return r; }
template <int K>
__device__ __forceinline__ DualN<K> operator+(double a, const DualN<K>& b) { return b + a; }
template <int K>
__device__ __forceinline__ DualN<K> operator-(const DualN<K>& a, double b) { DualN<K> r = a; r.v -= b; return r; }
template <int K>
__device__ __forceinline__ DualN<K> operator-(double a, const DualN<K>& b) { return (-b) + a; }
template <int K>
__device__ __forceinline__ DualN<K> operator/(const DualN<K>& a, const DualN<K>& b) {
  const double ib = 1.0 / b.v;
  DualN<K> r; r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <int K>
__device__ __forceinline__ DualN<K> operator/(const DualN<K>& a, double b) {
  const double ib = 1.0 / b;
  DualN<K> r; r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * ib;
  return r;
}
template <int K>
__device__ __forceinline__ DualN<K> operator/(double a, const DualN<K>& b) {
  const double ib = 1.0 / b.v;
  DualN<K> r; r.v = a * ib;
  const double s = -r.v * ib;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = s * b.d[i];
  return r;
}
template <int K>
__device__ __forceinline__ DualN<K>& operator+=(DualN<K>& a, const DualN<K>& b) { a = a + b; return a; }
template <int K>
__device__ __forceinline__ DualN<K>& operator-=(DualN<K>& a, const DualN<K>& b) { a = a - b; return a; }
template <int K>
__device__ __forceinline__ DualN<K>& operator*=(DualN<K>& a, const DualN<K>& b) { a = a * b; return a; }
template <int K>
__device__ __forceinline__ DualN<K>& operator*=(DualN<K>& a, double b) { a = a * b; return a; }

// fused multiply-add, exp, log, value part, and the warp-level all-reduce sum
__device__ __forceinline__ double sfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ Dual sfma(Dual a, Dual b, Dual c) {
  return Dual(fma(a.v, b.v, c.v), fma(a.v, b.d, fma(a.d, b.v, c.d)));
}
// ln x by table-driven reduction (Tang, ACM TOMS 16(4), 1990), in a variant with 256 table entries:
//   x = 2^k y, y in [1, 2); j = top 8 bits of y's fraction; u = y c_j - 1 with c_j the rounded reciprocal
//   of the centre of y's interval (1 and 2 for the first and last intervals), |u| <= 2^-8;
//   ln x = (k ln2_lead + lnF_lead_j) + (k ln2_trail + lnF_trail_j + log1p(u)), where lnF_j = -ln c_j
//   (so the rounding of c_j needs no correction) and the first sum is exact (leads on the grid 2^-43);
//   log1p(u) = u - u^2 (1/2 - u/3 + u^2/4 - u^3/5 + u^4/6 - u^5/7), truncation below 2^-59 relative.
// Thirteen FP64 operations; error about one ulp; ln of values near 1 keeps full relative accuracy.
// Zero, negative, subnormal, infinite and NaN arguments take the library log.
__device__ __forceinline__ double fast_log(double x) {
  const int hx = __double2hiint(x);
  if (hx < 0x00100000 || hx >= 0x7ff00000) return log(x);
  const int k = (hx >> 20) - 1023;
  const int j = (hx >> 12) & 0xff;
  const double y = __hiloint2double((hx & 0x000fffff) | 0x3ff00000, __double2loint(x));
  const double* tb = kLogTab[j];
  const double c = __ldg(tb), lead = __ldg(tb + 1), trail = __ldg(tb + 2);
  const double u = fma(y, c, -1.0);
  double q = fma(u, -1.0 / 7.0, 1.0 / 6.0);
  q = fma(u, q, -1.0 / 5.0);
  q = fma(u, q, 1.0 / 4.0);
  q = fma(u, q, -1.0 / 3.0);
  q = fma(u, q, 0.5);
  const double p = fma(-(u * u), q, u);
  // k as a double without a conversion instruction: 2^52 + 2^31 + k from its bits, minus 2^52 + 2^31
  const double kd = __hiloint2double(0x43300000, k ^ (int)0x80000000) - 0x1.00000800p52;
  const double t1 = fma(kd, kLn2Lead, lead);
  const double t2 = fma(kd, kLn2Trail, trail) + p;
  return t1 + t2;
}

__device__ __forceinline__ double sexp(double a) { return fast_exp(a); }
__device__ __forceinline__ Dual sexp(Dual a) {
  const double e = fast_exp(a.v);
  return Dual(e, a.d * e);
}
template <int K>
__device__ __forceinline__ DualN<K> sfma(const DualN<K>& a, const DualN<K>& b, const DualN<K>& c) {
  DualN<K> r; r.v = fma(a.v, b.v, c.v);
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = fma(a.v, b.d[i], fma(a.d[i], b.v, c.d[i]));
  return r;
}
template <int K>
__device__ __forceinline__ DualN<K> sexp(const DualN<K>& a) {
  DualN<K> r; r.v = fast_exp(a.v);
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * r.v;
  return r;
}
template <int K>
__device__ __forceinline__ DualN<K> slog(const DualN<K>& a) {
  DualN<K> r; r.v = fast_log(a.v);
  const double ia = 1.0 / a.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * ia;
  return r;
}
__device__ __forceinline__ double slog(double a) { return fast_log(a); }
__device__ __forceinline__ Dual slog(Dual a) { return Dual(fast_log(a.v), a.d / a.v); }
__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double val(Dual a) { return a.v; }
template <int K>
__device__ __forceinline__ double val(const DualN<K>& a) { return a.v; }
__device__ __forceinline__ double tangent(Dual a) { return a.d; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;   // identical on every lane (each butterfly stage adds the same pair of operands)
}
__device__ __forceinline__ Dual warp_sum(Dual a) { return Dual(warp_sum(a.v), warp_sum(a.d)); }
template <int K>
__device__ __forceinline__ DualN<K> warp_sum(DualN<K> a) {
  a.v = warp_sum(a.v);
#pragma unroll
  for (int i = 0; i < K; ++i) a.d[i] = warp_sum(a.d[i]);
  return a;
}

}  // namespace chemgb

// scalar.cuh -- scalar types of the device code: double, and a forward-mode dual number (value plus one
// directional derivative) used by the discrete adjoint for exact Hessian-vector and mixed
// parameter-state terms.  The helpers below reduce to the plain double operations for double, so the
// forward integrator's arithmetic is unchanged by the templating.
#pragma once

namespace chemgb {

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

// fused multiply-add, exp, log, value part, and the warp-level all-reduce sum
__device__ __forceinline__ double sfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ Dual sfma(Dual a, Dual b, Dual c) {
  return Dual(fma(a.v, b.v, c.v), fma(a.v, b.d, fma(a.d, b.v, c.d)));
}
__device__ __forceinline__ double sexp(double a) { return exp(a); }
__device__ __forceinline__ Dual sexp(Dual a) {
  const double e = exp(a.v);
  return Dual(e, a.d * e);
}
__device__ __forceinline__ double slog(double a) { return log(a); }
__device__ __forceinline__ Dual slog(Dual a) { return Dual(log(a.v), a.d / a.v); }
__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double val(Dual a) { return a.v; }
__device__ __forceinline__ double tangent(Dual a) { return a.d; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;   // identical on every lane (each butterfly stage adds the same pair of operands)
}
__device__ __forceinline__ Dual warp_sum(Dual a) { return Dual(warp_sum(a.v), warp_sum(a.d)); }

}  // namespace chemgb

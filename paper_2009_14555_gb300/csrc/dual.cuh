// dual.cuh - forward-mode dual numbers (value, derivative) for the adjoint.
//
// The adjoint sweep needs vector-Jacobian products of small local functions
// (one face flux of its 6-cell stencil, one cell's plastic and reactive
// update).  Each local Jacobian column is obtained by evaluating the same
// templated closure code on Dual numbers seeded along one input; comparisons
// and min/max act on the value, so the branch taken (limiter, BVD choice,
// Riemann region, radial return) is the forward one.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace dis {

// Keep the double overloads visible next to the Dual ones below (unqualified
// calls inside this namespace would otherwise see only the Dual versions).
using ::cbrt;
using ::copysign;
using ::cosh;
using ::exp;
using ::fabs;
using ::fmax;
using ::fmin;
using ::sqrt;
using ::tanh;

struct Dual {
  double v, d;
  __host__ __device__ Dual() : v(0.0), d(0.0) {}
  __host__ __device__ Dual(double x) : v(x), d(0.0) {}
  __host__ __device__ Dual(double x, double dx) : v(x), d(dx) {}
};

__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
// the value rounded on its own (physics.cuh: contact speed numerator)
__device__ __forceinline__ Dual mul_rn(Dual a, Dual b) { return Dual(__dmul_rn(a.v, b.v), a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
__device__ __forceinline__ Dual operator/(double a, Dual b) {
  const double q = a / b.v;
  return Dual(q, -q * b.d / b.v);
}
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
__device__ __forceinline__ Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
__device__ __forceinline__ Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }

__device__ __forceinline__ bool operator<(Dual a, Dual b) { return a.v < b.v; }
__device__ __forceinline__ bool operator>(Dual a, Dual b) { return a.v > b.v; }
__device__ __forceinline__ bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
__device__ __forceinline__ bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
__device__ __forceinline__ bool operator==(Dual a, Dual b) { return a.v == b.v; }
__device__ __forceinline__ bool operator!=(Dual a, Dual b) { return a.v != b.v; }
__device__ __forceinline__ bool operator<(Dual a, double b) { return a.v < b; }
__device__ __forceinline__ bool operator>(Dual a, double b) { return a.v > b; }
__device__ __forceinline__ bool operator<=(Dual a, double b) { return a.v <= b; }
__device__ __forceinline__ bool operator>=(Dual a, double b) { return a.v >= b; }
__device__ __forceinline__ bool operator==(Dual a, double b) { return a.v == b; }
__device__ __forceinline__ bool operator!=(Dual a, double b) { return a.v != b; }
__device__ __forceinline__ bool operator<(double a, Dual b) { return a < b.v; }
__device__ __forceinline__ bool operator>(double a, Dual b) { return a > b.v; }

__device__ __forceinline__ Dual sqrt(Dual a) {
  const double s = ::sqrt(a.v);
  return Dual(s, s > 0.0 ? a.d / (2.0 * s) : 0.0);
}
__device__ __forceinline__ Dual cbrt(Dual a) {
  const double c = ::cbrt(a.v);
  return Dual(c, a.d / (3.0 * c * c));
}
__device__ __forceinline__ Dual log(Dual a) { return Dual(::log(a.v), a.d / a.v); }
__device__ __forceinline__ Dual powr(Dual a, Dual b) {
  const double v = ::pow(a.v, b.v);
  return Dual(v, v * (b.d * ::log(a.v) + b.v * a.d / a.v));
}
__device__ __forceinline__ Dual exp(Dual a) {
  const double e = ::exp(a.v);
  return Dual(e, e * a.d);
}
__device__ __forceinline__ Dual tanh(Dual a) {
  const double t = ::tanh(a.v);
  return Dual(t, (1.0 - t * t) * a.d);
}
__device__ __forceinline__ Dual cosh(Dual a) { return Dual(::cosh(a.v), ::sinh(a.v) * a.d); }
// Non-differentiable points take the conventions of PyTorch's autograd (the
// float64 oracle's reverse mode): |x| has derivative 0 at 0, and min / max of
// two equal values pass half of the derivative to each argument.
__device__ __forceinline__ Dual fabs(Dual a) { return a.v < 0.0 ? -a : (a.v > 0.0 ? a : Dual(0.0, 0.0)); }
__device__ __forceinline__ Dual fmin(Dual a, Dual b) {
  return b.v < a.v ? b : (a.v < b.v ? a : Dual(a.v, 0.5 * (a.d + b.d)));
}
__device__ __forceinline__ Dual fmax(Dual a, Dual b) {
  return b.v > a.v ? b : (a.v > b.v ? a : Dual(a.v, 0.5 * (a.d + b.d)));
}
__device__ __forceinline__ Dual copysign(Dual a, Dual b) {
  return ((a.v < 0.0) != (b.v < 0.0)) ? -a : a;
}

__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(Dual x) { return x.v; }

}  // namespace dis

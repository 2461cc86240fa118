// First-order forward-mode dual numbers a + b eps (eps^2 = 0) for the device
// chemistry code.  Pushing a state y + eps K through the Jacobian code gives
// J(y) and its directional derivative dJ(y)[K] exactly (no differencing); the
// discrete adjoint uses that for the second-derivative terms of the
// Rosenbrock step.
#pragma once
#include "fastexp.cuh"

namespace df {

// keep the double overloads visible next to the Dual ones inside namespace df
using ::log;
using ::log10;
using ::sqrt;

struct Dual {
  double v, d;
  __host__ __device__ Dual() : v(0.0), d(0.0) {}
  __host__ __device__ Dual(double a) : v(a), d(0.0) {}
  __host__ __device__ Dual(double a, double b) : v(a), d(b) {}
  __device__ Dual& operator+=(const Dual& o) { v += o.v; d += o.d; return *this; }
  __device__ Dual& operator-=(const Dual& o) { v -= o.v; d -= o.d; return *this; }
  __device__ Dual& operator*=(const Dual& o) { d = d * o.v + v * o.d; v *= o.v; return *this; }
};

__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double iv = 1.0 / b.v;
  const double q = a.v * iv;
  return Dual(q, (a.d - q * b.d) * iv);
}
__device__ __forceinline__ Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
__device__ __forceinline__ Dual operator/(double a, Dual b) {
  const double q = a / b.v;
  return Dual(q, -q * b.d / b.v);
}

__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(const Dual& x) { return x.v; }

__device__ __forceinline__ Dual exp_tang(Dual x, const double2* tab) {
  const double e = exp_tang(x.v, tab);
  return Dual(e, e * x.d);
}
__device__ __forceinline__ Dual log(Dual x) { return Dual(::log(x.v), x.d / x.v); }
__device__ __forceinline__ Dual log10(Dual x) { return Dual(::log10(x.v), x.d / (x.v * 2.302585092994045684)); }
__device__ __forceinline__ Dual sqrt(Dual x) {
  const double s = ::sqrt(x.v);
  return Dual(s, 0.5 * x.d / s);
}

}  // namespace df

// Forward-mode differentiation of the force field by dual numbers x + eps x' (eps^2 = 0), in FP64.
// Running the force terms on positions q + eps v gives F(q) + eps J_F(q) v, where J_F = -H is minus
// the Hessian of V: the Hessian-vector product that the adjoint of the Langevin step needs.  Only the
// tangent part is accumulated (the value part is the ordinary force, known already).
#pragma once
#include "forcefield.cuh"

namespace grp {

struct Dual {
  double v, d;  // value, tangent
  __device__ __forceinline__ Dual() : v(0.0), d(0.0) {}
  __device__ __forceinline__ Dual(double x) : v(x), d(0.0) {}
  __device__ __forceinline__ Dual(double x, double t) : v(x), d(t) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual &operator+=(Dual &a, Dual b) { a = a + b; return a; }
__device__ __forceinline__ Dual &operator-=(Dual &a, Dual b) { a = a - b; return a; }
__device__ __forceinline__ Dual &operator*=(Dual &a, Dual b) { a = a * b; return a; }
__device__ __forceinline__ Dual &operator/=(Dual &a, Dual b) { a = a / b; return a; }
// comparisons look at the value only (branch decisions are those of the undifferentiated code)
__device__ __forceinline__ bool operator>(Dual a, Dual b) { return a.v > b.v; }
__device__ __forceinline__ bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
__device__ __forceinline__ bool operator<(Dual a, Dual b) { return a.v < b.v; }
// d sqrt(x) = dx / (2 sqrt x); d (1/x) = -dx / x^2; d atan2(y, x) = (x dy - y dx) / (x^2 + y^2)
__device__ __forceinline__ Dual gsqrt(Dual a) {
  const double s = sqrt(a.v);
  return {s, a.d / (2.0 * s)};
}
__device__ __forceinline__ Dual grcp(Dual a) {
  const double r = 1.0 / a.v;
  return {r, -a.d * r * r};
}
// d (x^-1/2) = -dx / (2 x^3/2)
__device__ __forceinline__ Dual grsqrt(Dual a) {
  const double r = 1.0 / sqrt(a.v);
  return {r, -0.5 * a.d * r * r * r};
}
__device__ __forceinline__ Dual gdiv(Dual a, Dual b) { return a / b; }
__device__ __forceinline__ Dual gatan2(Dual y, Dual x) {
  return {atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / (x.v * x.v + y.v * y.v)};
}

// Tangent accumulator: sum of the eps parts of the force contributions, 2^-40 fixed point.
struct AccTangent {
  long long *F;  // [3n]
  __device__ __forceinline__ void add(int a, V3<Dual> g, int *err) const {
    fix_add(&F[3 * a + 0], to_fix(g.x.d, err));
    fix_add(&F[3 * a + 1], to_fix(g.y.d, err));
    fix_add(&F[3 * a + 2], to_fix(g.z.d, err));
  }
  __device__ __forceinline__ long long efix(Dual, int *) const { return 0; }
};

struct PathTangent {
  using T = Dual;
  using Acc = AccTangent;
  static constexpr bool kMixed = false;
};

// Positions q + eps v (both [3n] FP64).
template <>
struct Pos<PathTangent> {
  const double *q, *v;
  __device__ __forceinline__ V3<Dual> diff(int i, int j) const {
    return {Dual(q[3 * i] - q[3 * j], v[3 * i] - v[3 * j]), Dual(q[3 * i + 1] - q[3 * j + 1], v[3 * i + 1] - v[3 * j + 1]),
            Dual(q[3 * i + 2] - q[3 * j + 2], v[3 * i + 2] - v[3 * j + 2])};
  }
};
template <>
struct Params<PathTangent> {
  const double4 *atom;
  const double2 *bond, *angle;
  const double4 *term;
  int rf;
  double krf, crf;
  double box[3], ibox[3], beta;
};

}  // namespace grp

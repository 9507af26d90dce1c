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

// ---- the same in FP32, for the adjoint of the mixed path: tangents of FP32 force terms, summed in the
// mixed path's split fixed point (2^-32 units, contributions below 2^18).
struct DualF {
  float v, d;  // value, tangent
  __device__ __forceinline__ DualF() : v(0.f), d(0.f) {}
  __device__ __forceinline__ DualF(float x) : v(x), d(0.f) {}
  __device__ __forceinline__ DualF(float x, float t) : v(x), d(t) {}
};
__device__ __forceinline__ DualF operator+(DualF a, DualF b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ DualF operator-(DualF a, DualF b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ DualF operator-(DualF a) { return {-a.v, -a.d}; }
__device__ __forceinline__ DualF operator*(DualF a, DualF b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ DualF operator/(DualF a, DualF b) {
  const float q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ DualF &operator+=(DualF &a, DualF b) { a = a + b; return a; }
__device__ __forceinline__ DualF &operator-=(DualF &a, DualF b) { a = a - b; return a; }
__device__ __forceinline__ DualF &operator*=(DualF &a, DualF b) { a = a * b; return a; }
__device__ __forceinline__ DualF &operator/=(DualF &a, DualF b) { a = a / b; return a; }
__device__ __forceinline__ bool operator>(DualF a, DualF b) { return a.v > b.v; }
__device__ __forceinline__ bool operator>=(DualF a, DualF b) { return a.v >= b.v; }
__device__ __forceinline__ bool operator<(DualF a, DualF b) { return a.v < b.v; }
__device__ __forceinline__ DualF gsqrt(DualF a) {
  const float s = sqrtf(a.v);
  return {s, a.d / (2.f * s)};
}
__device__ __forceinline__ DualF grcp(DualF a) {
  const float r = 1.f / a.v;
  return {r, -a.d * r * r};
}
__device__ __forceinline__ DualF grsqrt(DualF a) {
  const float r = rsqrtf(a.v);
  return {r, -0.5f * a.d * r * r * r};
}
__device__ __forceinline__ DualF gdiv(DualF a, DualF b) { return a / b; }
__device__ __forceinline__ DualF gatan2(DualF y, DualF x) {
  return {atan2f(y.v, x.v), (x.v * y.d - y.v * x.d) / (x.v * x.v + y.v * y.v)};
}

// Tangent accumulator of the mixed path: the eps parts in the split words ([3n] hi, then [3n] lo).
struct AccTangentF {
  int *hi;
  unsigned int *lo;
  __device__ __forceinline__ void add(int a, V3<DualF> g, int *err) const {
    split_add(hi, lo, 3 * a + 0, to_split(g.x.d, err));
    split_add(hi, lo, 3 * a + 1, to_split(g.y.d, err));
    split_add(hi, lo, 3 * a + 2, to_split(g.z.d, err));
  }
  __device__ __forceinline__ long long efix(DualF, int *) const { return 0; }
};

struct PathTangentF {
  using T = DualF;
  using Acc = AccTangentF;
  static constexpr bool kMixed = false;  // the generic (not double-single) term code, in FP32
};

// Positions q + eps v: differences taken in FP64 from the recomputed double-single state, then rounded
// to FP32 (q and v [3n] FP64).
template <>
struct Pos<PathTangentF> {
  const double *q, *v;
  __device__ __forceinline__ V3<DualF> diff(int i, int j) const {
    return {DualF((float)(q[3 * i] - q[3 * j]), (float)(v[3 * i] - v[3 * j])),
            DualF((float)(q[3 * i + 1] - q[3 * j + 1]), (float)(v[3 * i + 1] - v[3 * j + 1])),
            DualF((float)(q[3 * i + 2] - q[3 * j + 2]), (float)(v[3 * i + 2] - v[3 * j + 2]))};
  }
};
template <>
struct Params<PathTangentF> {
  const float4 *atom;
  const float2 *bond, *angle;
  const float4 *term;
  int rf;
  float krf, crf;
  float box[3], ibox[3], beta;
};

}  // namespace grp

// Force-field terms of the potential V of Eq. 1 evaluated by one thread per term, accumulated into
// fixed point in shared memory.  T = double (FP64 path) or float (mixed path).
#pragma once
#include "common.cuh"

#include <type_traits>

namespace grp {

template <class T>
struct V3 {
  T x, y, z;
};
template <class T>
__device__ __forceinline__ T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T>
__device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double gsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float gsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double gexp(double x) { return exp(x); }
__device__ __forceinline__ float gexp(float x) { return expf(x); }
__device__ __forceinline__ double gatan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float gatan2(float y, float x) { return atan2f(y, x); }
// reciprocal and quotient: IEEE in FP64, the hardware approximations (about 1 ulp) in FP32
__device__ __forceinline__ double grcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float grcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// reciprocal square root: IEEE-rounded quotient in FP64, the hardware approximation in FP32
__device__ __forceinline__ double grsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float grsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double gdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float gdiv(float a, float b) { return __fdividef(a, b); }

// FP64 path: int64 accumulators in 2^-40 units, updated as two 32-bit words with carry.
struct AccF64 {
  long long *F;  // [3n]
  static constexpr double kInv = kFixInv;
  __device__ __forceinline__ void add(int a, V3<double> g, int *err) const {
    fix_add(&F[3 * a + 0], to_fix(g.x, err));
    fix_add(&F[3 * a + 1], to_fix(g.y, err));
    fix_add(&F[3 * a + 2], to_fix(g.z, err));
  }
  __device__ __forceinline__ long long efix(double e, int *err) const { return to_fix(e, err); }
};
// Mixed path: split hi/lo words in 2^-32 units (see Split).
struct AccMixed {
  int *hi;           // [3n]
  unsigned int *lo;  // [3n]
  static constexpr double kInv = 2.3283064365386963e-10;  // 2^-32
  __device__ __forceinline__ void add(int a, V3<float> g, int *err) const {
    split_add(hi, lo, 3 * a + 0, to_split(g.x, err));
    split_add(hi, lo, 3 * a + 1, to_split(g.y, err));
    split_add(hi, lo, 3 * a + 2, to_split(g.z, err));
  }
  __device__ __forceinline__ long long efix(float e, int *err) const { return split_value(to_split(e, err)); }
};

// Precision traits.
struct PathF64 {
  using T = double;
  using Acc = AccF64;
  static constexpr bool kMixed = false;
};
struct PathMixed {
  using T = float;
  using Acc = AccMixed;
  static constexpr bool kMixed = true;
};

// Shared-memory view of one replica's positions.
template <class P>
struct Pos;
template <>
struct Pos<PathF64> {
  const double *q;  // [3n]
  __device__ __forceinline__ V3<double> diff(int i, int j) const {  // q_i - q_j
    return {q[3 * i] - q[3 * j], q[3 * i + 1] - q[3 * j + 1], q[3 * i + 2] - q[3 * j + 2]};
  }
  // one atom's position held in registers (tile loops)
  struct At {
    double x, y, z;
  };
  __device__ __forceinline__ At at(int i) const { return {q[3 * i], q[3 * i + 1], q[3 * i + 2]}; }
  __device__ __forceinline__ static V3<double> diff(const At &a, const At &b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
};
template <>
struct Pos<PathMixed> {
  const float4 *qh, *ql;  // [n] double-single positions
  __device__ __forceinline__ V3<float> diff(int i, int j) const {
    const float4 a = qh[i], b = qh[j], c = ql[i], d = ql[j];
    return {(a.x - b.x) + (c.x - d.x), (a.y - b.y) + (c.y - d.y), (a.z - b.z) + (c.z - d.z)};
  }
  struct At {
    float4 h, l;
  };
  __device__ __forceinline__ At at(int i) const { return {qh[i], ql[i]}; }
  __device__ __forceinline__ static V3<float> diff(const At &a, const At &b) {
    return {(a.h.x - b.h.x) + (a.l.x - b.l.x), (a.h.y - b.h.y) + (a.l.y - b.l.y), (a.h.z - b.h.z) + (a.l.z - b.l.z)};
  }
};

// Parameter arrays of a path (device pointers, FP64 or FP32 copies).
template <class P>
struct Params;
template <>
struct Params<PathF64> {
  const double4 *atom;  // (sigma/2, sqrt(eps), q sqrt(k_e/4), 1/m), may live in shared memory
  const double2 *bond, *angle;
  const double4 *term;
  int rf;               // Coulomb model: 0 eps = 4r, 1 reaction field (k_rf, c_rf), 2 Ewald real space
  double krf, crf;
  double box[3], ibox[3], beta;  // periodic box edges, their inverses, Ewald splitting parameter
};
template <>
struct Params<PathMixed> {
  const float4 *atom;
  const float2 *bond, *angle;
  const float4 *term;
  int rf;
  float krf, crf;
  float box[3], ibox[3], beta;
};

// Pair force factor -dE/dr / r and pair energy of Lennard-Jones (given eps_ij and (sigma_ij/r)^6) plus
// Coulomb (qq = k_e q_i q_j / 4).  Dielectric eps = 4r: E_C = qq / r^2, -dE_C/dr / r = 2 qq / r^4.
// Reaction field (eps_r = 1, a continuum of dielectric eps_rf beyond the cutoff r_c, as the
// non-periodic cutoff scheme of the paper's MD setups): E_C = 4 qq (1/r + k_rf r^2 - c_rf) with
// k_rf = (eps_rf - 1) / ((2 eps_rf + 1) r_c^3), c_rf = 1/r_c + k_rf r_c^2 (zero at the cutoff), and
// -dE_C/dr / r = 4 qq (1/r^3 - 2 k_rf).  Ewald real space (a periodic box, the rest of the lattice
// sum on the particle mesh): E_C = 4 qq erfc(beta r) / r and
// -dE_C/dr / r = 4 qq (erfc(beta r) / r + 2 beta / sqrt(pi) exp(-beta^2 r^2)) / r^2.
// kRF: 0 = eps = 4r, 1 = reaction field, 2 = Ewald real space, -1 = as par.rf says (decided per pair;
// the segment kernel fixes it per pass instead, keeping the branch out of its pair loops).
constexpr double kTwoOverSqrtPi = 1.1283791670955126;  // 2 / sqrt(pi)
// erfc(x) for x >= 0 given e = exp(-x^2): the library function in FP64; in FP32 the rational
// approximation of Abramowitz and Stegun (Handbook of Mathematical Functions, 1964, formula 7.1.26),
// erfc(x) = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2), t = 1 / (1 + p x), absolute error below
// 1.5e-7 (the FP32 rounding of the pair terms is ~6e-8 relative), which reuses the exponential the
// force needs anyway.
__device__ __forceinline__ double gerfc_e(double x, double) { return erfc(x); }
__device__ __forceinline__ float gerfc_e(float x, float e) {
  const float t = grcp(fmaf(0.3275911f, x, 1.0f));
  const float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                              0.254829592f);
  return poly * e;
}
__device__ __forceinline__ double gerf(double x) { return erf(x); }
__device__ __forceinline__ float gerf(float x) { return erff(x); }
__device__ __forceinline__ double gnearest(double x) { return rint(x); }
__device__ __forceinline__ float gnearest(float x) { return rintf(x); }

template <int kRF, class T, class Par>
__device__ __forceinline__ T pair_g(const Par &par, T eps, T s6, T qq, T r2, T inv_r2) {
  const int mode = kRF < 0 ? par.rf : kRF;
  if (mode == 0) return (T(24) * eps * (T(2) * s6 * s6 - s6) + T(2) * qq * inv_r2) * inv_r2;
  const T lj = T(24) * eps * (T(2) * s6 * s6 - s6) * inv_r2;
  if constexpr (std::is_floating_point<T>::value) {  // the tangent path never sees a periodic system
    if (mode == 2) {
      const T b = T(par.beta), ir = grsqrt(r2), e = gexp(-b * b * r2);
      return lj + T(4) * qq * (gerfc_e(b * r2 * ir, e) * ir + T(kTwoOverSqrtPi) * b * e) * inv_r2;
    }
  }
  return lj + T(4) * qq * (grsqrt(r2) * inv_r2 - T(2) * T(par.krf));
}
template <int kRF, class T, class Par>
__device__ __forceinline__ T pair_e(const Par &par, T eps, T s6, T qq, T r2, T inv_r2) {
  const int mode = kRF < 0 ? par.rf : kRF;
  if (mode == 0) return T(4) * eps * (s6 * s6 - s6) + qq * inv_r2;
  if constexpr (std::is_floating_point<T>::value) {
    if (mode == 2) {
      const T b = T(par.beta), ir = grsqrt(r2);
      return T(4) * eps * (s6 * s6 - s6) + T(4) * qq * gerfc_e(b * r2 * ir, gexp(-b * b * r2)) * ir;
    }
  }
  return T(4) * eps * (s6 * s6 - s6) + T(4) * qq * (grsqrt(r2) + T(par.krf) * r2 - T(par.crf));
}

// The nearest periodic image of a pair difference (Ewald real space; a no-op otherwise).
template <int kRF, class T, class Par>
__device__ __forceinline__ V3<T> pair_image(const Par &par, V3<T> d) {
  if constexpr (std::is_floating_point<T>::value) {
    const int mode = kRF < 0 ? par.rf : kRF;
    if (mode == 2) {
      d.x -= T(par.box[0]) * gnearest(d.x * T(par.ibox[0]));
      d.y -= T(par.box[1]) * gnearest(d.y * T(par.ibox[1]));
      d.z -= T(par.box[2]) * gnearest(d.z * T(par.ibox[2]));
    }
  }
  return d;
}

// Nonbonded parameters of an atom held in registers by the tile and row loops: sigma/2, sqrt(eps) and
// the scaled charge q sqrt(k_e/4).  The mixed path keeps sigma/2 and sqrt(eps) in the spare fourth
// words of the double-single position (State<PathMixed>::load), one shared-memory load fewer per pair
// in loops that are bound by shared-memory traffic; the charge comes from the parameter table.
template <class P>
__device__ __forceinline__ void nb_params(const typename Pos<P>::At &pa, const Params<P> &par, int a,
                                          typename P::T &sh, typename P::T &se, typename P::T &qc) {
  if constexpr (P::kMixed) {
    sh = pa.h.w;
    se = pa.l.w;
    qc = par.atom[a].z;
  } else {
    const auto p = par.atom[a];
    sh = p.x;
    se = p.y;
    qc = p.z;
  }
}

// Lennard-Jones (Lorentz-Berthelot) + Coulomb with eps(r) = 4r for the pair (i, j): force on i
// (minus the force on j) and the pair energy; false beyond the cutoff.
template <class P, int kRF = -1>
__device__ __forceinline__ bool pair_eval(const Pos<P> &pos, const Params<P> &par, int i, int j,
                                          typename P::T cutoff2, V3<typename P::T> &fi, typename P::T &e,
                                          bool want_e) {
  using T = typename P::T;
  const V3<T> d = pair_image<kRF>(par, pos.diff(i, j));
  const T r2 = dot(d, d);
  if (cutoff2 > T(0) && r2 >= cutoff2) return false;
  const auto ai = par.atom[i], aj = par.atom[j];
  const T sig = ai.x + aj.x, eps = ai.y * aj.y, qq = ai.z * aj.z;
  const T inv_r2 = grcp(r2);
  const T s2 = sig * sig * inv_r2;
  const T s6 = s2 * s2 * s2;
  // -dE/dr / r: 24 eps (2 s^12 - s^6) / r^2 + the Coulomb part (pair_g)
  const T g = pair_g<kRF>(par, eps, s6, qq, r2, inv_r2);
  fi = {g * d.x, g * d.y, g * d.z};
  if (want_e) e = pair_e<kRF>(par, eps, s6, qq, r2, inv_r2);
  return true;
}

template <class P, int kRF = -1>
__device__ __forceinline__ void pair_term(const Pos<P> &pos, const Params<P> &par, int i, int j,
                                          typename P::T cutoff2, const typename P::Acc &acc, bool want_e,
                                          long long &e_fix, int *err) {
  using T = typename P::T;
  V3<T> fi;
  T e = T(0);
  if (!pair_eval<P, kRF>(pos, par, i, j, cutoff2, fi, e, want_e)) return;
  acc.add(i, fi, err);
  acc.add(j, V3<T>{-fi.x, -fi.y, -fi.z}, err);
  if (want_e) e_fix += acc.efix(e, err);
}

// Tiled nonbonded pass: each warp takes tile pairs (I, J); lane l owns atom i = 32 I + l and, at
// rotation step s, meets atom j = 32 J + ((l + s) mod 32).  The force on i accumulates in registers;
// the force on j accumulates in registers that move down the lanes by warp shuffles, so that they
// always sit in the lane currently meeting atom j and end in known lanes.  In a periodic box (Ewald
// real space) each pair takes its nearest image.
// Off-diagonal tiles take s = 0..31; a diagonal tile takes s = 1..16 (lanes 16..31 skip s = 16), which
// meets every unordered pair once.  Per lane and tile pair the FP32 (FP64) sums are converted to fixed
// point once, so the result does not depend on which warp takes which tile pair, or in which order.
// With a cutoff, tile pairs whose bounding boxes are further apart than the cutoff are skipped; kCutoff =
// false drops the cutoff tests (the segment kernel's tile path, taken only by systems without a cutoff).
template <class P, bool kCutoff = true, int kRF = -1>
__device__ __forceinline__ void tile_pass(const SysDev &S, const Pos<P> &pos, const Params<P> &par,
                                          const typename P::Acc &acc, const float *boxes, bool want_e,
                                          long long &e_fix, int *err) {
  using T = typename P::T;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const T cut2 = (T)S.cutoff2;
  for (int tp = warp; tp < S.n_tile_pairs; tp += nwarps) {
    const uint32_t e = S.tile_pairs[tp];
    const int I = (int)(e & 0xFFFFu), J = (int)(e >> 16);
    if (kCutoff && boxes) {  // gap between the two tiles' boxes
      const float *a = boxes + 6 * I, *b = boxes + 6 * J;
      const float gx = fmaxf(0.f, fmaxf(a[0] - b[3], b[0] - a[3]));
      const float gy = fmaxf(0.f, fmaxf(a[1] - b[4], b[1] - a[4]));
      const float gz = fmaxf(0.f, fmaxf(a[2] - b[5], b[2] - a[5]));
      if (gx * gx + gy * gy + gz * gz >= (float)S.cutoff2) continue;
    }
    uint32_t mask = S.tile_masks[(size_t)tp * 32 + lane];
    const int i = I * 32 + lane, j0 = J * 32;
    const bool diag = I == J;
    // on a diagonal tile, step 16 meets lane l and lane l + 16 twice: lanes 16..31 drop that pair
    if (diag && lane >= 16) mask &= ~(1u << (lane - 16));
    const int s0 = diag ? 1 : 0, s1 = diag ? 17 : 32;
    V3<T> fi = {T(0), T(0), T(0)}, fja = {T(0), T(0), T(0)}, fjb = {T(0), T(0), T(0)};
    T en = T(0);
    // atom i in registers (padding lanes read a valid atom and have an empty mask)
    const int ic = i < S.n ? i : S.n - 1;
    const typename Pos<P>::At pi = pos.at(ic);
    T ash, ase, aqc;
    nb_params<P>(pi, par, ic, ash, ase, aqc);
    // Branch-free: a masked pair (excluded, padding, beyond the cutoff) evaluates atom i against itself
    // with r^2 = 1 and contributes g = 0, so that the two independent steps of a pair of steps carry no
    // divergent branches and their dependent chains can interleave (measured on the batched chains:
    // 12.0 -> 12.7 TFLOP/s).  kDense: every lane's mask is full and there is no cutoff, so the masking
    // selects drop out; the arithmetic of each pair is the same as on the masked path.
    auto meet = [&](auto dense, int s, V3<T> &fj) {
      constexpr bool kDense = decltype(dense)::value;
      const int m = (lane + s) & 31;
      const bool on0 = kDense || ((mask >> m) & 1u);
      const int j = on0 ? j0 + m : ic;
      const typename Pos<P>::At pj = pos.at(j);
      const V3<T> d = pair_image<kRF>(par, Pos<P>::diff(pi, pj));
      T r2 = dot(d, d);
      const bool on = on0 && (!kCutoff || !(cut2 > T(0) && r2 >= cut2));
      if constexpr (!kDense) r2 = on ? r2 : T(1);
      T bsh, bse, bqc;
      nb_params<P>(pj, par, j, bsh, bse, bqc);
      const T sig = ash + bsh, eps = ase * bse, qq = aqc * bqc;
      const T inv_r2 = grcp(r2);
      const T s2 = sig * sig * inv_r2;
      const T s6 = s2 * s2 * s2;
      T g = pair_g<kRF>(par, eps, s6, qq, r2, inv_r2);
      if constexpr (!kDense) g = on ? g : T(0);
      const V3<T> f = {g * d.x, g * d.y, g * d.z};
      fi.x += f.x; fi.y += f.y; fi.z += f.z;
      fj.x -= f.x; fj.y -= f.y; fj.z -= f.z;
      if (want_e && on) en += pair_e<kRF>(par, eps, s6, qq, r2, inv_r2);
    };
    // Steps go in pairs: the j forces of even steps ride in fja, those of odd steps in fjb, and both
    // move two lanes down after each pair, so each register waits on one shuffle per two steps
    // instead of one per step.  s1 - s0 is even (32, or 16 on a diagonal tile).
    auto rotate = [&](auto dense) {
#pragma unroll 2
      for (int s = s0; s < s1; s += 2) {
        meet(dense, s, fja);
        meet(dense, s + 1, fjb);
        fja.x = __shfl_sync(0xffffffffu, fja.x, (lane + 2) & 31);
        fja.y = __shfl_sync(0xffffffffu, fja.y, (lane + 2) & 31);
        fja.z = __shfl_sync(0xffffffffu, fja.z, (lane + 2) & 31);
        fjb.x = __shfl_sync(0xffffffffu, fjb.x, (lane + 2) & 31);
        fjb.y = __shfl_sync(0xffffffffu, fjb.y, (lane + 2) & 31);
        fjb.z = __shfl_sync(0xffffffffu, fjb.z, (lane + 2) & 31);
      }
    };
    // tile pairs of whole tiles away from the exclusions (a diagonal tile's mask is never full)
    if (!kCutoff && __all_sync(0xffffffffu, mask == 0xffffffffu)) rotate(std::true_type{});
    else rotate(std::false_type{});
    if (i < S.n) acc.add(i, fi, err);
    // after the last pair of steps lane l holds the j forces of atoms (l + s1) and (l + s1 + 1) mod 32
    const int ja = j0 + ((lane + s1) & 31), jb = j0 + ((lane + s1 + 1) & 31);
    if (ja < S.n) acc.add(ja, fja, err);
    if (jb < S.n) acc.add(jb, fjb, err);
    if (want_e) e_fix += acc.efix(en, err);
  }
}

// r - r0 of a bond for the mixed path in double-single arithmetic: the FP32 distance of a stiff bond
// (k = 3e5) loses ~1e-8 nm to rounding before the subtraction of r0, which would dominate the force
// error; here the difference vector, r^2 (exact products by fma) and one Newton step on sqrt keep
// r - r0 accurate to ~1e-7 of itself.  Returns r - r0 and the FP32 distance r.
__device__ __forceinline__ float bond_dr_ds(const Pos<PathMixed> &pos, int i, int j, float r0, float &r_out,
                                            V3<float> &d_out) {
  const float4 a = pos.qh[i], b = pos.qh[j], c = pos.ql[i], e = pos.ql[j];
  const float *ah = &a.x, *bh = &b.x, *al = &c.x, *bl = &e.x;
  float dh[3], dl[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const float s = __fsub_rn(ah[x], bh[x]);
    const float bp = __fsub_rn(s, ah[x]);
    const float err = __fadd_rn(__fsub_rn(ah[x], __fsub_rn(s, bp)), __fsub_rn(-bh[x], bp));  // TwoSum(a, -b)
    const float lo = __fadd_rn(err, __fsub_rn(al[x], bl[x]));
    dh[x] = __fadd_rn(s, lo);
    dl[x] = __fsub_rn(lo, __fsub_rn(dh[x], s));
  }
  // r^2 = sum (dh + dl)^2 as hi + lo
  float sh = 0.f, sl = 0.f;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const float p = __fmul_rn(dh[x], dh[x]);
    const float pe = __fmaf_rn(dh[x], dh[x], -p);
    const float t = __fadd_rn(sh, p);
    const float tb = __fsub_rn(t, sh);
    const float te = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, tb)), __fsub_rn(p, tb));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(te, __fmaf_rn(2.f * dh[x], dl[x], pe)));
  }
  const float r = sqrtf(sh);
  const float rr = __fmul_rn(r, r);
  const float rre = __fmaf_rn(r, r, -rr);
  const float resid = __fadd_rn(__fsub_rn(__fsub_rn(sh, rr), rre), sl);  // r^2 - r*r
  const float rlo = __fdividef(resid, 2.f * r);
  r_out = r;
  d_out = {dh[0], dh[1], dh[2]};
  return __fadd_rn(__fsub_rn(r, r0), rlo);
}

// Mixed path: bonds at least this stiff (kJ/mol/nm^2) take r - r0 in double-single arithmetic.
constexpr float kSoftBond = 1.0e4f;

// Harmonic bond 1/2 k (r - r0)^2: force on atom i (minus the force on j) and the energy.
template <class P>
__device__ __forceinline__ V3<typename P::T> bond_eval(const Pos<P> &pos, const Params<P> &par, int b, int i, int j,
                                                       typename P::T &e) {
  using T = typename P::T;
  const auto kp = par.bond[b];
  V3<T> d;
  T r, dr;
  if constexpr (P::kMixed) {
    if (kp.x >= kSoftBond) {
      dr = bond_dr_ds(pos, i, j, kp.y, r, d);
    } else {  // soft springs: the FP32 rounding of r moves the force by < 1e-6 of its thermal scale, so the
              // high words of the positions suffice (one 16-byte load per atom instead of two; on the
              // 2,030-atom elastic network the difference is 6e-8 of the largest force)
      const float4 a = pos.qh[i], c = pos.qh[j];
      d = {a.x - c.x, a.y - c.y, a.z - c.z};
      r = gsqrt(dot(d, d));
      dr = r - T(kp.y);
    }
  } else {
    d = pos.diff(i, j);
    r = gsqrt(dot(d, d));
    dr = r - T(kp.y);
  }
  const T g = -gdiv(T(kp.x) * dr, r);
  e = T(0.5) * T(kp.x) * dr * dr;
  return {g * d.x, g * d.y, g * d.z};
}

template <class P>
__device__ __forceinline__ void bond_term(const Pos<P> &pos, const Params<P> &par, int b, int i, int j,
                                          const typename P::Acc &acc, bool want_e, long long &e_fix, int *err) {
  using T = typename P::T;
  T e;
  const V3<T> fi = bond_eval<P>(pos, par, b, i, j, e);
  acc.add(i, fi, err);
  acc.add(j, V3<T>{-fi.x, -fi.y, -fi.z}, err);
  if (want_e) e_fix += acc.efix(e, err);
}

// Harmonic angle 1/2 k (theta - theta0)^2 at vertex j; theta = atan2(|u x v|, u.v) with
// u = q_i - q_j, v = q_k - q_j, d theta/d q_i = ((u.v)/|u|^2 u - v) / |u x v| and likewise for q_k.
template <class P>
__device__ __forceinline__ void angle_term(const Pos<P> &pos, const Params<P> &par, int t, int i, int j,
                                           int k, const typename P::Acc &acc, bool want_e, long long &e_fix,
                                           int *err) {
  using T = typename P::T;
  const auto kp = par.angle[t];
  const V3<T> u = pos.diff(i, j), v = pos.diff(k, j);
  const T uu = dot(u, u), vv = dot(v, v), c = dot(u, v);
  const V3<T> w = cross(u, v);
  T sn = gsqrt(dot(w, w));
  const T th = gatan2(sn, c);
  sn = sn > T(1e-30) ? sn : T(1e-30);
  const T dth = th - T(kp.y);
  const T s = -gdiv(T(kp.x) * dth, sn);  // F = -dE/dtheta * d theta/dq
  const T cu = gdiv(c, uu), cv = gdiv(c, vv);
  const V3<T> fi = {s * (cu * u.x - v.x), s * (cu * u.y - v.y), s * (cu * u.z - v.z)};
  const V3<T> fk = {s * (cv * v.x - u.x), s * (cv * v.y - u.y), s * (cv * v.z - u.z)};
  acc.add(i, fi, err);
  acc.add(k, fk, err);
  acc.add(j, V3<T>{-fi.x - fk.x, -fi.y - fk.y, -fi.z - fk.z}, err);
  if (want_e) e_fix += acc.efix(T(0.5) * T(kp.x) * dth * dth, err);
}

// Periodic dihedral terms sum_t k_t (1 + cos(n_t phi - delta_t)) of atoms (i, j, k, l), IUPAC sign;
// cos(n phi), sin(n phi) by the angle-addition recurrence; gradient of phi after Blondel & Karplus.
template <class P>
__device__ __forceinline__ void dihedral_term(const Pos<P> &pos, const Params<P> &par, int4 a, int2 terms,
                                              const typename P::Acc &acc, bool want_e, long long &e_fix,
                                              int *err) {
  using T = typename P::T;
  const V3<T> b1 = pos.diff(a.y, a.x), b2 = pos.diff(a.z, a.y), b3 = pos.diff(a.w, a.z);
  const V3<T> n1 = cross(b1, b2), n2 = cross(b2, b3);
  // reciprocal square roots (one hardware approximation each in FP32) instead of a square root followed by
  // a reciprocal: the dihedral terms are the longest items of small systems' force pass
  const T b2sq = dot(b2, b2), rb2 = grsqrt(b2sq), lb2 = b2sq * rb2;
  const T x = dot(n1, n2), y = lb2 * dot(b1, n2);
  const T irho = grsqrt(x * x + y * y);
  const T cph = x * irho, sph = y * irho;
  T dedphi = T(0), e = T(0);
  for (int t = terms.x; t < terms.y; ++t) {
    const auto tp = par.term[t];  // (k, n, cos delta, sin delta)
    const int nn = (int)tp.y;
    T cn = cph, sn = sph;
    for (int m = 1; m < nn; ++m) {
      const T c2 = cn * cph - sn * sph;
      sn = sn * cph + cn * sph;
      cn = c2;
    }
    const T sin_nd = sn * T(tp.z) - cn * T(tp.w);  // sin(n phi - delta)
    dedphi -= T(tp.x) * T(nn) * sin_nd;
    if (want_e) e += T(tp.x) * (T(1) + cn * T(tp.z) + sn * T(tp.w));
  }
  const T n1sq = dot(n1, n1), n2sq = dot(n2, n2);
  const T ib2 = rb2 * rb2;
  const T f12 = dot(b1, b2) * ib2, f32 = dot(b3, b2) * ib2;
  const T ci = gdiv(lb2, n1sq) * dedphi;   // F_i = -dE/dphi * (-|b2| n1/|n1|^2)
  const T cl = -gdiv(lb2, n2sq) * dedphi;  // F_l = -dE/dphi * ( |b2| n2/|n2|^2)
  const V3<T> fi = {ci * n1.x, ci * n1.y, ci * n1.z};
  const V3<T> fl = {cl * n2.x, cl * n2.y, cl * n2.z};
  // F_j = -(1 + f12) F_i + f32 F_l, F_k = f12 F_i - (1 + f32) F_l
  const V3<T> fj = {-(T(1) + f12) * fi.x + f32 * fl.x, -(T(1) + f12) * fi.y + f32 * fl.y,
                    -(T(1) + f12) * fi.z + f32 * fl.z};
  const V3<T> fk = {f12 * fi.x - (T(1) + f32) * fl.x, f12 * fi.y - (T(1) + f32) * fl.y,
                    f12 * fi.z - (T(1) + f32) * fl.z};
  acc.add(a.x, fi, err);
  acc.add(a.y, fj, err);
  acc.add(a.z, fk, err);
  acc.add(a.w, fl, err);
  if (want_e) e_fix += acc.efix(e, err);
}

// Nonbonded pairs of a Verlet list (i | j << 16), strided over the block's threads; pairs beyond the
// cutoff contribute nothing; in a periodic box (Ewald real space) each pair takes its nearest image.  The list lives in global memory (L2): each thread loads its next four
// entries before evaluating them, so that one load latency covers four pairs.  (Measured on the
// 2,030-atom ligand workload, this pair list with fixed-point atomics on both atoms beat per-atom
// neighbour rows evaluated from both ends by 1.36x, and rows holding each pair once by 7x.)
template <class P, int kRF = -1>
__device__ __forceinline__ void list_pass(const SysDev &S, const Pos<P> &pos, const Params<P> &par,
                                          const uint32_t *list, int count, const typename P::Acc &acc,
                                          bool want_e, long long &e_fix, int *err) {
  using T = typename P::T;
  const T cut2 = (T)S.cutoff2;
  const int bd = blockDim.x;
  for (int t = threadIdx.x; t < count; t += 4 * bd) {
    uint32_t pk[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) pk[u] = t + u * bd < count ? list[t + u * bd] : 0xFFFFFFFFu;  // written in this kernel: no .nc loads
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (pk[u] == 0xFFFFFFFFu) continue;
      const int i = (int)(pk[u] & 0xFFFFu), j = (int)(pk[u] >> 16);
      typename Pos<P>::At pi, pj;
      if constexpr (P::kMixed) {
        // screen on the high words alone (their distance is within ~1e-6 of the double-single one):
        // the list's pairs beyond the cutoff, about half of them, skip the low-word loads
        pi.h = pos.qh[i];
        pj.h = pos.qh[j];
        const V3<float> hd = pair_image<kRF>(par, V3<float>{pi.h.x - pj.h.x, pi.h.y - pj.h.y, pi.h.z - pj.h.z});
        if (dot(hd, hd) > cut2 * 1.0001f) continue;
        pi.l = pos.ql[i];
        pj.l = pos.ql[j];
      } else {
        pi = pos.at(i);
        pj = pos.at(j);
      }
      const V3<T> d = pair_image<kRF>(par, Pos<P>::diff(pi, pj));
      const T r2 = dot(d, d);
      if (!(r2 < cut2)) continue;
      T ash, ase, aqc, bsh, bse, bqc;
      nb_params<P>(pi, par, i, ash, ase, aqc);
      nb_params<P>(pj, par, j, bsh, bse, bqc);
      const T sig = ash + bsh, eps = ase * bse, qq = aqc * bqc;
      const T inv_r2 = grcp(r2);
      const T s2 = sig * sig * inv_r2;
      const T s6 = s2 * s2 * s2;
      const T g = pair_g<kRF>(par, eps, s6, qq, r2, inv_r2);
      const V3<T> f = {g * d.x, g * d.y, g * d.z};
      acc.add(i, f, err);
      acc.add(j, V3<T>{-f.x, -f.y, -f.z}, err);
      if (want_e) e_fix += acc.efix(pair_e<kRF>(par, eps, s6, qq, r2, inv_r2), err);
    }
  }
}

// Bonded terms by kind, without the item table (large systems, whose tables stay in global memory):
// each thread loads the indices and parameters of its next two bonds before evaluating them.
template <class P>
__device__ __forceinline__ void bonded_pass(const SysDev &S, const Pos<P> &pos, const Params<P> &par,
                                            const typename P::Acc &acc, bool want_e, long long &e_fix, int *err) {
  const int bd = blockDim.x;
  for (int b = threadIdx.x; b < S.n_bonds; b += 2 * bd) {
    const int b2 = b + bd;
    const int2 ij0 = S.bond_ij[b];
    const int2 ij1 = b2 < S.n_bonds ? S.bond_ij[b2] : make_int2(0, 0);
    bond_term<P>(pos, par, b, ij0.x, ij0.y, acc, want_e, e_fix, err);
    if (b2 < S.n_bonds) bond_term<P>(pos, par, b2, ij1.x, ij1.y, acc, want_e, e_fix, err);
  }
  for (int t = threadIdx.x; t < S.n_angles; t += bd) {
    const int4 ijk = S.angle_ijk[t];
    angle_term<P>(pos, par, t, ijk.x, ijk.y, ijk.z, acc, want_e, e_fix, err);
  }
  for (int t = threadIdx.x; t < S.n_dih; t += bd)
    dihedral_term<P>(pos, par, S.dih_ijkl[t], S.dih_terms[t], acc, want_e, e_fix, err);
}

// One pass over every force-field item of a replica, strided over the block's threads.  The item
// table groups pairs, bonds, angles and dihedrals, each group padded to a multiple of 32 entries, so
// that every warp runs a single kind of item (no serialised divergent paths) and the dihedrals, the
// longest items, land on the last warps rather than on warp 0, which also integrates atoms 0..31.
template <class P, int kRF = -1>
__device__ __forceinline__ void force_pass(const SysDev &S, const Pos<P> &pos, const Params<P> &par,
                                           const uint32_t *items, const uint32_t *pairs,
                                           const typename P::Acc &acc, bool want_e, long long &e_fix, int *err) {
  using T = typename P::T;
  const T cut2 = (T)S.cutoff2;
  for (int it = threadIdx.x; it < S.n_items; it += blockDim.x) {
    const uint32_t e = items[it];
    const uint32_t kind = e >> 28;
    const int idx = (int)(e & 0x0FFFFFFFu);
    if (kind == kItemPair) {
      const uint32_t pk = pairs[idx];
      pair_term<P, kRF>(pos, par, (int)(pk & 0xFFFFu), (int)(pk >> 16), cut2, acc, want_e, e_fix, err);
    } else if (kind == kItemBond) {
      const int2 ij = S.bond_ij[idx];
      bond_term<P>(pos, par, idx, ij.x, ij.y, acc, want_e, e_fix, err);
    } else if (kind == kItemAngle) {
      const int4 ijk = S.angle_ijk[idx];
      angle_term<P>(pos, par, idx, ijk.x, ijk.y, ijk.z, acc, want_e, e_fix, err);
    } else if (kind == kItemDihedral) {
      dihedral_term<P>(pos, par, S.dih_ijkl[idx], S.dih_terms[idx], acc, want_e, e_fix, err);
    }
  }
}

// Scalar fixed-point accumulators of a path: [m] values (the FP64 path's 2^-40 int64, the mixed
// path's split words).
template <class P>
struct ScalarAcc;
template <>
struct ScalarAcc<PathF64> {
  long long *v;
  static size_t bytes(int m) { return (size_t)m * 8; }
  __device__ void carve(unsigned char *&ptr, int m) { v = (long long *)ptr; ptr += (size_t)m * 8; }
  __device__ __forceinline__ void add(int i, double x, int *err) const { fix_add(&v[i], to_fix(x, err)); }
  __device__ __forceinline__ double get(int i) const { return (double)v[i] * kFixInv; }
  __device__ __forceinline__ void zero(int i) const { v[i] = 0; }
  __device__ __forceinline__ void set(int i, double x, int *err) const { v[i] = to_fix(x, err); }
};
template <>
struct ScalarAcc<PathMixed> {
  int *hi;
  unsigned int *lo;
  static size_t bytes(int m) { return (size_t)m * 8; }
  __device__ void carve(unsigned char *&ptr, int m) {
    hi = (int *)ptr; ptr += (size_t)m * 4;
    lo = (unsigned int *)ptr; ptr += (size_t)m * 4;
  }
  __device__ __forceinline__ void add(int i, float x, int *err) const { split_add(hi, lo, i, to_split(x, err)); }
  __device__ __forceinline__ float get(int i) const { return split_to_float(hi[i], lo[i]); }
  __device__ __forceinline__ void zero(int i) const { hi[i] = 0; lo[i] = 0u; }
  __device__ __forceinline__ void set(int i, float x, int *err) const {
    const Split s = to_split(x, err);
    hi[i] = s.hi;
    lo[i] = s.lo;
  }
};

}  // namespace grp

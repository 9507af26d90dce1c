// Shared-memory replica state of each precision path (positions, momenta, forces and noise scale
// of one replica held by one thread block), and the per-step noise.
#pragma once
#include "forcefield.cuh"

namespace grp {

// Noise amplitude sqrt((1 - c1^2) kT m) of the O step, with explicitly rounded operations so that
// every kernel computes the same bits (a contraction of 1 - c1^2 into an fma differs in the last bit).
__device__ __forceinline__ double noise_scale(double c1, double kT, double m) {
  return sqrt(__dmul_rn(__dmul_rn(__dadd_rn(1.0, -__dmul_rn(c1, c1)), kT), m));
}

__device__ __forceinline__ unsigned char *align32(unsigned char *p) {
  return (unsigned char *)(((uintptr_t)p + 31) & ~(uintptr_t)31);
}

__device__ __forceinline__ void normals4(const Philox4 &w, double xi[4]) { normals4_f64(w, xi); }
__device__ __forceinline__ void normals4(const Philox4 &w, float xi[4]) { normals4_f32(w, xi); }

// Normals for `steps` consecutive steps of one replica, [step][atom][3], spread over every thread of
// the block: the noise does not depend on the state, so it is generated off the per-step chain.
template <class T>
__device__ __forceinline__ void gen_noise(T *xi, int steps, long long t0, uint64_t seed, int r, int n) {
  const int items = steps * n;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int j = it / n, at = it - j * n;
    T z[4];
    normals4(philox_stream(seed, t0 + j, 0u, r, at), z);
    T *o = xi + (size_t)it * 3;
    o[0] = z[0]; o[1] = z[1]; o[2] = z[2];
  }
}

// ------------------------------------------------------------------------------------------------
// Shared-memory replica state of each precision path.
template <class P>
struct State;

template <>
struct State<PathF64> {
  double *q, *p, *f, *sd;  // [3n], [3n], [3n], [n]
  const double4 *atom;     // [n] parameters: a shared-memory copy, or the global table when lean
  bool own_atom;
  // lean: the atom parameters and the noise amplitudes are read from the system's global tables
  static size_t bytes(int n, bool lean) { return (size_t)n * (72 + (lean ? 0 : 8 + 32)); }
  __device__ void carve(unsigned char *&ptr, int n, const SysDev &S, bool lean) {
    own_atom = !lean;
    if (lean) atom = S.atom_d;
    else { atom = (const double4 *)ptr; ptr += (size_t)n * 32; }
    q = (double *)ptr; ptr += (size_t)n * 24;
    p = (double *)ptr; ptr += (size_t)n * 24;
    f = (double *)ptr; ptr += (size_t)n * 24;
    if (lean) sd = const_cast<double *>(S.sd_d);
    else { sd = (double *)ptr; ptr += (size_t)n * 8; }
  }
  static __device__ AccF64 acc(long long *F, int n) { return AccF64{F}; }
  __device__ void load(const SysDev &S, const double *gq, const double *gp, const double *gf, int n, double c1) {
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) { q[i] = gq[i]; p[i] = gp[i]; f[i] = gf[i]; }
    for (int at = threadIdx.x; at < n; at += blockDim.x) {
      if (own_atom) const_cast<double4 *>(atom)[at] = S.atom_d[at];
      if (own_atom) sd[at] = noise_scale(c1, S.kT, S.mass[at]);
    }
  }
  __device__ void store(double *gq, double *gp, double *gf, int n, int *err) const {
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
      gq[i] = q[i]; gp[i] = p[i]; gf[i] = f[i];
      if (!isfinite(q[i]) || !isfinite(p[i])) *err |= kErrNaN;
    }
  }
  __device__ Pos<PathF64> pos() const { return Pos<PathF64>{q}; }
  __device__ Params<PathF64> params(const SysDev &S) const {
    return Params<PathF64>{atom, S.bond_d, S.angle_d, S.term_d, S.coulomb_rf, S.krf, S.crf,
                           {S.box[0], S.box[1], S.box[2]}, {S.ibox[0], S.ibox[1], S.ibox[2]}, S.ewald_beta};
  }
  // B, A, O, A of BAOAB for one coordinate i = 3 atom + axis, and the final B with the new force,
  // written with explicitly rounded operations so that no kernel leaves contraction choices to the
  // compiler: every kernel that runs them (the segment, the adjoint's recomputation) reproduces the
  // same trajectory bit for bit.
  __device__ __forceinline__ void baoa_c(int i, double xi, double h, double c1) {
    const int at = i / 3;
    const double im = atom[at].w, s = sd[at];
    double pp = __fma_rn(h, f[i], p[i]);
    double qq = __fma_rn(__dmul_rn(h, pp), im, q[i]);
    pp = __fma_rn(c1, pp, __dmul_rn(s, xi));
    qq = __fma_rn(__dmul_rn(h, pp), im, qq);
    p[i] = pp;
    q[i] = qq;
  }
  __device__ __forceinline__ double bk_c(int i, const AccF64 &acc, double h) {
    const double im = atom[i / 3].w;
    const double fv = (double)acc.F[i] * kFixInv;
    acc.F[i] = 0;
    f[i] = fv;
    const double pp = __fma_rn(h, fv, p[i]);
    p[i] = pp;
    return __dmul_rn(__dmul_rn(0.5, __dmul_rn(pp, pp)), im);
  }
  // the same for the three coordinates of atom `at` (normals xi[0..2]); returns its kinetic energy
  __device__ __forceinline__ void baoa(int at, const double *xi, double h, double c1) {
#pragma unroll
    for (int x = 0; x < 3; ++x) baoa_c(3 * at + x, xi[x], h, c1);
  }
  __device__ __forceinline__ double bk(int at, const AccF64 &acc, double h) {
    double ke = 0;
#pragma unroll
    for (int x = 0; x < 3; ++x) ke += bk_c(3 * at + x, acc, h);
    return ke;
  }
  __device__ double coord(int i) const { return q[i]; }
  __device__ void get_f64(int at, double x[3]) const { x[0] = q[3 * at]; x[1] = q[3 * at + 1]; x[2] = q[3 * at + 2]; }
  __device__ void get_f32(int at, float x[3]) const {
    x[0] = (float)q[3 * at]; x[1] = (float)q[3 * at + 1]; x[2] = (float)q[3 * at + 2];
  }
  __device__ double mom(int i) const { return p[i]; }
};

template <>
struct State<PathMixed> {
  float4 *qh, *ql;   // [n] double-single positions; .w: sigma/2 (qh), sqrt(eps) (ql)
  float *ph, *pl;    // [3n] double-single momenta
  float *f, *sd;     // [3n], [n]
  const float4 *atom;  // [n] parameters: a shared-memory copy, or the global table when lean
  bool own_atom;
  static size_t bytes(int n, bool lean) { return (size_t)n * (32 + 24 + 12 + (lean ? 0 : 4 + 16)); }
  __device__ void carve(unsigned char *&ptr, int n, const SysDev &S, bool lean) {
    own_atom = !lean;
    qh = (float4 *)ptr; ptr += (size_t)n * 16;
    ql = (float4 *)ptr; ptr += (size_t)n * 16;
    if (lean) atom = S.atom_f;
    else { atom = (const float4 *)ptr; ptr += (size_t)n * 16; }
    ph = (float *)ptr; ptr += (size_t)n * 12;
    pl = (float *)ptr; ptr += (size_t)n * 12;
    f = (float *)ptr; ptr += (size_t)n * 12;
    if (lean) sd = const_cast<float *>(S.sd_f);
    else { sd = (float *)ptr; ptr += (size_t)n * 4; }
  }
  // the 8 bytes per force component hold the hi words [3n] then the lo words [3n]
  static __device__ AccMixed acc(long long *F, int n) {
    return AccMixed{(int *)F, (unsigned int *)F + 3 * n};
  }
  __device__ void load(const SysDev &S, const double *gq, const double *gp, const double *gf, int n, double c1) {
    for (int at = threadIdx.x; at < n; at += blockDim.x) {
      const ds x = ds_from_double(gq[3 * at]), y = ds_from_double(gq[3 * at + 1]),
               z = ds_from_double(gq[3 * at + 2]);
      const float4 pa = S.atom_f[at];
      qh[at] = make_float4(x.hi, y.hi, z.hi, pa.x);  // fourth words: sigma/2 and sqrt(eps) (nb_params)
      ql[at] = make_float4(x.lo, y.lo, z.lo, pa.y);
      if (own_atom) const_cast<float4 *>(atom)[at] = pa;
      if (own_atom) sd[at] = (float)noise_scale(c1, S.kT, S.mass[at]);
    }
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
      const ds v = ds_from_double(gp[i]);
      ph[i] = v.hi;
      pl[i] = v.lo;
      f[i] = (float)gf[i];
    }
  }
  __device__ void store(double *gq, double *gp, double *gf, int n, int *err) const {
    for (int at = threadIdx.x; at < n; at += blockDim.x) {
      const float4 a = qh[at], b = ql[at];
      gq[3 * at] = (double)a.x + (double)b.x;
      gq[3 * at + 1] = (double)a.y + (double)b.y;
      gq[3 * at + 2] = (double)a.z + (double)b.z;
      if (!isfinite(a.x) || !isfinite(a.y) || !isfinite(a.z)) *err |= kErrNaN;
    }
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
      gp[i] = (double)ph[i] + (double)pl[i];
      gf[i] = (double)f[i];
      if (!isfinite(ph[i])) *err |= kErrNaN;
    }
  }
  __device__ Pos<PathMixed> pos() const { return Pos<PathMixed>{qh, ql}; }
  __device__ Params<PathMixed> params(const SysDev &S) const {
    return Params<PathMixed>{atom, S.bond_f, S.angle_f, S.term_f, S.coulomb_rf, (float)S.krf, (float)S.crf,
                             {(float)S.box[0], (float)S.box[1], (float)S.box[2]},
                             {(float)S.ibox[0], (float)S.ibox[1], (float)S.ibox[2]}, (float)S.ewald_beta};
  }
  __device__ __forceinline__ void baoa(int at, const float *xi, float h, float c1) {
    const float im = atom[at].w, s = sd[at], hm = h * im;
    float4 a = qh[at], b = ql[at];
    float *qa = &a.x, *qb = &b.x;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const int i = 3 * at + x;
      ds P = {ph[i], pl[i]};
      ds Q = {qa[x], qb[x]};
      P = ds_add(P, h * f[i]);
      Q = ds_add(Q, hm * P.hi);
      P = ds_add(ds_scale(P, c1), s * xi[x]);
      Q = ds_add(Q, hm * P.hi);
      ph[i] = P.hi;
      pl[i] = P.lo;
      qa[x] = Q.hi;
      qb[x] = Q.lo;
    }
    qh[at] = a;
    ql[at] = b;
  }
  __device__ __forceinline__ float bk(int at, const AccMixed &acc, float h) {
    const float im = atom[at].w;
    float ke = 0.f;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const int i = 3 * at + x;
      const float fv = split_to_float(acc.hi[i], acc.lo[i]);
      acc.hi[i] = 0;
      acc.lo[i] = 0u;
      f[i] = fv;
      ds P = {ph[i], pl[i]};
      P = ds_add(P, h * fv);
      ph[i] = P.hi;
      pl[i] = P.lo;
      ke += 0.5f * P.hi * P.hi * im;
    }
    return ke;
  }
  __device__ __forceinline__ void baoa_c(int i, float xi, float h, float c1) {
    const int at = i / 3, x = i - 3 * at;
    const float im = atom[at].w, s = sd[at], hm = h * im;
    float *qa = &qh[at].x, *qb = &ql[at].x;
    ds P = {ph[i], pl[i]};
    ds Q = {qa[x], qb[x]};
    P = ds_add(P, h * f[i]);
    Q = ds_add(Q, hm * P.hi);
    P = ds_add(ds_scale(P, c1), s * xi);
    Q = ds_add(Q, hm * P.hi);
    ph[i] = P.hi;
    pl[i] = P.lo;
    qa[x] = Q.hi;
    qb[x] = Q.lo;
  }
  __device__ __forceinline__ float bk_c(int i, const AccMixed &acc, float h) {
    const float im = atom[i / 3].w;
    const float fv = split_to_float(acc.hi[i], acc.lo[i]);
    acc.hi[i] = 0;
    acc.lo[i] = 0u;
    f[i] = fv;
    ds P = {ph[i], pl[i]};
    P = ds_add(P, h * fv);
    ph[i] = P.hi;
    pl[i] = P.lo;
    return 0.5f * P.hi * P.hi * im;
  }
  __device__ float coord(int i) const { return (&qh[i / 3].x)[i % 3]; }
  __device__ void get_f64(int at, double x[3]) const {
    const float4 a = qh[at], b = ql[at];
    x[0] = (double)a.x + (double)b.x; x[1] = (double)a.y + (double)b.y; x[2] = (double)a.z + (double)b.z;
  }
  __device__ void get_f32(int at, float x[3]) const {
    const float4 a = qh[at];
    x[0] = a.x; x[1] = a.y; x[2] = a.z;
  }
  __device__ float mom(int i) const { return ph[i]; }
};

}  // namespace grp

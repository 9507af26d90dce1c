// Differentiation of the potential V of Eq. 1 with respect to the force-field parameters
// theta = (sigma_i, eps_i, k_t) (not in the paper: it serves gradient-based fitting of the force
// field that drives the dynamics).  Gradients with respect to the positions come from the force
// kernel; this file adds dV/d theta and the in-place update of the parameter tables.
//
// Per Lennard-Jones pair, with s = sig_ij / r, sig_ij = (sigma_i + sigma_j) / 2 and
// eps_ij = sqrt(eps_i eps_j):  dE/d sig_ij = 4 eps_ij (12 s^12 - 6 s^6) / sig_ij, d sig_ij / d sigma_i
// = 1/2;  dE/d eps_ij = 4 (s^12 - s^6), d eps_ij / d eps_i = sqrt(eps_j) / (2 sqrt(eps_i)).  Per
// dihedral term, dE/dk = 1 + cos(n phi - delta).  The sums use the 2^-40 fixed point of the FP64
// force path, so the result does not depend on the order in which threads add their terms.
#include <cfloat>

#include "dual.cuh"
#include "forcefield.cuh"
#include "kernels.h"
#include "state.cuh"

namespace grp {

// One block: validate theta, then rewrite (sigma/2, sqrt eps) of every atom and k of every dihedral
// term in both the FP64 and the FP32 tables.
__global__ void __launch_bounds__(256) set_params_kernel(SysDev S, int n_terms, const double *theta, int *bad) {
  const int n = S.n, nt = 2 * n + n_terms;
  int b = 0;
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    const double v = theta[i];
    if (!isfinite(v) || (i < n && !(v > 0.0)) || (i >= n && i < 2 * n && v < 0.0)) b = 1;
  }
  b = __syncthreads_or(b);
  if (threadIdx.x == 0) *bad = b;
  if (b) return;
  double4 *ad = const_cast<double4 *>(S.atom_d);
  float4 *af = const_cast<float4 *>(S.atom_f);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double4 a = ad[i];
    a.x = 0.5 * theta[i];
    a.y = sqrt(theta[n + i]);
    ad[i] = a;
    af[i] = make_float4((float)a.x, (float)a.y, (float)a.z, (float)a.w);
  }
  double4 *td = const_cast<double4 *>(S.term_d);
  float4 *tf = const_cast<float4 *>(S.term_f);
  for (int u = threadIdx.x; u < n_terms; u += blockDim.x) {
    const double k = theta[2 * n + S.term_src[u]];
    td[u].x = k;
    tf[u].x = (float)k;
  }
}

cudaError_t launch_set_params(const SysDev &S, int n_terms, const double *theta, int *bad, cudaStream_t st) {
  set_params_kernel<<<1, 256, 0, st>>>(S, n_terms, theta, bad);
  return cudaGetLastError();
}

template <class T>
__device__ __forceinline__ V3<T> qdiff(const double *q, int i, int j) {
  // differences taken in FP64, then rounded to the path's precision
  return {(T)(q[3 * i] - q[3 * j]), (T)(q[3 * i + 1] - q[3 * j + 1]), (T)(q[3 * i + 2] - q[3 * j + 2])};
}

// dE/d sig_ij (already halved: the share of each sigma) and the eps shares of atoms i and j.
template <class T, class A>
__device__ __forceinline__ bool lj_param_terms(const V3<T> &d, const A &ai, const A &aj, T cut2, T &dsig,
                                               T &dei, T &dej) {
  const T r2 = dot(d, d);
  if (cut2 > T(0) && r2 >= cut2) return false;
  const T sig = (T)ai.x + (T)aj.x, sei = (T)ai.y, sej = (T)aj.y;
  const T s2 = sig * sig * grcp(r2);
  const T s6 = s2 * s2 * s2;
  dsig = T(0.5) * gdiv(T(4) * sei * sej * (T(12) * s6 * s6 - T(6) * s6), sig);
  const T de = T(4) * (s6 * s6 - s6);
  dei = de * gdiv(sej, T(2) * sei);
  dej = de * gdiv(sei, T(2) * sej);
  return true;
}

// Accumulators of dV/d theta in the 2^-40 fixed point: the values, or the tangents (eps parts) when
// the positions are dual numbers q + eps v.
struct ParamAcc {
  long long *G;
  __device__ __forceinline__ void add(int k, double v, int *err) const { fix_add(&G[k], to_fix(v, err)); }
  __device__ __forceinline__ void add(int k, float v, int *err) const { fix_add(&G[k], to_fix((double)v, err)); }
};
struct ParamTangent {
  long long *G;
  __device__ __forceinline__ void add(int k, Dual v, int *err) const { fix_add(&G[k], to_fix(v.d, err)); }
  __device__ __forceinline__ void add(int k, DualF v, int *err) const { fix_add(&G[k], to_fix((double)v.d, err)); }
};

// dV/d theta of one configuration by the whole block; qd(i, j) gives q_i - q_j in type T.
template <class T, class A, class A4T, class QD, class PA>
__device__ __forceinline__ void param_pass(const SysDev &S, const A *atom, const A4T *term, QD qd, const PA &acc,
                                           int *err) {
  const int n = S.n;
  const T cut2 = (T)S.cutoff2;
  if (!S.tiled) {
    for (int t = threadIdx.x; t < S.n_pairs; t += blockDim.x) {
      const uint32_t pk = S.pairs[t];
      const int i = (int)(pk & 0xFFFFu), j = (int)(pk >> 16);
      T dsig, dei, dej;
      if (!lj_param_terms<T>(qd(i, j), atom[i], atom[j], cut2, dsig, dei, dej)) continue;
      acc.add(i, dsig, err);
      acc.add(j, dsig, err);
      acc.add(n + i, dei, err);
      acc.add(n + j, dej, err);
    }
  } else {
    // one warp per tile pair; at rotation step s lane l meets atom 32 J + ((l + s) mod 32), so the
    // lanes of a warp add to distinct j accumulators; a diagonal tile keeps j > i only
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int tp = warp; tp < S.n_tile_pairs; tp += nwarps) {
      const uint32_t e = S.tile_pairs[tp];
      const int I = (int)(e & 0xFFFFu), J = (int)(e >> 16);
      const uint32_t mask = S.tile_masks[(size_t)tp * 32 + lane];
      const int i = I * 32 + lane;
      T si = T(0), ei = T(0);
      for (int s = 0; s < 32; ++s) {
        const int m = (lane + s) & 31;
        if (!((mask >> m) & 1u) || (I == J && m <= lane)) continue;
        const int j = J * 32 + m;
        T dsig, dei, dej;
        if (!lj_param_terms<T>(qd(i, j), atom[i], atom[j], cut2, dsig, dei, dej)) continue;
        si += dsig;
        ei += dei;
        acc.add(j, dsig, err);
        acc.add(n + j, dej, err);
      }
      if (i < n) {
        acc.add(i, si, err);
        acc.add(n + i, ei, err);
      }
    }
  }
  // dihedral terms: dE/dk = 1 + cos(n phi - delta), cos and sin of n phi by the angle-addition recurrence
  for (int u = threadIdx.x; u < S.n_dih; u += blockDim.x) {
    const int4 a = S.dih_ijkl[u];
    const int2 tr = S.dih_terms[u];
    const V3<T> b1 = qd(a.y, a.x), b2 = qd(a.z, a.y), b3 = qd(a.w, a.z);
    const V3<T> n1 = cross(b1, b2), n2 = cross(b2, b3);
    const T x = dot(n1, n2), y = gsqrt(dot(b2, b2)) * dot(b1, n2);
    const T irho = grcp(gsqrt(x * x + y * y));
    const T cph = x * irho, sph = y * irho;
    for (int t = tr.x; t < tr.y; ++t) {
      const A4T tp = term[t];
      T cn = cph, sn = sph;
      for (int m = 1; m < (int)tp.y; ++m) {
        const T c2 = cn * cph - sn * sph;
        sn = sn * cph + cn * sph;
        cn = c2;
      }
      acc.add(2 * n + S.term_src[t], T(1) + cn * (T)tp.z + sn * (T)tp.w, err);
    }
  }
}

// One block per configuration b; G[2n + n_terms] fixed-point accumulators in shared memory.
template <class T, class A, class A4T>
__global__ void __launch_bounds__(256) param_grad_kernel(SysDev S, const A *atom, const A4T *term, int n_terms,
                                                         const double *q, const double *w, double *grad_q,
                                                         double *partial, int *errp) {
  extern __shared__ __align__(16) long long G[];
  const int n = S.n, nt = 2 * n + n_terms, b = blockIdx.x;
  const double *qb = q + (size_t)b * S.nd;
  for (int i = threadIdx.x; i < nt; i += blockDim.x) G[i] = 0;
  __syncthreads();
  int err = 0;
  param_pass<T>(S, atom, term, [&](int i, int j) { return qdiff<T>(qb, i, j); }, ParamAcc{G}, &err);
  __syncthreads();
  const double wb = w ? w[b] : 1.0;
  for (int i = threadIdx.x; i < nt; i += blockDim.x) partial[(size_t)b * nt + i] = wb * ((double)G[i] * kFixInv);
  if (grad_q)
    for (int i = threadIdx.x; i < S.nd; i += blockDim.x) grad_q[(size_t)b * S.nd + i] *= -wb;
  if (err) atomicOr(errp, err);
}

cudaError_t launch_param_grad(const SysDev &S, int n_terms, int n_conf, const double *q, const double *w,
                              double *grad_q, double *partial, int *err, cudaStream_t st) {
  if (n_conf <= 0) return cudaSuccess;
  if (S.potential != GRP_POT_FORCE_FIELD) return cudaErrorInvalidValue;
  const size_t smem = (size_t)(2 * S.n + n_terms) * 8;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e;
  if (S.precision == GRP_FP64) {
    auto k = param_grad_kernel<double, double4, double4>;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    k<<<n_conf, 256, smem, st>>>(S, S.atom_d, S.term_d, n_terms, q, w, grad_q, partial, err);
  } else {
    auto k = param_grad_kernel<float, float4, float4>;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    k<<<n_conf, 256, smem, st>>>(S, S.atom_f, S.term_f, n_terms, q, w, grad_q, partial, err);
  }
  return cudaGetLastError();
}

__global__ void scale_rows_kernel(double *x, int rows, int cols, const double *w, double alpha) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)rows * cols) return;
  const int r = (int)(i / cols);
  x[i] *= alpha * (w ? w[r] : 1.0);
}

cudaError_t launch_scale_rows(double *x, int rows, int cols, const double *w, double alpha, cudaStream_t st) {
  const size_t total = (size_t)rows * cols;
  if (total == 0) return cudaSuccess;
  scale_rows_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(x, rows, cols, w, alpha);
  return cudaGetLastError();
}

__global__ void column_sum_kernel(const double *partial, int rows, int cols, double *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0;
  for (int r = 0; r < rows; ++r) s += partial[(size_t)r * cols + c];
  out[c] = s;
}

cudaError_t launch_column_sum(const double *partial, int rows, int cols, double *out, cudaStream_t st) {
  if (cols <= 0) return cudaSuccess;
  column_sum_kernel<<<(cols + 127) / 128, 128, 0, st>>>(partial, rows, cols, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Adjoint of the FP64 BAOAB segment with the noise held fixed (common random numbers).
//
// One step maps (q_t, p_t) to (q_{t+1}, p_{t+1}), h = dt/2:  p' = p_t + h F(q_t);  q' = q_t + (h/m) p';
// p'' = c1 p' + s xi_t;  q_{t+1} = q' + (h/m) p'';  p_{t+1} = p'' + h F(q_{t+1}).  Its transpose,
// applied from the last step back to the first to the adjoints (lq, lp) of (q_{t+1}, p_{t+1}):
// lp'' = lp + (h/m) lq;  lp' = c1 lp'' + (h/m) lq;  (lq_t, lp_t) = (lq, lp').  Every configuration q_t
// meets two half kicks whose momentum adjoint is the same lp_t (the end of step t-1 and the start of
// step t), so each q_t contributes once with weight w = 2h (h at t = 0 and at t = k):
// lq_t += w J_F(q_t)^T lp_t = -w H(q_t) lp_t and dL/d theta -= w d/d theta (lp_t . grad V)(q_t).  Both
// come from one dual-number pass of the force field on q_t + eps lp_t (lp_t scaled to unit max-norm,
// so that the fixed-point tangents keep their relative precision).  A loss sample at step t adds
// 1/(R n_s) g'(O) dO/dq to lq_t.  States are recomputed forward from checkpoints every ck steps with
// the forward pass's own code and noise, and fixed-point force sums, so they are bit-identical.

// Block-wide maximum (every thread gets the result).
__device__ __forceinline__ double block_max_d(double v, double *red /* >= 33 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  const double m = red[32];
  __syncthreads();
  return m;
}

// Loss sample at configuration q (thread 0): returns g(O(q)) / (R n_s) and adds its gradient to lq.
__device__ double loss_sample(const AdjArgs &a, const double *q, double *lq) {
  const SysDev &S = a.S;
  const int *arg = a.obs_arg;
  double O = 0.0, u[3] = {0, 0, 0}, ca[3] = {0, 0, 0}, cb[3] = {0, 0, 0}, ma = 0, mb = 0;
  V3<double> gi{}, gj{}, gk{}, gl{};
  if (a.obs_kind == GRP_OBS_COORD) {
    O = q[3 * arg[0] + arg[1]];
  } else if (a.obs_kind == GRP_OBS_GROUP_DISTANCE) {
    for (int t = S.group_off[arg[0]]; t < S.group_off[arg[0] + 1]; ++t) {
      const int at = S.group_atoms[t];
      const double m = S.mass[at];
      ma += m;
      for (int x = 0; x < 3; ++x) ca[x] += m * q[3 * at + x];
    }
    for (int t = S.group_off[arg[1]]; t < S.group_off[arg[1] + 1]; ++t) {
      const int at = S.group_atoms[t];
      const double m = S.mass[at];
      mb += m;
      for (int x = 0; x < 3; ++x) cb[x] += m * q[3 * at + x];
    }
    for (int x = 0; x < 3; ++x) u[x] = ca[x] / ma - cb[x] / mb;
    O = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int x = 0; x < 3; ++x) u[x] = O > 0.0 ? u[x] / O : 0.0;
  } else {  // dihedral of arg[0..3] in radians; gradient after Blondel & Karplus
    auto d = [&](int i, int j) { return V3<double>{q[3 * i] - q[3 * j], q[3 * i + 1] - q[3 * j + 1], q[3 * i + 2] - q[3 * j + 2]}; };
    const V3<double> b1 = d(arg[1], arg[0]), b2 = d(arg[2], arg[1]), b3 = d(arg[3], arg[2]);
    const V3<double> n1 = cross(b1, b2), n2 = cross(b2, b3);
    const double lb2 = sqrt(dot(b2, b2));
    O = atan2(lb2 * dot(b1, n2), dot(n1, n2));
    const double ci = -lb2 / dot(n1, n1), cl = lb2 / dot(n2, n2);
    const double f12 = dot(b1, b2) / (lb2 * lb2), f32 = dot(b3, b2) / (lb2 * lb2);
    gi = {ci * n1.x, ci * n1.y, ci * n1.z};
    gl = {cl * n2.x, cl * n2.y, cl * n2.z};
    gj = {-(1 + f12) * gi.x + f32 * gl.x, -(1 + f12) * gi.y + f32 * gl.y, -(1 + f12) * gi.z + f32 * gl.z};
    gk = {f12 * gi.x - (1 + f32) * gl.x, f12 * gi.y - (1 + f32) * gl.y, f12 * gi.z - (1 + f32) * gl.z};
  }
  double g = O, gp = 1.0;
  if (a.transform == 1) {
    g = 1.0 / (1.0 + exp(-(O - a.center) / a.width));
    gp = g * (1.0 - g) / a.width;
  }
  const double c = a.inv_norm * gp;
  if (a.obs_kind == GRP_OBS_COORD) {
    lq[3 * arg[0] + arg[1]] += c;
  } else if (a.obs_kind == GRP_OBS_GROUP_DISTANCE) {
    for (int t = S.group_off[arg[0]]; t < S.group_off[arg[0] + 1]; ++t) {
      const int at = S.group_atoms[t];
      for (int x = 0; x < 3; ++x) lq[3 * at + x] += c * S.mass[at] / ma * u[x];
    }
    for (int t = S.group_off[arg[1]]; t < S.group_off[arg[1] + 1]; ++t) {
      const int at = S.group_atoms[t];
      for (int x = 0; x < 3; ++x) lq[3 * at + x] -= c * S.mass[at] / mb * u[x];
    }
  } else {
    const V3<double> *gs[4] = {&gi, &gj, &gk, &gl};
    for (int m = 0; m < 4; ++m) {
      lq[3 * arg[m] + 0] += c * gs[m]->x;
      lq[3 * arg[m] + 1] += c * gs[m]->y;
      lq[3 * arg[m] + 2] += c * gs[m]->z;
    }
  }
  return a.inv_norm * g;
}

// Precision of the adjoint: the recomputation runs the forward path's own arithmetic (PathF64, or the mixed
// path's FP32 forces into split fixed point with double-single integration), so that it reproduces the
// forward trajectory bit for bit; the reverse sweep's Hessian-vector products and mixed parameter
// derivatives come from dual numbers of that precision (Dual in FP64, DualF in FP32).  The tangent
// direction is scaled to a largest component of kTangentScale (1/16 on the mixed path, so that the
// stiff bonds' tangent contributions stay inside the split fixed point's 2^18 range).
template <class P>
struct AdjointTraits;
template <>
struct AdjointTraits<PathF64> {
  using TP = PathTangent;
  using Num = Dual;
  static constexpr double kTangentScale = 1.0;
  static __device__ AccTangent tacc(long long *DF, int) { return AccTangent{DF}; }
  static __device__ double tget(const long long *DF, int i, int) { return (double)DF[i] * kFixInv; }
  static __device__ Params<PathTangent> tpar(const SysDev &S) {
    return Params<PathTangent>{S.atom_d, S.bond_d, S.angle_d, S.term_d, S.coulomb_rf, S.krf, S.crf};
  }
};
template <>
struct AdjointTraits<PathMixed> {
  using TP = PathTangentF;
  using Num = DualF;
  static constexpr double kTangentScale = 1.0 / 16.0;
  static __device__ AccTangentF tacc(long long *DF, int nd) {
    return AccTangentF{(int *)DF, (unsigned int *)DF + nd};
  }
  static __device__ double tget(const long long *DF, int i, int nd) {
    return (double)split_to_float(((const int *)DF)[i], ((const unsigned int *)DF)[nd + i]);
  }
  static __device__ Params<PathTangentF> tpar(const SysDev &S) {
    return Params<PathTangentF>{S.atom_f, S.bond_f, S.angle_f, S.term_f, S.coulomb_rf, (float)S.krf, (float)S.crf};
  }
};

size_t adjoint_smem_bytes(const SysDev &S, int n_terms, int ck) {
  const size_t nd = (size_t)S.nd, nt = 2 * (size_t)S.n + n_terms;
  return nd * 8 * 2 + nt * 8 * 2 + nd * 8 * 3 + 33 * 8 + (size_t)(ck + 1) * nd * 8 + 32 +
         State<PathF64>::bytes(S.n, true) + 32;
}

template <class P>
__global__ void __launch_bounds__(256) adjoint_kernel(const AdjArgs a) {
  using Tr = AdjointTraits<P>;
  using TP = typename Tr::TP;
  using T = typename P::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const SysDev &S = a.S;
  const int r = blockIdx.x, n = S.n, nd = S.nd, nt = 2 * n + a.n_terms;
  unsigned char *ptr = smem;
  long long *F = (long long *)ptr; ptr += (size_t)nd * 8;
  long long *DF = (long long *)ptr; ptr += (size_t)nd * 8;
  long long *Gd = (long long *)ptr; ptr += (size_t)nt * 8;
  double *gth = (double *)ptr; ptr += (size_t)nt * 8;
  double *lq = (double *)ptr; ptr += (size_t)nd * 8;
  double *lp = (double *)ptr; ptr += (size_t)nd * 8;
  double *vn = (double *)ptr; ptr += (size_t)nd * 8;
  double *red = (double *)ptr; ptr += 33 * 8;
  ptr = align32(ptr);
  double *Qs = (double *)ptr; ptr += (size_t)(a.ck + 1) * nd * 8;
  State<P> st;
  ptr = align32(ptr);
  st.carve(ptr, n, S, true);
  for (int i = threadIdx.x; i < nd; i += blockDim.x) { lq[i] = 0.0; lp[i] = 0.0; F[i] = 0; }
  for (int k = threadIdx.x; k < nt; k += blockDim.x) gth[k] = 0.0;
  int err = 0;
  double loss = 0.0;
  const double h = a.h, c1 = a.c1;
  const typename P::Acc fa = State<P>::acc(F, n);
  const Params<TP> tpar = Tr::tpar(S);

  // the contribution of configuration q_t (see above)
  auto config = [&](const double *qt, long long t, double w) {
    if (t >= 1 && a.t_gr > 0 && (a.t_phase0 + t) % a.t_gr == 0) {
      if (threadIdx.x == 0) loss += loss_sample(a, qt, lq);
      __syncthreads();
    }
    double m = 0.0;
    for (int i = threadIdx.x; i < nd; i += blockDim.x) m = fmax(m, fabs(lp[i]));
    const double s = block_max_d(m, red) / Tr::kTangentScale;
    if (s > 0.0) {
      for (int i = threadIdx.x; i < nd; i += blockDim.x) { vn[i] = lp[i] / s; DF[i] = 0; }
      for (int k = threadIdx.x; k < nt; k += blockDim.x) Gd[k] = 0;
      __syncthreads();
      const Pos<TP> tpos{qt, vn};
      long long e = 0;
      force_pass<TP>(S, tpos, tpar, S.items, S.pairs, Tr::tacc(DF, nd), false, e, &err);
      param_pass<typename Tr::Num>(S, tpar.atom, tpar.term, [&](int i, int j) { return tpos.diff(i, j); },
                                   ParamTangent{Gd}, &err);
      __syncthreads();
      const double ws = w * s;
      for (int i = threadIdx.x; i < nd; i += blockDim.x) lq[i] += ws * Tr::tget(DF, i, nd);
      for (int k = threadIdx.x; k < nt; k += blockDim.x) gth[k] -= ws * kFixInv * (double)Gd[k];
      __syncthreads();
    }
  };

  for (int c = a.n_ck - 1; c >= 0; --c) {
    const int t0 = c * a.ck, len = min(a.ck, a.k - t0);
    const double *base = a.ckpt + ((size_t)r * a.n_ck + c) * 3 * nd;
    __syncthreads();
    st.load(S, base, base + nd, base + 2 * nd, n, c1);
    __syncthreads();
    for (int at = threadIdx.x; at < n; at += blockDim.x) st.get_f64(at, Qs + 3 * at);
    __syncthreads();  // the copy reads positions that the first drift below overwrites
    // forward recomputation of steps t0 .. t0 + len - 1, keeping every configuration
    for (int j = 0; j < len; ++j) {
      for (int at = threadIdx.x; at < n; at += blockDim.x) {
        T z[4];
        normals4(philox_stream(a.seed, a.t_global0 + t0 + j, 0u, r, at), z);
        st.baoa(at, z, (T)h, (T)c1);
      }
      __syncthreads();
      long long e = 0;
      force_pass<P>(S, st.pos(), st.params(S), S.items, S.pairs, fa, false, e, &err);
      __syncthreads();
      for (int at = threadIdx.x; at < n; at += blockDim.x) {
        st.bk(at, fa, (T)h);
        st.get_f64(at, Qs + (size_t)(j + 1) * nd + 3 * at);
      }
      __syncthreads();
    }
    // reverse sweep over configurations t0 + len .. t0 + 1 and the steps that led to them
    for (int j = len; j >= 1; --j) {
      const long long t = t0 + j;
      config(Qs + (size_t)j * nd, t, t == a.k ? h : 2.0 * h);
      for (int i = threadIdx.x; i < nd; i += blockDim.x) {
        const double hm = h * S.atom_d[i / 3].w;
        const double lpp = lp[i] + hm * lq[i];
        lp[i] = c1 * lpp + hm * lq[i];
      }
      __syncthreads();
    }
  }
  config(Qs, 0, h);  // q_0 (block 0 left it in Qs[0]): the first half kick
  for (int k = threadIdx.x; k < nt; k += blockDim.x) a.partial[(size_t)r * nt + k] = gth[k];
  if (a.grad_q0)
    for (int i = threadIdx.x; i < nd; i += blockDim.x) a.grad_q0[(size_t)r * nd + i] = lq[i];
  if (a.grad_p0)
    for (int i = threadIdx.x; i < nd; i += blockDim.x) a.grad_p0[(size_t)r * nd + i] = lp[i];
  if (threadIdx.x == 0) a.loss[r] = loss;
  if (err) atomicOr(a.err, err);
}

cudaError_t launch_adjoint(const AdjArgs &a, int n_rep, cudaStream_t st) {
  if (n_rep <= 0) return cudaSuccess;
  if (a.S.potential != GRP_POT_FORCE_FIELD || a.S.tiled) return cudaErrorInvalidValue;
  const size_t smem = adjoint_smem_bytes(a.S, a.n_terms, a.ck);
  if (smem > kMaxSmem) return cudaErrorInvalidValue;
  auto kern = a.S.precision == GRP_FP64 ? adjoint_kernel<PathF64> : adjoint_kernel<PathMixed>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n_rep, 256, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace grp

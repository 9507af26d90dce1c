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

#include "forcefield.cuh"
#include "kernels.h"

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
  const T cut2 = (T)S.cutoff2;
  if (!S.tiled) {
    for (int t = threadIdx.x; t < S.n_pairs; t += blockDim.x) {
      const uint32_t pk = S.pairs[t];
      const int i = (int)(pk & 0xFFFFu), j = (int)(pk >> 16);
      T dsig, dei, dej;
      if (!lj_param_terms<T>(qdiff<T>(qb, i, j), atom[i], atom[j], cut2, dsig, dei, dej)) continue;
      const long long fs = to_fix((double)dsig, &err);
      fix_add(&G[i], fs);
      fix_add(&G[j], fs);
      fix_add(&G[n + i], to_fix((double)dei, &err));
      fix_add(&G[n + j], to_fix((double)dej, &err));
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
        if (!lj_param_terms<T>(qdiff<T>(qb, i, j), atom[i], atom[j], cut2, dsig, dei, dej)) continue;
        si += dsig;
        ei += dei;
        fix_add(&G[j], to_fix((double)dsig, &err));
        fix_add(&G[n + j], to_fix((double)dej, &err));
      }
      if (i < n) {
        fix_add(&G[i], to_fix((double)si, &err));
        fix_add(&G[n + i], to_fix((double)ei, &err));
      }
    }
  }
  // dihedral terms: dE/dk = 1 + cos(n phi - delta), cos and sin of n phi by the angle-addition recurrence
  for (int u = threadIdx.x; u < S.n_dih; u += blockDim.x) {
    const int4 a = S.dih_ijkl[u];
    const int2 tr = S.dih_terms[u];
    const V3<T> b1 = qdiff<T>(qb, a.y, a.x), b2 = qdiff<T>(qb, a.z, a.y), b3 = qdiff<T>(qb, a.w, a.z);
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
      G[2 * n + S.term_src[t]] = to_fix((double)(T(1) + cn * (T)tp.z + sn * (T)tp.w), &err);
    }
  }
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

}  // namespace grp

// Generalized Born implicit solvent, OBC model II (the solvent model of the paper's protein-ligand MD
// setup, Section 4.2), for systems of the explicit item table (fewer than 64 atoms, no cutoff).
//
// Atom i has an offset radius a_i = rho_i - 0.009 nm and a descreening sphere of radius s_i = S_i a_i.
// Atom j descreens atom i by h_ij, twice (1/4 pi) the integral of |x|^-4 over sphere j outside the
// sphere of radius a_i around i: with L = max(a_i, |r - s_j|), U = r + s_j and a_i < U,
//   h = 1/L - 1/U + (r/4)(1/U^2 - 1/L^2) + (1/2r) ln(L/U) + (s_j^2/4r)(1/L^2 - 1/U^2)
//       [+ 2 (1/a_i - 1/L) when sphere j encloses atom i's sphere].
// I_i = (1/2) sum_j h_ij, psi = a_i I_i, 1/B_i = 1/a_i - tanh(psi - 0.8 psi^2 + 4.85 psi^3) / rho_i, and
//   E = -(tau/2) sum_i sum_j q_i q_j / f_ij,  f_ij = sqrt(r^2 + B_i B_j exp(-r^2 / 4 B_i B_j)), f_ii = B_i,
// tau = k_e (1/eps_in - 1/eps_out), over all pairs (bonded ones included).  Forces: the pair terms at
// fixed Born radii, then the chain rule through B_i(I_i(r_ij)) with the derivatives dh/dr that the first
// pass keeps per pair in shared memory.  Three passes over the pairs, separated
// by block barriers; sums go to fixed-point accumulators, so the result does not depend on the order.
#pragma once
#include "forcefield.cuh"

namespace grp {

// Shared-memory scratch of the solvent term: accumulators of I_i and dE/dB_i, Born radii and the
// per-atom chain-rule weights.
template <class P>
struct GbScratch {
  using T = typename P::T;
  ScalarAcc<P> acc;  // [0, n): sum_j h_ij;  [n, 2n): dE/dB_i
  T *born, *w;   // [n]
  T *dh;         // [2 n (n - 1) / 2]: dh_ij/dr and dh_ji/dr of every pair, from the first pass
  static size_t bytes(int n) {
    return ScalarAcc<P>::bytes(2 * n) + (size_t)2 * n * sizeof(T) + (size_t)n * (n - 1) * sizeof(T) + 32;
  }
  __device__ void carve(unsigned char *&ptr, int n) {
    acc.carve(ptr, 2 * n);
    ptr = (unsigned char *)(((uintptr_t)ptr + 15) & ~(uintptr_t)15);
    born = (T *)ptr; ptr += (size_t)n * sizeof(T);
    w = (T *)ptr; ptr += (size_t)n * sizeof(T);
    dh = (T *)ptr; ptr += (size_t)n * (n - 1) * sizeof(T);
  }
};

__device__ __forceinline__ double glog(double x) { return log(x); }
__device__ __forceinline__ float glog(float x) { return logf(x); }
__device__ __forceinline__ double gtanh(double x) { return tanh(x); }
__device__ __forceinline__ float gtanh(float x) { return tanhf(x); }

// h_ij and dh/dr for atom i (offset radius ai) descreened by a sphere of radius sj at distance r.
template <class T>
__device__ __forceinline__ T gb_hct(T r, T ai, T sj, T &dh) {
  const T U = r + sj;
  if (!(ai < U)) {
    dh = T(0);
    return T(0);
  }
  const T diff = r - sj, adiff = diff < T(0) ? -diff : diff;
  const bool lfix = ai > adiff;
  const T L = lfix ? ai : adiff, dL = lfix ? T(0) : (diff >= T(0) ? T(1) : T(-1));
  // reciprocals by grcp (the hardware approximation in FP32, an IEEE quotient in FP64)
  const T iL = grcp(L), iU = grcp(U), iL2 = iL * iL, iU2 = iU * iU, lg = glog(L * iU), s2 = sj * sj, ir = grcp(r);
  T h = iL - iU + T(0.25) * r * (iU2 - iL2) + T(0.5) * ir * lg + T(0.25) * s2 * ir * (iL2 - iU2);
  T d = -dL * iL2 + iU2 + T(0.25) * (iU2 - iL2) + T(0.25) * r * (T(-2) * iU2 * iU + T(2) * dL * iL2 * iL) -
        T(0.5) * ir * ir * lg + T(0.5) * ir * (dL * iL - iU) - T(0.25) * s2 * ir * ir * (iL2 - iU2) +
        T(0.25) * s2 * ir * (T(-2) * dL * iL2 * iL + T(2) * iU2 * iU);
  if (ai < sj - r) {
    h += T(2) * (grcp(ai) - iL);
    d += T(2) * dL * iL2;
  }
  dh = d;
  return h;
}

// Per-atom solvent parameters of a path: (a_i, 1/rho_i, s_i, q_i).
template <class P>
__device__ __forceinline__ auto gb_atom(const SysDev &S, int i) {
  if constexpr (P::kMixed) return S.gb_f[i];
  else return S.gb_d[i];
}

// The solvent forces (and energy when want_e) of one replica, added to the force accumulators; called
// by every thread of the block, with the positions final; returns after the last pass (the caller's
// barrier before reading the forces covers it).  The scratch accumulators are zero on entry and left
// zero.
template <class P>
__device__ void gb_forces(const SysDev &S, const Pos<P> &pos, const typename P::Acc &fa, const GbScratch<P> &g,
                          bool want_e, long long &e_fix, int *err) {
  using T = typename P::T;
  const int n = S.n, np = S.n_gb_pairs, bd = blockDim.x;
  const T tau = (T)S.gb_tau;
  // 1. descreening sums
  for (int t = threadIdx.x; t < np; t += bd) {
    const uint32_t pk = S.gb_pairs[t];
    const int i = (int)(pk & 0xFFFFu), j = (int)(pk >> 16);
    const V3<T> d = pos.diff(i, j);
    const T r = gsqrt(dot(d, d));
    const auto pi = gb_atom<P>(S, i), pj = gb_atom<P>(S, j);
    T dhij, dhji;
    g.acc.add(i, gb_hct<T>(r, (T)pi.x, (T)pj.z, dhij), err);
    g.acc.add(j, gb_hct<T>(r, (T)pj.x, (T)pi.z, dhji), err);
    g.dh[2 * t] = dhij;  // kept for the chain rule (pass 5)
    g.dh[2 * t + 1] = dhji;
  }
  __syncthreads();
  // 2. Born radii, dB/dI, the self terms of E and dE/dB
  for (int i = threadIdx.x; i < n; i += bd) {
    const auto p = gb_atom<P>(S, i);
    const T ai = (T)p.x, irho = (T)p.y, qi = (T)p.w;
    const T psi = ai * T(0.5) * g.acc.get(i);
    const T th = gtanh(psi - T(0.8) * psi * psi + T(4.85) * psi * psi * psi);
    const T B = T(1) / (T(1) / ai - th * irho);
    g.acc.zero(i);
    g.born[i] = B;
    g.w[i] = B * B * (T(1) - th * th) * irho * (T(1) - T(1.6) * psi + T(14.55) * psi * psi) * ai;  // dB/dI
    g.acc.set(n + i, T(0.5) * tau * qi * qi / (B * B), err);
    if (want_e) e_fix += fa.efix(T(-0.5) * tau * qi * qi / B, err);
  }
  __syncthreads();
  // 3. pair terms at fixed Born radii: forces and the pairs' parts of dE/dB
  for (int t = threadIdx.x; t < np; t += bd) {
    const uint32_t pk = S.gb_pairs[t];
    const int i = (int)(pk & 0xFFFFu), j = (int)(pk >> 16);
    const V3<T> d = pos.diff(i, j);
    const T r2 = dot(d, d);
    const T bi = g.born[i], bj = g.born[j], bb = bi * bj, D = r2 / (T(4) * bb), e = gexp(-D);
    const T f2 = r2 + bb * e, f = gsqrt(f2), qq = (T)gb_atom<P>(S, i).w * (T)gb_atom<P>(S, j).w;
    const T dEdf = tau * qq / f2;
    const T dBcommon = dEdf * e * (T(1) + D) / (T(2) * f);
    g.acc.add(n + i, dBcommon * bj, err);
    g.acc.add(n + j, dBcommon * bi, err);
    const T gr = -dEdf * (T(1) - T(0.25) * e) / f;  // -dE/dr / r
    fa.add(i, V3<T>{gr * d.x, gr * d.y, gr * d.z}, err);
    fa.add(j, V3<T>{-gr * d.x, -gr * d.y, -gr * d.z}, err);
    if (want_e) e_fix += fa.efix(-tau * qq / f, err);
  }
  __syncthreads();
  // 4. chain-rule weights w_i = dE/dB_i dB_i/dI_i / 2
  for (int i = threadIdx.x; i < n; i += bd) {
    g.w[i] = T(0.5) * g.acc.get(n + i) * g.w[i];
    g.acc.zero(n + i);
  }
  __syncthreads();
  // 5. forces through the Born radii
  for (int t = threadIdx.x; t < np; t += bd) {
    const uint32_t pk = S.gb_pairs[t];
    const int i = (int)(pk & 0xFFFFu), j = (int)(pk >> 16);
    const V3<T> d = pos.diff(i, j);
    const T r = gsqrt(dot(d, d));
    const T gr = -(g.w[i] * g.dh[2 * t] + g.w[j] * g.dh[2 * t + 1]) / r;
    fa.add(i, V3<T>{gr * d.x, gr * d.y, gr * d.z}, err);
    fa.add(j, V3<T>{-gr * d.x, -gr * d.y, -gr * d.z}, err);
  }
}

// The solvent forces of a system with a cutoff (Verlet-list systems, up to thousands of atoms): the five
// passes of gb_forces over the pairs within the cutoff (plain truncation: a pair at r >= r_c enters
// neither I_i nor the pair energy; the self terms always count).  `pairs(f)` calls f(i, j, k) for this
// thread's share of the candidate pairs (each unordered pair once), kGbBatch pairs at a time (slots with
// i < 0 are empty): the Verlet list, which holds every non-excluded pair within the cutoff, and the
// excluded pairs, which the solvent term includes; k is the pair's slot in `gr3` (the same in every
// pass), or -1 when `gr3` is null.  With a slot, pass 3 keeps its force factor -dE/dr / r there and
// pass 5 adds the pair's two force contributions at once (12 fixed-point additions fewer per pair).  Each pass loads the positions, parameters and Born
// quantities of a whole batch before evaluating it, so that the loads' latencies (the parameters and
// Born radii are in global memory) overlap instead of adding up pair by pair.  One shared-memory
// accumulator per atom serves I_i in passes 1-2 and dE/dB_i in passes 2-4; the Born radii and chain-rule
// weights of the replica live in `born` and `w` (global memory, [n] each, written and read by this
// block only).  dh/dr is recomputed in pass 5 instead of kept per pair.  Called by every thread of the
// block with the positions final; the scratch accumulator is zero on entry and left zero.
constexpr int kGbBatch = 4;
template <class P, class Pairs>
__device__ void gb_forces_cut(const SysDev &S, const Pos<P> &pos, const typename P::Acc &fa, const ScalarAcc<P> &acc,
                              typename P::T *born, typename P::T *w, typename P::T *gr3, Pairs pairs, bool want_e,
                              long long &e_fix, int *err) {
  using T = typename P::T;
  using GA = decltype(gb_atom<P>(S, 0));
  const int n = S.n, bd = blockDim.x;
  const T tau = (T)S.gb_tau, cut2 = (T)S.cutoff2;
  // 1. descreening sums
  pairs([&](const int (&I)[kGbBatch], const int (&J)[kGbBatch], const int (&K)[kGbBatch]) {
    V3<T> d[kGbBatch];
    GA pa[kGbBatch], pb[kGbBatch];
#pragma unroll
    for (int u = 0; u < kGbBatch; ++u) {  // an empty slot reads atom 0 and is skipped below
      const int i = I[u] < 0 ? 0 : I[u], j = I[u] < 0 ? 0 : J[u];
      d[u] = pos.diff(i, j);
      pa[u] = gb_atom<P>(S, i);
      pb[u] = gb_atom<P>(S, j);
    }
#pragma unroll
    for (int u = 0; u < kGbBatch; ++u) {
      const T r2 = dot(d[u], d[u]);
      if (I[u] < 0 || !(r2 < cut2)) continue;
      const T r = gsqrt(r2);
      T dh;
      acc.add(I[u], gb_hct<T>(r, (T)pa[u].x, (T)pb[u].z, dh), err);
      acc.add(J[u], gb_hct<T>(r, (T)pb[u].x, (T)pa[u].z, dh), err);
    }
  });
  __syncthreads();
  // 2. Born radii, dB/dI, the self terms of E and dE/dB
  for (int i = threadIdx.x; i < n; i += bd) {
    const auto p = gb_atom<P>(S, i);
    const T ai = (T)p.x, irho = (T)p.y, qi = (T)p.w;
    const T psi = ai * T(0.5) * acc.get(i);
    const T th = gtanh(psi - T(0.8) * psi * psi + T(4.85) * psi * psi * psi);
    const T B = T(1) / (T(1) / ai - th * irho);
    born[i] = B;
    w[i] = B * B * (T(1) - th * th) * irho * (T(1) - T(1.6) * psi + T(14.55) * psi * psi) * ai;  // dB/dI
    acc.set(i, T(0.5) * tau * qi * qi / (B * B), err);
    if (want_e) e_fix += fa.efix(T(-0.5) * tau * qi * qi / B, err);
  }
  __syncthreads();
  // 3. pair terms at fixed Born radii: forces and the pairs' parts of dE/dB
  pairs([&](const int (&I)[kGbBatch], const int (&J)[kGbBatch], const int (&K)[kGbBatch]) {
    V3<T> d[kGbBatch];
    T bi[kGbBatch], bj[kGbBatch], qq[kGbBatch];
#pragma unroll
    for (int u = 0; u < kGbBatch; ++u) {
      const int i = I[u] < 0 ? 0 : I[u], j = I[u] < 0 ? 0 : J[u];
      d[u] = pos.diff(i, j);
      bi[u] = born[i];
      bj[u] = born[j];
      qq[u] = (T)gb_atom<P>(S, i).w * (T)gb_atom<P>(S, j).w;
    }
#pragma unroll
    for (int u = 0; u < kGbBatch; ++u) {
      const T r2 = dot(d[u], d[u]);
      if (I[u] < 0 || !(r2 < cut2)) continue;
      const T bb = bi[u] * bj[u], D = T(0.25) * r2 * grcp(bb), e = gexp(-D);
      const T f2 = r2 + bb * e, rf = grsqrt(f2);
      const T dEdf = tau * qq[u] * rf * rf;
      const T dBcommon = T(0.5) * dEdf * e * (T(1) + D) * rf;
      acc.add(I[u], dBcommon * bj[u], err);
      acc.add(J[u], dBcommon * bi[u], err);
      const T gr = -dEdf * (T(1) - T(0.25) * e) * rf;  // -dE/dr / r
      if (K[u] >= 0) {
        gr3[K[u]] = gr;  // added with pass 5's factor
      } else {
        fa.add(I[u], V3<T>{gr * d[u].x, gr * d[u].y, gr * d[u].z}, err);
        fa.add(J[u], V3<T>{-gr * d[u].x, -gr * d[u].y, -gr * d[u].z}, err);
      }
      if (want_e) e_fix += fa.efix(-tau * qq[u] * rf, err);
    }
  });
  __syncthreads();
  // 4. chain-rule weights w_i = dE/dB_i dB_i/dI_i / 2
  for (int i = threadIdx.x; i < n; i += bd) {
    w[i] = T(0.5) * acc.get(i) * w[i];
    acc.zero(i);
  }
  __syncthreads();
  // 5. forces through the Born radii
  pairs([&](const int (&I)[kGbBatch], const int (&J)[kGbBatch], const int (&K)[kGbBatch]) {
    V3<T> d[kGbBatch];
    GA pa[kGbBatch], pb[kGbBatch];
    T wi[kGbBatch], wj[kGbBatch], g3[kGbBatch];
#pragma unroll
    for (int u = 0; u < kGbBatch; ++u) {
      const int i = I[u] < 0 ? 0 : I[u], j = I[u] < 0 ? 0 : J[u];
      d[u] = pos.diff(i, j);
      pa[u] = gb_atom<P>(S, i);
      pb[u] = gb_atom<P>(S, j);
      wi[u] = w[i];
      wj[u] = w[j];
      g3[u] = K[u] >= 0 ? gr3[K[u]] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kGbBatch; ++u) {
      const T r2 = dot(d[u], d[u]);
      if (I[u] < 0 || !(r2 < cut2)) continue;
      const T r = gsqrt(r2);
      T dhij, dhji;
      gb_hct<T>(r, (T)pa[u].x, (T)pb[u].z, dhij);
      gb_hct<T>(r, (T)pb[u].x, (T)pa[u].z, dhji);
      const T gr = g3[u] - (wi[u] * dhij + wj[u] * dhji) * grcp(r);
      fa.add(I[u], V3<T>{gr * d[u].x, gr * d[u].y, gr * d[u].z}, err);
      fa.add(J[u], V3<T>{-gr * d[u].x, -gr * d[u].y, -gr * d[u].z}, err);
    }
  });
}

}  // namespace grp

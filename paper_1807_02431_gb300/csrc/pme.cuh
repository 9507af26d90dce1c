// Smooth particle mesh Ewald (Essmann et al. 1995; the particle mesh Ewald method is among the
// optimisations the paper expects of an MD engine, Section 3.2) for one replica of an item-table system
// (fewer than 64 atoms) in an orthorhombic periodic box.
//
// The pair loop evaluates the real-space part k_e q_i q_j erfc(beta r)/r over minimum images within
// the cutoff.  This file adds the rest of the Ewald sum:
//   * excluded pairs: -k_e q_i q_j erf(beta r)/r (minimum image), removing what the reciprocal sum
//     gives the nearest image of a pair without Coulomb interaction;
//   * the reciprocal sum on a K0 x K1 x K2 grid.  Each charge is spread by cubic cardinal B-splines
//     (order 4) of its scaled fractional coordinates u_d = K_d frac(r_d / L_d): the weight of grid
//     point (floor(u) - t) mod K is M_4(u - floor(u) + t), t = 0..3.  The grid Q is transformed, each
//     coefficient multiplied by the influence function G(m) = B(m) exp(-pi^2 |m|^2/beta^2)/(pi V |m|^2)
//     (B the Euler exponential spline factor, G(0) = 0) and transformed back, which gives the
//     potential phi on the grid; E = 1/2 sum_k Q(k) phi(k), and F_i = -q_i sum_k grad W_i(k) phi(k);
//   * the self and neutralising-background energies, constants of the system.
// Charges enter scaled by sqrt(k_e / 4) (the atom table's third word), so the table holds 4 G.
//
// The grid is summed in fixed point (order-independent, like the force accumulators); the first
// transform pass reads it into a complex array in shared memory whose rows along the third axis are
// padded by one element (so that a warp's threads, each transforming one row, fall on different banks).  One thread transforms
// one line of K = 8 or 16 points in registers (radix-2, decimation in time).  The third axis runs
// last forward and first backward in one pass that applies G in between.
#pragma once
#include "forcefield.cuh"

namespace grp {

template <class P>
struct PmeCplx;
template <>
struct PmeCplx<PathF64> {
  using type = double2;
};
template <>
struct PmeCplx<PathMixed> {
  using type = float2;
};

// Shared-memory scratch of the mesh: the charge grid's fixed-point accumulators, the complex grid, and
// per atom and axis the grid cell floor(u) and the B-spline weights and derivatives at u.
// Strides of the fixed-point charge grid: rows of K2 + 1 words, planes of K1 (K2 + 1) words rounded up
// to 4 mod 32.  Spreading gives the 16 (t0, t1) offsets of one atom to 16 lanes, which then fall in 16
// distinct banks (t1 moves a row, 17 or 9 banks; t0 a plane, 4 banks); with planes of K1 K2 words all
// four t0 and two t1 offsets shared a bank (8-way conflicts on every fixed-point addition).
__host__ __device__ __forceinline__ void pme_acc_strides(int K1, int K2, int &rs, int &ps) {
  rs = K2 + 1;
  const int p = K1 * rs;
  ps = p + (36 - p % 32) % 32;
}

template <class P>
struct PmeScratch {
  using T = typename P::T;
  using C2 = typename PmeCplx<P>::type;
  ScalarAcc<P> acc;  // [K0][K1][K2] in padded rows and planes (pme_acc_strides)
  C2 *c;             // [K0][K1][K2 + 1]
  T *wm, *wd;        // [3n][4]: M_4(w + t), M_4'(w + t)
  int *cell;         // [3n]
  __host__ __device__ static int acc_points(const SysDev &S) {
    int rs, ps;
    pme_acc_strides(S.pme_K[1], S.pme_K[2], rs, ps);
    return S.pme_K[0] * ps;
  }
  static size_t bytes(const SysDev &S) {
    const size_t gc = (size_t)S.pme_K[0] * S.pme_K[1] * (S.pme_K[2] + 1);
    return ScalarAcc<P>::bytes(acc_points(S)) + 32 + gc * sizeof(C2) + (size_t)3 * S.n * (4 + 8 * sizeof(T)) + 32;
  }
  __device__ void carve(unsigned char *&ptr, const SysDev &S) {
    const int g = acc_points(S);
    acc.carve(ptr, g);
    ptr = (unsigned char *)(((uintptr_t)ptr + 15) & ~(uintptr_t)15);
    c = (C2 *)ptr;
    ptr += (size_t)S.pme_K[0] * S.pme_K[1] * (S.pme_K[2] + 1) * sizeof(C2);
    wm = (T *)ptr;
    ptr += (size_t)12 * S.n * sizeof(T);
    wd = (T *)ptr;
    ptr += (size_t)12 * S.n * sizeof(T);
    cell = (int *)ptr;
    ptr += (size_t)3 * S.n * 4;
    ptr = (unsigned char *)(((uintptr_t)ptr + 15) & ~(uintptr_t)15);
  }
  __device__ void zero(const SysDev &S) const {
    const int g = acc_points(S);
    for (int i = threadIdx.x; i < g; i += blockDim.x) acc.zero(i);
  }
};

// Coordinate x of atom i in FP64 (the mixed path's double-single pair summed).
template <class P>
__device__ __forceinline__ double pme_coord(const Pos<P> &pos, int i, int x) {
  if constexpr (P::kMixed) return (double)(&pos.qh[i].x)[x] + (double)(&pos.ql[i].x)[x];
  else return pos.q[3 * i + x];
}

// Cubic B-spline weights m[t] = M_4(w + t) and derivatives d[t] = M_4'(w + t), t = 0..3, for an offset
// w in [0, 1), built up from M_2 by the recursion M_n(x) = (x M_{n-1}(x) + (n - x) M_{n-1}(x - 1)) /
// (n - 1), and M_4'(x) = M_3(x) - M_3(x - 1).
template <class T>
__device__ __forceinline__ void bspline4(T w, T (&m)[4], T (&d)[4]) {
  m[0] = w;  // order 2: M_2(w), M_2(w + 1)
  m[1] = T(1) - w;
  m[2] = T(0.5) * (T(1) - w) * m[1];  // order 3, from the top index down
  m[1] = T(0.5) * ((w + T(1)) * m[1] + (T(2) - w) * m[0]);
  m[0] = T(0.5) * w * m[0];
  d[0] = m[0];
  d[1] = m[1] - m[0];
  d[2] = m[2] - m[1];
  d[3] = -m[2];
  const T c = T(1) / T(3);  // order 4
  m[3] = c * (T(1) - w) * m[2];
  m[2] = c * ((w + T(2)) * m[2] + (T(2) - w) * m[1]);
  m[1] = c * ((w + T(1)) * m[1] + (T(3) - w) * m[0]);
  m[0] = c * w * m[0];
}

// exp(2 pi i j / 16), j = 0..7: cos(pi/8) = sqrt(2 + sqrt 2)/2, sin(pi/8) = sqrt(2 - sqrt 2)/2.
__host__ __device__ constexpr double tw16_re(int j) {
  return j == 0 ? 1.0 : j == 1 ? 0.92387953251128674 : j == 2 ? 0.70710678118654752 : j == 3 ? 0.38268343236508977
       : j == 4 ? 0.0 : j == 5 ? -0.38268343236508977 : j == 6 ? -0.70710678118654752 : -0.92387953251128674;
}
__host__ __device__ constexpr double tw16_im(int j) {
  return j == 0 ? 0.0 : j == 1 ? 0.38268343236508977 : j == 2 ? 0.70710678118654752 : j == 3 ? 0.92387953251128674
       : j == 4 ? 1.0 : j == 5 ? 0.92387953251128674 : j == 6 ? 0.70710678118654752 : 0.38268343236508977;
}
// the low `bits` (3 or 4) bits of i reversed
__host__ __device__ constexpr int bitrev(int i, int bits) {
  return bits == 4 ? ((i & 1) << 3) | ((i & 2) << 1) | ((i & 4) >> 1) | ((i & 8) >> 3)
                   : ((i & 1) << 2) | (i & 2) | ((i & 4) >> 2);
}
template <int K>
struct Log2;
template <>
struct Log2<8> {
  static constexpr int value = 3;
};
template <>
struct Log2<16> {
  static constexpr int value = 4;
};

// In-register discrete Fourier transforms of K = 8 or 16 points, X(m) = sum_k x(k) exp(s 2 pi i m k / K),
// unnormalised, radix 2.  The forward transform (s = +1) decimates in time: it takes its input in
// bit-reversed order (x(bitrev(e)) in register e) and leaves X in natural order.  The backward one
// (s = -1) decimates in frequency: natural order in, bit-reversed order out.  The callers load and
// store at bit-reversed addresses, so no permutation happens in registers.
template <class T>
__device__ __forceinline__ void twiddle(T &re, T &im, int idx16, int sign) {
  if (idx16 == 4) {  // exp(+-i pi/2) = +-i: a swap and a sign, exact
    const T r = re;
    re = sign > 0 ? -im : im;
    im = sign > 0 ? r : -r;
    return;
  }
  const T wr = T(tw16_re(idx16)), wi = T(sign * tw16_im(idx16));
  const T r = re * wr - im * wi;
  im = re * wi + im * wr;
  re = r;
}
// One stage of butterflies of length kLen (decimation in time: twiddle, then sum and difference;
// in frequency: sum and difference, then twiddle), unrolled at compile time.
template <int K, int kLen, class T>
__device__ __forceinline__ void dit_stage(T (&re)[K], T (&im)[K]) {
  constexpr int kHalf = kLen / 2, kStep = 16 / kLen;
#pragma unroll
  for (int i = 0; i < K; i += kLen) {
#pragma unroll
    for (int j = 0; j < kHalf; ++j) {
      const int a = i + j, b = a + kHalf;
      T vr = re[b], vi = im[b];
      if (j > 0) twiddle(vr, vi, j * kStep, 1);
      re[b] = re[a] - vr;
      im[b] = im[a] - vi;
      re[a] += vr;
      im[a] += vi;
    }
  }
}
template <int K, int kLen, class T>
__device__ __forceinline__ void dif_stage(T (&re)[K], T (&im)[K]) {
  constexpr int kHalf = kLen / 2, kStep = 16 / kLen;
#pragma unroll
  for (int i = 0; i < K; i += kLen) {
#pragma unroll
    for (int j = 0; j < kHalf; ++j) {
      const int a = i + j, b = a + kHalf;
      const T ur = re[a], ui = im[a];
      re[a] = ur + re[b];
      im[a] = ui + im[b];
      T dr = ur - re[b], di = ui - im[b];
      if (j > 0) twiddle(dr, di, j * kStep, -1);
      re[b] = dr;
      im[b] = di;
    }
  }
}
template <int K, class T>
__device__ __forceinline__ void fft_fwd(T (&re)[K], T (&im)[K]) {
  dit_stage<K, 2>(re, im);
  dit_stage<K, 4>(re, im);
  dit_stage<K, 8>(re, im);
  if constexpr (K == 16) dit_stage<K, 16>(re, im);
}
template <int K, class T>
__device__ __forceinline__ void fft_bwd(T (&re)[K], T (&im)[K]) {
  if constexpr (K == 16) dif_stage<K, 16>(re, im);
  dif_stage<K, 8>(re, im);
  dif_stage<K, 4>(re, im);
  dif_stage<K, 2>(re, im);
}

// Transform every line of the complex grid along axis kAxis (0 or 1) in the first K0 planes of axis 0:
// forward (kSign = 1) or backward.
template <int K, int kAxis, int kSign, class C2, class T>
__device__ __forceinline__ void fft_lines(C2 *c, int K0, int K1, int K2) {
  constexpr int kBits = Log2<K>::value;
  const int rz = K2 + 1;  // padded row length along the third axis
  const int n_lines = (kAxis == 0 ? K1 : K0) * K2;
  const int stride = kAxis == 0 ? K1 * rz : rz;
  for (int l = threadIdx.x; l < n_lines; l += blockDim.x) {
    const int a = l / K2, k2 = l - a * K2;
    const int base = (kAxis == 0 ? a * rz : a * K1 * rz) + k2;
    T re[K], im[K];
#pragma unroll
    for (int e = 0; e < K; ++e) {
      const C2 v = c[base + (kSign > 0 ? bitrev(e, kBits) : e) * stride];
      re[e] = v.x;
      im[e] = v.y;
    }
    if (kSign > 0) fft_fwd<K>(re, im);
    else fft_bwd<K>(re, im);
#pragma unroll
    for (int e = 0; e < K; ++e) {
      C2 v;
      v.x = re[e];
      v.y = im[e];
      c[base + (kSign > 0 ? e : bitrev(e, kBits)) * stride] = v;
    }
  }
}
// The first pass, real to complex: the lines (k1, k2) and (k1, k2 + K2/2) along axis 0 of the real
// fixed-point charge grid (which they zero) are transformed together as z = a + i b; the spectra of the
// real lines follow from Z(m) and Z(K - m): A(m) = (Z(m) + conj Z(K-m)) / 2, B(m) = (Z(m) - conj Z(K-m)) / 2i.
// Only m = 0..K/2 is kept (A(K - m) = conj A(m)): planes 0..K0/2 of the complex grid.
template <int K, class P, class C2, class T>
__device__ __forceinline__ void fft_first_r2c(const ScalarAcc<P> &acc, C2 *c, int K1, int K2) {
  constexpr int kBits = Log2<K>::value;
  const int rz = K2 + 1, h2 = K2 >> 1;
  int rs, ps;
  pme_acc_strides(K1, K2, rs, ps);
  for (int l = threadIdx.x; l < K1 * h2; l += blockDim.x) {
    const int k1 = l / h2, k2 = l - k1 * h2;
    T re[K], im[K];
#pragma unroll
    for (int e = 0; e < K; ++e) {
      const int g = bitrev(e, kBits) * ps + k1 * rs + k2;
      re[e] = acc.get(g);
      im[e] = acc.get(g + h2);
      acc.zero(g);
      acc.zero(g + h2);
    }
    fft_fwd<K>(re, im);
#pragma unroll
    for (int m = 0; m <= K / 2; ++m) {
      const int mk = (K - m) & (K - 1);
      const T xr = re[m], xi = im[m], yr = re[mk], yi = im[mk];
      C2 a, b;
      a.x = T(0.5) * (xr + yr);
      a.y = T(0.5) * (xi - yi);
      b.x = T(0.5) * (xi + yi);
      b.y = T(0.5) * (yr - xr);
      c[(m * K1 + k1) * rz + k2] = a;
      c[(m * K1 + k1) * rz + k2 + h2] = b;
    }
  }
}

// The last pass, complex to real: the half spectra A, B (planes 0..K0/2) of the lines (k1, k2) and
// (k1, k2 + K2/2) are extended by A(K - m) = conj A(m) and transformed back together as A + i B, whose
// real and imaginary parts are the two real lines; they are stored in the real parts of the grid.
template <int K, class C2, class T>
__device__ __forceinline__ void fft_last_c2r(C2 *c, int K1, int K2) {
  constexpr int kBits = Log2<K>::value;
  const int rz = K2 + 1, h2 = K2 >> 1;
  for (int l = threadIdx.x; l < K1 * h2; l += blockDim.x) {
    const int k1 = l / h2, k2 = l - k1 * h2;
    T ar[K / 2 + 1], ai[K / 2 + 1], br[K / 2 + 1], bi[K / 2 + 1];
#pragma unroll
    for (int m = 0; m <= K / 2; ++m) {
      const C2 a = c[(m * K1 + k1) * rz + k2], b = c[(m * K1 + k1) * rz + k2 + h2];
      ar[m] = a.x;
      ai[m] = a.y;
      br[m] = b.x;
      bi[m] = b.y;
    }
    T re[K], im[K];
#pragma unroll
    for (int m = 0; m < K; ++m) {
      if (m <= K / 2) {
        re[m] = ar[m] - bi[m];
        im[m] = ai[m] + br[m];
      } else {
        const int mk = K - m;
        re[m] = ar[mk] + bi[mk];
        im[m] = br[mk] - ai[mk];
      }
    }
    fft_bwd<K>(re, im);
#pragma unroll
    for (int e = 0; e < K; ++e) {
      const int k0 = bitrev(e, kBits);
      c[(k0 * K1 + k1) * rz + k2].x = re[e];
      c[(k0 * K1 + k1) * rz + k2 + h2].x = im[e];
    }
  }
}

// Lines along axis 1 in planes 0..n0-1 of axis 0.
template <int kSign, class C2, class T>
__device__ __forceinline__ void fft_axis1(C2 *c, int n0, const int *K) {
  if (K[1] == 16) fft_lines<16, 1, kSign, C2, T>(c, n0, K[1], K[2]);
  else fft_lines<8, 1, kSign, C2, T>(c, n0, K[1], K[2]);
}

// The third axis in planes 0..K0/2 of axis 0: forward transform, multiplication by the influence table
// (and its energy 1/2 sum G |F|^2, planes 0 < m0 < K0/2 counted twice for their conjugates
// K0 - m0), backward transform.
template <int K, class C2, class T>
__device__ __forceinline__ T fft_third(C2 *c, const T *gtab, int K0, int K1, bool want_e) {
  constexpr int kBits = Log2<K>::value;
  const int rz = K + 1;
  T e = T(0);
  for (int l = threadIdx.x; l < (K0 / 2 + 1) * K1; l += blockDim.x) {
    const int base = l * rz, m0 = l / K1;
    const T wplane = (m0 == 0 || 2 * m0 == K0) ? T(0.5) : T(1);
    T re[K], im[K];
#pragma unroll
    for (int m = 0; m < K; ++m) {
      const C2 v = c[base + bitrev(m, kBits)];
      re[m] = v.x;
      im[m] = v.y;
    }
    fft_fwd<K>(re, im);
#pragma unroll
    for (int m = 0; m < K; ++m) {
      const T g = __ldg(gtab + l * K + m);
      if (want_e) e += wplane * g * (re[m] * re[m] + im[m] * im[m]);
      re[m] *= g;
      im[m] *= g;
    }
    fft_bwd<K>(re, im);
#pragma unroll
    for (int m = 0; m < K; ++m) {
      C2 v;
      v.x = re[m];
      v.y = im[m];
      c[base + bitrev(m, kBits)] = v;
    }
  }
  return e;
}

// The mesh part of the periodic electrostatics of one replica (everything but the real-space pairs),
// added to the force accumulators, and its energy when want_e; called by every thread of the block
// with the positions final.  The grid accumulators are zero on entry and left zero; returns after the
// gather (the caller's barrier before reading the forces covers it).
template <class P>
__device__ void pme_forces(const SysDev &S, const Pos<P> &pos, const Params<P> &par, const typename P::Acc &fa,
                           const PmeScratch<P> &g, bool want_e, long long &e_fix, int *err) {
  using T = typename P::T;
  using C2 = typename PmeCplx<P>::type;
  const int n = S.n, bd = blockDim.x;
  const int K0 = S.pme_K[0], K1 = S.pme_K[1], K2 = S.pme_K[2];
  // 1. grid cell and B-spline weights of every coordinate.  Unwrapped positions may lie many boxes out,
  // so the grid coordinate u = x K / L is formed at more than FP32 precision: in FP64 on the FP64 path;
  // on the mixed path in double-single from the position's two words and K / L's two words, with FP32
  // instructions only (FP64 instructions run at 1/64 of the FP32 rate on this part): t_hi + t_lo with
  // t_hi = x_hi c_hi and t_lo = its exact rounding error (fma) + x_hi c_lo + x_lo c_hi; the fractional
  // part t_hi - floor(t_hi) is exact, and adding t_lo leaves w within ~6e-8 of frac(u).
  for (int i = threadIdx.x; i < 3 * n; i += bd) {
    const int at = i / 3, x = i - 3 * at;
    int k;
    T w;
    if constexpr (P::kMixed) {
      const float xh = (&pos.qh[at].x)[x], xl = (&pos.ql[at].x)[x];
      const float ch = S.pme_kl[x][0], cl = S.pme_kl[x][1];
      const float th = xh * ch;
      const float tl = fmaf(xh, ch, -th) + fmaf(xh, cl, xl * ch);
      float nf = floorf(th);
      float wv = (th - nf) + tl;
      if (wv < 0.f) {
        wv += 1.f;
        nf -= 1.f;
      } else if (wv >= 1.f) {
        wv -= 1.f;
        nf += 1.f;
      }
      k = (int)nf % S.pme_K[x];
      k += k < 0 ? S.pme_K[x] : 0;
      w = wv;
    } else {
      const double t = pme_coord<P>(pos, at, x) * S.ibox[x];
      const double u = (t - floor(t)) * (double)S.pme_K[x];
      const double fl = floor(u);
      k = (int)fl;
      if (k >= S.pme_K[x]) k -= S.pme_K[x];
      w = (T)(u - fl);
    }
    g.cell[i] = k;
    T m[4], d[4];
    bspline4(w, m, d);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      g.wm[4 * i + t] = m[t];
      g.wd[4 * i + t] = d[t];
    }
  }
  // excluded pairs: E = -4 qq erf(b r)/r, -dE/dr / r = 4 qq (2 b/sqrt(pi) exp(-b^2 r^2) - erf(b r)/r) / r^2
  const T b = T(par.beta);
  for (int e = threadIdx.x; e < S.n_excl_pairs; e += bd) {
    const uint32_t pk = S.excl_pairs[e];
    const int i = (int)(pk & 0xFFFFu), j = (int)(pk >> 16);
    const V3<T> d = pair_image<2>(par, pos.diff(i, j));
    const T r2 = dot(d, d), ir = grsqrt(r2), qq = T(par.atom[i].z) * T(par.atom[j].z);
    const T erfr = gerf(b * r2 * ir) * ir;
    const T gr = T(4) * qq * (T(kTwoOverSqrtPi) * b * gexp(-b * b * r2) - erfr) * ir * ir;
    fa.add(i, V3<T>{gr * d.x, gr * d.y, gr * d.z}, err);
    fa.add(j, V3<T>{-gr * d.x, -gr * d.y, -gr * d.z}, err);
    if (want_e) e_fix += fa.efix(T(-4) * qq * erfr, err);
  }
  if (want_e && threadIdx.x == 0) e_fix += fa.efix((T)S.pme_e_const, err);
  __syncthreads();
  // 2. spread: one thread per (atom, t0, t1), four grid points along the third axis each
  int acc_rs, acc_ps;
  pme_acc_strides(K1, K2, acc_rs, acc_ps);
  for (int it = threadIdx.x; it < 16 * n; it += bd) {
    const int at = it >> 4, t0 = (it >> 2) & 3, t1 = it & 3;
    int k0 = g.cell[3 * at] - t0, k1 = g.cell[3 * at + 1] - t1;
    k0 += k0 < 0 ? K0 : 0;
    k1 += k1 < 0 ? K1 : 0;
    const T w = T(par.atom[at].z) * g.wm[12 * at + t0] * g.wm[12 * at + 4 + t1];
    const T *m2 = g.wm + 12 * at + 8;
    const int row = k0 * acc_ps + k1 * acc_rs, c2 = g.cell[3 * at + 2];
#pragma unroll
    for (int t2 = 0; t2 < 4; ++t2) {
      const int k2 = c2 - t2 + (c2 - t2 < 0 ? K2 : 0);
      g.acc.add(row + k2, w * m2[t2], err);
    }
  }
  __syncthreads();
  // 3. transforms: axis 0 forward from the fixed-point grid (left zero), axis 1 forward, axis 2
  // forward-G-backward, axes 1 and 0 backward
  const int n0 = K0 / 2 + 1;  // planes of axis 0 that the middle passes need (the grid is real)
  if (K0 == 16) fft_first_r2c<16, P, C2, T>(g.acc, g.c, K1, K2);
  else fft_first_r2c<8, P, C2, T>(g.acc, g.c, K1, K2);
  __syncthreads();
  fft_axis1<1, C2, T>(g.c, n0, S.pme_K);
  __syncthreads();
  const T *gtab;
  if constexpr (P::kMixed) gtab = S.pme_g_f;
  else gtab = S.pme_g_d;
  const T erec = K2 == 16 ? fft_third<16, C2, T>(g.c, gtab, K0, K1, want_e) : fft_third<8, C2, T>(g.c, gtab, K0, K1, want_e);
  if (want_e) e_fix += fa.efix(erec, err);
  __syncthreads();
  fft_axis1<-1, C2, T>(g.c, n0, S.pme_K);
  __syncthreads();
  if (K0 == 16) fft_last_c2r<16, C2, T>(g.c, K1, K2);
  else fft_last_c2r<8, C2, T>(g.c, K1, K2);
  __syncthreads();
  // 4. gather: one thread per (atom, t1); F_i = -q_i sum_k grad W_i(k) phi(k), dW/dr_d = K_d/L_d dW/du_d.
  // The four t1 threads of an atom are consecutive lanes reading rows one complex row apart (distinct
  // banks; with one thread per t0 the four lanes read planes 272 complex values apart, one bank); their
  // forces are summed by shuffles and added once.  Every thread runs the same number of rounds, so that
  // whole warps take part in the shuffles.
  for (int base = 0; base < 4 * n; base += bd) {
    const int it = base + threadIdx.x;
    const bool active = it < 4 * n;
    const int at = active ? it >> 2 : 0, t1 = it & 3;
    V3<T> f{T(0), T(0), T(0)};
    if (active) {
      const T *w0 = g.wm + 12 * at, *dw0 = g.wd + 12 * at, *m2 = g.wm + 12 * at + 8, *d2 = g.wd + 12 * at + 8;
      const int c0 = g.cell[3 * at], c2 = g.cell[3 * at + 2];
      int k1 = g.cell[3 * at + 1] - t1;
      k1 += k1 < 0 ? K1 : 0;
      T ax = T(0), ay = T(0), az = T(0);
#pragma unroll
      for (int t0 = 0; t0 < 4; ++t0) {
        const int k0 = c0 - t0 + (c0 - t0 < 0 ? K0 : 0);
        const int row = (k0 * K1 + k1) * (K2 + 1);
        T px = T(0), pz = T(0);  // sum over t2 of phi m2 and phi d2
#pragma unroll
        for (int t2 = 0; t2 < 4; ++t2) {
          const int k2 = c2 - t2 + (c2 - t2 < 0 ? K2 : 0);
          const T ph = g.c[row + k2].x;
          px += ph * m2[t2];
          pz += ph * d2[t2];
        }
        ax += dw0[t0] * px;
        ay += w0[t0] * px;
        az += w0[t0] * pz;
      }
      const T qi = T(par.atom[at].z);
      const T m1 = g.wm[12 * at + 4 + t1], d1 = g.wd[12 * at + 4 + t1];
      f = {-qi * m1 * ax * T(K0 * par.ibox[0]), -qi * d1 * ay * T(K1 * par.ibox[1]),
           -qi * m1 * az * T(K2 * par.ibox[2])};
    }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      f.x += __shfl_xor_sync(0xffffffffu, f.x, o);
      f.y += __shfl_xor_sync(0xffffffffu, f.y, o);
      f.z += __shfl_xor_sync(0xffffffffu, f.z, o);
    }
    if (active && t1 == 0) fa.add(at, f, err);
  }
}

}  // namespace grp

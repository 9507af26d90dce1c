// Shared device definitions of libgrp: system layout on the device, Philox4x32-10 noise,
// Box-Muller normals, 64-bit fixed-point force accumulation and double-single arithmetic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/grp.h"

namespace grp {

constexpr int kMaxObs = GRP_MAX_OBS;
constexpr int kMaxGroups = GRP_MAX_GROUPS;

// Error bits latched by kernels into the replica set's error word.
enum : int { kErrNaN = 1, kErrOverflow = 2, kErrList = 4, kErrConstraint = 8, kErrIndex = 16, kErrTimeout = 32 };

// Kinds of force-field work items.
enum : uint32_t { kItemPair = 0, kItemBond = 1, kItemAngle = 2, kItemDihedral = 3, kItemNone = 15 };

// FP64-path fixed point: one unit = 2^-40 of the force (or energy) unit, so that quantisation (9e-13)
// stays below FP64 rounding of typical forces.  Integer sums are exact modulo 2^64, so only a single
// contribution and the final sum must fit: contributions are bounded by 2^22 (larger ones set the
// overflow flag), and a sum is exact while its magnitude stays below 2^23.
constexpr double kFixScale = 1099511627776.0;       // 2^40
constexpr double kFixInv = 1.0 / 1099511627776.0;
constexpr double kFixLimit = 4194304.0;               // 2^22

// Device copy of a system.  All arrays are device memory owned by grp_system.  Parameters exist in
// FP64 (FP64 path) and FP32 (mixed path) copies.
struct SysDev {
  int n, dim, nd, potential, precision;
  double dw_a, dw_b;
  double kT, gamma, dt;
  const double *mass;      // [n]
  const double4 *atom_d;   // [n] (sigma/2, sqrt(eps), q sqrt(k_e/4), 1/m)
  const float4 *atom_f;
  const double *sd_d;      // [n] noise amplitudes sqrt((1 - c1^2) kT m) of the O step (large systems)
  const float *sd_f;
  int n_pairs;             // explicit non-excluded pair list (i | j << 16), i < j
  const uint32_t *pairs;
  int n_items;             // force-field work items, (kind << 28) | index, each kind padded to a
  const uint32_t *items;   // multiple of 32 entries so that a warp runs a single kind of item
  // Tiled nonbonded path (tiled = 1): atoms in tiles of 32; every tile pair I <= J with, per lane
  // of tile I, a 32-bit mask of the atoms of tile J it interacts with (exclusions, padding and, on
  // the diagonal, i != j removed); the explicit pair items are then not in the item table.
  int tiled;
  int n_tiles, n_tile_pairs;
  const uint32_t *tile_pairs;  // I | J << 16
  const uint32_t *tile_masks;  // [n_tile_pairs][32]
  double cutoff2;          // 0: no cutoff
  int coulomb_rf;          // Coulomb model: 0 dielectric eps = 4r, 1 reaction field (eps_r = 1),
                           // 2 periodic: Ewald real space on pairs plus particle mesh Ewald
  int gb;                  // 1: Generalized Born (OBC II) implicit solvent
  int n_cons;              // bond constraints, in the description's order
  const int2 *con_ij;
  const double *con_len;
  double con_tol;          // relative tolerance of SHAKE / RATTLE
  int con_max_iter;
  const unsigned char *con_atom;  // [n] 1 for atoms of a constraint
  int n_cgroups;           // connected groups of constraints (independent of each other)
  const int *cgroup_off;   // [n_cgroups + 1] into cgroup_cons and cgroup_atoms_off
  const int *cgroup_cons;  // constraint indices of each group, ascending
  const int *cgroup_aoff;  // [n_cgroups + 1] into cgroup_atoms
  const int *cgroup_atoms; // atoms of each group
  int n_gb_pairs;          // every pair i < j (i | j << 16) (systems of the item table)
  const uint32_t *gb_pairs;
  int n_gb_xpairs;         // the excluded pairs i < j (systems with Verlet lists, whose lists omit them)
  const uint32_t *gb_xpairs;
  double gb_tau;           // k_e (1/eps_in - 1/eps_out)
  const double4 *gb_d;     // per atom (rho - 0.009, 1/rho, S (rho - 0.009), q)
  const float4 *gb_f;
  double krf, crf;         // reaction-field constants k_rf, c_rf (per nm^3, per nm)
  // Periodic electrostatics by smooth particle mesh Ewald (coulomb_rf = 2)
  double box[3], ibox[3];  // orthorhombic box edges (nm) and their inverses
  double ewald_beta;       // splitting parameter (per nm)
  int pme_K[3];            // grid points per axis (8 or 16)
  float pme_kl[3][2];      // K_d / L_d as a double-single pair (the mixed path's grid coordinates)
  double pme_e_const;      // self and neutralising-background energy
  int n_excl_pairs;        // excluded pairs (i | j << 16): minus the smooth part of their Coulomb
  const uint32_t *excl_pairs;
  const double *pme_g_d;   // [K0][K1][K2] 4 B(m) exp(-pi^2 |m|^2 / beta^2) / (pi V |m|^2), 0 at m = 0
  const float *pme_g_f;
  // Verlet lists (tiled systems with a cutoff): pairs closer than cutoff + skin, rebuilt when an atom
  // has moved more than skin/2 since the last build
  int use_list;
  float list_cut2;         // (cutoff + skin)^2
  float half_skin2;        // (skin / 2)^2
  int n_bonds;
  const int2 *bond_ij;
  const double2 *bond_d;   // (k, r0)
  const float2 *bond_f;
  int n_angles;
  const int4 *angle_ijk;
  const double2 *angle_d;  // (k, theta0)
  const float2 *angle_f;
  int n_dih;               // dihedral items: 4 atoms, terms [dih_terms.x, dih_terms.y)
  const int4 *dih_ijkl;
  const int2 *dih_terms;
  const double4 *term_d;   // (k, n, cos delta, sin delta)
  const float4 *term_f;
  const int *term_src;     // [terms] index of each term in the description's dihedral list
  int cv_kind;
  int cv_atoms[8];
  double cv_params[8];
  int n_groups;
  int group_off[kMaxGroups + 1];
  const int *group_atoms;
  int n_obs;
  int obs_kind[kMaxObs];
  int obs_arg[kMaxObs][4];
};

// ------------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).
// Counter = (t_global low 32 bits, t_global bits 32..55 | stream << 24, replica, atom), key = seed.
// Stream 0: BAOAB noise; stream 1: Fleming-Viot branching draw.
struct Philox4 {
  uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                  uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  Philox4 r;
  r.v[0] = c0; r.v[1] = c1; r.v[2] = c2; r.v[3] = c3;
  return r;
}

__device__ __forceinline__ Philox4 philox_stream(uint64_t seed, int64_t step, uint32_t stream,
                                                 int replica, int atom) {
  const uint64_t st = (uint64_t)step;
  return philox4x32_10((uint32_t)st, (uint32_t)((st >> 32) & 0x00FFFFFFu) | (stream << 24),
                       (uint32_t)replica, (uint32_t)atom, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Box-Muller on word pairs (w0, w1), (w2, w3) with u = (w + 1/2) 2^-32.
__device__ __forceinline__ void normals4_f64(const Philox4 &w, double xi[4]) {
#pragma unroll
  for (int pr = 0; pr < 2; ++pr) {
    const double u1 = ((double)w.v[2 * pr] + 0.5) * 0x1p-32;
    const double u2 = ((double)w.v[2 * pr + 1] + 0.5) * 0x1p-32;
    const double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    xi[2 * pr] = rad * c;
    xi[2 * pr + 1] = rad * s;
  }
}

__device__ __forceinline__ void normals4_f32(const Philox4 &w, float xi[4]) {
#pragma unroll
  for (int pr = 0; pr < 2; ++pr) {
    const float u1 = fmaf((float)w.v[2 * pr], 0x1p-32f, 0x1p-33f);
    const float u2 = fmaf((float)w.v[2 * pr + 1], 0x1p-32f, 0x1p-33f);
    const float rad = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    xi[2 * pr] = rad * c;
    xi[2 * pr + 1] = rad * s;
  }
}

// ------------------------------------------------------------------------------------------------
// Fixed-point accumulation: contributions converted with round-to-nearest; integer sums are exact
// and independent of order, so results do not depend on the thread decomposition.
__device__ __forceinline__ long long to_fix(double v, int *err) {
  if (!(fabs(v) < kFixLimit)) { *err |= kErrOverflow; return 0; }
  return __double2ll_rn(v * kFixScale);
}
// Mixed-path force accumulator: fixed point with 2^-32 units kept as two 32-bit words that are
// summed separately with non-returning atomics (no carry between them; the 64-bit integer
// conversions would run on the FP64 pipe, 1/64 of the FP32 rate on GB300): a contribution v 2^32 is
// split as hi 2^20 + lo with lo in [0, 2^20].  The lo word holds up to 4,095 contributions without
// wrapping; the hi word is summed modulo 2^32, exact as long as the total |F| < 2^19.  The value is
// hi_sum 2^20 + lo_sum, the same integer whatever the order of the additions.  Single contributions
// are bounded by 2^18 (larger ones, or NaN, set the overflow flag).
constexpr float kSplitHiScale = 4096.0f;       // 2^32 / 2^20
constexpr float kSplitLoScale = 1048576.0f;    // 2^20
constexpr float kSplitInv = 2.3283064365386963e-10f;  // 2^-32
constexpr float kSplitLimit = 262144.0f;       // 2^18
struct Split {
  int hi;
  unsigned int lo;
};
// hi = floor(v 2^12) (one rounding-down conversion), r = v 2^12 - hi in [0, 1) (exact: |v 2^12| <
// 2^27 keeps hi exactly representable), lo = round(r 2^20) in [0, 2^20]; lo = 2^20 (r rounding up)
// is a valid split of the same integer, so the lo word holds at most 4,095 contributions.  A
// contribution at or beyond the fixed-point limit (or NaN) sets the overflow flag.
__device__ __forceinline__ Split to_split(float v, int *err) {
  const float a = v * kSplitHiScale;
  Split s;
  s.hi = __float2int_rd(a);
  s.lo = __float2uint_rn((a - (float)s.hi) * kSplitLoScale);
  *err |= (fabsf(v) < kSplitLimit) ? 0 : kErrOverflow;
  return s;
}
__device__ __forceinline__ long long split_value(Split s) { return (long long)s.hi * (1ll << 20) + (long long)s.lo; }
__device__ __forceinline__ void split_add(int *hi, unsigned int *lo, int idx, Split s) {
  atomicAdd(&hi[idx], s.hi);
  atomicAdd(&lo[idx], s.lo);
}
__device__ __forceinline__ float split_to_float(int hi_sum, unsigned int lo_sum) {
  return fmaf((float)hi_sum, kSplitLoScale, (float)lo_sum) * kSplitInv;
}
// 64-bit shared-memory atomics are not native on sm_103a (measured: 5x slower than 32-bit, 140x
// under a 32-way address conflict), so the int64 accumulator is updated as two 32-bit words: the low
// word's atomic returns its previous value, which gives this addition's carry into the high word.
// Every addition changes the 64-bit value by exactly v (mod 2^64) whatever the interleaving.
__device__ __forceinline__ void fix_add(long long *dst, long long v) {
  unsigned int *w = reinterpret_cast<unsigned int *>(dst);  // little endian: w[0] low, w[1] high
  const unsigned long long u = (unsigned long long)v;
  const unsigned int lo = (unsigned int)u, hi = (unsigned int)(u >> 32);
  const unsigned int old = atomicAdd(&w[0], lo);
  const unsigned int carry = (unsigned int)(old + lo < old);
  atomicAdd(&w[1], hi + carry);
}

// ------------------------------------------------------------------------------------------------
// Double-single numbers x = hi + lo (|lo| <= ulp(hi)/2): Knuth's TwoSum and Dekker's Fast2Sum keep
// about 48 significant bits with FP32 instructions only.
struct ds {
  float hi, lo;
};
__device__ __forceinline__ ds ds_from_double(double x) {
  ds r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}
__device__ __forceinline__ double ds_to_double(ds x) { return (double)x.hi + (double)x.lo; }
// x + d for a float d
__device__ __forceinline__ ds ds_add(ds x, float d) {
  const float s = __fadd_rn(x.hi, d);
  const float bp = __fsub_rn(s, x.hi);
  const float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bp)), __fsub_rn(d, bp));
  const float lo = __fadd_rn(x.lo, e);
  ds r;
  r.hi = __fadd_rn(s, lo);
  r.lo = __fsub_rn(lo, __fsub_rn(r.hi, s));
  return r;
}
// c * x for a float c
__device__ __forceinline__ ds ds_scale(ds x, float c) {
  const float ph = __fmul_rn(c, x.hi);
  const float pl = __fmaf_rn(c, x.hi, -ph);  // exact error of the product
  const float lo = __fmaf_rn(c, x.lo, pl);
  ds r;
  r.hi = __fadd_rn(ph, lo);
  r.lo = __fsub_rn(lo, __fsub_rn(r.hi, ph));
  return r;
}

// x + y and x - y of two double-single numbers (TwoSum of the high words, the low words added to the
// error, renormalised by Fast2Sum; about 2^-46 relative), and x * y (Dekker's product of the high words
// by an fma, the cross terms in FP32).
__device__ __forceinline__ ds ds_add2(ds x, ds y) {
  const float s = __fadd_rn(x.hi, y.hi);
  const float bp = __fsub_rn(s, x.hi);
  const float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bp)), __fsub_rn(y.hi, bp));
  const float lo = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  ds r;
  r.hi = __fadd_rn(s, lo);
  r.lo = __fsub_rn(lo, __fsub_rn(r.hi, s));
  return r;
}
__device__ __forceinline__ ds ds_sub2(ds x, ds y) { return ds_add2(x, ds{-y.hi, -y.lo}); }
__device__ __forceinline__ ds ds_mul2(ds x, ds y) {
  const float ph = __fmul_rn(x.hi, y.hi);
  const float pl = __fmaf_rn(x.hi, y.hi, -ph);
  const float lo = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, pl));
  ds r;
  r.hi = __fadd_rn(ph, lo);
  r.lo = __fsub_rn(lo, __fsub_rn(r.hi, ph));
  return r;
}

// Block-wide sum of int64 values (every thread contributes; result valid in thread 0).
__device__ __forceinline__ long long block_sum_ll(long long v, long long *scratch /* >= 32 */) {
  const int kThreads = (int)blockDim.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  long long t = 0;
  if (warp == 0) {
    t = (lane < (kThreads + 31) / 32) ? scratch[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

// Two block-wide int64 sums in one pass (scratch >= 64 entries); the results are valid in thread 0.
__device__ __forceinline__ void block_sum2_ll(long long &a, long long &b, long long *scratch) {
  const int kThreads = (int)blockDim.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { scratch[warp] = a; scratch[32 + warp] = b; }
  __syncthreads();
  if (warp == 0) {
    const bool in = lane < (kThreads + 31) / 32;
    a = in ? scratch[lane] : 0;
    b = in ? scratch[32 + lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
  }
}

}  // namespace grp

// Fused segment kernels: k BAOAB steps of Eq. 1 per replica with the replica's state held on chip,
// observable sampling every t_GR (Section 2.4.1) and the exit test at the end of the segment
// (Section 3.3).  One thread block per replica for force-field systems; one thread per replica for
// the analytic 2-D double well.
#include <cfloat>

#include <type_traits>

#include "forcefield.cuh"
#include "constraints.cuh"
#include "gb.cuh"
#include "pme.cuh"
#include "kernels.h"
#include "state.cuh"

namespace grp {

// ------------------------------------------------------------------------------------------------
// FP64 state functions (Section 3.3) on positions given by an accessor get(a, double[3]).
template <class Get>
__device__ double dihedral_rad_f64(Get get, int i, int j, int k, int l) {
  double qi[3], qj[3], qk[3], ql[3];
  get(i, qi); get(j, qj); get(k, qk); get(l, ql);
  const V3<double> b1 = {qj[0] - qi[0], qj[1] - qi[1], qj[2] - qi[2]};
  const V3<double> b2 = {qk[0] - qj[0], qk[1] - qj[1], qk[2] - qj[2]};
  const V3<double> b3 = {ql[0] - qk[0], ql[1] - qk[1], ql[2] - qk[2]};
  const V3<double> n1 = cross(b1, b2), n2 = cross(b2, b3);
  return atan2(sqrt(dot(b2, b2)) * dot(b1, n2), dot(n1, n2));
}

template <class Get>
__device__ void group_com_f64(const SysDev &S, Get get, int g, double com[3]) {
  double mt = 0, c[3] = {0, 0, 0};
  for (int t = S.group_off[g]; t < S.group_off[g + 1]; ++t) {
    const int at = S.group_atoms[t];
    const double m = S.mass[at];
    double x[3];
    get(at, x);
    mt += m;
    c[0] += m * x[0]; c[1] += m * x[1]; c[2] += m * x[2];
  }
  com[0] = c[0] / mt; com[1] = c[1] / mt; com[2] = c[2] / mt;
}

// Returns the state index containing the configuration (-1: none); *out_exited = outside omega.
template <class Get>
__device__ int state_check_f64(const SysDev &S, Get get, int omega, int *out_exited) {
  if (S.cv_kind == GRP_CV_DOUBLE_WELL) {
    double x[3];
    get(0, x);
    const double w = S.cv_params[0];
    *out_exited = omega == 0 ? (x[0] >= 0.0) : (x[0] < 0.0);
    return x[0] < -w ? 0 : (x[0] > w ? 1 : -1);
  }
  if (S.cv_kind == GRP_CV_ROTAMERS) {
    // base-3 index of the torsions' wells (gauche+ [0, 120), trans, gauche- [-120, 0) degrees); in a
    // state when every torsion is within w of its well's centre; outside omega when a well differs
    const int *c = S.cv_atoms;
    const int m = (int)S.cv_params[0];
    const double w = S.cv_params[1], deg = 57.295779513082320876798154814105;
    int label = 0, scale = 1, core = 1, ex = 0, rest = omega;
    for (int t = 0; t < m; ++t, rest /= 3, scale *= 3) {
      const double phi = deg * dihedral_rad_f64(get, c[t], c[t + 1], c[t + 2], c[t + 3]);
      const int well = (phi >= 0.0 && phi < 120.0) ? 0 : ((phi >= -120.0 && phi < 0.0) ? 2 : 1);
      const double off = well == 0 ? fabs(phi - 60.0) : (well == 2 ? fabs(phi + 60.0) : 180.0 - fabs(phi));
      core &= off < w ? 1 : 0;
      label += well * scale;
      ex |= well != rest % 3 ? 1 : 0;
    }
    *out_exited = ex;
    return core ? label : -1;
  }
  int label;
  if (S.cv_kind == GRP_CV_DIHEDRAL_RECT) {
    const int *c = S.cv_atoms;
    const double deg = 57.295779513082320876798154814105;
    const double phi = deg * dihedral_rad_f64(get, c[0], c[1], c[2], c[3]);
    const double psi = deg * dihedral_rad_f64(get, c[1], c[2], c[3], c[4]);
    const bool in = phi >= S.cv_params[0] && phi <= S.cv_params[1] && psi >= S.cv_params[2] &&
                    psi <= S.cv_params[3];
    label = in ? 0 : 1;
  } else {
    double c0[3], c1[3];
    group_com_f64(S, get, 0, c0);
    group_com_f64(S, get, 1, c1);
    const double dx = c0[0] - c1[0], dy = c0[1] - c1[1], dz = c0[2] - c1[2];
    label = sqrt(dx * dx + dy * dy + dz * dz) < S.cv_params[0] ? 0 : 1;
  }
  *out_exited = label != omega;
  return label;
}

__device__ __forceinline__ void acc_add(double *acc, double v) {
  // acc = (shift c, sum (O - c), sum (O - c)^2, n); the first sample sets the shift.
  if (acc[3] == 0.0) acc[0] = v;
  const double d = v - acc[0];
  acc[1] += d;
  acc[2] += d * d;
  acc[3] += 1.0;
}

// A parallel-step segment of check M is skipped when an exit was already recorded at an earlier
// check (segments are queued ahead of the readback); an exit at the same check M must not stop the
// other replicas of check M, whose exits may carry a lower index k.
__device__ __forceinline__ bool exit_seen_before(const SegArgs &a) {
  return (*(volatile unsigned long long *)a.exit_key >> 32) < (unsigned long long)a.M;
}

__device__ __forceinline__ void record_check(const SegArgs &a, int r, int label, int ex) {
  a.labels[r] = (int8_t)label;
  a.exited[r] = (uint8_t)ex;
  if (ex && a.exit_key)
    atomicMin(a.exit_key, ((unsigned long long)a.M << 32) | (unsigned long long)(unsigned)r);
}

// Observable j (Section 2.4.1) in the path's precision, from shared-memory state.
template <class P>
__device__ typename P::T observable_ff(const SysDev &S, const State<P> &st, int j, typename P::T v_pot,
                                       typename P::T v_kin) {
  using T = typename P::T;
  const int *arg = S.obs_arg[j];
  const Pos<P> pos = st.pos();
  switch (S.obs_kind[j]) {
    case GRP_OBS_POTENTIAL: return v_pot;
    case GRP_OBS_KINETIC: return v_kin;
    case GRP_OBS_COORD: {
      double x[3];
      if constexpr (P::kMixed) {
        const float4 a = st.qh[arg[0]], b = st.ql[arg[0]];
        return (&a.x)[arg[1]] + (&b.x)[arg[1]];
      } else {
        st.get_f64(arg[0], x);
        return x[arg[1]];
      }
    }
    case GRP_OBS_DIHEDRAL: {
      const V3<T> b1 = pos.diff(arg[1], arg[0]), b2 = pos.diff(arg[2], arg[1]), b3 = pos.diff(arg[3], arg[2]);
      const V3<T> n1 = cross(b1, b2), n2 = cross(b2, b3);
      return gatan2(gsqrt(dot(b2, b2)) * dot(b1, n2), dot(n1, n2));
    }
    case GRP_OBS_GROUP_DISTANCE: {
      // centre of mass difference relative to the first atom of group a (keeps FP32 sums small)
      const int ref = S.group_atoms[S.group_off[arg[0]]];
      T c[2][3] = {{0, 0, 0}, {0, 0, 0}};
      for (int g = 0; g < 2; ++g) {
        T mt = 0;
        for (int t = S.group_off[arg[g]]; t < S.group_off[arg[g] + 1]; ++t) {
          const int at = S.group_atoms[t];
          const T m = (T)S.mass[at];
          const V3<T> d = pos.diff(at, ref);
          c[g][0] += m * d.x; c[g][1] += m * d.y; c[g][2] += m * d.z;
          mt += m;
        }
        c[g][0] /= mt; c[g][1] /= mt; c[g][2] /= mt;
      }
      const T dx = c[0][0] - c[1][0], dy = c[0][1] - c[1][1], dz = c[0][2] - c[1][2];
      return gsqrt(dx * dx + dy * dy + dz * dz);
    }
    case GRP_OBS_RMS_VELOCITY: {
      T s = 0;
      int cnt = 0;
      for (int t = S.group_off[arg[0]]; t < S.group_off[arg[0] + 1]; ++t) {
        const int at = S.group_atoms[t];
        const T im = (T)st.atom[at].w;
        for (int x = 0; x < 3; ++x) {
          const T v = (T)st.mom(3 * at + x) * im;
          s += v * v;
        }
        ++cnt;
      }
      return gsqrt(s / (T)cnt);
    }
  }
  return T(0);
}

// Bounding box of every tile of 32 atoms, [n_tiles][min xyz, max xyz], padded by 1e-3 length units
// (the boxes only decide which tile pairs to skip under a cutoff).  One warp per tile.
template <class P>
__device__ void tile_boxes(const SysDev &S, const State<P> &st, float *boxes) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int t = warp; t < S.n_tiles; t += nwarps) {
    const int a = t * 32 + lane;
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    if (a < S.n) {
      float x[3];
      st.get_f32(a, x);
      for (int c = 0; c < 3; ++c) { lo[c] = x[c]; hi[c] = x[c]; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      for (int c = 0; c < 3; ++c) {
        lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
        hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
      }
    if (lane < 6) {
      const float v = lane == 0 ? lo[0] : lane == 1 ? lo[1] : lane == 2 ? lo[2] : lane == 3 ? hi[0] : lane == 4 ? hi[1] : hi[2];
      boxes[6 * t + lane] = lane < 3 ? v - 1e-3f : v + 1e-3f;
    }
  }
}

// Verlet list of one replica (systems with a cutoff): every non-excluded pair closer than cutoff +
// skin, found by the tiled scan over tile pairs whose bounding boxes are that close (the same lane
// rotation as tile_pass, so each unordered pair is met once).  Each warp appends to chunks of
// kListChunk entries that it reserves with one shared atomic, so that a rotation step's ballot is
// written without a round trip to the shared counter; the unused tail of a warp's last chunk is filled
// with 0xFFFFFFFF, which the list's readers skip.  The positions at the build are kept for the
// displacement test.  Returns the entry count, padding included (a list longer than `cap` sets kErrList
// and is cut).  Called by every thread of the block.
constexpr int kListChunk = 256;
template <class P>
__device__ int build_list(const SysDev &S, const State<P> &st, float *boxes, uint32_t *list, int cap,
                          float4 *qref, int *cnt, int *err) {
  tile_boxes<P>(S, st, boxes);
  for (int at = threadIdx.x; at < S.n; at += blockDim.x) {
    float x[3];
    st.get_f32(at, x);
    qref[at] = make_float4(x[0], x[1], x[2], 0.f);
  }
  if (threadIdx.x == 0) *cnt = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const float lc2 = S.list_cut2;
  // periodic box: tile gaps and pair distances over nearest images (cutoff + skin is at most half the
  // shortest edge, so a pair within it has one nearest image)
  const bool per = S.coulomb_rf == 2;
  const float L[3] = {(float)S.box[0], (float)S.box[1], (float)S.box[2]};
  const float iL[3] = {(float)S.ibox[0], (float)S.ibox[1], (float)S.ibox[2]};
  int wpos = 0, wleft = 0;  // this warp's next free entry and the room left in its chunk (warp-uniform)
  for (int tp = warp; tp < S.n_tile_pairs; tp += nwarps) {
    const uint32_t e = S.tile_pairs[tp];
    const int I = (int)(e & 0xFFFFu), J = (int)(e >> 16);
    const float *ba = boxes + 6 * I, *bb = boxes + 6 * J;
    float g2 = 0.f;
    for (int x = 0; x < 3; ++x) {
      float g;
      if (per) {  // centre distance to the nearest image minus both half extents
        float dc = 0.5f * ((ba[x] + ba[x + 3]) - (bb[x] + bb[x + 3]));
        dc -= L[x] * rintf(dc * iL[x]);
        g = fmaxf(0.f, fabsf(dc) - 0.5f * ((ba[x + 3] - ba[x]) + (bb[x + 3] - bb[x])));
      } else {
        g = fmaxf(0.f, fmaxf(ba[x] - bb[x + 3], bb[x] - ba[x + 3]));
      }
      g2 += g * g;
    }
    if (g2 >= lc2) continue;
    const uint32_t mask = S.tile_masks[(size_t)tp * 32 + lane];
    const int i = I * 32 + lane;
    const bool diag = I == J;
    const int s0 = diag ? 1 : 0, s1 = diag ? 17 : 32;
    float xi[3] = {0.f, 0.f, 0.f};
    if (i < S.n) st.get_f32(i, xi);
    for (int s = s0; s < s1; ++s) {
      const int m = (lane + s) & 31;
      bool take = false;
      if (((mask >> m) & 1u) && !(diag && s == 16 && lane >= 16)) {
        float xj[3];
        st.get_f32(J * 32 + m, xj);
        float dx = xi[0] - xj[0], dy = xi[1] - xj[1], dz = xi[2] - xj[2];
        if (per) {
          dx -= L[0] * rintf(dx * iL[0]);
          dy -= L[1] * rintf(dy * iL[1]);
          dz -= L[2] * rintf(dz * iL[2]);
        }
        take = dx * dx + dy * dy + dz * dz < lc2;
      }
      const unsigned b = __ballot_sync(0xffffffffu, take);
      if (b) {
        const int nb = __popc(b);
        if (nb > wleft) {  // pad the rest of the chunk and reserve a new one
          for (int t = lane; t < wleft; t += 32)
            if (wpos + t < cap) list[wpos + t] = 0xFFFFFFFFu;
          int base = 0;
          if (lane == 0) base = atomicAdd(cnt, kListChunk);
          wpos = __shfl_sync(0xffffffffu, base, 0);
          wleft = kListChunk;
        }
        const int idx = wpos + __popc(b & ((1u << lane) - 1u));
        if (take && idx < cap) list[idx] = (uint32_t)i | ((uint32_t)(J * 32 + m) << 16);
        wpos += nb;
        wleft -= nb;
      }
    }
  }
  for (int t = lane; t < wleft; t += 32)
    if (wpos + t < cap) list[wpos + t] = 0xFFFFFFFFu;
  __syncthreads();
  int c = *cnt;
  if (c > cap) {
    *err |= kErrList;
    c = cap;
  }
  return c;
}

// Fixed-point sum (2^-40 units on the FP64 path, 2^-32 on the mixed path) to the path's precision,
// the mixed path with 32-bit conversions only.
__device__ __forceinline__ double fix_value(long long x, double) { return (double)x * kFixInv; }
__device__ __forceinline__ float fix_value(long long x, float) {
  return fmaf((float)(int)(x >> 32), 4294967296.0f, (float)(unsigned int)x) * kSplitInv;
}

// Samples of one observable within a segment, accumulated by the thread that owns the observable.
// FP64 path: straight into the FP64 accumulators.  Mixed path: on chip in double-single arithmetic
// (no FP64 instruction per sample: on GB300 each costs ~64 cycles on the critical path), folded into
// the FP64 accumulators once at the end of the segment, re-expressed relative to the stored shift:
// sum (v - c) = S1 + n d and sum (v - c)^2 = S2 + 2 d S1 + n d^2 with d = c_chip - c.
template <class P>
struct ObsAcc {
  __device__ void begin(const double *) {}
  __device__ void add(double *acc4, double v) { acc_add(acc4, v); }
  __device__ void end(double *) {}
};
template <>
struct ObsAcc<PathMixed> {
  float c;
  ds s1, s2;
  int n;
  bool have_c;
  __device__ void begin(const double *acc4) {
    have_c = acc4[3] > 0.0;
    c = have_c ? (float)acc4[0] : 0.f;
    s1 = ds{0.f, 0.f};
    s2 = ds{0.f, 0.f};
    n = 0;
  }
  __device__ void add(double *, float v) {
    if (!have_c) { c = v; have_c = true; }
    const float d = v - c;
    s1 = ds_add(s1, d);
    s2 = ds_add(s2, d * d);
    ++n;
  }
  __device__ void end(double *acc4) {
    if (n == 0) return;
    const double cs = acc4[3] == 0.0 ? (double)c : acc4[0];
    const double dd = (double)c - cs;
    const double S1 = ds_to_double(s1), S2 = ds_to_double(s2);
    acc4[0] = cs;
    acc4[1] += S1 + n * dd;
    acc4[2] += S2 + 2.0 * dd * S1 + n * dd * dd;
    acc4[3] += (double)n;
  }
};

// Whether an atom of constraint group g has moved more than skin/2 since the last Verlet-list build.
template <class P>
__device__ __forceinline__ int group_moved(const SysDev &S, const State<P> &st, int g, const float4 *qref) {
  int mv = 0;
  for (int t = S.cgroup_aoff[g]; t < S.cgroup_aoff[g + 1]; ++t) {
    const int at = S.cgroup_atoms[t];
    float x[3];
    st.get_f32(at, x);
    const float4 o = qref[at];
    const float dx = x[0] - o.x, dy = x[1] - o.y, dz = x[2] - o.z;
    mv |= dx * dx + dy * dy + dz * dz > S.half_skin2;
  }
  return mv;
}

// ------------------------------------------------------------------------------------------------
// One segment of replica r by the whole thread block (the block's shared memory holds its state).
// Force-field paths of the segment kernel, fixed at compile time so that each kernel carries only
// the code of its path (a kernel with every path inlined ran 9 % slower on the 22-bead chain).
enum : int {
  kModeAny = -1,   // decided per launch (the batched kernel, whose runs may differ)
  kModeItems = 0,  // explicit item table (fewer than 64 atoms)
  kModeTiles = 1,  // 32x32 atom tiles, no cutoff
  kModeList = 2    // Verlet lists built from the tiles (cutoff)
};

// kFF: the nonbonded model compiled into the step loop, 0 = Coulomb with eps = 4r, 1 = reaction field,
// 2 = eps = 4r plus Generalized Born solvent, 3 = eps = 4r with bond constraints, 4 = periodic box with
// particle mesh Ewald (2, 3 and 4 on the item table and the Verlet lists), 5 = solvent and constraints
// (Verlet lists), -1 = eps = 4r or reaction field
// decided per launch (the batched kernel, whose runs may differ; implicit solvent is not batched).
// The single-run kernels are compiled for one model, which keeps one copy of the force passes and no
// unused solvent code in the step loop.
template <class P, int kMode, int kFF>
__device__ __forceinline__ void segment_body(const SegArgs &a, const int r, unsigned char *smem) {
  using T = typename P::T;
  const SysDev &S = a.S;
  const int kThreads = (int)blockDim.x;
  const int n = S.n, nd = 3 * n, no = S.n_obs, NB = a.noise_batch;
  unsigned char *ptr = smem;
  long long *F = (long long *)ptr; ptr += (size_t)nd * 8;
  long long *red = (long long *)ptr; ptr += 64 * 8;
  double *acc = (double *)ptr; ptr += kMaxObs * 4 * 8;
  long long *ek = (long long *)ptr; ptr += 2 * 8;
  int *lcount = (int *)ptr; ptr += 8;
  State<P> st;
  ptr = align32(ptr);
  st.carve(ptr, n, S, a.lean != 0);
  ptr = align32(ptr);
  T *xi = (T *)ptr; ptr += (size_t)NB * nd * sizeof(T);  // NB = 0: noise drawn inline per atom
  float *boxes = nullptr;  // tile bounding boxes, only with tiles and a cutoff
  if (S.tiled && S.cutoff2 > 0) { boxes = (float *)ptr; ptr += (size_t)S.n_tiles * 6 * 4; }
  // kFF = 5 (Verlet lists only): solvent and bond constraints together, the paper's protein-ligand setup
  constexpr bool kGB = kMode == kModeItems && kFF == 2;
  constexpr bool kGBL = kMode == kModeList && (kFF == 2 || kFF == 5);  // solvent with a cutoff on the list
  constexpr bool kCon = (kMode == kModeItems && kFF == 3) || (kMode == kModeList && (kFF == 3 || kFF == 5));
  constexpr bool kPME = (kMode == kModeItems || kMode == kModeList) && kFF == 4;
  constexpr int kRF = kFF == 4 ? 2 : (kFF >= 2 ? 0 : kFF);
  GbScratch<P> gbs;  // implicit solvent (item-table systems only)
  if constexpr (kGB) {
    ptr = align32(ptr);
    gbs.carve(ptr, n);
    for (int i = threadIdx.x; i < 2 * n; i += kThreads) gbs.acc.zero(i);
  }
  ScalarAcc<P> gbl_acc;  // solvent with a cutoff: one accumulator per atom; radii and weights in global memory
  T *gbl_born = nullptr, *gbl_w = nullptr, *gbl_gr = nullptr;
  if constexpr (kGBL) {
    ptr = align32(ptr);
    gbl_acc.carve(ptr, n);
    for (int i = threadIdx.x; i < n; i += kThreads) gbl_acc.zero(i);
    gbl_born = reinterpret_cast<T *>(a.gb_glob + (size_t)r * 2 * n);
    gbl_w = gbl_born + n;
    if (a.gb_gr) gbl_gr = reinterpret_cast<T *>(a.gb_gr) + (size_t)r * a.gb_gr_stride;
  }
  PmeScratch<P> pms;  // particle mesh (periodic systems: item table or Verlet lists)
  if constexpr (kPME) {
    ptr = align32(ptr);
    pms.carve(ptr, S);
    pms.zero(S);
  }
  PairDsConst *kds = nullptr;  // the mixed path's single-bond constraint groups: constants per group
  if constexpr (kCon && P::kMixed) {
    ptr = align32(ptr);
    kds = (PairDsConst *)ptr;
    ptr += (size_t)S.n_cgroups * sizeof(PairDsConst);
    for (int g = threadIdx.x; g < S.n_cgroups; g += kThreads)
      if (S.cgroup_off[g + 1] - S.cgroup_off[g] == 1) pair_ds_const(S, g, a.h, a.c1, kds[g]);
  }

  const uint32_t *pairs = S.pairs, *items = S.items;
  if (a.pairs_in_smem) {
    ptr = align32(ptr);
    uint32_t *sp = (uint32_t *)ptr;
    for (int i = threadIdx.x; i < S.n_pairs; i += kThreads) sp[i] = S.pairs[i];
    pairs = sp;
    uint32_t *si = sp + S.n_pairs;
    for (int i = threadIdx.x; i < S.n_items; i += kThreads) si[i] = S.items[i];
    items = si;
  }
  const size_t off = (size_t)r * nd;
  st.load(S, a.q + off, a.p + off, a.f + off, n, a.c1);
  for (int i = threadIdx.x; i < nd; i += kThreads) F[i] = 0;
  if (threadIdx.x < no * 4) acc[threadIdx.x] = a.acc[(size_t)r * no * 4 + threadIdx.x];
  __syncthreads();
  ObsAcc<P> oacc;
  if (threadIdx.x < no) oacc.begin(acc + 4 * threadIdx.x);
  const bool use_list = kMode == kModeList || (kMode == kModeAny && a.nbl != nullptr);
  const bool tiled = kMode == kModeTiles || kMode == kModeList || (kMode == kModeAny && S.tiled);
  const bool lean = kMode != kModeItems && a.lean;
  uint32_t *list = use_list ? a.nbl + (size_t)r * a.nbl_cap : nullptr;
  float4 *qref = use_list ? a.qref + (size_t)r * n : nullptr;
  int n_list = 0;

  int err = 0;
  if (use_list) n_list = build_list<P>(S, st, boxes, list, a.nbl_cap, qref, lcount, &err);
  const T h = (T)a.h, c1 = (T)a.c1;
  const Pos<P> pos = st.pos();
  const Params<P> par = st.params(S);
  const typename P::Acc fa = State<P>::acc(F, n);
  // steps until the next sample: (t_phase0 + s + 1) % t_gr == 0
  int until = a.t_gr > 0 ? (int)(a.t_gr - a.t_phase0 % a.t_gr) : 0x7fffffff;
  int j = 0;  // step index inside the current noise batch
  for (int s = 0; s < a.k; ++s, ++j) {
    int moved = 0;
    if (kMode == kModeItems || NB > 0) {
      if (j == NB) j = 0;
      if (j == 0) {
        gen_noise<T>(xi, min(NB, a.k - s), a.t_global0 + s, a.seed, r + a.rep0, n);
        __syncthreads();
      }
      // one thread per coordinate; with a Verlet list, an atom is taken to have moved more than skin/2
      // when one of its coordinates moved more than skin / (2 sqrt 3) (a sufficient test)
      const T *xs = xi + (size_t)j * nd;
      for (int i = threadIdx.x; i < nd; i += kThreads) {
        if constexpr (kCon) {
          if (S.con_atom[i / 3]) continue;  // integrated with its constraint group below
        }
        st.baoa_c(i, xs[i], h, c1);
        if (use_list) {
          const float d = (float)st.coord(i) - (&qref[i / 3].x)[i % 3];
          moved |= 3.f * d * d > S.half_skin2;
        }
      }
      if constexpr (kCon)
        for (int g = threadIdx.x; g < S.n_cgroups; g += kThreads) {
          con_baoa<P>(S, st, g, [&](int at, T z3[3]) { z3[0] = xs[3 * at]; z3[1] = xs[3 * at + 1]; z3[2] = xs[3 * at + 2]; },
                      a.h, a.c1, &err, kds);
          if (use_list) moved |= group_moved(S, st, g, qref);
        }
    } else {
      if constexpr (kCon)  // constrained atoms: their groups, with the noise drawn from the same stream
        for (int g = threadIdx.x; g < S.n_cgroups; g += kThreads) {
          con_baoa<P>(S, st, g, [&](int at, T z3[3]) {
            T z[4];
            normals4(philox_stream(a.seed, a.t_global0 + s, 0u, r + a.rep0, at), z);
            z3[0] = z[0]; z3[1] = z[1]; z3[2] = z[2];
          }, a.h, a.c1, &err, kds);
          if (use_list) moved |= group_moved(S, st, g, qref);
        }
      for (int at = threadIdx.x; at < n; at += kThreads) {
        if constexpr (kCon) {
          if (S.con_atom[at]) continue;
        }
        T z[4];
        normals4(philox_stream(a.seed, a.t_global0 + s, 0u, r + a.rep0, at), z);
        st.baoa(at, z, h, c1);
        if (use_list) {  // Verlet list: rebuilt when some atom has moved more than skin/2
          float x[3];
          st.get_f32(at, x);
          const float4 o = qref[at];
          const float dx = x[0] - o.x, dy = x[1] - o.y, dz = x[2] - o.z;
          moved |= dx * dx + dy * dy + dz * dz > S.half_skin2;
        }
      }
    }
    if (use_list) {
      if (__syncthreads_or(moved)) n_list = build_list<P>(S, st, boxes, list, a.nbl_cap, qref, lcount, &err);
    } else {
      __syncthreads();
    }
    if (tiled && !use_list && boxes) {
      tile_boxes<P>(S, st, boxes);
      __syncthreads();
    }
    const bool sample = --until == 0;
    if (sample) until = a.t_gr;
    long long e_fix = 0;
    if constexpr (kGB) gb_forces<P>(S, pos, fa, gbs, sample, e_fix, &err);
    if constexpr (kGBL) {
      const int nl = n_list;
      // batches of kGbBatch entries per thread (list entries t, t + kThreads, ...), padding entries and
      // the tail as empty slots
      // the slot of a pair in the gr3 row: its list position, or nbl_cap + its index among the excluded pairs
      gb_forces_cut<P>(S, pos, fa, gbl_acc, gbl_born, gbl_w, gbl_gr, [&](auto f) {
        auto batches = [&](const uint32_t *src, int cnt, int slot0) {
          for (int t = threadIdx.x; t < cnt; t += kGbBatch * kThreads) {
            int I[kGbBatch], J[kGbBatch], K[kGbBatch];
#pragma unroll
            for (int u = 0; u < kGbBatch; ++u) {
              const uint32_t pk = t + u * kThreads < cnt ? src[t + u * kThreads] : 0xFFFFFFFFu;
              I[u] = pk == 0xFFFFFFFFu ? -1 : (int)(pk & 0xFFFFu);
              J[u] = (int)(pk >> 16);
              K[u] = (gbl_gr && I[u] >= 0) ? slot0 + t + u * kThreads : -1;  // empty slots and the tail: none
            }
            f(I, J, K);
          }
        };
        batches(list, nl, 0);
        batches(S.gb_xpairs, S.n_gb_xpairs, a.nbl_cap);
      }, sample, e_fix, &err);
    }
    if constexpr (kPME) pme_forces<P>(S, pos, par, fa, pms, sample, e_fix, &err);
    auto passes = [&](auto rf) {
      constexpr int R = decltype(rf)::value;
      if (lean) bonded_pass<P>(S, pos, par, fa, sample, e_fix, &err);
      else force_pass<P, R>(S, pos, par, items, pairs, fa, sample, e_fix, &err);
      if (use_list) list_pass<P, R>(S, pos, par, list, n_list, fa, sample, e_fix, &err);
      else if (tiled) tile_pass<P, false, R>(S, pos, par, fa, boxes, sample, e_fix, &err);  // tiles: no cutoff
    };
    if constexpr (kRF >= 0) {
      passes(std::integral_constant<int, kRF>{});
    } else if (par.rf) {
      passes(std::integral_constant<int, 1>{});
    } else {
      passes(std::integral_constant<int, 0>{});
    }
    __syncthreads();
    long long k_fix = 0;
    if (kMode == kModeItems || NB > 0) {
      for (int i = threadIdx.x; i < nd; i += kThreads) {
        if constexpr (kCon) {
          if (S.con_atom[i / 3]) continue;
        }
        const T ke = st.bk_c(i, fa, h);
        if (sample) k_fix += fa.efix(ke, &err);
      }
      if constexpr (kCon)
        for (int g = threadIdx.x; g < S.n_cgroups; g += kThreads) {
          const double ke = con_b<P>(S, st, fa, g, a.h, &err, kds);
          if (sample) k_fix += fa.efix((T)ke, &err);
        }
    } else {  // the same thread owns each atom in both halves of the step
      for (int at = threadIdx.x; at < n; at += kThreads) {
        if constexpr (kCon) {
          if (S.con_atom[at]) continue;
        }
        const T ke = st.bk(at, fa, h);
        if (sample) k_fix += fa.efix(ke, &err);
      }
      if constexpr (kCon)
        for (int g = threadIdx.x; g < S.n_cgroups; g += kThreads) {
          const double ke = con_b<P>(S, st, fa, g, a.h, &err, kds);
          if (sample) k_fix += fa.efix((T)ke, &err);
        }
    }
    if (sample) {
      block_sum2_ll(e_fix, k_fix, red);
      if (threadIdx.x == 0) { ek[0] = e_fix; ek[1] = k_fix; }
      __syncthreads();
      if (threadIdx.x < no)
        oacc.add(acc + 4 * threadIdx.x,
                 observable_ff<P>(S, st, threadIdx.x, fix_value(ek[0], T(0)), fix_value(ek[1], T(0))));
      __syncthreads();
    }
  }
  if (threadIdx.x < no) oacc.end(acc + 4 * threadIdx.x);
  __syncthreads();  // the write-back reads coordinates owned by other threads
  st.store(a.q + off, a.p + off, a.f + off, n, &err);
  if (threadIdx.x < no * 4) a.acc[(size_t)r * no * 4 + threadIdx.x] = acc[threadIdx.x];
  if (a.do_check && threadIdx.x == 0) {
    int ex;
    const int label = state_check_f64(S, [&](int at, double x[3]) { st.get_f64(at, x); }, a.omega, &ex);
    record_check(a, r, label, ex);
  }
  if (err) atomicOr(a.err, err);
}

// kMaxThreads/kMinBlocks: blocks of up to 320 threads keep two resident per SM (256 replica blocks
// on 152 SMs then run in one wave); larger systems use up to 512 threads, one block per SM.
template <class P, int kMaxThreads, int kMinBlocks, int kMode, int kFF>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocks) ff_segment_kernel(const SegArgs a) {
  if (a.skip_if_exit && exit_seen_before(a)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  segment_body<P, kMode, kFF>(a, blockIdx.x, smem);
}

// Batched segments: a persistent grid of blocks takes (run, replica) units from a queue sorted by
// decreasing system size, so that the largest replicas start first and the small ones fill in.
// Each unit's launch arguments are copied into shared memory before its segment runs.
template <class P>
// (Launch bounds (512, 1), up to 128 registers: measured on the batched chains against (256, 3), (256, 4)
// and (384, 2), which trade registers for resident blocks, 12.7 vs 11.4-11.6 TFLOP/s.)
__global__ void __launch_bounds__(512, 1) ff_segment_batch_kernel(const SegArgs *runs, const uint2 *units,
                                                                  int n_units, int *counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SegArgs sa;
  __shared__ int su;
  for (;;) {
    if (threadIdx.x == 0) {
      // units of replicas beyond a run's n_active (a transient advances replica 0 alone, a finished
      // run none) and of runs whose parallel step saw an exit at an earlier check are passed over
      int u = atomicAdd(counter, 1);
      while (u < n_units) {
        const uint2 un = units[u];
        const SegArgs &g = runs[un.x];
        if ((int)un.y < g.n_active && !(g.skip_if_exit && exit_seen_before(g))) break;
        u = atomicAdd(counter, 1);
      }
      su = u;
    }
    __syncthreads();
    const int u = su;
    if (u >= n_units) break;
    const uint2 un = units[u];
    const int *src = reinterpret_cast<const int *>(runs + un.x);
    int *dst = reinterpret_cast<int *>(&sa);
    for (int i = threadIdx.x; i < (int)(sizeof(SegArgs) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    segment_body<P, kModeAny, -1>(sa, (int)un.y, smem);
    __syncthreads();
  }
}

// Analytic 2-D double well: one thread per replica, FP64 (dim = 2, one particle).
__global__ void __launch_bounds__(64) dw_segment_kernel(const SegArgs a) {
  const SysDev &S = a.S;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.n_active) return;
  if (a.skip_if_exit && exit_seen_before(a)) return;
  double x = a.q[2 * r], y = a.q[2 * r + 1], px = a.p[2 * r], py = a.p[2 * r + 1];
  double fx = a.f[2 * r], fy = a.f[2 * r + 1];
  const int no = S.n_obs;
  double acc[kMaxObs][4];
  for (int j = 0; j < no; ++j)
    for (int c = 0; c < 4; ++c) acc[j][c] = a.acc[((size_t)r * no + j) * 4 + c];
  const double h = a.h, c1 = a.c1, im = 1.0 / S.mass[0];
  const double sd = sqrt((1.0 - c1 * c1) * S.kT * S.mass[0]);
  int until = a.t_gr > 0 ? (int)(a.t_gr - a.t_phase0 % a.t_gr) : 0x7fffffff;
  for (int s = 0; s < a.k; ++s) {
    double xi[4];
    normals4_f64(philox_stream(a.seed, a.t_global0 + s, 0u, r + a.rep0, 0), xi);
    px += h * fx; py += h * fy;
    x += h * px * im; y += h * py * im;
    px = c1 * px + sd * xi[0]; py = c1 * py + sd * xi[1];
    x += h * px * im; y += h * py * im;
    fx = -S.dw_a * 4.0 * x * (x * x - 1.0);
    fy = -S.dw_b * 2.0 * y;
    px += h * fx; py += h * fy;
    if (--until == 0) {
      until = a.t_gr;
      for (int j = 0; j < no; ++j) {
        double v;
        const int kind = S.obs_kind[j];
        if (kind == GRP_OBS_COORD) v = S.obs_arg[j][1] == 0 ? x : y;
        else if (kind == GRP_OBS_POTENTIAL) v = S.dw_a * (x * x - 1.0) * (x * x - 1.0) + S.dw_b * y * y;
        else v = 0.5 * (px * px + py * py) * im;
        acc_add(acc[j], v);
      }
    }
  }
  a.q[2 * r] = x; a.q[2 * r + 1] = y; a.p[2 * r] = px; a.p[2 * r + 1] = py;
  a.f[2 * r] = fx; a.f[2 * r + 1] = fy;
  for (int j = 0; j < no; ++j)
    for (int c = 0; c < 4; ++c) a.acc[((size_t)r * no + j) * 4 + c] = acc[j][c];
  if (!isfinite(x) || !isfinite(y) || !isfinite(px) || !isfinite(py)) atomicOr(a.err, (int)kErrNaN);
  if (a.do_check) {
    int ex;
    const int label = state_check_f64(S, [&](int, double v[3]) { v[0] = x; v[1] = y; v[2] = 0; }, a.omega, &ex);
    record_check(a, r, label, ex);
  }
}

// Noise amplitudes of every atom (the tables that lean replica states read), with the arithmetic of
// the states that keep them in shared memory, so that both give the same bits.
__global__ void noise_sd_kernel(int n, double c1, double kT, const double *mass, double *sd_d, float *sd_f) {
  const int at = blockIdx.x * blockDim.x + threadIdx.x;
  if (at >= n) return;
  const double v = noise_scale(c1, kT, mass[at]);
  sd_d[at] = v;
  sd_f[at] = (float)v;
}

cudaError_t launch_noise_sd(const SysDev &S, double c1, double *sd_d, float *sd_f, cudaStream_t st) {
  if (S.n <= 0) return cudaSuccess;
  noise_sd_kernel<<<(S.n + 127) / 128, 128, 0, st>>>(S.n, c1, S.kT, S.mass, sd_d, sd_f);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
static size_t ff_smem_bytes(const SysDev &S, int pairs_in_smem, int noise_batch, int lean) {
  const int n = S.n;
  const size_t real = S.precision == GRP_FP64 ? 8 : 4;
  size_t b = (size_t)3 * n * 8 + 64 * 8 + kMaxObs * 4 * 8 + 16 + 8 + 96;  // + alignment padding
  b += S.precision == GRP_FP64 ? State<PathF64>::bytes(n, lean) : State<PathMixed>::bytes(n, lean);
  b += (size_t)noise_batch * 3 * n * real;
  if (S.tiled && S.cutoff2 > 0) b += (size_t)S.n_tiles * 6 * 4;
  if (pairs_in_smem) b += (size_t)(S.n_pairs + S.n_items) * 4 + 32;
  if (S.gb && S.use_list) b += 32 + ScalarAcc<PathF64>::bytes(n);  // one 8-byte accumulator per atom
  else if (S.gb) b += 32 + (S.precision == GRP_FP64 ? GbScratch<PathF64>::bytes(n) : GbScratch<PathMixed>::bytes(n));
  if (S.coulomb_rf == 2)
    b += 32 + (S.precision == GRP_FP64 ? PmeScratch<PathF64>::bytes(S) : PmeScratch<PathMixed>::bytes(S));
  if (S.n_cons > 0 && S.precision != GRP_FP64) b += 32 + (size_t)S.n_cgroups * sizeof(PairDsConst);
  return b;
}

SegConfig segment_config(const SysDev &S, int threads_hint) {
  SegConfig c{};
  if (S.potential == GRP_POT_DOUBLE_WELL_2D) {
    c.threads = 64;
    c.smem = 0;
    c.noise_batch = 1;
    return c;
  }
  // one thread per (padded) item, or one warp per tile pair, up to 512 threads per replica, a
  // multiple of 32, at least 64
  int t = threads_hint;
  if (t <= 0) {
    t = ((S.n_items + 31) / 32) * 32;
    if (S.tiled && 32 * S.n_tile_pairs > t) t = 32 * S.n_tile_pairs;
  }
  t = t < 64 ? 64 : (t > 512 ? 512 : ((t + 31) / 32) * 32);
  // the mixed path's particle mesh and constraints: 320 threads, two replicas per SM (the mesh's 256
  // lines per transform pass take one round of the block; the constraint groups run on one warp, and
  // two blocks per SM run two such warps at once and 256 replicas in one wave); the FP64 transforms and
  // groups need the registers of the 512-thread variant
  if ((S.coulomb_rf == 2 || S.n_cons > 0) && S.precision != GRP_FP64 && threads_hint <= 0 && t > 320 && !S.tiled)
    t = 320;
  c.threads = t;
  // noise for up to 64 steps at a time (one barrier per batch), within 32 KB; beyond 16 steps only where
  // the block keeps to half an SM's shared memory, so that a larger batch costs no occupancy (the
  // counter-based noise is the same whatever the batch)
  const size_t real = S.precision == GRP_FP64 ? 8 : 4;
  int nb = 64;
  while (nb > 1 && (size_t)nb * 3 * S.n * real > 32 * 1024) nb /= 2;
  while (nb > 16 && ff_smem_bytes(S, 1, nb, 0) > 113 * 1024) nb /= 2;
  c.noise_batch = nb;
  c.lean = 0;
  // large systems: atom parameters read from the global table and noise drawn inline, so that the
  // replica state alone fills the shared memory
  if (ff_smem_bytes(S, 0, nb, 0) > kMaxSmem) {
    c.lean = 1;
    c.noise_batch = nb = 0;
  }
  c.pairs_in_smem = ff_smem_bytes(S, 1, nb, c.lean) <= 160 * 1024 ? 1 : 0;
  c.smem = ff_smem_bytes(S, c.pairs_in_smem, nb, c.lean);
  return c;
}

template <class P>
static cudaError_t launch_ff_p(const SegArgs &a, const SegConfig &c, cudaStream_t st) {
  if (c.threads < 32 || c.threads > 512 || c.threads % 32) return cudaErrorInvalidValue;
  const int mode = a.S.use_list ? kModeList : (a.S.tiled ? kModeTiles : kModeItems);
  const bool small = c.threads <= 320;
  // tiles are taken only without a cutoff, so never with the reaction field; implicit solvent only on
  // the item table (and never with a cutoff)
  const bool rf = a.S.coulomb_rf == 1, gb = a.S.gb != 0, con = a.S.n_cons > 0, pme = a.S.coulomb_rf == 2;
  auto kern = mode == kModeItems
                  ? (pme  ? (small ? ff_segment_kernel<P, 320, 2, kModeItems, 4> : ff_segment_kernel<P, 512, 1, kModeItems, 4>)
                     : con ? (small ? ff_segment_kernel<P, 320, 2, kModeItems, 3> : ff_segment_kernel<P, 512, 1, kModeItems, 3>)
                     : gb ? (small ? ff_segment_kernel<P, 320, 2, kModeItems, 2> : ff_segment_kernel<P, 512, 1, kModeItems, 2>)
                     : rf ? (small ? ff_segment_kernel<P, 320, 2, kModeItems, 1> : ff_segment_kernel<P, 512, 1, kModeItems, 1>)
                          : (small ? ff_segment_kernel<P, 320, 2, kModeItems, 0> : ff_segment_kernel<P, 512, 1, kModeItems, 0>))
            : mode == kModeTiles
                  ? (small ? ff_segment_kernel<P, 320, 2, kModeTiles, 0> : ff_segment_kernel<P, 512, 1, kModeTiles, 0>)
                  : pme ? ff_segment_kernel<P, 512, 1, kModeList, 4>  // periodic (the mesh's registers)
                  : (rf ? (small ? ff_segment_kernel<P, 320, 2, kModeList, 1> : ff_segment_kernel<P, 512, 1, kModeList, 1>)
                     : (gb && con) ? (small ? ff_segment_kernel<P, 320, 2, kModeList, 5> : ff_segment_kernel<P, 512, 1, kModeList, 5>)
                     : gb ? (small ? ff_segment_kernel<P, 320, 2, kModeList, 2> : ff_segment_kernel<P, 512, 1, kModeList, 2>)
                     : con ? (small ? ff_segment_kernel<P, 320, 2, kModeList, 3> : ff_segment_kernel<P, 512, 1, kModeList, 3>)
                          : (small ? ff_segment_kernel<P, 320, 2, kModeList, 0> : ff_segment_kernel<P, 512, 1, kModeList, 0>));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
  if (e != cudaSuccess) return e;
  kern<<<a.n_active, c.threads, c.smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_segment_batch(const SegArgs *d_runs, const uint2 *d_units, int n_units, int *d_counter,
                                 int precision, int threads, size_t smem, cudaStream_t st, int *blocks_used) {
  if (n_units <= 0) return cudaSuccess;
  if (threads < 32 || threads > 512 || threads % 32) return cudaErrorInvalidValue;
  auto kern = precision == GRP_FP64 ? ff_segment_batch_kernel<PathF64> : ff_segment_batch_kernel<PathMixed>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int blocks = sms * per_sm;
  if (blocks > n_units) blocks = n_units;
  if ((e = cudaMemsetAsync(d_counter, 0, sizeof(int), st)) != cudaSuccess) return e;
  kern<<<blocks, threads, smem, st>>>(d_runs, d_units, n_units, d_counter);
  if (blocks_used) *blocks_used = blocks;
  return cudaGetLastError();
}

cudaError_t launch_segment(const SegArgs &a0, const SegConfig &c, cudaStream_t st) {
  SegArgs a = a0;
  a.pairs_in_smem = c.pairs_in_smem;
  a.noise_batch = c.noise_batch;
  a.lean = c.lean;
  if (a.n_active <= 0) return cudaSuccess;
  if (a.S.potential == GRP_POT_DOUBLE_WELL_2D) {
    dw_segment_kernel<<<(a.n_active + 63) / 64, 64, 0, st>>>(a);
    return cudaGetLastError();
  }
  return a.S.precision == GRP_FP64 ? launch_ff_p<PathF64>(a, c, st) : launch_ff_p<PathMixed>(a, c, st);
}

// ------------------------------------------------------------------------------------------------
// Energies and forces of independent configurations (one block per configuration).
template <class P>
__global__ void __launch_bounds__(256) energy_forces_kernel(SysDev S, const double *q, double *energy,
                                                            double *forces, int *errp, int lean, double *gb_glob) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = S.n, nd = 3 * n, b = blockIdx.x;
  unsigned char *ptr = smem;
  long long *F = (long long *)ptr; ptr += (size_t)nd * 8;
  long long *red = (long long *)ptr; ptr += 32 * 8;
  State<P> st;
  ptr = align32(ptr);
  st.carve(ptr, n, S, lean != 0);
  GbScratch<P> gbs;
  ScalarAcc<P> gbl_acc;  // solvent with a cutoff: radii and weights in global memory (gb_glob [conf][2n])
  if (S.gb && S.use_list) {
    ptr = align32(ptr);
    gbl_acc.carve(ptr, n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) gbl_acc.zero(i);
  } else if (S.gb) {
    ptr = align32(ptr);
    gbs.carve(ptr, n);
    for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) gbs.acc.zero(i);
  }
  PmeScratch<P> pms;
  if (S.coulomb_rf == 2) {
    ptr = align32(ptr);
    pms.carve(ptr, S);
    pms.zero(S);
  }
  // positions only: momenta and forces are not used
  for (int at = threadIdx.x; at < n; at += blockDim.x) {
    if constexpr (P::kMixed) {
      const ds x = ds_from_double(q[(size_t)b * nd + 3 * at]), y = ds_from_double(q[(size_t)b * nd + 3 * at + 1]),
               z = ds_from_double(q[(size_t)b * nd + 3 * at + 2]);
      const float4 pa = S.atom_f[at];
      st.qh[at] = make_float4(x.hi, y.hi, z.hi, pa.x);  // as State<PathMixed>::load
      st.ql[at] = make_float4(x.lo, y.lo, z.lo, pa.y);
      if (!lean) const_cast<float4 *>(st.atom)[at] = pa;
    } else {
      for (int x = 0; x < 3; ++x) st.q[3 * at + x] = q[(size_t)b * nd + 3 * at + x];
      if (!lean) const_cast<double4 *>(st.atom)[at] = S.atom_d[at];
    }
  }
  for (int i = threadIdx.x; i < nd; i += blockDim.x) F[i] = 0;
  __syncthreads();
  int err = 0;
  long long e_fix = 0;
  const typename P::Acc fa = State<P>::acc(F, n);
  if (S.gb && S.use_list) {
    // every pair i < j, the cutoff applied inside: rows i, i + blockDim.x, ... per thread
    using T = typename P::T;
    T *born = reinterpret_cast<T *>(gb_glob + (size_t)b * 2 * n);
    gb_forces_cut<P>(S, st.pos(), fa, gbl_acc, born, born + n, nullptr, [&](auto f) {
      for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int j = i + 1; j < n; j += kGbBatch) {
          int I[kGbBatch], J[kGbBatch], K[kGbBatch];
#pragma unroll
          for (int u = 0; u < kGbBatch; ++u) {
            I[u] = j + u < n ? i : -1;
            J[u] = j + u;
            K[u] = -1;
          }
          f(I, J, K);
        }
    }, energy != nullptr, e_fix, &err);
    __syncthreads();
  } else if (S.gb) {
    gb_forces<P>(S, st.pos(), fa, gbs, energy != nullptr, e_fix, &err);
  }
  if (S.coulomb_rf == 2) pme_forces<P>(S, st.pos(), st.params(S), fa, pms, energy != nullptr, e_fix, &err);
  force_pass<P>(S, st.pos(), st.params(S), S.items, S.pairs, fa, energy != nullptr, e_fix, &err);
  if (S.tiled) tile_pass<P>(S, st.pos(), st.params(S), fa, nullptr, energy != nullptr, e_fix, &err);
  __syncthreads();
  if (forces) {
    for (int i = threadIdx.x; i < nd; i += blockDim.x) {
      long long v;
      if constexpr (P::kMixed) v = (long long)fa.hi[i] * (1ll << 20) + (long long)fa.lo[i];
      else v = F[i];
      forces[(size_t)b * nd + i] = (double)v * P::Acc::kInv;
    }
  }
  const long long es = block_sum_ll(e_fix, red);
  if (energy && threadIdx.x == 0) energy[b] = (double)es * P::Acc::kInv;
  if (err) atomicOr(errp, err);
}

__global__ void dw_energy_forces_kernel(SysDev S, int nc, const double *q, double *energy, double *forces) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nc) return;
  const double x = q[2 * b], y = q[2 * b + 1];
  if (energy) energy[b] = S.dw_a * (x * x - 1.0) * (x * x - 1.0) + S.dw_b * y * y;
  if (forces) {
    forces[2 * b] = -S.dw_a * 4.0 * x * (x * x - 1.0);
    forces[2 * b + 1] = -S.dw_b * 2.0 * y;
  }
}

cudaError_t launch_energy_forces(const SysDev &S, int n_conf, const double *q, double *energy,
                                 double *forces, int *err, cudaStream_t st) {
  if (n_conf <= 0) return cudaSuccess;
  if (S.potential == GRP_POT_DOUBLE_WELL_2D) {
    dw_energy_forces_kernel<<<(n_conf + 127) / 128, 128, 0, st>>>(S, n_conf, q, energy, forces);
    return cudaGetLastError();
  }
  auto bytes = [&](bool lean) {
    size_t b = (size_t)3 * S.n * 8 + 32 * 8 + 32 +
               (S.precision == GRP_FP64 ? State<PathF64>::bytes(S.n, lean) : State<PathMixed>::bytes(S.n, lean));
    if (S.gb && S.use_list) b += 32 + ScalarAcc<PathF64>::bytes(S.n);
    else if (S.gb) b += 32 + (S.precision == GRP_FP64 ? GbScratch<PathF64>::bytes(S.n) : GbScratch<PathMixed>::bytes(S.n));
    if (S.coulomb_rf == 2)
      b += 32 + (S.precision == GRP_FP64 ? PmeScratch<PathF64>::bytes(S) : PmeScratch<PathMixed>::bytes(S));
    return b;
  };
  const int lean = bytes(false) > kMaxSmem ? 1 : 0;
  const size_t smem = bytes(lean);
  if (smem > kMaxSmem) return cudaErrorInvalidValue;
  cudaError_t e;
  double *gb_glob = nullptr;  // Born radii and weights of every configuration (solvent with a cutoff)
  if (S.gb && S.use_list) {
    e = cudaMallocAsync((void **)&gb_glob, (size_t)n_conf * 2 * S.n * sizeof(double), st);
    if (e != cudaSuccess) return e;
  }
  if (S.precision == GRP_FP64) {
    e = cudaFuncSetAttribute(energy_forces_kernel<PathF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) energy_forces_kernel<PathF64><<<n_conf, 256, smem, st>>>(S, q, energy, forces, err, lean, gb_glob);
  } else {
    e = cudaFuncSetAttribute(energy_forces_kernel<PathMixed>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) energy_forces_kernel<PathMixed><<<n_conf, 256, smem, st>>>(S, q, energy, forces, err, lean, gb_glob);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (gb_glob) {
    const cudaError_t e2 = cudaFreeAsync(gb_glob, st);
    if (e == cudaSuccess) e = e2;
  }
  return e;
}

// ------------------------------------------------------------------------------------------------
// Stand-alone state check (Section 3.3) from the FP64 state in memory, one thread per replica.
__global__ void check_kernel(SysDev S, const double *q, int n_rep, int omega, int8_t *labels, uint8_t *exited,
                             unsigned long long *exit_key, long long M) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rep) return;
  const double *qr = q + (size_t)r * S.nd;
  const int dim = S.dim;
  int ex;
  const int label = state_check_f64(
      S, [&](int at, double x[3]) { x[0] = qr[dim * at]; x[1] = qr[dim * at + 1]; x[2] = dim == 3 ? qr[dim * at + 2] : 0.0; },
      omega, &ex);
  if (labels) labels[r] = (int8_t)label;
  if (exited) exited[r] = (uint8_t)ex;
  if (ex && exit_key) atomicMin(exit_key, ((unsigned long long)M << 32) | (unsigned long long)(unsigned)r);
}

cudaError_t launch_check(const SysDev &S, const double *q, int n_rep, int omega, int8_t *labels,
                         uint8_t *exited, unsigned long long *exit_key, long long M, cudaStream_t st) {
  check_kernel<<<(n_rep + 127) / 128, 128, 0, st>>>(S, q, n_rep, omega, labels, exited, exit_key, M);
  return cudaGetLastError();
}

}  // namespace grp

// Bond constraints in the BAOAB step (the paper's MD setups hold the bonds of hydrogens fixed,
// Section 4): every sub-step of the unconstrained step is followed by its projection -- positions by
// SHAKE along the bond vectors before the A step, momenta by RATTLE onto the tangent space (no relative
// velocity along any bond).  The constraints form independent groups (connected components); one thread
// integrates a whole group in FP64 (the mixed path's single-bond groups in double-single, below), with
// Gauss-Seidel sweeps over the group's
// constraints in their order until a sweep moves nothing beyond the tolerance, so that the result is
// that of sweeping over every constraint of the system.  Item-table systems only.
#pragma once
#include "state.cuh"

namespace grp {

constexpr int kMaxGroupAtoms = 16;
constexpr int kMaxGroupCons = 16;

// One group in registers and local memory, positions, momenta, forces in FP64.
struct ConGroup {
  int na, nc;
  int atom[kMaxGroupAtoms];
  int ci[kMaxGroupCons], cj[kMaxGroupCons];  // local atom indices of each constraint
  double d[kMaxGroupCons];
  double w[kMaxGroupAtoms];                  // 1 / m
  double q[kMaxGroupAtoms][3], p[kMaxGroupAtoms][3];
};

// FP64 views of a replica's shared-memory state, per coordinate i = 3 atom + axis.
__device__ __forceinline__ double st_q(const State<PathF64> &st, int i) { return st.q[i]; }
__device__ __forceinline__ double st_p(const State<PathF64> &st, int i) { return st.p[i]; }
__device__ __forceinline__ double st_f(const State<PathF64> &st, int i) { return st.f[i]; }
__device__ __forceinline__ void st_set_q(State<PathF64> &st, int i, double v) { st.q[i] = v; }
__device__ __forceinline__ void st_set_p(State<PathF64> &st, int i, double v) { st.p[i] = v; }
__device__ __forceinline__ double st_q(const State<PathMixed> &st, int i) {
  return (double)(&st.qh[i / 3].x)[i % 3] + (double)(&st.ql[i / 3].x)[i % 3];
}
__device__ __forceinline__ double st_p(const State<PathMixed> &st, int i) {
  return (double)st.ph[i] + (double)st.pl[i];
}
__device__ __forceinline__ double st_f(const State<PathMixed> &st, int i) { return (double)st.f[i]; }
__device__ __forceinline__ void st_set_q(State<PathMixed> &st, int i, double v) {
  const ds x = ds_from_double(v);
  (&st.qh[i / 3].x)[i % 3] = x.hi;
  (&st.ql[i / 3].x)[i % 3] = x.lo;
}
__device__ __forceinline__ void st_set_p(State<PathMixed> &st, int i, double v) {
  const ds x = ds_from_double(v);
  st.ph[i] = x.hi;
  st.pl[i] = x.lo;
}

__device__ __forceinline__ int local_atom(const ConGroup &G, int a) {
  for (int u = 0; u < G.na; ++u)
    if (G.atom[u] == a) return u;
  return 0;  // unreachable: the group lists every atom of its constraints
}

template <class P>
__device__ void con_load(const SysDev &S, const State<P> &st, int g, ConGroup &G) {
  const int a0 = S.cgroup_aoff[g], a1 = S.cgroup_aoff[g + 1], k0 = S.cgroup_off[g], k1 = S.cgroup_off[g + 1];
  G.na = a1 - a0;
  G.nc = k1 - k0;
  for (int u = 0; u < G.na; ++u) {
    const int a = S.cgroup_atoms[a0 + u];
    G.atom[u] = a;
    G.w[u] = 1.0 / S.mass[a];
    for (int x = 0; x < 3; ++x) {
      G.q[u][x] = st_q(st, 3 * a + x);
      G.p[u][x] = st_p(st, 3 * a + x);
    }
  }
  for (int c = 0; c < G.nc; ++c) {
    const int k = S.cgroup_cons[k0 + c];
    const int2 ij = S.con_ij[k];
    G.ci[c] = local_atom(G, ij.x);
    G.cj[c] = local_atom(G, ij.y);
    G.d[c] = S.con_len[k];
  }
}

// RATTLE: remove each bond's relative velocity until |r . v| <= tol d^2 / dt for all; false when the
// sweeps ran out.
__device__ bool con_rattle(const SysDev &S, ConGroup &G) {
  for (int it = 0; it < S.con_max_iter; ++it) {
    bool moved = false;
    for (int c = 0; c < G.nc; ++c) {
      const int i = G.ci[c], j = G.cj[c];
      const double wi = G.w[i], wj = G.w[j], d = G.d[c];
      const double r[3] = {G.q[i][0] - G.q[j][0], G.q[i][1] - G.q[j][1], G.q[i][2] - G.q[j][2]};
      double rv = 0.0, rr = 0.0;
      for (int x = 0; x < 3; ++x) {
        rv += r[x] * (G.p[i][x] * wi - G.p[j][x] * wj);
        rr += r[x] * r[x];
      }
      if (fabs(rv) <= S.con_tol * d * d / S.dt) continue;
      const double mu = rv / ((wi + wj) * rr);
      for (int x = 0; x < 3; ++x) {
        G.p[i][x] -= mu * r[x];
        G.p[j][x] += mu * r[x];
      }
      moved = true;
    }
    if (!moved) return true;
  }
  return false;
}

// SHAKE after an A step from q_old: move each pair along its bond vector at q_old until
// | |r|^2 - d^2 | <= tol d^2, adding the matching impulses (displacement times m / h) to the momenta.
__device__ bool con_shake(const SysDev &S, ConGroup &G, const double (*q_old)[3], double h) {
  for (int it = 0; it < S.con_max_iter; ++it) {
    bool moved = false;
    for (int c = 0; c < G.nc; ++c) {
      const int i = G.ci[c], j = G.cj[c];
      const double wi = G.w[i], wj = G.w[j], d = G.d[c];
      double rr = 0.0, sr = 0.0, so[3];
      for (int x = 0; x < 3; ++x) {
        const double r = G.q[i][x] - G.q[j][x];
        so[x] = q_old[i][x] - q_old[j][x];
        rr += r * r;
        sr += so[x] * r;
      }
      const double diff = d * d - rr;
      if (fabs(diff) <= S.con_tol * d * d) continue;
      const double gam = diff / (2.0 * (wi + wj) * sr);
      for (int x = 0; x < 3; ++x) {
        G.q[i][x] += gam * wi * so[x];
        G.q[j][x] -= gam * wj * so[x];
        G.p[i][x] += gam / h * so[x];
        G.p[j][x] -= gam / h * so[x];
      }
      moved = true;
    }
    if (!moved) return true;
  }
  return false;
}

__device__ __forceinline__ void con_a_step(const SysDev &S, ConGroup &G, double h, int *err) {
  double q_old[kMaxGroupAtoms][3];
  for (int u = 0; u < G.na; ++u)
    for (int x = 0; x < 3; ++x) {
      q_old[u][x] = G.q[u][x];
      G.q[u][x] += h * G.p[u][x] * G.w[u];
    }
  if (!con_shake(S, G, q_old, h)) *err |= kErrConstraint;
  if (!con_rattle(S, G)) *err |= kErrConstraint;
}

// The same for a group of one constraint (two atoms: the common case of one hydrogen on a heavy
// atom), in registers: the same sweeps, tests and updates as the general group code, without its
// local arrays and atom lookups.
struct ConPair {
  int a, b;
  double wa, wb, d, tq, tv;  // 1/m, length, SHAKE and RATTLE thresholds (tol d^2, tol d^2 / dt)
  double q[2][3], p[2][3];
};

__device__ __forceinline__ bool pair_rattle(const SysDev &S, ConPair &C) {
  for (int it = 0; it < S.con_max_iter; ++it) {
    const double r[3] = {C.q[0][0] - C.q[1][0], C.q[0][1] - C.q[1][1], C.q[0][2] - C.q[1][2]};
    double rv = 0.0, rr = 0.0;
    for (int x = 0; x < 3; ++x) {
      rv += r[x] * (C.p[0][x] * C.wa - C.p[1][x] * C.wb);
      rr += r[x] * r[x];
    }
    if (fabs(rv) <= C.tv) return true;
    const double mu = rv / ((C.wa + C.wb) * rr);
    for (int x = 0; x < 3; ++x) {
      C.p[0][x] -= mu * r[x];
      C.p[1][x] += mu * r[x];
    }
  }
  return false;
}

__device__ __forceinline__ void pair_a_step(const SysDev &S, ConPair &C, double h, double ih, int *err) {
  double so[3];
  for (int x = 0; x < 3; ++x) {
    so[x] = C.q[0][x] - C.q[1][x];
    C.q[0][x] += h * C.p[0][x] * C.wa;
    C.q[1][x] += h * C.p[1][x] * C.wb;
  }
  bool ok = false;
  for (int it = 0; it < S.con_max_iter && !ok; ++it) {
    double rr = 0.0, sr = 0.0;
    for (int x = 0; x < 3; ++x) {
      const double r = C.q[0][x] - C.q[1][x];
      rr += r * r;
      sr += so[x] * r;
    }
    const double diff = C.d * C.d - rr;
    if (fabs(diff) <= C.tq) { ok = true; break; }
    const double gam = diff / (2.0 * (C.wa + C.wb) * sr);
    for (int x = 0; x < 3; ++x) {
      C.q[0][x] += gam * C.wa * so[x];
      C.q[1][x] -= gam * C.wb * so[x];
      C.p[0][x] += gam * ih * so[x];
      C.p[1][x] -= gam * ih * so[x];
    }
  }
  if (!ok) *err |= kErrConstraint;
  if (!pair_rattle(S, C)) *err |= kErrConstraint;
}

template <class P>
__device__ __forceinline__ void pair_load(const SysDev &S, const State<P> &st, int g, ConPair &C) {
  const int k = S.cgroup_cons[S.cgroup_off[g]];
  const int2 ij = S.con_ij[k];
  C.a = ij.x;
  C.b = ij.y;
  C.wa = 1.0 / S.mass[C.a];
  C.wb = 1.0 / S.mass[C.b];
  C.d = S.con_len[k];
  C.tq = S.con_tol * C.d * C.d;
  C.tv = C.tq / S.dt;
  for (int x = 0; x < 3; ++x) {
    C.q[0][x] = st_q(st, 3 * C.a + x);
    C.q[1][x] = st_q(st, 3 * C.b + x);
    C.p[0][x] = st_p(st, 3 * C.a + x);
    C.p[1][x] = st_p(st, 3 * C.b + x);
  }
}

// The mixed path's groups of one constraint in double-single arithmetic (FP32 instructions: each FP64
// warp instruction costs GB300 ~64 cycles, and one warp carries every group of the block).  Positions,
// momenta, inverse masses and d^2 are double-single; the SHAKE residual d^2 - |r|^2 and the RATTLE
// residual r . (v_a - v_b) are evaluated in double-single, so the tolerances are those of the FP64 code;
// the drift h p / m is double-single too; the corrections (a Newton step on each residual) are computed in
// FP32 and added in double-single, so a sweep may take one more iteration.  Per-group constants, computed once per launch in FP64, sit in
// shared memory: PairDsConst.
struct PairDsConst {
  ds wa, wb, ha, hb, d2;  // 1/m, h/m (h half a step), d^2
  float tq, tv, sa, sb;   // SHAKE and RATTLE thresholds, noise amplitudes sqrt((1 - c1^2) kT m)
  float h, ih, c1;        // h, 1/h and c1 in FP32 (no FP64 division or conversion in the step loop)
};
__device__ __forceinline__ void pair_ds_const(const SysDev &S, int g, double h, double c1, PairDsConst &K) {
  const int k = S.cgroup_cons[S.cgroup_off[g]];
  const int2 ij = S.con_ij[k];
  const double d = S.con_len[k];
  K.wa = ds_from_double(1.0 / S.mass[ij.x]);
  K.wb = ds_from_double(1.0 / S.mass[ij.y]);
  K.ha = ds_from_double(h / S.mass[ij.x]);
  K.hb = ds_from_double(h / S.mass[ij.y]);
  K.d2 = ds_from_double(d * d);
  K.tq = (float)(S.con_tol * d * d);
  K.tv = (float)(S.con_tol * d * d / S.dt);
  K.sa = (float)noise_scale(c1, S.kT, S.mass[ij.x]);
  K.sb = (float)noise_scale(c1, S.kT, S.mass[ij.y]);
  K.h = (float)h;
  K.ih = (float)(1.0 / h);
  K.c1 = (float)c1;
}

struct ConPairDs {
  int a, b;
  ds q[2][3], p[2][3];
};

__device__ __forceinline__ void pair_load_ds(const SysDev &S, const State<PathMixed> &st, int g, ConPairDs &C) {
  const int2 ij = S.con_ij[S.cgroup_cons[S.cgroup_off[g]]];
  C.a = ij.x;
  C.b = ij.y;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    C.q[0][x] = ds{(&st.qh[C.a].x)[x], (&st.ql[C.a].x)[x]};
    C.q[1][x] = ds{(&st.qh[C.b].x)[x], (&st.ql[C.b].x)[x]};
    C.p[0][x] = ds{st.ph[3 * C.a + x], st.pl[3 * C.a + x]};
    C.p[1][x] = ds{st.ph[3 * C.b + x], st.pl[3 * C.b + x]};
  }
}
__device__ __forceinline__ void pair_store_ds(State<PathMixed> &st, const ConPairDs &C, bool positions) {
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    if (positions) {
      (&st.qh[C.a].x)[x] = C.q[0][x].hi;
      (&st.ql[C.a].x)[x] = C.q[0][x].lo;
      (&st.qh[C.b].x)[x] = C.q[1][x].hi;
      (&st.ql[C.b].x)[x] = C.q[1][x].lo;
    }
    st.ph[3 * C.a + x] = C.p[0][x].hi;
    st.pl[3 * C.a + x] = C.p[0][x].lo;
    st.ph[3 * C.b + x] = C.p[1][x].hi;
    st.pl[3 * C.b + x] = C.p[1][x].lo;
  }
}

// RATTLE for one bond: until |r . (p_a w_a - p_b w_b)| <= tv, p_a -= mu r, p_b += mu r with
// mu = r . v / ((w_a + w_b) |r|^2).
__device__ __forceinline__ bool pair_rattle_ds(const SysDev &S, const PairDsConst &K, ConPairDs &C) {
  float r[3];
  ds rd[3];
  float rr = 0.f;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    rd[x] = ds_sub2(C.q[0][x], C.q[1][x]);
    r[x] = rd[x].hi;
    rr = fmaf(r[x], r[x], rr);
  }
  const float den = (K.wa.hi + K.wb.hi) * rr;
  for (int it = 0; it < S.con_max_iter; ++it) {
    ds rv{0.f, 0.f};
#pragma unroll
    for (int x = 0; x < 3; ++x)
      rv = ds_add2(rv, ds_mul2(rd[x], ds_sub2(ds_mul2(C.p[0][x], K.wa), ds_mul2(C.p[1][x], K.wb))));
    if (fabsf(rv.hi) <= K.tv) return true;
    const float mu = rv.hi / den;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      C.p[0][x] = ds_add(C.p[0][x], -mu * r[x]);
      C.p[1][x] = ds_add(C.p[1][x], mu * r[x]);
    }
  }
  return false;
}

// A (half a step of drift) then SHAKE along the bond vector s_o before the drift: until
// |d^2 - |r|^2| <= tq, q_a += g w_a s_o, q_b -= g w_b s_o with g = (d^2 - |r|^2) / (2 (w_a + w_b) s_o . r),
// and the momenta by the matching impulse g s_o / h; then RATTLE.
__device__ __forceinline__ void pair_a_step_ds(const SysDev &S, const PairDsConst &K, ConPairDs &C, float ih,
                                               int *err) {
  float so[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) {  // the drift h p / m in double-single (a hydrogen's is large)
    so[x] = ds_sub2(C.q[0][x], C.q[1][x]).hi;
    C.q[0][x] = ds_add2(C.q[0][x], ds_mul2(C.p[0][x], K.ha));
    C.q[1][x] = ds_add2(C.q[1][x], ds_mul2(C.p[1][x], K.hb));
  }
  bool ok = false;
  for (int it = 0; it < S.con_max_iter && !ok; ++it) {
    ds rr{0.f, 0.f};
    float sr = 0.f;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const ds r = ds_sub2(C.q[0][x], C.q[1][x]);
      rr = ds_add2(rr, ds_mul2(r, r));
      sr = fmaf(so[x], r.hi, sr);
    }
    const float diff = ds_sub2(K.d2, rr).hi;
    if (fabsf(diff) <= K.tq) { ok = true; break; }
    const float gam = diff / (2.f * (K.wa.hi + K.wb.hi) * sr);
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const float gs = gam * so[x];
      C.q[0][x] = ds_add(C.q[0][x], gs * K.wa.hi);
      C.q[1][x] = ds_add(C.q[1][x], -gs * K.wb.hi);
      C.p[0][x] = ds_add(C.p[0][x], gs * ih);
      C.p[1][x] = ds_add(C.p[1][x], -gs * ih);
    }
  }
  if (!ok) *err |= kErrConstraint;
  if (!pair_rattle_ds(S, K, C)) *err |= kErrConstraint;
}

// B, A, O, A of one constrained group (the force of the previous step in the state's f; noise(atom, z)
// writes the three normals of this step for an atom: from a noise batch, or drawn from the counter-based
// stream, which give the same values).
template <class P, class Noise>
__device__ void con_baoa(const SysDev &S, State<P> &st, int g, Noise noise, double h, double c1, int *err,
                         const PairDsConst *kds = nullptr) {
  using T = typename P::T;
  if constexpr (P::kMixed) {
    if (kds && S.cgroup_off[g + 1] - S.cgroup_off[g] == 1) {  // one bond, double-single
      const PairDsConst &K = kds[g];
      ConPairDs C;
      pair_load_ds(S, st, g, C);
      T za[3], zb[3];
      noise(C.a, za);
      noise(C.b, zb);
      const float hf = K.h, ih = K.ih, c1f = K.c1;
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        C.p[0][x] = ds_add(C.p[0][x], hf * st.f[3 * C.a + x]);
        C.p[1][x] = ds_add(C.p[1][x], hf * st.f[3 * C.b + x]);
      }
      if (!pair_rattle_ds(S, K, C)) *err |= kErrConstraint;
      pair_a_step_ds(S, K, C, ih, err);
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        C.p[0][x] = ds_add(ds_scale(C.p[0][x], c1f), K.sa * za[x]);
        C.p[1][x] = ds_add(ds_scale(C.p[1][x], c1f), K.sb * zb[x]);
      }
      if (!pair_rattle_ds(S, K, C)) *err |= kErrConstraint;
      pair_a_step_ds(S, K, C, ih, err);
      pair_store_ds(st, C, true);
      return;
    }
  }
  if (S.cgroup_off[g + 1] - S.cgroup_off[g] == 1) {  // one constraint, two atoms
    ConPair C;
    pair_load<P>(S, st, g, C);
    const double ih = 1.0 / h;
    for (int x = 0; x < 3; ++x) {
      C.p[0][x] += h * st_f(st, 3 * C.a + x);
      C.p[1][x] += h * st_f(st, 3 * C.b + x);
    }
    if (!pair_rattle(S, C)) *err |= kErrConstraint;
    pair_a_step(S, C, h, ih, err);
    const double sa = noise_scale(c1, S.kT, S.mass[C.a]), sb = noise_scale(c1, S.kT, S.mass[C.b]);
    T za[3], zb[3];
    noise(C.a, za);
    noise(C.b, zb);
    for (int x = 0; x < 3; ++x) {
      C.p[0][x] = c1 * C.p[0][x] + sa * (double)za[x];
      C.p[1][x] = c1 * C.p[1][x] + sb * (double)zb[x];
    }
    if (!pair_rattle(S, C)) *err |= kErrConstraint;
    pair_a_step(S, C, h, ih, err);
    for (int x = 0; x < 3; ++x) {
      st_set_q(st, 3 * C.a + x, C.q[0][x]);
      st_set_q(st, 3 * C.b + x, C.q[1][x]);
      st_set_p(st, 3 * C.a + x, C.p[0][x]);
      st_set_p(st, 3 * C.b + x, C.p[1][x]);
    }
    return;
  }
  ConGroup G;
  con_load<P>(S, st, g, G);
  for (int u = 0; u < G.na; ++u)
    for (int x = 0; x < 3; ++x) G.p[u][x] += h * st_f(st, 3 * G.atom[u] + x);
  if (!con_rattle(S, G)) *err |= kErrConstraint;
  con_a_step(S, G, h, err);
  for (int u = 0; u < G.na; ++u) {
    const double sd = noise_scale(c1, S.kT, S.mass[G.atom[u]]);
    T z[3];
    noise(G.atom[u], z);
    for (int x = 0; x < 3; ++x) G.p[u][x] = c1 * G.p[u][x] + sd * (double)z[x];
  }
  if (!con_rattle(S, G)) *err |= kErrConstraint;
  con_a_step(S, G, h, err);
  for (int u = 0; u < G.na; ++u)
    for (int x = 0; x < 3; ++x) {
      st_set_q(st, 3 * G.atom[u] + x, G.q[u][x]);
      st_set_p(st, 3 * G.atom[u] + x, G.p[u][x]);
    }
}

// The closing B of a constrained group with the new forces (taken from the fixed-point accumulators,
// which are cleared, and kept in the state's f), then RATTLE; returns the group's kinetic energy.
__device__ __forceinline__ double con_take_force(State<PathF64> &st, const AccF64 &fa, int i) {
  const double v = (double)fa.F[i] * kFixInv;
  fa.F[i] = 0;
  st.f[i] = v;
  return v;
}
__device__ __forceinline__ double con_take_force(State<PathMixed> &st, const AccMixed &fa, int i) {
  const float v = split_to_float(fa.hi[i], fa.lo[i]);
  fa.hi[i] = 0;
  fa.lo[i] = 0u;
  st.f[i] = v;
  return (double)v;
}

template <class P>
__device__ double con_b(const SysDev &S, State<P> &st, const typename P::Acc &fa, int g, double h, int *err,
                        const PairDsConst *kds = nullptr) {
  if constexpr (P::kMixed) {
    if (kds && S.cgroup_off[g + 1] - S.cgroup_off[g] == 1) {
      const PairDsConst &K = kds[g];
      ConPairDs C;
      pair_load_ds(S, st, g, C);
      const float hf = K.h;
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        C.p[0][x] = ds_add(C.p[0][x], hf * (float)con_take_force(st, fa, 3 * C.a + x));
        C.p[1][x] = ds_add(C.p[1][x], hf * (float)con_take_force(st, fa, 3 * C.b + x));
      }
      if (!pair_rattle_ds(S, K, C)) *err |= kErrConstraint;
      pair_store_ds(st, C, false);
      float ke = 0.f;
#pragma unroll
      for (int x = 0; x < 3; ++x)
        ke += 0.5f * (C.p[0][x].hi * C.p[0][x].hi * K.wa.hi + C.p[1][x].hi * C.p[1][x].hi * K.wb.hi);
      return (double)ke;
    }
  }
  if (S.cgroup_off[g + 1] - S.cgroup_off[g] == 1) {
    ConPair C;
    pair_load<P>(S, st, g, C);
    for (int x = 0; x < 3; ++x) {
      C.p[0][x] += h * con_take_force(st, fa, 3 * C.a + x);
      C.p[1][x] += h * con_take_force(st, fa, 3 * C.b + x);
    }
    if (!pair_rattle(S, C)) *err |= kErrConstraint;
    double ke = 0.0;
    for (int x = 0; x < 3; ++x) {
      st_set_p(st, 3 * C.a + x, C.p[0][x]);
      st_set_p(st, 3 * C.b + x, C.p[1][x]);
      ke += 0.5 * (C.p[0][x] * C.p[0][x] * C.wa + C.p[1][x] * C.p[1][x] * C.wb);
    }
    return ke;
  }
  ConGroup G;
  con_load<P>(S, st, g, G);
  for (int u = 0; u < G.na; ++u)
    for (int x = 0; x < 3; ++x) G.p[u][x] += h * con_take_force(st, fa, 3 * G.atom[u] + x);
  if (!con_rattle(S, G)) *err |= kErrConstraint;
  double ke = 0.0;
  for (int u = 0; u < G.na; ++u)
    for (int x = 0; x < 3; ++x) {
      st_set_p(st, 3 * G.atom[u] + x, G.p[u][x]);
      ke += 0.5 * G.p[u][x] * G.p[u][x] * G.w[u];
    }
  return ke;
}

}  // namespace grp

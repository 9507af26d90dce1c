// C ABI of libgrp (include/grp.h): argument validation, device buffers, and the host driver of the
// Gen. ParRep loop of Fig. 1.  Every step of the hot path runs in the kernels of segment.cu and
// fvgr.cu; the host only launches them and reads a few bytes per exit test.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"

using namespace grp;

namespace {
// NVTX range over one host call (the phases of Fig. 1 as they appear on a profiler's timeline);
// without a profiler attached the calls return at once.
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};
}  // namespace

namespace {
thread_local std::string g_last_error;

grp_status fail(grp_status code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CU(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(GRP_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <class T>
grp_status upload(std::vector<void *> &owned, const T *h, size_t n, const T **out) {
  *out = nullptr;
  if (n == 0) return GRP_OK;
  void *d = nullptr;
  cudaError_t e = cudaMalloc(&d, n * sizeof(T));
  if (e != cudaSuccess) return fail(GRP_ENOMEM, "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
  owned.push_back(d);
  e = cudaMemcpy(d, h, n * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(GRP_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
  *out = (const T *)d;
  return GRP_OK;
}
}  // namespace

struct grp_system {
  SysDev dev{};
  SegConfig seg{};
  std::vector<void *> owned;
  int device = 0;
  // force-field parameters theta = (sigma_i, eps_i, k of each dihedral term in description order)
  int n_terms = 0;
  double *theta = nullptr;  // device [2n + n_terms], owned
  std::vector<uint8_t> excl;  // host [n][n] exclusion matrix of systems with Verlet lists
};

struct grp_replicas {
  grp_system *sys = nullptr;
  int R = 0;
  uint64_t seed = 0;
  double *q = nullptr, *p = nullptr, *f = nullptr, *acc = nullptr;
  int8_t *labels = nullptr;
  uint8_t *exited = nullptr;
  int32_t *src = nullptr;
  unsigned long long *exit_key = nullptr;
  int *err = nullptr;
  int *n_branched = nullptr;
  double *rhat = nullptr;
  uint32_t *nbl = nullptr;  // [R][nbl_cap] Verlet lists
  float4 *qref = nullptr;   // [R][n]
  int nbl_cap = 0;
  long long t_global = 0, t_phase = 0;
  // shard of a run sharded over processes: global index of replica 0 and the run's replica count
  // (rep0 = 0, n_global = R for a set that is the whole run)
  int rep0 = 0, n_global = 0;
  double *d_gr = nullptr;  // [3 GRP_MAX_OBS] Gelman-Rubin sums of the shard
  double *gb_glob = nullptr;  // [R][2n] Born radii and weights (solvent on Verlet lists)
  void *gb_gr = nullptr;      // [R][gb_gr_stride] the solvent's pass-3 force factor per candidate pair
  int gb_gr_stride = 0;
  // one-launch status readback (branch count, reference label and exit flag, ratios, error word,
  // first-exit key): the set's arrays for the status kernel, its output and a pinned copy
  RunArrays *d_run = nullptr;
  BatchStatus *d_status = nullptr, *h_status = nullptr;
  // pinned host mirror of the small per-check readback
  struct Readback {
    unsigned long long exit_key;
    int err;
    int n_branched;
    int8_t label0;
    uint8_t exited0;
    int8_t pad[6];
    double rhat[GRP_MAX_OBS];
    int dephase[2];  // replicas dephased, restarts (original ParRep)
  } *hb = nullptr;
};

extern "C" const char *grp_last_error(void) { return g_last_error.c_str(); }

// Shared with noalloc.cu.
grp::SysDev grp_system_device_view(const grp_system *s) { return s->dev; }
int grp_system_device_index(const grp_system *s) { return s->device; }
void grp_set_last_error(const char *msg) { g_last_error = msg; }

// ------------------------------------------------------------------------------------------------
// Periodic electrostatics by smooth particle mesh Ewald: validation and the device tables (box,
// excluded pairs, the self and background energies, the influence function on the grid).
static double host_bspline(int p, double x) {  // cardinal B-spline M_p, support (0, p)
  if (x <= 0.0 || x >= p) return 0.0;
  if (p == 2) return 1.0 - std::fabs(x - 1.0);
  return (x * host_bspline(p - 1, x) + (p - x) * host_bspline(p - 1, x - 1.0)) / (p - 1);
}

static grp_status setup_pme(const grp_system_desc *d, const std::vector<uint8_t> &excl, grp_system *s) {
  SysDev &D = s->dev;
  const int n = d->n_atoms;
  const double pi = 3.14159265358979323846;
  for (int x = 0; x < 3; ++x)
    if (!(d->box[x] > 0) || !std::isfinite(d->box[x])) return fail(GRP_EINVAL, "box edge %d must be positive", x);
  if (!(d->ewald_beta > 0) || !std::isfinite(d->ewald_beta)) return fail(GRP_EINVAL, "ewald_beta must be positive");
  const double lmin = std::min(d->box[0], std::min(d->box[1], d->box[2]));
  if (!(d->cutoff > 0) || d->cutoff > 0.5 * lmin)
    return fail(GRP_EINVAL, "particle mesh Ewald needs 0 < cutoff <= half the shortest box edge");
  // systems of 64 atoms and more keep a Verlet list (skin = cutoff / 6) over minimum images: each pair
  // within cutoff + skin must have one nearest image
  if (n >= 64 && 7.0 / 6.0 * d->cutoff > 0.5 * lmin)
    return fail(GRP_EINVAL, "particle mesh Ewald on %d atoms needs cutoff + skin (7/6 cutoff) <= half the shortest box edge", n);
  for (int x = 0; x < 3; ++x)
    if (d->pme_grid[x] != 8 && d->pme_grid[x] != 16)
      return fail(GRP_ENOTIMPL, "particle mesh Ewald grids of 8 or 16 points per axis (axis %d: %d)", x, d->pme_grid[x]);
  if (d->pme_order != 4) return fail(GRP_ENOTIMPL, "particle mesh Ewald with B-splines of order 4 (got %d)", d->pme_order);
  if (d->gb_radius || d->n_constraints > 0)
    return fail(GRP_ENOTIMPL, "particle mesh Ewald without implicit solvent or constraints");
  D.coulomb_rf = 2;
  D.ewald_beta = d->ewald_beta;
  for (int x = 0; x < 3; ++x) {
    D.box[x] = d->box[x];
    D.ibox[x] = 1.0 / d->box[x];
    D.pme_K[x] = d->pme_grid[x];
    const double kl = d->pme_grid[x] / d->box[x];
    D.pme_kl[x][0] = (float)kl;
    D.pme_kl[x][1] = (float)(kl - (double)D.pme_kl[x][0]);
  }
  const double V = d->box[0] * d->box[1] * d->box[2], b = d->ewald_beta, ke = d->coulomb_k;
  double q2 = 0.0, qt = 0.0;
  for (int i = 0; i < n; ++i) {
    q2 += d->charge[i] * d->charge[i];
    qt += d->charge[i];
  }
  D.pme_e_const = -ke * b / std::sqrt(pi) * q2 - ke * pi * qt * qt / (2.0 * V * b * b);
  std::vector<uint32_t> ex;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (excl[(size_t)i * n + j]) ex.push_back((uint32_t)i | ((uint32_t)j << 16));
  D.n_excl_pairs = (int)ex.size();
  grp_status st = GRP_OK;
  if (!ex.empty() && (st = upload(s->owned, ex.data(), ex.size(), &D.excl_pairs)) != GRP_OK) return st;
  // influence function times 4 (charges enter the grid scaled by sqrt(k_e/4)):
  // 4 B(m) exp(-pi^2 |m|^2 / beta^2) / (pi V |m|^2), B(m) = prod_d |sum_{k<p-1} M_p(k+1) e^{2 pi i m_d k/K_d}|^-2
  const int p = d->pme_order, *K = d->pme_grid;
  std::vector<double> bmod[3];
  for (int x = 0; x < 3; ++x) {
    bmod[x].resize(K[x]);
    for (int m = 0; m < K[x]; ++m) {
      double re = 0.0, im = 0.0;
      for (int k = 0; k + 1 < p; ++k) {
        const double a = 2.0 * pi * m * k / K[x], w = host_bspline(p, k + 1.0);
        re += w * std::cos(a);
        im += w * std::sin(a);
      }
      bmod[x][m] = 1.0 / (re * re + im * im);
    }
  }
  const size_t G = (size_t)K[0] * K[1] * K[2];
  std::vector<double> gd(G);
  std::vector<float> gf(G);
  for (int a = 0; a < K[0]; ++a)
    for (int c = 0; c < K[1]; ++c)
      for (int e = 0; e < K[2]; ++e) {
        const int mi[3] = {a, c, e};
        double m2 = 0.0;
        for (int x = 0; x < 3; ++x) {
          const double mx = (mi[x] <= K[x] / 2 ? mi[x] : mi[x] - K[x]) / d->box[x];
          m2 += mx * mx;
        }
        const size_t t = ((size_t)a * K[1] + c) * K[2] + e;
        gd[t] = m2 > 0.0 ? 4.0 * bmod[0][a] * bmod[1][c] * bmod[2][e] * std::exp(-pi * pi * m2 / (b * b)) / (pi * V * m2) : 0.0;
        gf[t] = (float)gd[t];
      }
  if ((st = upload(s->owned, gd.data(), G, &D.pme_g_d)) != GRP_OK) return st;
  return upload(s->owned, gf.data(), G, &D.pme_g_f);
}

extern "C" grp_status grp_create_system(const grp_system_desc *d, grp_system **out) {
  if (!d || !out) return fail(GRP_EINVAL, "grp_create_system: null argument");
  *out = nullptr;
  const int n = d->n_atoms;
  if (d->potential != GRP_POT_DOUBLE_WELL_2D && d->potential != GRP_POT_FORCE_FIELD)
    return fail(GRP_EINVAL, "unknown potential %d", d->potential);
  if (d->precision != GRP_FP64 && d->precision != GRP_MIXED)
    return fail(GRP_EINVAL, "unknown precision %d", d->precision);
  if (d->potential == GRP_POT_DOUBLE_WELL_2D) {
    if (n != 1 || d->dim != 2) return fail(GRP_EINVAL, "double well needs n_atoms = 1, dim = 2");
  } else if (d->dim != 3 || n < 1 || n > 65535) {
    return fail(GRP_EINVAL, "force field needs dim = 3 and 1 <= n_atoms <= 65535 (got %d, %d)", d->dim, n);
  }
  if (!d->mass) return fail(GRP_EINVAL, "mass is null");
  for (int i = 0; i < n; ++i)
    if (!(d->mass[i] > 0)) return fail(GRP_EINVAL, "mass[%d] must be > 0", i);
  if (!(d->kT > 0) || !(d->dt > 0) || !(d->gamma >= 0)) return fail(GRP_EINVAL, "need kT > 0, dt > 0, gamma >= 0");
  if (d->n_obs < 0 || d->n_obs > GRP_MAX_OBS) return fail(GRP_EINVAL, "n_obs must be in [0, %d]", GRP_MAX_OBS);
  if (d->n_groups < 0 || d->n_groups > GRP_MAX_GROUPS) return fail(GRP_EINVAL, "n_groups out of range");
  for (int g = 0; g < d->n_groups; ++g)
    if (d->group_offsets[g] < 0 || d->group_offsets[g + 1] <= d->group_offsets[g])
      return fail(GRP_EINVAL, "group %d is empty or offsets decrease", g);
  const int n_group_atoms = d->n_groups > 0 ? d->group_offsets[d->n_groups] : 0;
  if (n_group_atoms > 0 && !d->group_atoms) return fail(GRP_EINVAL, "group_atoms is null");
  for (int t = 0; t < n_group_atoms; ++t)
    if (d->group_atoms[t] < 0 || d->group_atoms[t] >= n) return fail(GRP_EINVAL, "group atom %d out of range", t);
  auto bad_atom = [&](int a) { return a < 0 || a >= n; };
  for (int j = 0; j < d->n_obs; ++j) {
    const int k = d->obs_kind[j];
    const int *a = d->obs_arg[j];
    if (k == GRP_OBS_COORD) {
      if (bad_atom(a[0]) || a[1] < 0 || a[1] >= d->dim) return fail(GRP_EINVAL, "observable %d: bad atom/axis", j);
    } else if (k == GRP_OBS_DIHEDRAL) {
      if (d->dim != 3 || bad_atom(a[0]) || bad_atom(a[1]) || bad_atom(a[2]) || bad_atom(a[3]))
        return fail(GRP_EINVAL, "observable %d: bad dihedral atoms", j);
    } else if (k == GRP_OBS_GROUP_DISTANCE) {
      if (d->dim != 3 || a[0] < 0 || a[0] >= d->n_groups || a[1] < 0 || a[1] >= d->n_groups)
        return fail(GRP_EINVAL, "observable %d: bad groups", j);
    } else if (k == GRP_OBS_RMS_VELOCITY) {
      if (d->dim != 3 || a[0] < 0 || a[0] >= d->n_groups) return fail(GRP_EINVAL, "observable %d: bad group", j);
    } else if (k != GRP_OBS_POTENTIAL && k != GRP_OBS_KINETIC) {
      return fail(GRP_EINVAL, "observable %d: unknown kind %d", j, k);
    }
    if (d->potential == GRP_POT_DOUBLE_WELL_2D && k != GRP_OBS_COORD && k != GRP_OBS_POTENTIAL && k != GRP_OBS_KINETIC)
      return fail(GRP_EINVAL, "observable %d: not available for the double well", j);
  }
  if (d->cv_kind == GRP_CV_DOUBLE_WELL) {
    if (d->potential != GRP_POT_DOUBLE_WELL_2D) return fail(GRP_EINVAL, "double-well states need the double-well potential");
  } else if (d->cv_kind == GRP_CV_DIHEDRAL_RECT) {
    if (d->dim != 3) return fail(GRP_EINVAL, "dihedral states need dim = 3");
    for (int t = 0; t < 5; ++t)
      if (bad_atom(d->cv_atoms[t])) return fail(GRP_EINVAL, "cv_atoms[%d] out of range", t);
  } else if (d->cv_kind == GRP_CV_COM_DISTANCE) {
    if (d->dim != 3 || d->n_groups < 2) return fail(GRP_EINVAL, "COM-distance states need two groups");
  } else if (d->cv_kind == GRP_CV_ROTAMERS) {
    const double m = d->cv_params[0], w = d->cv_params[1];
    if (d->dim != 3) return fail(GRP_EINVAL, "rotamer states need dim = 3");
    if (!(m >= 1.0 && m <= 4.0) || m != (double)(int)m)
      return fail(GRP_EINVAL, "rotamer states: cv_params[0] (torsions) must be an integer in [1, 4]");
    if (!(w > 0.0 && w <= 60.0)) return fail(GRP_EINVAL, "rotamer states: core half-width cv_params[1] must be in (0, 60]");
    for (int t = 0; t < (int)m + 3; ++t)
      if (bad_atom(d->cv_atoms[t])) return fail(GRP_EINVAL, "cv_atoms[%d] out of range", t);
  } else {
    return fail(GRP_EINVAL, "unknown cv_kind %d", d->cv_kind);
  }

  grp_system *s = new grp_system();
  CU(cudaGetDevice(&s->device));
  SysDev &D = s->dev;
  D.n = n;
  D.dim = d->dim;
  D.nd = n * d->dim;
  D.potential = d->potential;
  D.precision = d->precision;
  D.dw_a = d->dw_a;
  D.dw_b = d->dw_b;
  D.kT = d->kT;
  D.gamma = d->gamma;
  D.dt = d->dt;
  D.cv_kind = d->cv_kind;
  for (int t = 0; t < 8; ++t) { D.cv_atoms[t] = d->cv_atoms[t]; D.cv_params[t] = d->cv_params[t]; }
  D.n_groups = d->n_groups;
  for (int g = 0; g <= GRP_MAX_GROUPS; ++g) D.group_off[g] = g <= d->n_groups ? d->group_offsets[g] : n_group_atoms;
  D.n_obs = d->n_obs;
  for (int j = 0; j < GRP_MAX_OBS; ++j) {
    D.obs_kind[j] = d->obs_kind[j];
    for (int t = 0; t < 4; ++t) D.obs_arg[j][t] = d->obs_arg[j][t];
  }
  grp_status st = GRP_OK;
#define UP(h, cnt, out)                                   \
  do {                                                    \
    st = upload(s->owned, h, cnt, out);                   \
    if (st != GRP_OK) { grp_destroy_system(s); return st; } \
  } while (0)
  UP(d->mass, (size_t)n, &D.mass);
  if (n_group_atoms > 0) UP(d->group_atoms, (size_t)n_group_atoms, &D.group_atoms);

  if (d->potential == GRP_POT_FORCE_FIELD) {
    if (!d->sigma || !d->epsilon || !d->charge) { grp_destroy_system(s); return fail(GRP_EINVAL, "sigma/epsilon/charge null"); }
    std::vector<double4> ad(n);
    std::vector<float4> af(n);
    const double ck = std::sqrt(std::max(d->coulomb_k, 0.0) / 4.0);
    for (int i = 0; i < n; ++i) {
      if (!(d->epsilon[i] >= 0)) { grp_destroy_system(s); return fail(GRP_EINVAL, "epsilon[%d] < 0", i); }
      ad[i] = make_double4(0.5 * d->sigma[i], std::sqrt(d->epsilon[i]), d->charge[i] * ck, 1.0 / d->mass[i]);
      af[i] = make_float4((float)ad[i].x, (float)ad[i].y, (float)ad[i].z, (float)ad[i].w);
    }
    // noise amplitudes sqrt((1 - c1^2) kT m) per atom, computed on the device as the states compute them
    {
      std::vector<double> zd(n, 0.0);
      std::vector<float> zf(n, 0.f);
      UP(zd.data(), (size_t)n, &D.sd_d);
      UP(zf.data(), (size_t)n, &D.sd_f);
      const cudaError_t e = launch_noise_sd(D, std::exp(-d->gamma * d->dt), const_cast<double *>(D.sd_d),
                                            const_cast<float *>(D.sd_f), 0);
      if (e != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        grp_destroy_system(s);
        return fail(GRP_ECUDA, "noise amplitude table: %s", cudaGetErrorString(e));
      }
    }
    UP(ad.data(), (size_t)n, &D.atom_d);
    UP(af.data(), (size_t)n, &D.atom_f);
    // explicit list of non-excluded pairs
    std::vector<uint8_t> excl((size_t)n * n, 0);
    if (d->n_excl > 0 && !d->excl) { grp_destroy_system(s); return fail(GRP_EINVAL, "excl is null"); }
    for (int e = 0; e < d->n_excl; ++e) {
      const int i = d->excl[2 * e], j = d->excl[2 * e + 1];
      if (bad_atom(i) || bad_atom(j) || i == j) { grp_destroy_system(s); return fail(GRP_EINVAL, "exclusion %d invalid", e); }
      excl[(size_t)i * n + j] = excl[(size_t)j * n + i] = 1;
    }
    D.cutoff2 = d->cutoff > 0 ? d->cutoff * d->cutoff : 0.0;
    if (d->coulomb_mode == GRP_COULOMB_REACTION_FIELD) {
      if (!(d->cutoff > 0)) { grp_destroy_system(s); return fail(GRP_EINVAL, "the reaction field needs cutoff > 0"); }
      if (!(d->rf_dielectric == 0.0 || d->rf_dielectric >= 1.0)) {
        grp_destroy_system(s);
        return fail(GRP_EINVAL, "rf_dielectric must be >= 1 (or 0 for a conductor)");
      }
      const double rc = d->cutoff, er = d->rf_dielectric;
      D.coulomb_rf = 1;
      D.krf = (er == 0.0 ? 0.5 : (er - 1.0) / (2.0 * er + 1.0)) / (rc * rc * rc);
      D.crf = 1.0 / rc + D.krf * rc * rc;
    } else if (d->coulomb_mode == GRP_COULOMB_PME) {
      const grp_status ps = setup_pme(d, excl, s);
      if (ps != GRP_OK) { grp_destroy_system(s); return ps; }
    } else if (d->coulomb_mode != GRP_COULOMB_EPS4R) {
      grp_destroy_system(s);
      return fail(GRP_EINVAL, "unknown coulomb_mode %d", d->coulomb_mode);
    }
    // Small systems: an explicit list of non-excluded pairs, one thread per pair.  From 64 atoms on:
    // tiles of 32 atoms, every tile pair I <= J with per-lane interaction masks; with a cutoff, the
    // segment kernel keeps a Verlet list per replica (skin = cutoff / 6) built from the tiles.
    D.tiled = n >= 64 ? 1 : 0;
    if (D.tiled && d->cutoff > 0) {
      const double skin = d->cutoff / 6.0;
      D.use_list = 1;
      D.list_cut2 = (float)((d->cutoff + skin) * (d->cutoff + skin));
      D.half_skin2 = (float)(0.25 * skin * skin);
      s->excl = excl;
    }
    std::vector<uint32_t> pairs;
    if (!D.tiled) {
      // Pairs in round-robin order (the circle method: each round pairs every atom once), so that the
      // 32 pairs of a warp touch each atom a few times at most: the fixed-point additions of a warp to
      // the same accumulator are serialised, and the row-major order put ~20 lanes on atom i.
      pairs.reserve((size_t)n * (n - 1) / 2);
      const int m = n + (n & 1);  // with a dummy atom n when n is odd
      std::vector<int> ring(m);
      for (int r = 0; r < m - 1; ++r) {
        ring[0] = 0;
        for (int k = 1; k < m; ++k) ring[k] = 1 + (k - 1 + r) % (m - 1);
        for (int k = 0; k < m / 2; ++k) {
          const int i = std::min(ring[k], ring[m - 1 - k]), j = std::max(ring[k], ring[m - 1 - k]);
          if (j < n && !excl[(size_t)i * n + j]) pairs.push_back((uint32_t)i | ((uint32_t)j << 16));
        }
      }
    } else {
      const int nt = (n + 31) / 32;
      std::vector<uint32_t> tps, masks;
      for (int I = 0; I < nt; ++I)
        for (int J = I; J < nt; ++J) {
          tps.push_back((uint32_t)I | ((uint32_t)J << 16));
          for (int l = 0; l < 32; ++l) {
            const int i = I * 32 + l;
            uint32_t m = 0;
            for (int k = 0; k < 32; ++k) {
              const int j = J * 32 + k;
              if (i < n && j < n && i != j && !excl[(size_t)i * n + j]) m |= 1u << k;
            }
            masks.push_back(m);
          }
        }
      D.n_tiles = nt;
      D.n_tile_pairs = (int)tps.size();
      UP(tps.data(), tps.size(), &D.tile_pairs);
      UP(masks.data(), masks.size(), &D.tile_masks);
    }
    D.n_pairs = (int)pairs.size();
    if (!pairs.empty()) UP(pairs.data(), pairs.size(), &D.pairs);
    // bonds
    if (d->n_bonds > 0 && (!d->bond_atoms || !d->bond_k || !d->bond_r0)) { grp_destroy_system(s); return fail(GRP_EINVAL, "bond arrays null"); }
    std::vector<int2> bij(d->n_bonds);
    std::vector<double2> bd(d->n_bonds);
    std::vector<float2> bf(d->n_bonds);
    for (int b = 0; b < d->n_bonds; ++b) {
      const int i = d->bond_atoms[2 * b], j = d->bond_atoms[2 * b + 1];
      if (bad_atom(i) || bad_atom(j) || i == j) { grp_destroy_system(s); return fail(GRP_EINVAL, "bond %d invalid", b); }
      bij[b] = make_int2(i, j);
      bd[b] = make_double2(d->bond_k[b], d->bond_r0[b]);
      bf[b] = make_float2((float)bd[b].x, (float)bd[b].y);
    }
    // Large systems evaluate their bonds straight from these arrays, 32 consecutive bonds per warp: order
    // them in greedy rounds of atom-disjoint bonds, so that a warp's fixed-point additions go to distinct
    // atoms (the elastic network's springs come atom by atom, and consecutive springs of one atom made
    // the lanes of a warp add to the same words: 90,000 -> 63,000 cycles per step of the ligand's
    // bonded pass).  The sums are exact, so the order changes no result.
    if (D.tiled && d->n_bonds > 1) {
      std::vector<int> left(d->n_bonds), order;
      for (int b = 0; b < d->n_bonds; ++b) left[b] = b;
      std::vector<int> used(n, -1);
      for (int round = 0; !left.empty(); ++round) {
        std::vector<int> later;
        for (int b : left) {
          if (used[bij[b].x] == round || used[bij[b].y] == round) { later.push_back(b); continue; }
          used[bij[b].x] = used[bij[b].y] = round;
          order.push_back(b);
        }
        left.swap(later);
      }
      std::vector<int2> bij2(order.size());
      std::vector<double2> bd2(order.size());
      std::vector<float2> bf2(order.size());
      for (size_t u = 0; u < order.size(); ++u) { bij2[u] = bij[order[u]]; bd2[u] = bd[order[u]]; bf2[u] = bf[order[u]]; }
      bij.swap(bij2);
      bd.swap(bd2);
      bf.swap(bf2);
    }
    D.n_bonds = d->n_bonds;
    UP(bij.data(), bij.size(), &D.bond_ij);
    UP(bd.data(), bd.size(), &D.bond_d);
    UP(bf.data(), bf.size(), &D.bond_f);
    // angles
    if (d->n_angles > 0 && (!d->angle_atoms || !d->angle_k || !d->angle_theta0)) { grp_destroy_system(s); return fail(GRP_EINVAL, "angle arrays null"); }
    std::vector<int4> aijk(d->n_angles);
    std::vector<double2> angd(d->n_angles);
    std::vector<float2> angf(d->n_angles);
    for (int t = 0; t < d->n_angles; ++t) {
      const int *a = d->angle_atoms + 3 * t;
      if (bad_atom(a[0]) || bad_atom(a[1]) || bad_atom(a[2])) { grp_destroy_system(s); return fail(GRP_EINVAL, "angle %d invalid", t); }
      aijk[t] = make_int4(a[0], a[1], a[2], 0);
      angd[t] = make_double2(d->angle_k[t], d->angle_theta0[t]);
      angf[t] = make_float2((float)angd[t].x, (float)angd[t].y);
    }
    D.n_angles = d->n_angles;
    UP(aijk.data(), aijk.size(), &D.angle_ijk);
    UP(angd.data(), angd.size(), &D.angle_d);
    UP(angf.data(), angf.size(), &D.angle_f);
    // dihedrals: entries with the same four atoms form one item whose terms share the geometry
    if (d->n_dihedrals > 0 && (!d->dihedral_atoms || !d->dihedral_n || !d->dihedral_k || !d->dihedral_delta)) {
      grp_destroy_system(s);
      return fail(GRP_EINVAL, "dihedral arrays null");
    }
    std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;
    std::vector<std::tuple<int, int, int, int>> order;
    for (int t = 0; t < d->n_dihedrals; ++t) {
      const int *a = d->dihedral_atoms + 4 * t;
      if (bad_atom(a[0]) || bad_atom(a[1]) || bad_atom(a[2]) || bad_atom(a[3]) || d->dihedral_n[t] < 1 ||
          d->dihedral_n[t] > 6) {
        grp_destroy_system(s);
        return fail(GRP_EINVAL, "dihedral %d invalid (atoms or multiplicity outside 1..6)", t);
      }
      auto key = std::make_tuple(a[0], a[1], a[2], a[3]);
      if (!groups.count(key)) order.push_back(key);
      groups[key].push_back(t);
    }
    std::vector<int4> dijkl;
    std::vector<int2> dterms;
    std::vector<double4> td;
    std::vector<float4> tf;
    std::vector<int> tsrc;
    // Small systems on the mixed path (item table, idle lanes): one item per term, so that the terms
    // of a torsion run in parallel; the FP64 path and larger systems: one item per torsion whose terms
    // share the geometry (measured on the 22-bead chain: per term 0.85 ms mixed / 8.8 ms FP64 per
    // 500-step launch, per torsion 0.88 / 8.1 ms: the FP64 geometry is worth sharing).
    // (per term, the items run term-major -- every torsion's first term, then every second term -- so
    // that the terms of one torsion, which add to the same four atoms, fall in different warps.)
    const bool per_term = !D.tiled && d->precision == GRP_MIXED;
    size_t max_terms = 0;
    for (auto &key : order) max_terms = std::max(max_terms, groups[key].size());
    for (size_t level = 0; level < (per_term ? max_terms : 1); ++level)
      for (auto &key : order) {
        const int4 ijkl = make_int4(std::get<0>(key), std::get<1>(key), std::get<2>(key), std::get<3>(key));
        const std::vector<int> &g = groups[key];
        if (per_term && level >= g.size()) continue;
        const int t0 = (int)td.size();
        for (size_t u = per_term ? level : 0; u < (per_term ? level + 1 : g.size()); ++u) {
          const int t = g[u];
          td.push_back(make_double4(d->dihedral_k[t], (double)d->dihedral_n[t], std::cos(d->dihedral_delta[t]),
                                    std::sin(d->dihedral_delta[t])));
          tf.push_back(make_float4((float)td.back().x, (float)td.back().y, (float)td.back().z, (float)td.back().w));
          tsrc.push_back(t);
        }
        dijkl.push_back(ijkl);
        dterms.push_back(make_int2(t0, (int)td.size()));
      }
    D.n_dih = (int)dijkl.size();
    // work items: pairs, bonds, angles, dihedrals, each kind padded to a multiple of 32 entries
    // Within a kind the items run in greedy rounds of atom-disjoint items (like the round-robin pairs),
    // so that neighbouring lanes rarely add to the same atom's accumulator.
    std::vector<uint32_t> items;
    auto add_kind = [&](uint32_t kind, int count, auto atoms_of) {
      std::vector<int> left(count);
      for (int i = 0; i < count; ++i) left[i] = i;
      std::vector<int> used(n, -1);
      for (int round = 0; !left.empty(); ++round) {
        std::vector<int> later;
        for (int it : left) {
          const int4 a = atoms_of(it);
          const int at[4] = {a.x, a.y, a.z, a.w};
          bool free = true;
          for (int u = 0; u < 4; ++u) free = free && (at[u] < 0 || used[at[u]] != round);
          if (!free) { later.push_back(it); continue; }
          for (int u = 0; u < 4; ++u) if (at[u] >= 0) used[at[u]] = round;
          items.push_back((kind << 28) | (uint32_t)it);
        }
        left.swap(later);
      }
      while (items.size() % 32) items.push_back((uint32_t)kItemNone << 28);
    };
    add_kind(kItemPair, D.n_pairs, [&](int t) {
      return make_int4((int)(pairs[t] & 0xFFFFu), (int)(pairs[t] >> 16), -1, -1);
    });
    add_kind(kItemBond, D.n_bonds, [&](int t) { return make_int4(bij[t].x, bij[t].y, -1, -1); });
    add_kind(kItemAngle, D.n_angles, [&](int t) { return make_int4(aijk[t].x, aijk[t].y, aijk[t].z, -1); });
    add_kind(kItemDihedral, D.n_dih, [&](int t) { return dijkl[t]; });
    if (D.n_pairs >= (1 << 28) || items.size() >= (size_t)1 << 31) {
      grp_destroy_system(s);
      return fail(GRP_ENOTIMPL, "too many force-field items (%zu)", items.size());
    }
    D.n_items = (int)items.size();
    UP(items.data(), items.size(), &D.items);
    // Generalized Born implicit solvent (OBC II): every pair, per-atom radii and scales
    if (d->gb_radius) {
      if (!d->gb_scale) { grp_destroy_system(s); return fail(GRP_EINVAL, "gb_scale is null"); }
      // the item table (fewer than 64 atoms, every pair), or Verlet lists with the cutoff applied to the
      // solvent sums too (eps = 4r Coulomb)
      const bool gb_items = n < 64 && !(d->cutoff > 0);
      const bool gb_list = D.use_list && d->coulomb_mode == GRP_COULOMB_EPS4R;
      if (!gb_items && !gb_list) {
        grp_destroy_system(s);
        return fail(GRP_ENOTIMPL, "implicit solvent is implemented for systems of fewer than 64 atoms without a cutoff, "
                                  "and for systems of 64 atoms or more with a cutoff and the eps = 4r Coulomb model");
      }
      if (!(d->gb_solute_dielectric > 0) || !(d->gb_solvent_dielectric > 0)) {
        grp_destroy_system(s);
        return fail(GRP_EINVAL, "gb dielectric constants must be positive");
      }
      std::vector<double4> gd(n);
      std::vector<float4> gf(n);
      for (int i = 0; i < n; ++i) {
        const double a = d->gb_radius[i] - 0.009;
        if (!(a > 0) || !(d->gb_scale[i] >= 0)) {
          grp_destroy_system(s);
          return fail(GRP_EINVAL, "gb atom %d: radius must exceed 0.009 nm and the scale be >= 0", i);
        }
        gd[i] = make_double4(a, 1.0 / d->gb_radius[i], d->gb_scale[i] * a, d->charge[i]);
        gf[i] = make_float4((float)gd[i].x, (float)gd[i].y, (float)gd[i].z, (float)gd[i].w);
      }
      std::vector<uint32_t> gp, gx;
      if (gb_items) {
        gp.reserve((size_t)n * (n - 1) / 2);
        const int m = n + (n & 1);  // round-robin order, as the nonbonded pairs
        std::vector<int> ring(m);
        for (int rr = 0; rr < m - 1; ++rr) {
          ring[0] = 0;
          for (int k = 1; k < m; ++k) ring[k] = 1 + (k - 1 + rr) % (m - 1);
          for (int k = 0; k < m / 2; ++k) {
            const int i = std::min(ring[k], ring[m - 1 - k]), j = std::max(ring[k], ring[m - 1 - k]);
            if (j < n) gp.push_back((uint32_t)i | ((uint32_t)j << 16));
          }
        }
      } else {  // the solvent term includes the excluded pairs, which the Verlet lists leave out
        std::vector<uint32_t> all;
        for (int i = 0; i < n; ++i)
          for (int j = i + 1; j < n; ++j)
            if (s->excl[(size_t)i * n + j]) all.push_back((uint32_t)i | ((uint32_t)j << 16));
        // in greedy rounds of atom-disjoint pairs, as the bonds of large systems
        std::vector<int> used(n, -1);
        for (int round = 0; !all.empty(); ++round) {
          std::vector<uint32_t> later;
          for (uint32_t pk : all) {
            const int i = (int)(pk & 0xFFFFu), j = (int)(pk >> 16);
            if (used[i] == round || used[j] == round) { later.push_back(pk); continue; }
            used[i] = used[j] = round;
            gx.push_back(pk);
          }
          all.swap(later);
        }
      }
      D.gb = 1;
      D.n_gb_xpairs = (int)gx.size();
      if (!gx.empty()) UP(gx.data(), gx.size(), &D.gb_xpairs);
      D.n_gb_pairs = (int)gp.size();
      D.gb_tau = d->coulomb_k * (1.0 / d->gb_solute_dielectric - 1.0 / d->gb_solvent_dielectric);
      UP(gd.data(), gd.size(), &D.gb_d);
      UP(gf.data(), gf.size(), &D.gb_f);
      if (!gp.empty()) UP(gp.data(), gp.size(), &D.gb_pairs);
    }
    // bond constraints: independent groups (connected components of the constraint graph)
    if (d->n_constraints > 0) {
      if (!d->constraint_atoms || !d->constraint_length) { grp_destroy_system(s); return fail(GRP_EINVAL, "constraint arrays null"); }
      // the item table (eps = 4r, no solvent), or Verlet lists (eps = 4r, with or without the solvent: the
      // paper's protein-ligand setup)
      const bool con_items = !D.tiled && !D.coulomb_rf && !D.gb;
      const bool con_list = D.use_list && !D.coulomb_rf;
      if (!con_items && !con_list) {
        grp_destroy_system(s);
        return fail(GRP_ENOTIMPL, "bond constraints are implemented with the eps = 4r Coulomb model for systems of fewer "
                                  "than 64 atoms without implicit solvent, and for systems with Verlet lists");
      }
      if (!(d->constraint_tol > 0) || d->constraint_max_iter < 1) {
        grp_destroy_system(s);
        return fail(GRP_EINVAL, "constraint_tol must be > 0 and constraint_max_iter >= 1");
      }
      const int nc = d->n_constraints;
      std::vector<int> parent(n);
      for (int i = 0; i < n; ++i) parent[i] = i;
      auto root = [&](int x) { while (parent[x] != x) x = parent[x] = parent[parent[x]]; return x; };
      std::vector<int2> cij(nc);
      std::vector<unsigned char> flag(n, 0);
      for (int k = 0; k < nc; ++k) {
        const int i = d->constraint_atoms[2 * k], j = d->constraint_atoms[2 * k + 1];
        if (bad_atom(i) || bad_atom(j) || i == j || !(d->constraint_length[k] > 0)) {
          grp_destroy_system(s);
          return fail(GRP_EINVAL, "constraint %d invalid", k);
        }
        cij[k] = make_int2(i, j);
        flag[i] = flag[j] = 1;
        parent[root(i)] = root(j);
      }
      std::map<int, int> gid;  // root -> group, numbered by first constraint
      std::vector<std::vector<int>> gcons, gatoms;
      for (int k = 0; k < nc; ++k) {
        const int rk = root(cij[k].x);
        if (!gid.count(rk)) { gid[rk] = (int)gcons.size(); gcons.emplace_back(); gatoms.emplace_back(); }
        const int g = gid[rk];
        gcons[g].push_back(k);
        for (int a : {cij[k].x, cij[k].y})
          if (std::find(gatoms[g].begin(), gatoms[g].end(), a) == gatoms[g].end()) gatoms[g].push_back(a);
      }
      std::vector<int> off{0}, cons, aoff{0}, atoms;
      for (size_t g = 0; g < gcons.size(); ++g) {
        if (gcons[g].size() > 16 || gatoms[g].size() > 16) {
          grp_destroy_system(s);
          return fail(GRP_ENOTIMPL, "a group of coupled constraints holds more than 16 constraints or atoms");
        }
        cons.insert(cons.end(), gcons[g].begin(), gcons[g].end());
        off.push_back((int)cons.size());
        atoms.insert(atoms.end(), gatoms[g].begin(), gatoms[g].end());
        aoff.push_back((int)atoms.size());
      }
      D.n_cons = nc;
      D.con_tol = d->constraint_tol;
      D.con_max_iter = d->constraint_max_iter;
      D.n_cgroups = (int)gcons.size();
      UP(cij.data(), cij.size(), &D.con_ij);
      UP(d->constraint_length, (size_t)nc, &D.con_len);
      UP(flag.data(), flag.size(), &D.con_atom);
      UP(off.data(), off.size(), &D.cgroup_off);
      UP(cons.data(), cons.size(), &D.cgroup_cons);
      UP(aoff.data(), aoff.size(), &D.cgroup_aoff);
      UP(atoms.data(), atoms.size(), &D.cgroup_atoms);
    }
    UP(dijkl.data(), dijkl.size(), &D.dih_ijkl);
    UP(dterms.data(), dterms.size(), &D.dih_terms);
    UP(td.data(), td.size(), &D.term_d);
    UP(tf.data(), tf.size(), &D.term_f);
    UP(tsrc.data(), tsrc.size(), &D.term_src);
    // theta as given, for grp_get_params
    s->n_terms = (int)td.size();
    std::vector<double> th(2 * (size_t)n + s->n_terms);
    for (int i = 0; i < n; ++i) { th[i] = d->sigma[i]; th[n + i] = d->epsilon[i]; }
    for (int t = 0; t < s->n_terms; ++t) th[2 * n + t] = d->dihedral_k[t];
    const double *dth = nullptr;
    UP(th.data(), th.size(), &dth);
    s->theta = const_cast<double *>(dth);
  }
#undef UP
  s->seg = segment_config(D, 0);
  if (s->seg.smem > kMaxSmem) {
    grp_destroy_system(s);
    return fail(GRP_ENOTIMPL, "system of %d atoms needs %zu bytes of shared memory per replica", n, s->seg.smem);
  }
  *out = s;
  return GRP_OK;
}

extern "C" void grp_destroy_system(grp_system *s) {
  if (!s) return;
  for (void *p : s->owned) cudaFree(p);
  delete s;
}

// ------------------------------------------------------------------------------------------------
static grp_status latch_errors(grp_replicas *r, cudaStream_t st) {
  CU(cudaMemcpyAsync(&r->hb->err, r->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  const int e = r->hb->err;
  if (e) {
    CU(cudaMemsetAsync(r->err, 0, sizeof(int), st));
    if (e & kErrNaN) return fail(GRP_ENAN, "non-finite position or momentum");
    if (e & kErrList) return fail(GRP_ENOMEM, "a Verlet list outgrew its capacity (twice the pairs of the first configuration, at least 65,536 or every pair)");
    if (e & kErrConstraint) return fail(GRP_ETIMEOUT, "SHAKE or RATTLE did not converge within constraint_max_iter sweeps");
    if (e & kErrIndex) return fail(GRP_EINVAL, "a row index outside the replica set");
    if (e & kErrTimeout) return fail(GRP_ETIMEOUT, "a bulk copy of the branching did not complete within its time limit");
    return fail(GRP_EOVERFLOW, "force or energy term outside the fixed-point range (2^22 FP64, 2^18 mixed) or not finite");
  }
  return GRP_OK;
}

// The calls that treat the set as a whole run (its replica 0 the reference walker, its replicas all
// the workers) refuse a shard of a larger run.
static bool sharded(const grp_replicas *r) { return r->rep0 != 0 || r->n_global != r->R; }
#define NOT_SHARDED(r, name)                                                                          \
  do {                                                                                                \
    if (sharded(r)) return fail(GRP_EINVAL, "%s: the replica set is a shard of a larger run (use the " \
                                            "shard calls)", name);                                    \
  } while (0)

static grp_status compute_forces(grp_replicas *r, cudaStream_t st) {
  CU(launch_energy_forces(r->sys->dev, r->R, r->q, nullptr, r->f, r->err, st));
  return GRP_OK;
}

extern "C" grp_status grp_init_replicas(grp_system *s, int32_t n_replicas, uint64_t seed, const double *h_q0,
                                        const double *h_p0, int32_t per_replica, void *stream, grp_replicas **out) {
  if (!s || !out || !h_q0 || !h_p0) return fail(GRP_EINVAL, "grp_init_replicas: null argument");
  *out = nullptr;
  if (n_replicas < 1 || n_replicas > (1 << 24)) return fail(GRP_EINVAL, "n_replicas must be in [1, 2^24]");
  cudaStream_t st = (cudaStream_t)stream;
  grp_replicas *r = new grp_replicas();
  r->sys = s;
  r->R = n_replicas;
  r->n_global = n_replicas;
  r->seed = seed;
  const SysDev &D = s->dev;
  const size_t nd = (size_t)D.nd, R = (size_t)n_replicas, nacc = (size_t)D.n_obs * 4;
  auto alloc = [&](void **p, size_t bytes) -> grp_status {
    cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 8);
    if (e != cudaSuccess) return fail(GRP_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    return GRP_OK;
  };
  grp_status stt = GRP_OK;
#define AL(p, b)                                                  \
  do {                                                            \
    stt = alloc((void **)&(p), (b));                              \
    if (stt != GRP_OK) { grp_destroy_replicas(r); return stt; }   \
  } while (0)
  AL(r->q, R * nd * 8);
  AL(r->p, R * nd * 8);
  AL(r->f, R * nd * 8);
  AL(r->acc, R * nacc * 8);
  AL(r->labels, R);
  AL(r->exited, R);
  AL(r->src, R * 4);
  AL(r->exit_key, 8);
  AL(r->err, 4);
  AL(r->n_branched, 4);
  AL(r->rhat, GRP_MAX_OBS * 8);
  AL(r->d_gr, 3 * GRP_MAX_OBS * 8);
  if (D.use_list) {
    // capacity: twice the non-excluded pairs within cutoff + skin in the first configuration (over
    // nearest images in a periodic box), see below
    const int n = D.n;
    const double lc2 = (double)D.list_cut2;
    const bool per = D.coulomb_rf == 2;
    size_t cnt = 0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) {
        if (s->excl[(size_t)i * n + j]) continue;
        double d2 = 0;
        for (int x = 0; x < 3; ++x) {
          double dx = h_q0[3 * i + x] - h_q0[3 * j + x];
          if (per) dx -= D.box[x] * std::nearbyint(dx * D.ibox[x]);
          d2 += dx * dx;
        }
        cnt += d2 < lc2;
      }
    const size_t all = (size_t)n * (n - 1) / 2;
    // at least 65,536 entries (every pair, for systems of up to ~360 atoms, whose density may still
    // change a lot: ions condensing in a periodic box), + the padding of the warps' partly filled chunks
    // (16 warps of a 512-thread block, 256 entries each)
    r->nbl_cap = (int)(std::min(all, std::max(2 * cnt + 1024, (size_t)65536)) + 16 * 256);
    AL(r->nbl, R * (size_t)r->nbl_cap * 4);
    AL(r->qref, R * (size_t)n * 16);
    if (D.gb) {
      AL(r->gb_glob, R * (size_t)n * 2 * 8);
      r->gb_gr_stride = r->nbl_cap + D.n_gb_xpairs;
      AL(r->gb_gr, R * (size_t)r->gb_gr_stride * (D.precision == GRP_FP64 ? 8 : 4));
    }
  }
  AL(r->d_run, sizeof(RunArrays));
  AL(r->d_status, sizeof(BatchStatus));
#undef AL
  if (cudaMallocHost((void **)&r->h_status, sizeof(BatchStatus)) != cudaSuccess) {
    grp_destroy_replicas(r);
    return fail(GRP_ENOMEM, "cudaMallocHost failed");
  }
  {
    RunArrays ra{};
    ra.q = r->q; ra.p = r->p; ra.f = r->f; ra.acc = r->acc; ra.exited = r->exited; ra.labels = r->labels;
    ra.src = r->src; ra.n_branched = r->n_branched; ra.rhat = r->rhat; ra.err = r->err;
    ra.nd = D.nd; ra.nacc = D.n_obs * 4; ra.n_rep = n_replicas; ra.n_obs = D.n_obs;
    ra.seed = seed; ra.exit_key = r->exit_key;
    if (cudaMemcpy(r->d_run, &ra, sizeof(ra), cudaMemcpyHostToDevice) != cudaSuccess) {
      grp_destroy_replicas(r);
      return fail(GRP_ECUDA, "grp_init_replicas: upload failed");
    }
  }
  if (cudaMallocHost((void **)&r->hb, sizeof(*r->hb)) != cudaSuccess) {
    grp_destroy_replicas(r);
    return fail(GRP_ENOMEM, "cudaMallocHost failed");
  }
  if (per_replica) {
    CU(cudaMemcpyAsync(r->q, h_q0, R * nd * 8, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(r->p, h_p0, R * nd * 8, cudaMemcpyHostToDevice, st));
  } else {
    for (size_t i = 0; i < R; ++i) {
      CU(cudaMemcpyAsync(r->q + i * nd, h_q0, nd * 8, cudaMemcpyHostToDevice, st));
      CU(cudaMemcpyAsync(r->p + i * nd, h_p0, nd * 8, cudaMemcpyHostToDevice, st));
    }
  }
  if (nacc > 0) CU(cudaMemsetAsync(r->acc, 0, R * nacc * 8, st));
  CU(cudaMemsetAsync(r->labels, 0, R, st));
  CU(cudaMemsetAsync(r->exited, 0, R, st));
  CU(cudaMemsetAsync(r->err, 0, 4, st));
  CU(cudaMemsetAsync(r->exit_key, 0xff, 8, st));
  grp_status e = compute_forces(r, st);
  if (e == GRP_OK) e = latch_errors(r, st);
  if (e != GRP_OK) { grp_destroy_replicas(r); return e; }
  *out = r;
  return GRP_OK;
}

extern "C" void grp_destroy_replicas(grp_replicas *r) {
  if (!r) return;
  cudaFree(r->q); cudaFree(r->p); cudaFree(r->f); cudaFree(r->acc);
  cudaFree(r->labels); cudaFree(r->exited); cudaFree(r->src); cudaFree(r->exit_key);
  cudaFree(r->err); cudaFree(r->n_branched); cudaFree(r->rhat); cudaFree(r->d_gr);
  cudaFree(r->nbl); cudaFree(r->qref); cudaFree(r->gb_glob); cudaFree(r->gb_gr);
  if (r->hb) cudaFreeHost(r->hb);
  cudaFree(r->d_run); cudaFree(r->d_status);
  if (r->h_status) cudaFreeHost(r->h_status);
  delete r;
}

// ------------------------------------------------------------------------------------------------
static SegArgs seg_args(grp_replicas *r, int k, int t_gr, int n_active) {
  SegArgs a{};
  a.S = r->sys->dev;
  a.rep0 = r->rep0;
  a.q = r->q; a.p = r->p; a.f = r->f; a.acc = r->acc;
  a.labels = r->labels; a.exited = r->exited; a.exit_key = r->exit_key; a.err = r->err;
  a.nbl = r->nbl;
  a.qref = r->qref;
  a.nbl_cap = r->nbl_cap;
  a.gb_glob = r->gb_glob;
  a.gb_gr = r->gb_gr;
  a.gb_gr_stride = r->gb_gr_stride;
  a.seed = r->seed;
  a.t_global0 = r->t_global;
  a.t_phase0 = r->t_phase;
  a.k = k;
  a.t_gr = t_gr;
  a.n_active = n_active;
  a.h = 0.5 * a.S.dt;
  a.c1 = std::exp(-a.S.gamma * a.S.dt);
  return a;
}

// k steps in launches of at most kMaxSegment steps, so that one launch stays short.
static constexpr long long kMaxSegment = 20000;

static grp_status run_steps(grp_replicas *r, long long k, int t_gr, int n_active, int do_check, int omega,
                            long long M, int skip, cudaStream_t st) {
  while (k > 0) {
    const int kk = (int)std::min(k, kMaxSegment);
    SegArgs a = seg_args(r, kk, t_gr, n_active);
    a.do_check = (k == kk) ? do_check : 0;
    a.omega = omega;
    a.M = M;
    a.skip_if_exit = skip;
    CU(launch_segment(a, r->sys->seg, st));
    r->t_global += kk;
    r->t_phase += kk;
    k -= kk;
  }
  return GRP_OK;
}

extern "C" grp_status grp_step_k(grp_replicas *r, int64_t k, int32_t t_gr, int32_t n_active, void *stream) {
  const Range range("grp_step_k");
  if (!r) return fail(GRP_EINVAL, "grp_step_k: null handle");
  if (k < 0 || t_gr < 0 || n_active < 0 || n_active > r->R) return fail(GRP_EINVAL, "grp_step_k: bad k/t_gr/n_active");
  return run_steps(r, k, t_gr, n_active ? n_active : r->R, 0, 0, 0, 0, (cudaStream_t)stream);
}

extern "C" grp_status grp_check_states(grp_replicas *r, int32_t omega, int8_t *d_labels, uint8_t *d_exited, void *stream) {
  if (!r) return fail(GRP_EINVAL, "grp_check_states: null handle");
  cudaStream_t st = (cudaStream_t)stream;
  CU(launch_check(r->sys->dev, r->q, r->R, omega, r->labels, r->exited, nullptr, 0, st));
  if (d_labels) CU(cudaMemcpyAsync(d_labels, r->labels, r->R, cudaMemcpyDeviceToDevice, st));
  if (d_exited) CU(cudaMemcpyAsync(d_exited, r->exited, r->R, cudaMemcpyDeviceToDevice, st));
  return GRP_OK;
}

extern "C" grp_status grp_fv_branch(grp_replicas *r, const uint8_t *d_exited, int32_t *d_src, int32_t *h_n_branched,
                                    void *stream) {
  if (!r) return fail(GRP_EINVAL, "grp_fv_branch: null handle");
  NOT_SHARDED(r, "grp_fv_branch");
  cudaStream_t st = (cudaStream_t)stream;
  const SysDev &D = r->sys->dev;
  CU(launch_fv_branch(D, r->R, r->q, r->p, r->f, r->acc, d_exited ? d_exited : r->exited, r->src, r->n_branched,
                      r->seed, r->t_global, st, r->err));
  if (d_src) CU(cudaMemcpyAsync(d_src, r->src, (size_t)r->R * 4, cudaMemcpyDeviceToDevice, st));
  if (h_n_branched) {
    CU(cudaMemcpyAsync(&r->hb->n_branched, r->n_branched, 4, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    *h_n_branched = r->hb->n_branched;
  }
  return GRP_OK;
}

extern "C" grp_status grp_gelman_rubin(grp_replicas *r, double tol, double *h_rhat, int32_t *h_converged, void *stream) {
  if (!r) return fail(GRP_EINVAL, "grp_gelman_rubin: null handle");
  NOT_SHARDED(r, "grp_gelman_rubin");
  if (r->R < 2) return fail(GRP_EINVAL, "grp_gelman_rubin: needs at least one F-V worker (R >= 2)");
  cudaStream_t st = (cudaStream_t)stream;
  const SysDev &D = r->sys->dev;
  CU(launch_gelman_rubin(D, r->R, r->acc, tol, r->rhat, nullptr, st));
  CU(cudaMemcpyAsync(r->hb->rhat, r->rhat, sizeof(double) * D.n_obs, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  int conv = 1;
  for (int j = 0; j < D.n_obs; ++j) {
    if (h_rhat) h_rhat[j] = r->hb->rhat[j];
    if (!(r->hb->rhat[j] < 1.0 + tol)) conv = 0;
  }
  if (h_converged) *h_converged = conv;
  return GRP_OK;
}

// ------------------------------------------------------------------------------------------------
// Batched runs.
struct grp_batch {
  std::vector<grp_replicas *> runs;
  int precision = 0;
  int threads = 0;
  size_t smem = 0;
  int n_units = 0, n_branch_units = 0, n_gr_units = 0;
  SegArgs *d_args = nullptr, *h_args = nullptr;      // [n_runs], h_ pinned
  RunArrays *d_arrays = nullptr, *h_arrays = nullptr;  // [n_runs], h_ pinned
  uint2 *d_units = nullptr, *d_branch_units = nullptr, *d_gr_units = nullptr;
  int *d_counter = nullptr, *d_nb = nullptr;
  BatchStatus *d_status = nullptr, *h_status = nullptr;  // h_ pinned
  long long ticks = 0, graph_ticks = 0;                  // of the last grp_batch_run
};

extern "C" void grp_batch_destroy(grp_batch *b) {
  if (!b) return;
  cudaFree(b->d_args); cudaFree(b->d_arrays); cudaFree(b->d_units); cudaFree(b->d_branch_units);
  cudaFree(b->d_gr_units); cudaFree(b->d_counter); cudaFree(b->d_nb); cudaFree(b->d_status);
  if (b->h_args) cudaFreeHost(b->h_args);
  if (b->h_arrays) cudaFreeHost(b->h_arrays);
  if (b->h_status) cudaFreeHost(b->h_status);
  delete b;
}

extern "C" grp_status grp_batch_create(grp_replicas *const *runs, int32_t n_runs, grp_batch **out) {
  if (!runs || !out || n_runs < 1) return fail(GRP_EINVAL, "grp_batch_create: need n_runs >= 1 runs");
  *out = nullptr;
  for (int i = 0; i < n_runs; ++i) {
    if (!runs[i]) return fail(GRP_EINVAL, "grp_batch_create: run %d is null", i);
    if (sharded(runs[i])) return fail(GRP_EINVAL, "grp_batch_create: run %d is a shard of a larger run", i);
    if (runs[i]->sys->dev.potential != GRP_POT_FORCE_FIELD)
      return fail(GRP_ENOTIMPL, "grp_batch_create: batches hold force-field systems");
    if (runs[i]->sys->dev.gb || runs[i]->sys->dev.n_cons || runs[i]->sys->dev.coulomb_rf == 2)
      return fail(GRP_ENOTIMPL, "grp_batch_create: systems in implicit solvent, with constraints or periodic run alone");
    if (runs[i]->sys->dev.precision != runs[0]->sys->dev.precision)
      return fail(GRP_EINVAL, "grp_batch_create: runs must share one precision");
  }
  grp_batch *b = new grp_batch();
  b->runs.assign(runs, runs + n_runs);
  b->precision = runs[0]->sys->dev.precision;
  std::vector<uint2> units, bunits, gunits;
  for (int i = 0; i < n_runs; ++i) {
    const grp_replicas *r = runs[i];
    b->threads = std::max(b->threads, r->sys->seg.threads);
    b->smem = std::max(b->smem, r->sys->seg.smem);
    for (int k = 0; k < r->R; ++k) { units.push_back(make_uint2(i, k)); bunits.push_back(make_uint2(i, k)); }
    for (int j = 0; j < r->sys->dev.n_obs; ++j) gunits.push_back(make_uint2(i, j));
  }
  // largest systems first
  std::stable_sort(units.begin(), units.end(), [&](const uint2 &x, const uint2 &y) {
    return runs[x.x]->sys->dev.n > runs[y.x]->sys->dev.n;
  });
  b->threads = std::min(512, b->threads);
  b->n_units = (int)units.size();
  b->n_branch_units = (int)bunits.size();
  b->n_gr_units = (int)gunits.size();
  auto dalloc = [&](void **p, size_t bytes) { return cudaMalloc(p, bytes > 0 ? bytes : 8) == cudaSuccess; };
  bool ok = dalloc((void **)&b->d_args, sizeof(SegArgs) * n_runs) && dalloc((void **)&b->d_arrays, sizeof(RunArrays) * n_runs) &&
            dalloc((void **)&b->d_units, sizeof(uint2) * units.size()) &&
            dalloc((void **)&b->d_branch_units, sizeof(uint2) * bunits.size()) &&
            dalloc((void **)&b->d_gr_units, sizeof(uint2) * gunits.size()) && dalloc((void **)&b->d_counter, 8) &&
            dalloc((void **)&b->d_nb, sizeof(int) * n_runs) && dalloc((void **)&b->d_status, sizeof(BatchStatus) * n_runs) &&
            cudaMallocHost((void **)&b->h_args, sizeof(SegArgs) * n_runs) == cudaSuccess &&
            cudaMallocHost((void **)&b->h_arrays, sizeof(RunArrays) * n_runs) == cudaSuccess &&
            cudaMallocHost((void **)&b->h_status, sizeof(BatchStatus) * n_runs) == cudaSuccess;
  if (!ok) { grp_batch_destroy(b); return fail(GRP_ENOMEM, "grp_batch_create: allocation failed"); }
  if (cudaMemcpy(b->d_units, units.data(), sizeof(uint2) * units.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_branch_units, bunits.data(), sizeof(uint2) * bunits.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      (!gunits.empty() &&
       cudaMemcpy(b->d_gr_units, gunits.data(), sizeof(uint2) * gunits.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
    grp_batch_destroy(b);
    return fail(GRP_ECUDA, "grp_batch_create: upload failed");
  }
  *out = b;
  return GRP_OK;
}

// What one batched segment does for one run: replicas advanced (0: none), sampling period, fused
// exit test against omega, parallel-step check index M and early return after an earlier exit.
struct RunTick {
  int n_active, t_gr, do_check, omega, skip;
  long long M;
};

// One batched segment of k steps (k <= kMaxSegment), each run as its tick says.
// Host half of a batched segment: the argument block of every run (pinned memory, read by the copy
// that enqueue_segment queues) and the runs' step counters.
static void fill_args(grp_batch *b, int k, const RunTick *ticks) {
  const int nr = (int)b->runs.size();
  for (int i = 0; i < nr; ++i) {
    grp_replicas *r = b->runs[i];
    const RunTick &t = ticks[i];
    SegArgs a = seg_args(r, k, t.t_gr, t.n_active);
    a.do_check = t.do_check;
    a.omega = t.omega;
    a.M = t.M;
    a.skip_if_exit = t.skip;
    a.pairs_in_smem = r->sys->seg.pairs_in_smem;
    a.noise_batch = r->sys->seg.noise_batch;
    a.lean = r->sys->seg.lean;
    b->h_args[i] = a;
  }
  for (int i = 0; i < nr; ++i) {
    if (ticks[i].n_active <= 0) continue;
    b->runs[i]->t_global += k;
    b->runs[i]->t_phase += k;
  }
}

static grp_status enqueue_segment(grp_batch *b, cudaStream_t st) {
  CU(cudaMemcpyAsync(b->d_args, b->h_args, sizeof(SegArgs) * b->runs.size(), cudaMemcpyHostToDevice, st));
  CU(launch_segment_batch(b->d_args, b->d_units, b->n_units, b->d_counter, b->precision, b->threads, b->smem, st,
                          nullptr));
  return GRP_OK;
}

// One batched segment of k steps (k <= kMaxSegment), each run as its tick says.
static grp_status batch_launch(grp_batch *b, int k, const RunTick *ticks, cudaStream_t st) {
  CU(cudaStreamSynchronize(st));  // the pinned argument block may still be read by a queued copy
  fill_args(b, k, ticks);
  return enqueue_segment(b, st);
}

// Every replica of every run, with or without the fused exit test.
static grp_status batch_segment(grp_batch *b, int k, int t_gr, int do_check, const int32_t *omega, cudaStream_t st) {
  std::vector<RunTick> ticks(b->runs.size());
  for (size_t i = 0; i < ticks.size(); ++i)
    ticks[i] = RunTick{b->runs[i]->R, t_gr, do_check, omega ? omega[i] : 0, 0, 0};
  return batch_launch(b, k, ticks.data(), st);
}

// Host half of a batched status: the runs' arrays with their branching and Gelman-Rubin flags.
static void fill_arrays(grp_batch *b, const int *branch, const int *gr) {
  const int nr = (int)b->runs.size();
  for (int i = 0; i < nr; ++i) {
    grp_replicas *r = b->runs[i];
    const SysDev &D = r->sys->dev;
    RunArrays a;
    a.q = r->q; a.p = r->p; a.f = r->f; a.acc = r->acc; a.exited = r->exited; a.labels = r->labels;
    a.src = r->src; a.n_branched = b->d_nb + i; a.rhat = r->rhat; a.err = r->err;
    a.nd = D.nd; a.nacc = D.n_obs * 4; a.n_rep = r->R; a.n_obs = D.n_obs;
    a.seed = r->seed; a.t_global = r->t_global;
    a.exit_key = r->exit_key;
    a.branch = branch[i];
    a.gr = gr[i];
    b->h_arrays[i] = a;
  }
}

static grp_status enqueue_status(grp_batch *b, cudaStream_t st) {
  const int nr = (int)b->runs.size();
  CU(cudaMemcpyAsync(b->d_arrays, b->h_arrays, sizeof(RunArrays) * nr, cudaMemcpyHostToDevice, st));
  CU(cudaMemsetAsync(b->d_nb, 0, sizeof(int) * nr, st));
  CU(launch_fv_branch_batch(b->d_arrays, b->d_branch_units, b->n_branch_units, st));
  CU(launch_gelman_rubin_batch(b->d_arrays, b->d_gr_units, b->n_gr_units, st));
  CU(launch_collect_status(b->d_arrays, nr, b->d_status, st));
  CU(cudaMemcpyAsync(b->h_status, b->d_status, sizeof(BatchStatus) * nr, cudaMemcpyDeviceToHost, st));
  return GRP_OK;
}

// After a batched exit test: branching of the runs with branch[i], Gelman-Rubin ratios of those with
// gr[i], and one readback of every run's status into b->h_status.
static grp_status batch_status(grp_batch *b, const int *branch, const int *gr, cudaStream_t st) {
  fill_arrays(b, branch, gr);
  grp_status e = enqueue_status(b, st);
  if (e != GRP_OK) return e;
  CU(cudaStreamSynchronize(st));
  return GRP_OK;
}

// One tick of the batched loop as a CUDA graph: the segment, branching, Gelman-Rubin ratios and the
// status readback, captured once per grp_batch_run call.  Every node reads fixed buffers (the pinned
// argument blocks are refilled before each launch), so the graph is replayed as captured.
struct TickGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~TickGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
  // false (and no graph) when capture is unavailable; the caller then launches the nodes one by one
  bool capture(grp_batch *b) {
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); return false; }
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    const bool queued = ok && enqueue_segment(b, cs) == GRP_OK && enqueue_status(b, cs) == GRP_OK;
    if (ok) ok = cudaStreamEndCapture(cs, &graph) == cudaSuccess && queued;
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    cudaStreamDestroy(cs);
    if (!ok) {
      cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      graph = nullptr;
      exec = nullptr;
    }
    return ok;
  }
};

extern "C" grp_status grp_batch_step_k(grp_batch *b, int64_t k, int32_t t_gr, void *stream) {
  const Range range("grp_batch_step_k");
  if (!b || k < 0 || t_gr < 0) return fail(GRP_EINVAL, "grp_batch_step_k: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  while (k > 0) {
    const int kk = (int)std::min<long long>(k, kMaxSegment);
    grp_status e = batch_segment(b, kk, t_gr, 0, nullptr, st);
    if (e != GRP_OK) return e;
    k -= kk;
  }
  return GRP_OK;  // device error words stay latched until the next synchronising call
}

extern "C" grp_status grp_batch_fv_check(grp_batch *b, const int32_t *h_omega, int32_t t_check, int32_t t_gr,
                                         double tol, int64_t min_fv_steps, grp_fv_status *h_out, void *stream) {
  const Range range("grp_batch_fv_check (exit test)");
  if (!b || !h_omega || !h_out || t_check < 1 || t_check > kMaxSegment || t_gr < 0)
    return fail(GRP_EINVAL, "grp_batch_fv_check: bad argument (t_check must be in [1, %lld])", kMaxSegment);
  cudaStream_t st = (cudaStream_t)stream;
  const int nr = (int)b->runs.size();
  grp_status e = batch_segment(b, t_check, t_gr, 1, h_omega, st);
  if (e != GRP_OK) return e;
  const std::vector<int> all(nr, 1);
  if ((e = batch_status(b, all.data(), all.data(), st)) != GRP_OK) return e;
  for (int i = 0; i < nr; ++i) {
    const grp_replicas *r = b->runs[i];
    const BatchStatus &s = b->h_status[i];
    grp_fv_status &o = h_out[i];
    const int no = r->sys->dev.n_obs;
    const bool want_gr = r->t_phase >= min_fv_steps && r->R > 1 && no > 0;
    o.ref_exited = s.exited0;
    o.label0 = s.label0;
    o.n_branched = s.n_branched;
    o.gr_evaluated = want_gr ? 1 : 0;
    o.t_phase = r->t_phase;
    o.pad = 0;
    int conv = want_gr ? 1 : 0;
    for (int j = 0; j < GRP_MAX_OBS; ++j) {
      o.rhat[j] = (want_gr && j < no) ? s.rhat[j] : 0.0;
      if (want_gr && j < no && !(s.rhat[j] < 1.0 + tol)) conv = 0;
    }
    o.converged = conv;
  }
  for (int i = 0; i < nr; ++i) {
    if (b->h_status[i].err) {  // latched by a kernel of run i: report it and clear it
      e = latch_errors(b->runs[i], st);
      if (e != GRP_OK) return e;
    }
  }
  return GRP_OK;
}

extern "C" grp_status grp_batch_stats(const grp_batch *b, int64_t *h_ticks, int64_t *h_graph_ticks) {
  if (!b) return fail(GRP_EINVAL, "grp_batch_stats: null batch");
  if (h_ticks) *h_ticks = b->ticks;
  if (h_graph_ticks) *h_graph_ticks = b->graph_ticks;
  return GRP_OK;
}

extern "C" grp_status grp_batch_autotune(grp_batch *b, int32_t t_gr, void *stream, int32_t *h_threads) {
  if (!b) return fail(GRP_EINVAL, "grp_batch_autotune: null batch");
  cudaStream_t st = (cudaStream_t)stream;
  // snapshot every run's state and counters
  struct Snap {
    double *q, *p, *f, *acc;
    size_t nq, na;
    long long tg, tp;
  };
  std::vector<Snap> snaps;
  for (grp_replicas *r : b->runs) {
    Snap s{};
    s.nq = (size_t)r->R * r->sys->dev.nd * 8;
    s.na = (size_t)r->R * r->sys->dev.n_obs * 4 * 8;
    if (cudaMalloc((void **)&s.q, s.nq) != cudaSuccess || cudaMalloc((void **)&s.p, s.nq) != cudaSuccess ||
        cudaMalloc((void **)&s.f, s.nq) != cudaSuccess || cudaMalloc((void **)&s.acc, s.na + 8) != cudaSuccess) {
      for (Snap &x : snaps) { cudaFree(x.q); cudaFree(x.p); cudaFree(x.f); cudaFree(x.acc); }
      return fail(GRP_ENOMEM, "grp_batch_autotune: snapshot allocation failed");
    }
    cudaMemcpyAsync(s.q, r->q, s.nq, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(s.p, r->p, s.nq, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(s.f, r->f, s.nq, cudaMemcpyDeviceToDevice, st);
    if (s.na) cudaMemcpyAsync(s.acc, r->acc, s.na, cudaMemcpyDeviceToDevice, st);
    s.tg = r->t_global;
    s.tp = r->t_phase;
    snaps.push_back(s);
  }
  const int candidates[] = {128, 256, 384, 512};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = b->threads;
  float best_ms = 1e30f;
  grp_status status = GRP_OK;
  for (int c : candidates) {
    b->threads = c;
    if (batch_segment(b, 10, t_gr, 0, nullptr, st) != GRP_OK) continue;  // warm-up
    cudaEventRecord(e0, st);
    status = batch_segment(b, 50, t_gr, 0, nullptr, st);
    cudaEventRecord(e1, st);
    if (status != GRP_OK) break;
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) { best_ms = ms; best = c; }
  }
  b->threads = best;
  for (size_t i = 0; i < b->runs.size(); ++i) {
    grp_replicas *r = b->runs[i];
    Snap &s = snaps[i];
    cudaMemcpyAsync(r->q, s.q, s.nq, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(r->p, s.p, s.nq, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(r->f, s.f, s.nq, cudaMemcpyDeviceToDevice, st);
    if (s.na) cudaMemcpyAsync(r->acc, s.acc, s.na, cudaMemcpyDeviceToDevice, st);
    r->t_global = s.tg;
    r->t_phase = s.tp;
  }
  cudaStreamSynchronize(st);
  for (Snap &s : snaps) { cudaFree(s.q); cudaFree(s.p); cudaFree(s.f); cudaFree(s.acc); }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (h_threads) *h_threads = best;
  return status;
}

// Parallel phase: segments of t_check steps with the exit test fused at the end; batches of
// segments are queued before the exit key is read back (segments after an exit return at once).
static grp_status parallel_phase(grp_replicas *r, int omega, int t_check, long long max_checks, grp_exit *out,
                                 cudaStream_t st) {
  CU(cudaMemsetAsync(r->exit_key, 0xff, 8, st));
  const long long tg0 = r->t_global, tp0 = r->t_phase;
  long long M = 0;
  int batch = 1;
  while (M < max_checks) {
    const long long nb = std::min<long long>(batch, max_checks - M);
    for (long long i = 0; i < nb; ++i) {
      ++M;
      grp_status e = run_steps(r, t_check, 0, r->R, 1, omega, M, 1, st);
      if (e != GRP_OK) return e;
    }
    // the first-exit key and the label of that replica in one launch and one copy
    CU(launch_collect_status(r->d_run, 1, r->d_status, st));
    CU(cudaMemcpyAsync(r->h_status, r->d_status, sizeof(BatchStatus), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    const unsigned long long key = r->h_status->exit_key;
    if (key != ~0ull) {
      const long long Mx = (long long)(key >> 32);
      const int k0 = (int)(key & 0xffffffffu);
      r->t_global = tg0 + Mx * t_check;
      r->t_phase = tp0 + Mx * t_check;
      out->M = Mx;
      out->k = k0 + 1;
      out->label_to = r->h_status->label_k;
      out->tau_steps = ((long long)r->R * (Mx - 1) + (k0 + 1)) * (long long)t_check;
      return GRP_OK;
    }
    batch = std::min(batch * 2, 16);
  }
  return GRP_NOEXIT;
}

extern "C" grp_status grp_run_parallel_phase(grp_replicas *r, int32_t omega, int32_t t_check, int64_t max_checks,
                                             grp_exit *h_out, void *stream) {
  const Range range("grp_run_parallel_phase (Eq. 5)");
  if (!r || !h_out) return fail(GRP_EINVAL, "grp_run_parallel_phase: null argument");
  NOT_SHARDED(r, "grp_run_parallel_phase");
  if (t_check < 1 || max_checks < 1) return fail(GRP_EINVAL, "grp_run_parallel_phase: t_check, max_checks >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  grp_status e = parallel_phase(r, omega, t_check, max_checks, h_out, st);
  grp_status e2 = latch_errors(r, st);
  return e2 != GRP_OK ? e2 : e;
}

extern "C" grp_status grp_broadcast(grp_replicas *r, int32_t src, void *stream) {
  if (!r) return fail(GRP_EINVAL, "grp_broadcast: null handle");
  if (src < 0 || src >= r->R) return fail(GRP_EINVAL, "grp_broadcast: src out of range");
  CU(launch_copy_replica(r->sys->dev, r->R, r->q, r->p, r->f, r->acc, src, -1, 1, (cudaStream_t)stream));
  r->t_phase = 0;
  return GRP_OK;
}

// One exit test of the convergence step: segment with the fused exit test, branching of exited
// workers, Gelman-Rubin ratios when t_phase >= min_fv_steps, and one readback of the status.
static grp_status fv_check(grp_replicas *r, int omega, int t_check, int t_gr, double tol, long long min_fv_steps,
                           grp_fv_status *out, cudaStream_t st) {
  const SysDev &D = r->sys->dev;
  const int R = r->R;
  grp_status e = run_steps(r, t_check, t_gr, R, 1, omega, 0, 0, st);
  if (e != GRP_OK) return e;
  CU(launch_fv_branch(D, R, r->q, r->p, r->f, r->acc, r->exited, r->src, r->n_branched, r->seed, r->t_global, st,
                      r->err));
  const bool want_gr = r->t_phase >= min_fv_steps && R > 1 && D.n_obs > 0;
  if (want_gr) CU(launch_gelman_rubin(D, R, r->acc, tol, r->rhat, nullptr, st));
  // the whole status in one launch and one copy
  CU(launch_collect_status(r->d_run, 1, r->d_status, st));
  CU(cudaMemcpyAsync(r->h_status, r->d_status, sizeof(BatchStatus), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  const BatchStatus &bs = *r->h_status;
  out->ref_exited = bs.exited0;
  out->label0 = bs.label0;
  out->n_branched = bs.n_branched;
  out->gr_evaluated = want_gr ? 1 : 0;
  out->t_phase = r->t_phase;
  out->pad = 0;
  int conv = want_gr ? 1 : 0;
  for (int j = 0; j < GRP_MAX_OBS; ++j) {
    out->rhat[j] = (want_gr && j < D.n_obs) ? bs.rhat[j] : 0.0;
    if (want_gr && j < D.n_obs && !(bs.rhat[j] < 1.0 + tol)) conv = 0;
  }
  out->converged = conv;
  if (bs.err) return latch_errors(r, st);  // a kernel latched an error during this check
  return GRP_OK;
}

extern "C" grp_status grp_fv_check(grp_replicas *r, int32_t omega, int32_t t_check, int32_t t_gr, double tol,
                                   int64_t min_fv_steps, grp_fv_status *h_out, void *stream) {
  const Range range("grp_fv_check (convergence step)");
  if (!r || !h_out) return fail(GRP_EINVAL, "grp_fv_check: null argument");
  NOT_SHARDED(r, "grp_fv_check");
  if (t_check < 1 || t_gr < 0) return fail(GRP_EINVAL, "grp_fv_check: need t_check >= 1, t_gr >= 0");
  return fv_check(r, omega, t_check, t_gr, tol, min_fv_steps, h_out, (cudaStream_t)stream);
}

// ------------------------------------------------------------------------------------------------
// Event log of a run: the host array, its capacity and the clock t_sim (Eq. 6).
struct EventLog {
  grp_event *h;
  int max, n = 0;
  long long tsim = 0;
  void add(int kind, int omega, int to, int k, long long M, long long steps, long long nb) {
    if (n < max) {
      grp_event &e = h[n];
      e.kind = kind; e.omega = omega; e.label_to = to; e.k = k; e.M = M; e.steps = steps;
      e.t_sim = tsim; e.n_branch = nb;
    }
    ++n;
  }
};

// State label of replica 0 and whether it is outside omega.
static grp_status ref_label(grp_replicas *r, int omega, int *label, int *exited, cudaStream_t st) {
  CU(launch_check(r->sys->dev, r->q, 1, omega, r->labels, r->exited, nullptr, 0, st));
  CU(cudaMemcpyAsync(&r->hb->label0, r->labels, 1, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(&r->hb->exited0, r->exited, 1, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  *label = r->hb->label0;
  *exited = r->hb->exited0;
  return GRP_OK;
}

// Transient propagation of the reference walker until a check finds it in a state (Section 2.4.1,
// task 1); *omega = -1 when max_steps came first.
static grp_status transient(grp_replicas *r, int t_check, long long max_steps, EventLog &L, int *omega,
                            cudaStream_t st) {
  long long treach = 0;
  int ex;
  grp_status e = ref_label(r, 0, omega, &ex, st);
  while (e == GRP_OK && *omega < 0 && r->t_global < max_steps) {
    if ((e = run_steps(r, t_check, 0, 1, 0, 0, 0, 0, st)) != GRP_OK) return e;
    treach += t_check;
    e = ref_label(r, 0, omega, &ex, st);
  }
  if (e == GRP_OK && *omega >= 0 && treach > 0) {
    L.tsim += treach;
    L.add(GRP_EV_TRANSIENT, -1, *omega, 0, 0, treach, 0);
  }
  return e;
}

// Parallel dynamics step (Eq. 5) ending a visit of omega; the exit configuration becomes replica 0.
// *found = 0 when max_steps came first.
static grp_status parallel_step(grp_replicas *r, int omega, int t_check, long long max_steps, EventLog &L,
                                int *found, cudaStream_t st) {
  *found = 0;
  const long long left = (max_steps - r->t_global + t_check - 1) / t_check;
  if (left < 1) return GRP_OK;
  grp_exit ex_out{};
  grp_status e = parallel_phase(r, omega, t_check, left, &ex_out, st);
  if (e == GRP_NOEXIT) return GRP_OK;
  if (e != GRP_OK) return e;
  L.tsim += ex_out.tau_steps;
  L.add(GRP_EV_PARALLEL_EXIT, omega, ex_out.label_to, ex_out.k, ex_out.M, ex_out.tau_steps, 0);
  if (ex_out.k != 1) CU(launch_copy_replica(r->sys->dev, r->R, r->q, r->p, r->f, r->acc, ex_out.k - 1, 0, 0, st));
  *found = 1;
  return GRP_OK;
}

extern "C" grp_status grp_run(grp_replicas *r, const grp_run_params *p, grp_event *h_events, int32_t max_events,
                              int32_t *h_n_events, int64_t *h_t_sim, void *stream) {
  const Range range("grp_run (Fig. 1)");
  if (!r || !p || (max_events > 0 && !h_events)) return fail(GRP_EINVAL, "grp_run: null argument");
  NOT_SHARDED(r, "grp_run");
  if (p->t_gr < 1 || p->t_check < 1 || !(p->tol > 0)) return fail(GRP_EINVAL, "grp_run: need t_gr, t_check >= 1, tol > 0");
  cudaStream_t st = (cudaStream_t)stream;
  const SysDev &D = r->sys->dev;
  const int R = r->R;
  int nexit = 0;
  EventLog L{h_events, max_events};
  grp_status e = GRP_OK;
  while (nexit < p->max_exits && r->t_global < p->max_steps && L.n < max_events) {
    // 1. transient propagation of the reference walker
    int omega;
    if ((e = transient(r, p->t_check, p->max_steps, L, &omega, st)) != GRP_OK) return e;
    if (omega < 0) break;
    // 2. convergence step
    CU(launch_copy_replica(D, R, r->q, r->p, r->f, r->acc, 0, -1, 1, st));
    r->t_phase = 0;
    long long nbranch = 0;
    int converged = 0, ref_exit = 0;
    while (r->t_global < p->max_steps) {
      grp_fv_status fs;
      if ((e = fv_check(r, omega, p->t_check, p->t_gr, p->tol, p->min_fv_steps, &fs, st)) != GRP_OK) return e;
      // (a) the reference walker left omega: the F-V workers are discarded
      if (fs.ref_exited) {
        L.tsim += r->t_phase;
        L.add(GRP_EV_REF_EXIT, omega, fs.label0, 0, 0, r->t_phase, nbranch);
        ++nexit;
        ref_exit = 1;
        break;
      }
      // (b) branching (done on the device)
      if (fs.n_branched > 0 && fs.n_branched == R - 1)
        L.add(GRP_EV_FV_ALL_EXITED, omega, omega, 0, 0, r->t_phase, fs.n_branched);
      nbranch += fs.n_branched;
      // (c) Gelman-Rubin test, Eq. 4
      if (fs.gr_evaluated && fs.converged) { converged = 1; break; }
    }
    if (ref_exit) continue;
    if (!converged) break;
    L.tsim += r->t_phase;
    L.add(GRP_EV_FV_CONVERGED, omega, omega, 0, 0, r->t_phase, nbranch);
    // 3. parallel dynamics step
    int found;
    if ((e = parallel_step(r, omega, p->t_check, p->max_steps, L, &found, st)) != GRP_OK) return e;
    if (!found) break;
    ++nexit;
  }
  if (h_n_events) *h_n_events = std::min(L.n, max_events);
  if (h_t_sim) *h_t_sim = L.tsim;
  return latch_errors(r, st);
}

// ------------------------------------------------------------------------------------------------
// Original ParRep (Section 2.4.3).  Device scratch of one call: the samples (slot r the dephased
// state of replica r, slot R the decorrelated reference), each replica's stay, done flags, counters.
struct DephaseScratch {
  double *sq = nullptr, *sp = nullptr, *sf = nullptr;
  long long *stay = nullptr;
  uint8_t *done = nullptr;
  int *cnt = nullptr;
  ~DephaseScratch() {
    cudaFree(sq); cudaFree(sp); cudaFree(sf); cudaFree(stay); cudaFree(done); cudaFree(cnt);
  }
};

// Dephasing of one visit: returns in *dsteps the steps it took (all replicas in lockstep), in
// *restarts the restarts from the decorrelated reference, *ok = 0 when max_steps came first.
static grp_status dephase(grp_replicas *r, int omega, const grp_original_params *p, DephaseScratch &S,
                          long long *dsteps, long long *restarts, int *ok, cudaStream_t st) {
  const SysDev &D = r->sys->dev;
  const int R = r->R;
  const size_t row = (size_t)D.nd * 8;
  const size_t ref = row / 8 * (size_t)R;
  CU(cudaMemcpyAsync(S.sq + ref, r->q, row, cudaMemcpyDeviceToDevice, st));
  CU(cudaMemcpyAsync(S.sp + ref, r->p, row, cudaMemcpyDeviceToDevice, st));
  CU(cudaMemcpyAsync(S.sf + ref, r->f, row, cudaMemcpyDeviceToDevice, st));
  CU(launch_copy_replica(D, R, r->q, r->p, r->f, r->acc, 0, -1, 1, st));
  CU(cudaMemsetAsync(S.stay, 0, sizeof(long long) * R, st));
  CU(cudaMemsetAsync(S.done, 0, R, st));
  CU(cudaMemsetAsync(S.cnt, 0, 2 * sizeof(int), st));
  r->t_phase = 0;
  *dsteps = 0;
  *restarts = 0;
  int n_done = 0;
  while (n_done < R && r->t_global < p->max_steps) {
    grp_status e = run_steps(r, p->t_check, 0, R, 1, omega, 0, 0, st);
    if (e != GRP_OK) return e;
    *dsteps += p->t_check;
    CU(launch_dephase(D, R, r->q, r->p, r->f, S.sq, S.sp, S.sf, r->exited, S.stay, S.done, p->t_check,
                      p->t_phase, S.cnt, st));
    CU(cudaMemcpyAsync(r->hb->dephase, S.cnt, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&r->hb->err, r->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (r->hb->err) return latch_errors(r, st);
    n_done = r->hb->dephase[0];
    *restarts = r->hb->dephase[1];
  }
  *ok = n_done == R;
  if (!*ok) return GRP_OK;
  const size_t all = row * (size_t)R;
  CU(cudaMemcpyAsync(r->q, S.sq, all, cudaMemcpyDeviceToDevice, st));
  CU(cudaMemcpyAsync(r->p, S.sp, all, cudaMemcpyDeviceToDevice, st));
  CU(cudaMemcpyAsync(r->f, S.sf, all, cudaMemcpyDeviceToDevice, st));
  return GRP_OK;
}

static grp_status run_original(grp_replicas *r, const grp_original_params *p, EventLog &L, DephaseScratch &S,
                               cudaStream_t st) {
  int nexit = 0;
  grp_status e = GRP_OK;
  while (nexit < p->max_exits && r->t_global < p->max_steps && L.n < L.max) {
    // 1. transient propagation of the reference walker
    int omega;
    if ((e = transient(r, p->t_check, p->max_steps, L, &omega, st)) != GRP_OK) return e;
    if (omega < 0) break;
    // 2. decorrelation: replica 0 alone, checked every t_check, must stay t_corr steps in omega
    long long d = 0;
    int ref_exit = 0;
    while (d < p->t_corr && r->t_global < p->max_steps) {
      if ((e = run_steps(r, p->t_check, 0, 1, 0, 0, 0, 0, st)) != GRP_OK) return e;
      d += p->t_check;
      int label, ex;
      if ((e = ref_label(r, omega, &label, &ex, st)) != GRP_OK) return e;
      if (ex) {
        L.tsim += d;
        L.add(GRP_EV_REF_EXIT, omega, label, 0, 0, d, 0);
        ++nexit;
        ref_exit = 1;
        break;
      }
    }
    if (ref_exit) continue;
    if (d < p->t_corr) break;
    L.tsim += d;
    L.add(GRP_EV_DECORRELATED, omega, omega, 0, 0, d, 0);
    // 3. dephasing (not counted in the clock)
    long long dsteps, restarts;
    int ok;
    if ((e = dephase(r, omega, p, S, &dsteps, &restarts, &ok, st)) != GRP_OK) return e;
    if (!ok) break;
    L.add(GRP_EV_DEPHASED, omega, omega, 0, 0, dsteps, restarts);
    // 4. parallel dynamics step
    int found;
    if ((e = parallel_step(r, omega, p->t_check, p->max_steps, L, &found, st)) != GRP_OK) return e;
    if (!found) break;
    ++nexit;
  }
  return GRP_OK;
}

extern "C" grp_status grp_run_original(grp_replicas *r, const grp_original_params *p, grp_event *h_events,
                                       int32_t max_events, int32_t *h_n_events, int64_t *h_t_sim, void *stream) {
  const Range range("grp_run_original (Section 2.4.3)");
  if (!r || !p || (max_events > 0 && !h_events)) return fail(GRP_EINVAL, "grp_run_original: null argument");
  NOT_SHARDED(r, "grp_run_original");
  if (p->t_check < 1 || p->t_corr < 0 || p->t_phase < 0)
    return fail(GRP_EINVAL, "grp_run_original: need t_check >= 1, t_corr >= 0, t_phase >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t R = (size_t)r->R, bytes = (R + 1) * (size_t)r->sys->dev.nd * 8;
  DephaseScratch S;
  if (cudaMalloc(&S.sq, bytes) != cudaSuccess || cudaMalloc(&S.sp, bytes) != cudaSuccess ||
      cudaMalloc(&S.sf, bytes) != cudaSuccess || cudaMalloc(&S.stay, R * sizeof(long long)) != cudaSuccess ||
      cudaMalloc(&S.done, R) != cudaSuccess || cudaMalloc(&S.cnt, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(GRP_ENOMEM, "grp_run_original: cudaMalloc of the dephasing samples (%zu bytes) failed", 3 * bytes);
  }
  EventLog L{h_events, max_events};
  grp_status e = run_original(r, p, L, S, st);
  if (e == GRP_OK) {
    if (h_n_events) *h_n_events = std::min(L.n, max_events);
    if (h_t_sim) *h_t_sim = L.tsim;
  }
  cudaStreamSynchronize(st);  // the scratch is freed below: nothing may still use it
  grp_status e2 = latch_errors(r, st);
  return e != GRP_OK ? e : e2;
}

// ------------------------------------------------------------------------------------------------
// The loop of Fig. 1 for every run of a batch, each run in its own phase: one batched segment of
// t_check steps per tick (replica 0 alone for a transient, every replica for a convergence or a
// parallel step, none for a finished run), then batched branching and Gelman-Rubin ratios for the
// runs in their convergence step and one readback of all statuses.  Each run's decisions and event
// log are those of grp_run on that run alone.
namespace {
struct RunLoop {
  enum Phase { kTransient, kFv, kParallel, kDone } phase = kTransient;
  int omega = -1, nexit = 0;
  long long treach = 0, nbranch = 0, M = 0, left = 0;
  EventLog L{nullptr, 0};
};
}  // namespace

extern "C" grp_status grp_batch_run(grp_batch *b, const grp_run_params *p, grp_event *h_events, int32_t max_events,
                                    int32_t *h_n_events, int64_t *h_t_sim, void *stream) {
  const Range range("grp_batch_run (Fig. 1, every run)");
  if (!b || !p || (max_events > 0 && !h_events)) return fail(GRP_EINVAL, "grp_batch_run: null argument");
  if (p->t_gr < 1 || p->t_check < 1 || p->t_check > kMaxSegment || !(p->tol > 0))
    return fail(GRP_EINVAL, "grp_batch_run: need t_gr >= 1, t_check in [1, %lld], tol > 0", kMaxSegment);
  cudaStream_t st = (cudaStream_t)stream;
  const int nr = (int)b->runs.size();
  std::vector<RunLoop> run(nr);
  for (int i = 0; i < nr; ++i) run[i].L = EventLog{h_events ? h_events + (size_t)i * max_events : nullptr, max_events};

  auto finish = [&](int i) { run[i].phase = RunLoop::kDone; };
  // a new visit from the current configuration of replica 0, whose state label is `label`
  auto begin_fv = [&](int i, int omega) -> grp_status {
    grp_replicas *r = b->runs[i];
    CU(launch_copy_replica(r->sys->dev, r->R, r->q, r->p, r->f, r->acc, 0, -1, 1, st));
    r->t_phase = 0;
    run[i].omega = omega;
    run[i].nbranch = 0;
    run[i].phase = RunLoop::kFv;
    return GRP_OK;
  };
  auto start_visit = [&](int i, int label) -> grp_status {
    RunLoop &u = run[i];
    const grp_replicas *r = b->runs[i];
    if (!(u.nexit < p->max_exits && r->t_global < p->max_steps && u.L.n < max_events)) { finish(i); return GRP_OK; }
    u.treach = 0;
    if (label >= 0) return begin_fv(i, label);
    u.phase = RunLoop::kTransient;
    return GRP_OK;
  };

  // the label of every run's replica 0 before the first tick
  for (int i = 0; i < nr; ++i) {
    grp_replicas *r = b->runs[i];
    CU(launch_check(r->sys->dev, r->q, 1, 0, r->labels, r->exited, nullptr, 0, st));
    CU(cudaMemcpyAsync(&r->hb->label0, r->labels, 1, cudaMemcpyDeviceToHost, st));
  }
  CU(cudaStreamSynchronize(st));
  grp_status e = GRP_OK;
  for (int i = 0; i < nr && e == GRP_OK; ++i) e = start_visit(i, b->runs[i]->hb->label0);
  if (e != GRP_OK) return e;

  std::vector<RunTick> ticks(nr);
  std::vector<int> branch(nr), gr(nr);
  TickGraph tick;
  bool graphs = true;
  long long n_ticks = 0;
  b->ticks = b->graph_ticks = 0;
  for (;;) {
    int busy = 0;
    for (int i = 0; i < nr; ++i) {
      RunLoop &u = run[i];
      grp_replicas *r = b->runs[i];
      // the convergence step runs while t_global < max_steps (as in grp_run)
      if (u.phase == RunLoop::kFv && r->t_global >= p->max_steps) finish(i);
      RunTick t{0, 0, 1, 0, 0, 0};
      branch[i] = gr[i] = 0;
      if (u.phase == RunLoop::kTransient) {
        t.n_active = 1;
      } else if (u.phase == RunLoop::kFv) {
        t = RunTick{r->R, p->t_gr, 1, u.omega, 0, 0};
        branch[i] = 1;
        gr[i] = (r->t_phase + p->t_check >= p->min_fv_steps && r->R > 1 && r->sys->dev.n_obs > 0) ? 1 : 0;
      } else if (u.phase == RunLoop::kParallel) {
        t = RunTick{r->R, 0, 1, u.omega, 1, ++u.M};
      }
      ticks[i] = t;
      busy += t.n_active > 0;
    }
    if (!busy) break;
    // the first tick runs node by node (it also sets the kernels' attributes); the graph is captured
    // before the second and replayed from then on
    if (graphs && n_ticks == 1 && !tick.capture(b)) graphs = false;
    fill_args(b, p->t_check, ticks.data());
    fill_arrays(b, branch.data(), gr.data());
    if (graphs && tick.exec) {
      CU(cudaGraphLaunch(tick.exec, st));
      ++b->graph_ticks;
    } else {
      if ((e = enqueue_segment(b, st)) != GRP_OK) return e;
      if ((e = enqueue_status(b, st)) != GRP_OK) return e;
    }
    CU(cudaStreamSynchronize(st));
    ++n_ticks;
    ++b->ticks;
    for (int i = 0; i < nr; ++i) {
      if (b->h_status[i].err && (e = latch_errors(b->runs[i], st)) != GRP_OK) return e;
    }
    for (int i = 0; i < nr; ++i) {
      RunLoop &u = run[i];
      grp_replicas *r = b->runs[i];
      const BatchStatus &s = b->h_status[i];
      if (ticks[i].n_active == 0) continue;
      if (u.phase == RunLoop::kTransient) {
        u.treach += p->t_check;
        if (s.label0 >= 0) {
          if (u.treach > 0) {
            u.L.tsim += u.treach;
            u.L.add(GRP_EV_TRANSIENT, -1, s.label0, 0, 0, u.treach, 0);
          }
          if ((e = begin_fv(i, s.label0)) != GRP_OK) return e;
        } else if (r->t_global >= p->max_steps) {
          finish(i);
        }
      } else if (u.phase == RunLoop::kFv) {
        if (s.exited0) {  // the reference walker left omega: the F-V workers are discarded
          u.L.tsim += r->t_phase;
          u.L.add(GRP_EV_REF_EXIT, u.omega, s.label0, 0, 0, r->t_phase, u.nbranch);
          ++u.nexit;
          if ((e = start_visit(i, s.label0)) != GRP_OK) return e;
          continue;
        }
        if (s.n_branched > 0 && s.n_branched == r->R - 1)
          u.L.add(GRP_EV_FV_ALL_EXITED, u.omega, u.omega, 0, 0, r->t_phase, s.n_branched);
        u.nbranch += s.n_branched;
        int conv = gr[i];
        for (int j = 0; j < r->sys->dev.n_obs && conv; ++j) conv = s.rhat[j] < 1.0 + p->tol;
        if (conv) {
          u.L.tsim += r->t_phase;
          u.L.add(GRP_EV_FV_CONVERGED, u.omega, u.omega, 0, 0, r->t_phase, u.nbranch);
          u.left = (p->max_steps - r->t_global + p->t_check - 1) / p->t_check;
          if (u.left < 1) { finish(i); continue; }
          CU(cudaMemsetAsync(r->exit_key, 0xff, 8, st));
          u.M = 0;
          u.phase = RunLoop::kParallel;
        }
      } else if (u.phase == RunLoop::kParallel) {
        if (s.exit_key != ~0ull) {
          const int k0 = (int)(s.exit_key & 0xffffffffu);
          const long long tau = ((long long)r->R * (u.M - 1) + (k0 + 1)) * (long long)p->t_check;
          u.L.tsim += tau;
          u.L.add(GRP_EV_PARALLEL_EXIT, u.omega, s.label_k, k0 + 1, u.M, tau, 0);
          ++u.nexit;
          // the exit configuration becomes the reference walker
          if (k0 != 0) CU(launch_copy_replica(r->sys->dev, r->R, r->q, r->p, r->f, r->acc, k0, 0, 0, st));
          if ((e = start_visit(i, s.label_k)) != GRP_OK) return e;
        } else if (u.M >= u.left) {
          finish(i);
        }
      }
    }
  }
  for (int i = 0; i < nr; ++i) {
    if (h_n_events) h_n_events[i] = std::min(run[i].L.n, max_events);
    if (h_t_sim) h_t_sim[i] = run[i].L.tsim;
  }
  for (int i = 0; i < nr; ++i)
    if ((e = latch_errors(b->runs[i], st)) != GRP_OK) return e;
  return GRP_OK;
}

// ------------------------------------------------------------------------------------------------
extern "C" grp_status grp_get_state(grp_replicas *r, double *h_q, double *h_p, double *h_acc, grp_counters *h_ctr,
                                    void *stream) {
  if (!r) return fail(GRP_EINVAL, "grp_get_state: null handle");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nd = (size_t)r->sys->dev.nd * r->R, na = (size_t)r->sys->dev.n_obs * 4 * r->R;
  if (h_q) CU(cudaMemcpyAsync(h_q, r->q, nd * 8, cudaMemcpyDeviceToHost, st));
  if (h_p) CU(cudaMemcpyAsync(h_p, r->p, nd * 8, cudaMemcpyDeviceToHost, st));
  if (h_acc && na) CU(cudaMemcpyAsync(h_acc, r->acc, na * 8, cudaMemcpyDeviceToHost, st));
  if (h_ctr) { h_ctr->t_global = r->t_global; h_ctr->t_phase = r->t_phase; }
  return latch_errors(r, st);
}

extern "C" grp_status grp_set_state(grp_replicas *r, const double *h_q, const double *h_p, const double *h_acc,
                                    const grp_counters *h_ctr, void *stream) {
  if (!r) return fail(GRP_EINVAL, "grp_set_state: null handle");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nd = (size_t)r->sys->dev.nd * r->R, na = (size_t)r->sys->dev.n_obs * 4 * r->R;
  if (h_q) CU(cudaMemcpyAsync(r->q, h_q, nd * 8, cudaMemcpyHostToDevice, st));
  if (h_p) CU(cudaMemcpyAsync(r->p, h_p, nd * 8, cudaMemcpyHostToDevice, st));
  if (h_acc && na) CU(cudaMemcpyAsync(r->acc, h_acc, na * 8, cudaMemcpyHostToDevice, st));
  if (h_ctr) {
    if (h_ctr->t_global < 0 || h_ctr->t_phase < 0) return fail(GRP_EINVAL, "grp_set_state: negative counters");
    r->t_global = h_ctr->t_global;
    r->t_phase = h_ctr->t_phase;
  }
  if (h_q) {
    grp_status e = compute_forces(r, st);
    if (e != GRP_OK) return e;
  }
  return latch_errors(r, st);
}

// ------------------------------------------------------------------------------------------------
// Runs sharded over several processes (Section 3.1 distributes the replicas over processes).
extern "C" grp_status grp_set_shard(grp_replicas *r, int32_t first, int32_t n_global) {
  if (!r) return fail(GRP_EINVAL, "grp_set_shard: null handle");
  if (first < 0 || n_global < 1 || (long long)first + r->R > n_global)
    return fail(GRP_EINVAL, "grp_set_shard: need 0 <= first and first + R <= n_global (first %d, R %d, n_global %d)",
                first, r->R, n_global);
  r->rep0 = first;
  r->n_global = n_global;
  return GRP_OK;
}

extern "C" grp_status grp_fv_plan(grp_replicas *r, const uint8_t *d_exited_global, int32_t *d_src, void *stream) {
  if (!r || !d_exited_global || !d_src) return fail(GRP_EINVAL, "grp_fv_plan: null argument");
  CU(launch_fv_plan(r->R, r->rep0, r->n_global, d_exited_global, d_src, r->seed, r->t_global, (cudaStream_t)stream));
  return GRP_OK;
}

static grp_status pack_rows(grp_replicas *r, int32_t n, const int32_t *d_idx, double *d_buf, int unpack,
                            const char *name, cudaStream_t st) {
  if (!r || n < 0 || (n > 0 && (!d_idx || !d_buf))) return fail(GRP_EINVAL, "%s: bad argument", name);
  CU(launch_pack_rows(r->sys->dev, r->R, r->q, r->p, r->f, r->acc, n, d_idx, d_buf, unpack, r->err, st));
  return GRP_OK;
}

extern "C" grp_status grp_pack_rows(grp_replicas *r, int32_t n, const int32_t *d_idx, double *d_buf, void *stream) {
  return pack_rows(r, n, d_idx, d_buf, 0, "grp_pack_rows", (cudaStream_t)stream);
}

extern "C" grp_status grp_unpack_rows(grp_replicas *r, int32_t n, const int32_t *d_idx, const double *d_buf,
                                      void *stream) {
  return pack_rows(r, n, d_idx, const_cast<double *>(d_buf), 1, "grp_unpack_rows", (cudaStream_t)stream);
}

extern "C" grp_status grp_gr_partials(grp_replicas *r, int32_t pass, const double *h_sums1, double *h_out,
                                      void *stream) {
  if (!r || !h_out || (pass != 1 && pass != 2) || (pass == 2 && !h_sums1))
    return fail(GRP_EINVAL, "grp_gr_partials: need pass 1, or pass 2 with the summed pass-1 sums, and h_out");
  cudaStream_t st = (cudaStream_t)stream;
  const SysDev &D = r->sys->dev;
  GrGrand g{};
  if (pass == 2)
    for (int j = 0; j < D.n_obs; ++j) {
      const double nw = h_sums1[3 * j + 1] + h_sums1[3 * j + 2];
      g.v[j] = nw > 0 ? h_sums1[3 * j] / nw : 0.0;
    }
  CU(launch_gr_partials(D, r->R, r->rep0, r->acc, pass, g, r->d_gr, st));
  const size_t bytes = sizeof(double) * (size_t)D.n_obs * (pass == 1 ? 3 : 2);
  if (bytes) CU(cudaMemcpyAsync(h_out, r->d_gr, bytes, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return latch_errors(r, st);
}

extern "C" grp_status grp_gr_combine(int32_t n_obs, const double *h_sums1, const double *h_sums2, double tol,
                                     double *h_rhat, int32_t *h_converged) {
  if (n_obs < 0 || n_obs > GRP_MAX_OBS || (n_obs > 0 && (!h_sums1 || !h_sums2)))
    return fail(GRP_EINVAL, "grp_gr_combine: bad argument");
  int conv = n_obs > 0 ? 1 : 0;
  for (int j = 0; j < n_obs; ++j) {
    const double good = h_sums1[3 * j + 1], bad = h_sums1[3 * j + 2], nw = good + bad;
    const double B = h_sums2[2 * j] / nw, W = h_sums2[2 * j + 1] / nw;
    const double R = (nw < 1 || bad > 0 || !(W > 0)) ? INFINITY : 1.0 + B / W;
    if (h_rhat) h_rhat[j] = R;
    if (!(R < 1.0 + tol)) conv = 0;
  }
  if (h_converged) *h_converged = conv;
  return GRP_OK;
}

extern "C" grp_status grp_get_device_view(grp_replicas *r, grp_device_view *out) {
  if (!r || !out) return fail(GRP_EINVAL, "grp_get_device_view: null argument");
  out->q = r->q; out->p = r->p; out->f = r->f; out->acc = r->acc;
  out->labels = r->labels; out->exited = r->exited;
  return GRP_OK;
}

extern "C" grp_status grp_energy_forces(grp_system *s, int32_t n_conf, const double *d_q, double *d_energy,
                                        double *d_forces, void *stream) {
  if (!s || !d_q || n_conf < 0) return fail(GRP_EINVAL, "grp_energy_forces: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  int *err = nullptr;
  CU(cudaMallocAsync((void **)&err, 4, st));
  CU(cudaMemsetAsync(err, 0, 4, st));
  CU(launch_energy_forces(s->dev, n_conf, d_q, d_energy, d_forces, err, st));
  int h = 0;
  CU(cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  CU(cudaFreeAsync(err, st));
  if (h & kErrOverflow) return fail(GRP_EOVERFLOW, "force contribution outside the fixed-point range");
  return GRP_OK;
}

// ------------------------------------------------------------------------------------------------
// Differentiation with respect to positions and force-field parameters.
extern "C" grp_status grp_param_count(const grp_system *s, int32_t *h_n_theta) {
  if (!s || !h_n_theta) return fail(GRP_EINVAL, "grp_param_count: null argument");
  *h_n_theta = s->dev.potential == GRP_POT_FORCE_FIELD ? 2 * s->dev.n + s->n_terms : 0;
  return GRP_OK;
}

extern "C" grp_status grp_get_params(const grp_system *s, double *d_theta, void *stream) {
  if (!s || !d_theta) return fail(GRP_EINVAL, "grp_get_params: null argument");
  if (s->dev.potential != GRP_POT_FORCE_FIELD) return fail(GRP_EINVAL, "grp_get_params: no force-field parameters");
  const size_t nt = 2 * (size_t)s->dev.n + s->n_terms;
  CU(cudaMemcpyAsync(d_theta, s->theta, nt * 8, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return GRP_OK;
}

extern "C" grp_status grp_set_params(grp_system *s, const double *d_theta, void *stream) {
  if (!s || !d_theta) return fail(GRP_EINVAL, "grp_set_params: null argument");
  if (s->dev.potential != GRP_POT_FORCE_FIELD) return fail(GRP_EINVAL, "grp_set_params: no force-field parameters");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nt = 2 * (size_t)s->dev.n + s->n_terms;
  int *bad = nullptr;
  CU(cudaMallocAsync((void **)&bad, 4, st));
  CU(launch_set_params(s->dev, s->n_terms, d_theta, bad, st));
  int h = 0;
  CU(cudaMemcpyAsync(&h, bad, 4, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  CU(cudaFreeAsync(bad, st));
  if (h) return fail(GRP_EINVAL, "grp_set_params: sigma must be > 0, epsilon >= 0 and every value finite");
  CU(cudaMemcpyAsync(s->theta, d_theta, nt * 8, cudaMemcpyDeviceToDevice, st));
  return GRP_OK;
}

extern "C" grp_status grp_energy_grad(grp_system *s, int32_t n_conf, const double *d_q, const double *d_w,
                                      double *d_energy, double *d_grad_q, double *d_grad_theta, void *stream) {
  if (!s || !d_q || n_conf < 0) return fail(GRP_EINVAL, "grp_energy_grad: bad argument");
  if (d_grad_theta && s->dev.potential != GRP_POT_FORCE_FIELD)
    return fail(GRP_EINVAL, "grp_energy_grad: no force-field parameters to differentiate");
  if (s->dev.coulomb_rf == 2) return fail(GRP_ENOTIMPL, "grp_energy_grad: periodic systems are not differentiated");
  cudaStream_t st = (cudaStream_t)stream;
  const int nt = 2 * s->dev.n + s->n_terms;
  if (d_grad_theta && (size_t)nt * 8 > kMaxSmem)
    return fail(GRP_ENOTIMPL, "grp_energy_grad: %d parameters exceed one block's shared memory", nt);
  if (n_conf == 0) {
    if (d_grad_theta) CU(cudaMemsetAsync(d_grad_theta, 0, (size_t)nt * 8, st));
    return GRP_OK;
  }
  int *err = nullptr;
  double *partial = nullptr;
  CU(cudaMallocAsync((void **)&err, 4, st));
  CU(cudaMemsetAsync(err, 0, 4, st));
  if (d_energy || d_grad_q) CU(launch_energy_forces(s->dev, n_conf, d_q, d_energy, d_grad_q, err, st));
  if (d_grad_theta) {
    CU(cudaMallocAsync((void **)&partial, (size_t)n_conf * nt * 8, st));
    CU(launch_param_grad(s->dev, s->n_terms, n_conf, d_q, d_w, d_grad_q, partial, err, st));
    CU(launch_column_sum(partial, n_conf, nt, d_grad_theta, st));
    CU(cudaFreeAsync(partial, st));
  } else if (d_grad_q) {
    CU(launch_scale_rows(d_grad_q, n_conf, s->dev.nd, d_w, -1.0, st));
  }
  int h = 0;
  CU(cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  CU(cudaFreeAsync(err, st));
  if (h) return fail(GRP_EOVERFLOW, "grp_energy_grad: a term outside the fixed-point range or not finite");
  return GRP_OK;
}

extern "C" grp_status grp_adjoint_segment(grp_replicas *r, int32_t k, int32_t t_gr, int32_t checkpoint,
                                          const grp_loss *loss, double *h_loss, double *d_grad_theta,
                                          double *d_grad_q0, double *d_grad_p0, void *stream) {
  const Range range("grp_adjoint_segment");
  if (!r || !loss || k < 1 || t_gr < 1 || checkpoint < 1 || k > (1 << 30))
    return fail(GRP_EINVAL, "grp_adjoint_segment: bad argument");
  const grp_system *s = r->sys;
  const SysDev &D = s->dev;
  if (D.potential != GRP_POT_FORCE_FIELD || D.tiled || D.gb || D.n_cons || D.coulomb_rf == 2)
    return fail(GRP_ENOTIMPL, "grp_adjoint_segment: needs a force-field system of fewer than 64 atoms in vacuum");
  if (loss->obs < 0 || loss->obs >= D.n_obs) return fail(GRP_EINVAL, "grp_adjoint_segment: bad observable index");
  const int kind = D.obs_kind[loss->obs];
  if (kind != GRP_OBS_COORD && kind != GRP_OBS_GROUP_DISTANCE && kind != GRP_OBS_DIHEDRAL)
    return fail(GRP_ENOTIMPL, "grp_adjoint_segment: the loss observable must be a coordinate, a group distance or a dihedral");
  if (loss->transform != GRP_LOSS_IDENTITY && loss->transform != GRP_LOSS_LOGISTIC)
    return fail(GRP_EINVAL, "grp_adjoint_segment: unknown transform");
  if (loss->transform == GRP_LOSS_LOGISTIC && !(loss->width > 0))
    return fail(GRP_EINVAL, "grp_adjoint_segment: logistic width must be > 0");
  const long long n_s = (r->t_phase + k) / t_gr - r->t_phase / t_gr;
  if (n_s < 1) return fail(GRP_EINVAL, "grp_adjoint_segment: no sampling step in the segment");
  const int ck = std::min(checkpoint, k);
  if (adjoint_smem_bytes(D, s->n_terms, ck) > 180 * 1024)
    return fail(GRP_EINVAL, "grp_adjoint_segment: checkpoint interval %d needs too much shared memory", ck);
  cudaStream_t st = (cudaStream_t)stream;
  const int R = r->R, nd = D.nd, nt = 2 * D.n + s->n_terms;
  const int n_ck = (k + ck - 1) / ck;
  AdjArgs a{};
  a.S = D;
  a.n_ck = n_ck;
  a.ck = ck;
  a.k = k;
  a.seed = r->seed;
  a.t_global0 = r->t_global;
  a.t_phase0 = r->t_phase;
  a.t_gr = t_gr;
  a.obs_kind = kind;
  for (int t = 0; t < 4; ++t) a.obs_arg[t] = D.obs_arg[loss->obs][t];
  a.transform = loss->transform;
  a.center = loss->center;
  a.width = loss->width;
  a.inv_norm = 1.0 / ((double)R * (double)n_s);
  a.h = 0.5 * D.dt;
  a.c1 = std::exp(-D.gamma * D.dt);
  a.n_terms = s->n_terms;
  a.grad_q0 = d_grad_q0;
  a.grad_p0 = d_grad_p0;
  double *ckpt = nullptr, *partial = nullptr, *lossr = nullptr, *lsum = nullptr;
  int *err = nullptr;
  auto release = [&]() {
    if (ckpt) cudaFreeAsync(ckpt, st);
    if (partial) cudaFreeAsync(partial, st);
    if (lossr) cudaFreeAsync(lossr, st);
    if (lsum) cudaFreeAsync(lsum, st);
    if (err) cudaFreeAsync(err, st);
  };
#define CUA(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      release();                                                                                    \
      return fail(GRP_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));                       \
    }                                                                                               \
  } while (0)
  CUA(cudaMallocAsync((void **)&ckpt, (size_t)R * n_ck * 3 * nd * 8, st));
  CUA(cudaMallocAsync((void **)&partial, (size_t)R * nt * 8, st));
  CUA(cudaMallocAsync((void **)&lossr, (size_t)R * 8, st));
  CUA(cudaMallocAsync((void **)&lsum, 8, st));
  CUA(cudaMallocAsync((void **)&err, 4, st));
  CUA(cudaMemsetAsync(err, 0, 4, st));
  // forces of the current parameters at the starting configurations
  {
    const grp_status e = compute_forces(r, st);
    if (e != GRP_OK) { release(); return e; }
  }
  // forward pass: save (q, p, f) of every replica before each block of ck steps, then advance it
  const size_t pitch = (size_t)n_ck * 3 * nd * 8;
  for (int c = 0; c < n_ck; ++c) {
    const double *src[3] = {r->q, r->p, r->f};
    for (int x = 0; x < 3; ++x)
      CUA(cudaMemcpy2DAsync(ckpt + ((size_t)c * 3 + x) * nd, pitch, src[x], (size_t)nd * 8, (size_t)nd * 8, R,
                            cudaMemcpyDeviceToDevice, st));
    const grp_status e = run_steps(r, std::min(ck, k - c * ck), 0, R, 0, 0, 0, 0, st);
    if (e != GRP_OK) { release(); return e; }
  }
  a.ckpt = ckpt;
  a.partial = partial;
  a.loss = lossr;
  a.err = err;
  CUA(launch_adjoint(a, R, st));
  if (d_grad_theta) CUA(launch_column_sum(partial, R, nt, d_grad_theta, st));
  CUA(launch_column_sum(lossr, R, 1, lsum, st));
  double hl = 0.0;
  int he = 0;
  CUA(cudaMemcpyAsync(&hl, lsum, 8, cudaMemcpyDeviceToHost, st));
  CUA(cudaMemcpyAsync(&he, err, 4, cudaMemcpyDeviceToHost, st));
  CUA(cudaStreamSynchronize(st));
  release();
#undef CUA
  if (he) return fail(GRP_EOVERFLOW, "grp_adjoint_segment: a term outside the fixed-point range or not finite");
  if (h_loss) *h_loss = hl;
  return latch_errors(r, st);
}

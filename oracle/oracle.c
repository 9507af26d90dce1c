/*
 * Oracle for Gen. ParRep dynamics — TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain FP64 C, no blocking, fusion or reordering beyond what the definitions state.  Each function
 * names the passage of the paper (Hedin & Lelievre, gen.parRep) or the published method it follows.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct orc_ctx {
  orc_system s;
  uint8_t *excluded; /* [n][n] 1 when the nonbonded pair is excluded */
  int64_t unconverged; /* SHAKE or RATTLE projections that ran out of sweeps (the state goes on) */
};

orc_ctx *orc_create(const orc_system *sys) {
  orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  if (!c) return NULL;
  c->s = *sys;
  int n = sys->n_atoms;
  c->excluded = (uint8_t *)calloc((size_t)n * (size_t)n, 1);
  if (!c->excluded) { free(c); return NULL; }
  for (int e = 0; e < sys->n_excl; ++e) {
    int i = sys->excl[2 * e], j = sys->excl[2 * e + 1];
    c->excluded[(size_t)i * n + j] = 1;
    c->excluded[(size_t)j * n + i] = 1;
  }
  return c;
}

int64_t orc_unconverged(const orc_ctx *c) { return c->unconverged; }

void orc_destroy(orc_ctx *c) {
  if (!c) return;
  free(c->excluded);
  free(c);
}

/* ---------------------------------------------------------------- vector helpers (3-D) */
static void sub3(const double *a, const double *b, double *r) { r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* Dihedral angle of atoms (i, j, k, l) in radians, (-pi, pi]: the signed angle between the planes
 * (i, j, k) and (j, k, l), positive for a right-handed rotation about j->k. */
static double dihedral_angle(const double *qi, const double *qj, const double *qk, const double *ql) {
  double b1[3], b2[3], b3[3], n1[3], n2[3];
  sub3(qj, qi, b1); sub3(qk, qj, b2); sub3(ql, qk, b3);
  cross3(b1, b2, n1); cross3(b2, b3, n2);
  return atan2(norm3(b2) * dot3(b1, n2), dot3(n1, n2));
}

static void group_com(const orc_ctx *c, int g, const double *q, double *com) {
  const orc_system *s = &c->s;
  double mt = 0, acc[3] = {0, 0, 0};
  for (int t = s->group_offsets[g]; t < s->group_offsets[g + 1]; ++t) {
    int a = s->group_atoms[t];
    double m = s->mass[a];
    mt += m;
    for (int d = 0; d < 3; ++d) acc[d] += m * q[3 * a + d];
  }
  for (int d = 0; d < 3; ++d) com[d] = acc[d] / mt;
}

/* Reaction-field constants (eps_r = 1): k_rf = (eps_rf - 1) / ((2 eps_rf + 1) r_c^3) and
 * c_rf = 1/r_c + k_rf r_c^2, so that the pair energy k_e q_i q_j (1/r + k_rf r^2 - c_rf) vanishes at
 * the cutoff r_c; eps_rf = 0 stands for a conductor (eps_rf -> infinity, k_rf = 1 / (2 r_c^3)). */
static void rf_constants(const orc_system *s, double *krf, double *crf) {
  const double rc = s->cutoff, er = s->rf_dielectric;
  *krf = (er == 0.0 ? 0.5 : (er - 1.0) / (2.0 * er + 1.0)) / (rc * rc * rc);
  *crf = 1.0 / rc + *krf * rc * rc;
}

/* ---------------------------------------------------------------- Generalized Born, OBC model II
 * Each atom i has an offset radius a_i = rho_i - 0.009 nm.  Atom j, a sphere of radius s_j = S_j a_j
 * at distance r, descreens atom i by h_ij = 2 x (1/4 pi) x the integral of |x|^-4 over the part of that
 * sphere outside the sphere of radius a_i around atom i (the pairwise approximation of Hawkins, Cramer
 * and Truhlar).  With L = max(a_i, |r - s_j|) and U = r + s_j, for a_i < U:
 *   h = 1/L - 1/U + (r/4)(1/U^2 - 1/L^2) + (1/2r) ln(L/U) + (s_j^2/4r)(1/L^2 - 1/U^2),
 *   plus 2 (1/a_i - 1/L) when sphere j encloses atom i's sphere (a_i < s_j - r); h = 0 otherwise.
 * I_i = (1/2) sum_j h_ij, psi_i = a_i I_i, and the Born radius (Onufriev, Bashford and Case, model II:
 * alpha, beta, gamma = 1, 0.8, 4.85) is 1/B_i = 1/a_i - tanh(alpha psi - beta psi^2 + gamma psi^3) / rho_i.
 * The energy, over all pairs including bonded ones and each atom with itself, is
 *   E = -(1/2) k_e (1/eps_in - 1/eps_out) sum_i sum_j q_i q_j / f_ij,
 *   f_ij = sqrt(r^2 + B_i B_j exp(-r^2 / (4 B_i B_j))), f_ii = B_i.
 * With a cutoff r_c (a system whose nonbonded terms are truncated, as the paper's protein-ligand setup
 * in a non-periodic cutoff scheme), a pair i != j at r >= r_c enters neither the descreening sums nor
 * the pair energy (plain truncation, like the Lennard-Jones and Coulomb terms of such a system); the
 * self terms always count. */
static const double kGbOffset = 0.009, kGbAlpha = 1.0, kGbBeta = 0.8, kGbGamma = 4.85;

/* Whether the pair at squared distance r2 enters the solvent sums. */
static int gb_in_range(const orc_system *s, double r2) {
  return !(s->cutoff > 0 && r2 >= s->cutoff * s->cutoff);
}

/* h_ij and its derivative dh/dr (L and U depend on r). */
static double gb_hct(double r, double ai, double sj, double *dh) {
  const double U = r + sj;
  if (!(ai < U)) { *dh = 0.0; return 0.0; }
  const double diff = r - sj;
  double L, dL;
  if (ai > fabs(diff)) { L = ai; dL = 0.0; }
  else { L = fabs(diff); dL = diff >= 0.0 ? 1.0 : -1.0; }
  const double iL = 1.0 / L, iU = 1.0 / U, iL2 = iL * iL, iU2 = iU * iU, lg = log(L / U), s2 = sj * sj;
  double h = iL - iU + 0.25 * r * (iU2 - iL2) + 0.5 / r * lg + 0.25 * s2 / r * (iL2 - iU2);
  double d = -dL * iL2 + iU2                                  /* d(1/L - 1/U) */
             + 0.25 * (iU2 - iL2) + 0.25 * r * (-2.0 * iU2 * iU + 2.0 * dL * iL2 * iL)
             - 0.5 / (r * r) * lg + 0.5 / r * (dL * iL - iU)
             - 0.25 * s2 / (r * r) * (iL2 - iU2) + 0.25 * s2 / r * (-2.0 * dL * iL2 * iL + 2.0 * iU2 * iU);
  if (ai < sj - r) {
    h += 2.0 * (1.0 / ai - iL);
    d += 2.0 * dL * iL2;
  }
  *dh = d;
  return h;
}

/* Born radii, their derivatives dB_i / dI_i (dbdi, optional) and the sums I_i. */
static void gb_radii(const orc_ctx *c, const double *q, double *born, double *dbdi, double *integral) {
  const orc_system *s = &c->s;
  const int n = s->n_atoms;
  for (int i = 0; i < n; ++i) {
    const double ai = s->gb_radius[i] - kGbOffset;
    double sum = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3], dh;
      sub3(q + 3 * i, q + 3 * j, d);
      if (!gb_in_range(s, dot3(d, d))) continue;
      sum += gb_hct(norm3(d), ai, s->gb_scale[j] * (s->gb_radius[j] - kGbOffset), &dh);
    }
    const double I = 0.5 * sum, psi = ai * I;
    const double x = kGbAlpha * psi - kGbBeta * psi * psi + kGbGamma * psi * psi * psi;
    const double t = tanh(x);
    const double B = 1.0 / (1.0 / ai - t / s->gb_radius[i]);
    born[i] = B;
    if (integral) integral[i] = I;
    if (dbdi) dbdi[i] = B * B * (1.0 - t * t) / s->gb_radius[i] * (kGbAlpha - 2.0 * kGbBeta * psi + 3.0 * kGbGamma * psi * psi) * ai;
  }
}

void orc_gb_born(const orc_ctx *c, const double *q, double *born, double *integral) {
  gb_radii(c, q, born, NULL, integral);
}

static double gb_tau(const orc_system *s) {
  return s->coulomb_k * (1.0 / s->gb_solute_dielectric - 1.0 / s->gb_solvent_dielectric);
}

static double gb_energy(const orc_ctx *c, const double *q) {
  const orc_system *s = &c->s;
  const int n = s->n_atoms;
  double *B = (double *)malloc(sizeof(double) * (size_t)n);
  gb_radii(c, q, B, NULL, NULL);
  double sum = 0.0;
  for (int i = 0; i < n; ++i) {
    sum += s->charge[i] * s->charge[i] / B[i];
    for (int j = i + 1; j < n; ++j) {
      double d[3];
      sub3(q + 3 * i, q + 3 * j, d);
      const double r2 = dot3(d, d), bb = B[i] * B[j];
      if (!gb_in_range(s, r2)) continue;
      sum += 2.0 * s->charge[i] * s->charge[j] / sqrt(r2 + bb * exp(-r2 / (4.0 * bb)));
    }
  }
  free(B);
  return -0.5 * gb_tau(s) * sum;
}

/* Forces -dE/dq: the pair terms at fixed Born radii, then the chain rule through B_i(I_i(r_ij)). */
static void gb_forces(const orc_ctx *c, const double *q, double *f) {
  const orc_system *s = &c->s;
  const int n = s->n_atoms;
  const double tau = gb_tau(s);
  double *B = (double *)malloc(sizeof(double) * (size_t)n), *dBdI = (double *)malloc(sizeof(double) * (size_t)n);
  double *dEdB = (double *)calloc((size_t)n, sizeof(double));
  gb_radii(c, q, B, dBdI, NULL);
  for (int i = 0; i < n; ++i) dEdB[i] = 0.5 * tau * s->charge[i] * s->charge[i] / (B[i] * B[i]);
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double d[3];
      sub3(q + 3 * i, q + 3 * j, d);
      const double r2 = dot3(d, d);
      if (!gb_in_range(s, r2)) continue;
      const double r = sqrt(r2), bb = B[i] * B[j], D = r2 / (4.0 * bb), e = exp(-D);
      const double fij = sqrt(r2 + bb * e), qq = s->charge[i] * s->charge[j];
      /* E_pair = -tau qq / f: dE/df = tau qq / f^2 */
      const double dEdf = tau * qq / (fij * fij);
      const double dfdr = r * (1.0 - 0.25 * e) / fij;
      dEdB[i] += dEdf * B[j] * e * (1.0 + D) / (2.0 * fij);
      dEdB[j] += dEdf * B[i] * e * (1.0 + D) / (2.0 * fij);
      const double g = dEdf * dfdr / r; /* dE/dr / r */
      for (int x = 0; x < 3; ++x) {
        f[3 * i + x] -= g * d[x];
        f[3 * j + x] += g * d[x];
      }
    }
  for (int i = 0; i < n; ++i) {
    const double ai = s->gb_radius[i] - kGbOffset;
    const double w = dEdB[i] * dBdI[i] * 0.5; /* dE/dh_ij for every j: I_i = (1/2) sum_j h_ij */
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double d[3], dh;
      sub3(q + 3 * i, q + 3 * j, d);
      if (!gb_in_range(s, dot3(d, d))) continue;
      const double r = norm3(d);
      gb_hct(r, ai, s->gb_scale[j] * (s->gb_radius[j] - kGbOffset), &dh);
      const double g = w * dh / r;
      for (int x = 0; x < 3; ++x) {
        f[3 * i + x] -= g * d[x];
        f[3 * j + x] += g * d[x];
      }
    }
  }
  free(B); free(dBdI); free(dEdB);
}

/* ---------------------------------------------------------------- periodic electrostatics
 * Ewald's splitting of the lattice sum of k_e q_i q_j / r over all periodic images, the sum that the
 * particle mesh Ewald method (cited in Section 3.2 among the optimisations an engine should offer)
 * approximates.  With beta the splitting parameter, V the box volume and Q the net charge:
 *   E = sum_{i<j, not excluded, r_ij < r_c} k_e q_i q_j erfc(beta r_ij) / r_ij       (minimum image)
 *     - sum_{excluded i<j} k_e q_i q_j erf(beta r_ij) / r_ij                          (minimum image)
 *     - k_e beta / sqrt(pi) sum_i q_i^2
 *     + k_e / (2 pi V) sum_{m != 0} exp(-pi^2 |m|^2 / beta^2) / |m|^2 |S(m)|^2
 *     - k_e pi Q^2 / (2 V beta^2),
 * S(m) = sum_j q_j exp(2 pi i m.r_j), m = (k_0/L_0, k_1/L_1, k_2/L_2) over integer k != 0.  The
 * excluded pairs' erf term removes what the reciprocal sum adds for the nearest image of a pair that
 * has no Coulomb interaction; their other images keep theirs. */
static const double kPi = 3.14159265358979323846;

static int periodic(const orc_system *s) { return s->coulomb_mode == 2 || s->coulomb_mode == 3; }

/* q_i - q_j, at the nearest image in a periodic system */
static void pair_vec(const orc_system *s, const double *q, int i, int j, double *d) {
  sub3(q + 3 * i, q + 3 * j, d);
  if (periodic(s))
    for (int x = 0; x < 3; ++x) d[x] -= s->box[x] * nearbyint(d[x] / s->box[x]);
}

static double box_volume(const orc_system *s) { return s->box[0] * s->box[1] * s->box[2]; }

/* Excluded pairs, the self term and the background: energy, and their forces added to f (if not
 * NULL).  parts[1], parts[2], parts[4] as in orc_ewald_parts. */
static void ewald_corrections(const orc_ctx *c, const double *q, double *f, double parts[5]) {
  const orc_system *s = &c->s;
  const int n = s->n_atoms;
  const double b = s->ewald_beta, ke = s->coulomb_k;
  double ex = 0.0, q2 = 0.0, qt = 0.0;
  for (int i = 0; i < n; ++i) {
    q2 += s->charge[i] * s->charge[i];
    qt += s->charge[i];
    for (int j = i + 1; j < n; ++j) {
      if (!c->excluded[(size_t)i * n + j]) continue;
      double d[3];
      pair_vec(s, q, i, j, d);
      const double r2 = dot3(d, d), r = sqrt(r2), kqq = ke * s->charge[i] * s->charge[j];
      ex -= kqq * erf(b * r) / r;
      if (f) {
        /* E = -kqq erf(b r)/r: -dE/dr / r = kqq (2 b/sqrt(pi) exp(-b^2 r^2) - erf(b r)/r) / r^2 */
        const double g = kqq * (2.0 * b / sqrt(kPi) * exp(-b * b * r2) - erf(b * r) / r) / r2;
        for (int x = 0; x < 3; ++x) {
          f[3 * i + x] += g * d[x];
          f[3 * j + x] -= g * d[x];
        }
      }
    }
  }
  parts[1] = ex;
  parts[2] = -ke * b / sqrt(kPi) * q2;
  parts[4] = -ke * kPi * qt * qt / (2.0 * box_volume(s) * b * b);
}

/* Reciprocal sum of the plain Ewald method over |k_d| <= ewald_kmax; forces added to f (if not
 * NULL): F_i = (2 k_e q_i / V) sum_m g(m) m (C(m) sin(2 pi m.r_i) - S(m) cos(2 pi m.r_i)) with
 * S(m) = C(m) + i S(m) split into its real and imaginary parts and g = exp(-pi^2 m^2/beta^2)/m^2. */
static double ewald_reciprocal(const orc_ctx *c, const double *q, double *f) {
  const orc_system *s = &c->s;
  const int n = s->n_atoms, K = s->ewald_kmax;
  const double V = box_volume(s), b = s->ewald_beta, ke = s->coulomb_k;
  double e = 0.0;
  for (int k0 = -K; k0 <= K; ++k0)
    for (int k1 = -K; k1 <= K; ++k1)
      for (int k2 = -K; k2 <= K; ++k2) {
        if (k0 == 0 && k1 == 0 && k2 == 0) continue;
        const double m[3] = {k0 / s->box[0], k1 / s->box[1], k2 / s->box[2]};
        const double m2 = dot3(m, m), g = exp(-kPi * kPi * m2 / (b * b)) / m2;
        double sc = 0.0, ss = 0.0;
        for (int j = 0; j < n; ++j) {
          const double th = 2.0 * kPi * dot3(m, q + 3 * j);
          sc += s->charge[j] * cos(th);
          ss += s->charge[j] * sin(th);
        }
        e += g * (sc * sc + ss * ss);
        if (f)
          for (int i = 0; i < n; ++i) {
            const double th = 2.0 * kPi * dot3(m, q + 3 * i);
            const double w = 2.0 * ke * s->charge[i] / V * g * (sc * sin(th) - ss * cos(th));
            for (int x = 0; x < 3; ++x) f[3 * i + x] += w * m[x];
          }
      }
  return ke * e / (2.0 * kPi * V);
}

/* Cardinal B-spline M_p (Essmann et al. 1995): M_2(x) = 1 - |x - 1| on [0, 2], and
 * M_p(x) = (x M_{p-1}(x) + (p - x) M_{p-1}(x - 1)) / (p - 1), supported on (0, p). */
static double bspline(int p, double x) {
  if (x <= 0.0 || x >= (double)p) return 0.0;
  if (p == 2) return 1.0 - fabs(x - 1.0);
  return (x * bspline(p - 1, x) + ((double)p - x) * bspline(p - 1, x - 1.0)) / (double)(p - 1);
}
/* dM_p/dx = M_{p-1}(x) - M_{p-1}(x - 1) */
static double bspline_d(int p, double x) { return bspline(p - 1, x) - bspline(p - 1, x - 1.0); }

/* Interpolation weights of one coordinate on a periodic axis of K points: u = K r / L taken into
 * [0, K); w[k] = sum over images n of M_p(u - k - n K), dw[k] its derivative in u. */
static void spline_weights(int p, int K, double L, double r, double *w, double *dw) {
  double u = (double)K * (r / L - floor(r / L));
  for (int k = 0; k < K; ++k) {
    w[k] = dw[k] = 0.0;
    for (int img = -2; img <= 2; ++img) {
      const double x = u - k - (double)img * K;
      w[k] += bspline(p, x);
      dw[k] += bspline_d(p, x);
    }
  }
}

/* One-dimensional discrete Fourier transform of every line along axis ax of a complex grid
 * [K0][K1][K2]: X(m) = sum_k x(k) exp(sign 2 pi i m k / K_ax), in place. */
static void dft_lines(double *re, double *im, const int *K, int ax, int sign) {
  const int stride[3] = {K[1] * K[2], K[2], 1};
  const int Ka = K[ax], oa = (ax + 1) % 3, ob = (ax + 2) % 3;
  double *tr = (double *)malloc(sizeof(double) * Ka), *ti = (double *)malloc(sizeof(double) * Ka);
  for (int a = 0; a < K[oa]; ++a)
    for (int c2 = 0; c2 < K[ob]; ++c2) {
      const size_t base = (size_t)a * stride[oa] + (size_t)c2 * stride[ob];
      for (int m = 0; m < Ka; ++m) {
        double xr = 0.0, xi = 0.0;
        for (int k = 0; k < Ka; ++k) {
          const double th = sign * 2.0 * kPi * (double)m * (double)k / (double)Ka;
          const double vr = re[base + (size_t)k * stride[ax]], vi = im[base + (size_t)k * stride[ax]];
          xr += vr * cos(th) - vi * sin(th);
          xi += vr * sin(th) + vi * cos(th);
        }
        tr[m] = xr;
        ti[m] = xi;
      }
      for (int m = 0; m < Ka; ++m) {
        re[base + (size_t)m * stride[ax]] = tr[m];
        im[base + (size_t)m * stride[ax]] = ti[m];
      }
    }
  free(tr);
  free(ti);
}

/* Smooth particle mesh Ewald reciprocal sum (Essmann et al. 1995, Section 3 and Eq. 4.7):
 *   Q(k) = sum_i q_i w_0i(k_0) w_1i(k_1) w_2i(k_2)   (the charges spread by B-splines of order p),
 *   F(m) = sum_k Q(k) exp(2 pi i sum_d m_d k_d / K_d),
 *   E = (k_e/2) sum_m G(m) |F(m)|^2,  G(m) = B(m) exp(-pi^2 |m'|^2 / beta^2) / (pi V |m'|^2), G(0) = 0,
 * with m'_d = m_d / L_d for m_d <= K_d/2, (m_d - K_d) / L_d otherwise, and the Euler exponential
 * spline factor B(m) = prod_d |sum_{k=0}^{p-2} M_p(k+1) exp(2 pi i m_d k / K_d)|^-2.  Forces:
 * phi(k) = sum_m G(m) F(m) exp(-2 pi i m.k/K) is dE/dQ(k) / k_e, and F_i = -k_e sum_k dQ(k)/dr_i phi(k). */
static double pme_reciprocal(const orc_ctx *c, const double *q, double *f) {
  const orc_system *s = &c->s;
  const int n = s->n_atoms, p = s->pme_order;
  const int *K = s->pme_grid;
  const size_t ng = (size_t)K[0] * K[1] * K[2];
  const double V = box_volume(s), b = s->ewald_beta, ke = s->coulomb_k;
  double *w[3], *dw[3];
  for (int d = 0; d < 3; ++d) {
    w[d] = (double *)malloc(sizeof(double) * (size_t)n * K[d]);
    dw[d] = (double *)malloc(sizeof(double) * (size_t)n * K[d]);
    for (int i = 0; i < n; ++i)
      spline_weights(p, K[d], s->box[d], q[3 * i + d], w[d] + (size_t)i * K[d], dw[d] + (size_t)i * K[d]);
  }
  double *re = (double *)calloc(ng, sizeof(double)), *im = (double *)calloc(ng, sizeof(double));
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < K[0]; ++a)
      for (int bb = 0; bb < K[1]; ++bb)
        for (int cc = 0; cc < K[2]; ++cc)
          re[((size_t)a * K[1] + bb) * K[2] + cc] +=
              s->charge[i] * w[0][(size_t)i * K[0] + a] * w[1][(size_t)i * K[1] + bb] * w[2][(size_t)i * K[2] + cc];
  for (int d = 0; d < 3; ++d) dft_lines(re, im, K, d, +1);
  /* B(m) per axis */
  double *bmod[3];
  for (int d = 0; d < 3; ++d) {
    bmod[d] = (double *)malloc(sizeof(double) * K[d]);
    for (int m = 0; m < K[d]; ++m) {
      double dr = 0.0, di = 0.0;
      for (int k = 0; k <= p - 2; ++k) {
        const double th = 2.0 * kPi * (double)m * (double)k / (double)K[d];
        dr += bspline(p, k + 1.0) * cos(th);
        di += bspline(p, k + 1.0) * sin(th);
      }
      bmod[d][m] = 1.0 / (dr * dr + di * di);
    }
  }
  double e = 0.0;
  for (int a = 0; a < K[0]; ++a)
    for (int bb = 0; bb < K[1]; ++bb)
      for (int cc = 0; cc < K[2]; ++cc) {
        const size_t t = ((size_t)a * K[1] + bb) * K[2] + cc;
        const int mi[3] = {a, bb, cc};
        double m2 = 0.0;
        for (int d = 0; d < 3; ++d) {
          const double md = (mi[d] <= K[d] / 2 ? mi[d] : mi[d] - K[d]) / s->box[d];
          m2 += md * md;
        }
        double G = 0.0;
        if (m2 > 0.0) G = bmod[0][a] * bmod[1][bb] * bmod[2][cc] * exp(-kPi * kPi * m2 / (b * b)) / (kPi * V * m2);
        e += 0.5 * ke * G * (re[t] * re[t] + im[t] * im[t]);
        re[t] *= G;
        im[t] *= G;
      }
  if (f) {
    for (int d = 0; d < 3; ++d) dft_lines(re, im, K, d, -1); /* re = phi */
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < K[0]; ++a)
        for (int bb = 0; bb < K[1]; ++bb)
          for (int cc = 0; cc < K[2]; ++cc) {
            const double ph = re[((size_t)a * K[1] + bb) * K[2] + cc];
            const double w0 = w[0][(size_t)i * K[0] + a], w1 = w[1][(size_t)i * K[1] + bb], w2 = w[2][(size_t)i * K[2] + cc];
            const double d0 = dw[0][(size_t)i * K[0] + a], d1 = dw[1][(size_t)i * K[1] + bb], d2 = dw[2][(size_t)i * K[2] + cc];
            const double kq = -ke * s->charge[i] * ph;
            f[3 * i + 0] += kq * K[0] / s->box[0] * d0 * w1 * w2;
            f[3 * i + 1] += kq * K[1] / s->box[1] * w0 * d1 * w2;
            f[3 * i + 2] += kq * K[2] / s->box[2] * w0 * w1 * d2;
          }
  }
  for (int d = 0; d < 3; ++d) { free(w[d]); free(dw[d]); free(bmod[d]); }
  free(re);
  free(im);
  return e;
}

static double periodic_reciprocal(const orc_ctx *c, const double *q, double *f) {
  return c->s.coulomb_mode == 2 ? pme_reciprocal(c, q, f) : ewald_reciprocal(c, q, f);
}

void orc_ewald_parts(const orc_ctx *c, const double *q, double parts[5]) {
  const orc_system *s = &c->s;
  const int n = s->n_atoms;
  double dir = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      if (c->excluded[(size_t)i * n + j]) continue;
      double d[3];
      pair_vec(s, q, i, j, d);
      const double r2 = dot3(d, d);
      if (s->cutoff > 0 && r2 >= s->cutoff * s->cutoff) continue;
      const double r = sqrt(r2);
      dir += s->coulomb_k * s->charge[i] * s->charge[j] * erfc(s->ewald_beta * r) / r;
    }
  ewald_corrections(c, q, NULL, parts);
  parts[0] = dir;
  parts[3] = periodic_reciprocal(c, q, NULL);
}

/* ---------------------------------------------------------------- potential V(q), Eq. 1 */
double orc_potential(const orc_ctx *c, const double *q) {
  const orc_system *s = &c->s;
  if (s->potential == ORC_POT_DOUBLE_WELL_2D) {
    double x = q[0], y = q[1];
    return s->dw_a * (x * x - 1.0) * (x * x - 1.0) + s->dw_b * y * y;
  }
  int n = s->n_atoms;
  double e = 0.0;
  for (int b = 0; b < s->n_bonds; ++b) {
    const int *a = s->bond_atoms + 2 * b;
    double d[3];
    sub3(q + 3 * a[0], q + 3 * a[1], d);
    double r = norm3(d);
    e += 0.5 * s->bond_k[b] * (r - s->bond_r0[b]) * (r - s->bond_r0[b]);
  }
  for (int t = 0; t < s->n_angles; ++t) {
    const int *a = s->angle_atoms + 3 * t;
    double u[3], v[3], w[3];
    sub3(q + 3 * a[0], q + 3 * a[1], u);
    sub3(q + 3 * a[2], q + 3 * a[1], v);
    cross3(u, v, w);
    double th = atan2(norm3(w), dot3(u, v));
    e += 0.5 * s->angle_k[t] * (th - s->angle_theta0[t]) * (th - s->angle_theta0[t]);
  }
  for (int t = 0; t < s->n_dihedrals; ++t) {
    const int *a = s->dihedral_atoms + 4 * t;
    double phi = dihedral_angle(q + 3 * a[0], q + 3 * a[1], q + 3 * a[2], q + 3 * a[3]);
    e += s->dihedral_k[t] * (1.0 + cos(s->dihedral_n[t] * phi - s->dihedral_delta[t]));
  }
  for (int i = 0; i < n; ++i) {
    for (int j = i + 1; j < n; ++j) {
      if (c->excluded[(size_t)i * n + j]) continue;
      double d[3];
      pair_vec(s, q, i, j, d);
      double r2 = dot3(d, d);
      if (s->cutoff > 0 && r2 >= s->cutoff * s->cutoff) continue;
      double sig = 0.5 * (s->sigma[i] + s->sigma[j]);
      double eps = sqrt(s->epsilon[i] * s->epsilon[j]);
      double sr6 = pow(sig * sig / r2, 3);
      e += 4.0 * eps * (sr6 * sr6 - sr6);
      const double kqq = s->coulomb_k * s->charge[i] * s->charge[j];
      if (periodic(s)) {
        /* real-space part of the Ewald sum */
        const double r = sqrt(r2);
        e += kqq * erfc(s->ewald_beta * r) / r;
      } else if (s->coulomb_mode == 1) {
        /* reaction field: E = k_e q_i q_j (1/r + k_rf r^2 - c_rf) */
        double krf, crf;
        rf_constants(s, &krf, &crf);
        e += kqq * (1.0 / sqrt(r2) + krf * r2 - crf);
      } else {
        /* dielectric eps(r) = 4 r: E = k_e q_i q_j / (4 r * r) */
        e += kqq / (4.0 * r2);
      }
    }
  }
  if (s->gb_radius) e += gb_energy(c, q);
  if (periodic(s)) {
    double parts[5];
    ewald_corrections(c, q, NULL, parts);
    e += parts[1] + parts[2] + parts[4] + periodic_reciprocal(c, q, NULL);
  }
  return e;
}

/* ---------------------------------------------------------------- forces F = -grad V */
void orc_forces(const orc_ctx *c, const double *q, double *f) {
  const orc_system *s = &c->s;
  if (s->potential == ORC_POT_DOUBLE_WELL_2D) {
    double x = q[0], y = q[1];
    f[0] = -s->dw_a * 4.0 * x * (x * x - 1.0);
    f[1] = -s->dw_b * 2.0 * y;
    return;
  }
  int n = s->n_atoms;
  memset(f, 0, sizeof(double) * 3 * (size_t)n);
  /* bonds: dE/dr = k (r - r0); F_i = -dE/dr * (q_i - q_j)/r */
  for (int b = 0; b < s->n_bonds; ++b) {
    const int *a = s->bond_atoms + 2 * b;
    double d[3];
    sub3(q + 3 * a[0], q + 3 * a[1], d);
    double r = norm3(d);
    double g = s->bond_k[b] * (r - s->bond_r0[b]) / r;
    for (int x = 0; x < 3; ++x) {
      f[3 * a[0] + x] -= g * d[x];
      f[3 * a[1] + x] += g * d[x];
    }
  }
  /* angles: theta = atan2(|u x v|, u.v) with u = q_i - q_j, v = q_k - q_j;
   * d theta / d q_i = (cos(theta) u/|u| - v/|v|) / (|u| sin(theta)), likewise for q_k. */
  for (int t = 0; t < s->n_angles; ++t) {
    const int *a = s->angle_atoms + 3 * t;
    double u[3], v[3], w[3];
    sub3(q + 3 * a[0], q + 3 * a[1], u);
    sub3(q + 3 * a[2], q + 3 * a[1], v);
    cross3(u, v, w);
    double lu = norm3(u), lv = norm3(v);
    double th = atan2(norm3(w), dot3(u, v));
    double ct = cos(th), st = sin(th);
    if (st < 1e-12) st = 1e-12;
    double dedth = s->angle_k[t] * (th - s->angle_theta0[t]);
    for (int x = 0; x < 3; ++x) {
      double dthi = (ct * u[x] / lu - v[x] / lv) / (lu * st);
      double dthk = (ct * v[x] / lv - u[x] / lu) / (lv * st);
      f[3 * a[0] + x] -= dedth * dthi;
      f[3 * a[2] + x] -= dedth * dthk;
      f[3 * a[1] + x] += dedth * (dthi + dthk);
    }
  }
  /* dihedrals (Blondel & Karplus 1996 gradient of the dihedral angle):
   * d phi/d q_i = -|b2| n1/|n1|^2, d phi/d q_l = |b2| n2/|n2|^2,
   * d phi/d q_j = -(1 + b1.b2/|b2|^2) d phi/d q_i + (b3.b2/|b2|^2) d phi/d q_l,
   * d phi/d q_k = (b1.b2/|b2|^2) d phi/d q_i - (1 + b3.b2/|b2|^2) d phi/d q_l
   * (the four gradients sum to zero: translation invariance). */
  for (int t = 0; t < s->n_dihedrals; ++t) {
    const int *a = s->dihedral_atoms + 4 * t;
    const double *qi = q + 3 * a[0], *qj = q + 3 * a[1], *qk = q + 3 * a[2], *ql = q + 3 * a[3];
    double b1[3], b2[3], b3[3], n1[3], n2[3];
    sub3(qj, qi, b1); sub3(qk, qj, b2); sub3(ql, qk, b3);
    cross3(b1, b2, n1); cross3(b2, b3, n2);
    double lb2 = norm3(b2);
    double phi = atan2(lb2 * dot3(b1, n2), dot3(n1, n2));
    double dedphi = -s->dihedral_k[t] * s->dihedral_n[t] * sin(s->dihedral_n[t] * phi - s->dihedral_delta[t]);
    double n1sq = dot3(n1, n1), n2sq = dot3(n2, n2);
    double f12 = dot3(b1, b2) / (lb2 * lb2), f32 = dot3(b3, b2) / (lb2 * lb2);
    for (int x = 0; x < 3; ++x) {
      double gi = -lb2 * n1[x] / n1sq;
      double gl = lb2 * n2[x] / n2sq;
      double gj = -(1.0 + f12) * gi + f32 * gl;
      double gk = f12 * gi - (1.0 + f32) * gl;
      f[3 * a[0] + x] -= dedphi * gi;
      f[3 * a[1] + x] -= dedphi * gj;
      f[3 * a[2] + x] -= dedphi * gk;
      f[3 * a[3] + x] -= dedphi * gl;
    }
  }
  /* Lennard-Jones (Lorentz-Berthelot) and Coulomb with eps(r) = 4r over non-excluded pairs */
  for (int i = 0; i < n; ++i) {
    for (int j = i + 1; j < n; ++j) {
      if (c->excluded[(size_t)i * n + j]) continue;
      double d[3];
      pair_vec(s, q, i, j, d);
      double r2 = dot3(d, d);
      if (s->cutoff > 0 && r2 >= s->cutoff * s->cutoff) continue;
      double sig = 0.5 * (s->sigma[i] + s->sigma[j]);
      double eps = sqrt(s->epsilon[i] * s->epsilon[j]);
      double sr6 = pow(sig * sig / r2, 3);
      /* -dE_LJ/dr / r = 24 eps (2 (s/r)^12 - (s/r)^6) / r^2 */
      double g = 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r2;
      const double kqq = s->coulomb_k * s->charge[i] * s->charge[j];
      if (periodic(s)) {
        /* E = kqq erfc(b r)/r: -dE/dr / r = kqq (erfc(b r)/r + 2 b/sqrt(pi) exp(-b^2 r^2)) / r^2 */
        const double r = sqrt(r2), b = s->ewald_beta;
        g += kqq * (erfc(b * r) / r + 2.0 * b / sqrt(kPi) * exp(-b * b * r2)) / r2;
      } else if (s->coulomb_mode == 1) {
        /* reaction field: -dE_C/dr / r = k_e q_i q_j (1/r^2 - 2 k_rf r) / r */
        double krf, crf;
        rf_constants(s, &krf, &crf);
        g += kqq * (1.0 / (r2 * sqrt(r2)) - 2.0 * krf);
      } else {
        /* -dE_C/dr / r = 2 k_e q_i q_j / (4 r^3) / r */
        g += 2.0 * kqq / (4.0 * r2 * r2);
      }
      for (int x = 0; x < 3; ++x) {
        f[3 * i + x] += g * d[x];
        f[3 * j + x] -= g * d[x];
      }
    }
  }
  if (s->gb_radius) gb_forces(c, q, f);
  if (periodic(s)) {
    double parts[5];
    ewald_corrections(c, q, f, parts);
    periodic_reciprocal(c, q, f);
  }
}

/* ---------------------------------------------------------------- dV/d theta
 * Pair (i, j): E = 4 e (s^12 - s^6) with s = sig / r, sig = (sigma_i + sigma_j) / 2 and
 * e = sqrt(epsilon_i epsilon_j).  dE/d sig = 4 e (12 s^12 - 6 s^6) / sig and d sig / d sigma_i = 1/2;
 * dE/d e = 4 (s^12 - s^6) and d e / d epsilon_i = epsilon_j / (2 e).  Coulomb does not depend on
 * theta.  Dihedral term t: E = k_t (1 + cos(n_t phi - delta_t)), so dE/dk_t = 1 + cos(n_t phi - delta_t). */
void orc_param_grad(const orc_ctx *c, const double *q, double *g) {
  const orc_system *s = &c->s;
  int n = s->n_atoms;
  int nt = 2 * n + s->n_dihedrals;
  memset(g, 0, sizeof(double) * (size_t)nt);
  if (s->potential != ORC_POT_FORCE_FIELD) return;
  for (int i = 0; i < n; ++i) {
    for (int j = i + 1; j < n; ++j) {
      if (c->excluded[(size_t)i * n + j]) continue;
      double d[3];
      pair_vec(s, q, i, j, d);
      double r2 = dot3(d, d);
      if (s->cutoff > 0 && r2 >= s->cutoff * s->cutoff) continue;
      double sig = 0.5 * (s->sigma[i] + s->sigma[j]);
      double eps = sqrt(s->epsilon[i] * s->epsilon[j]);
      double sr6 = pow(sig * sig / r2, 3);
      double de_dsig = 4.0 * eps * (12.0 * sr6 * sr6 - 6.0 * sr6) / sig;
      double de_deps = 4.0 * (sr6 * sr6 - sr6);
      g[i] += 0.5 * de_dsig;
      g[j] += 0.5 * de_dsig;
      g[n + i] += de_deps * s->epsilon[j] / (2.0 * eps);
      g[n + j] += de_deps * s->epsilon[i] / (2.0 * eps);
    }
  }
  for (int t = 0; t < s->n_dihedrals; ++t) {
    const int *a = s->dihedral_atoms + 4 * t;
    double phi = dihedral_angle(q + 3 * a[0], q + 3 * a[1], q + 3 * a[2], q + 3 * a[3]);
    g[2 * n + t] = 1.0 + cos(s->dihedral_n[t] * phi - s->dihedral_delta[t]);
  }
}

/* ---------------------------------------------------------------- Philox4x32-10 */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, x0, &hi0, &lo0);
    mulhilo32(0xCD9E8D57u, x2, &hi1, &lo1);
    uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u; /* Weyl sequence key schedule */
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Counter layout: (step low 32 bits, step bits 32..55 | stream << 24, replica, atom); key = seed. */
static void philox_words(uint64_t seed, int64_t step, uint32_t stream, int32_t replica, int32_t atom,
                         uint32_t out[4]) {
  uint64_t st = (uint64_t)step;
  uint32_t ctr[4] = {(uint32_t)st, (uint32_t)((st >> 32) & 0x00FFFFFFu) | (stream << 24),
                     (uint32_t)replica, (uint32_t)atom};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* Box-Muller (1958): (sqrt(-2 ln u1) cos 2 pi u2, sqrt(-2 ln u1) sin 2 pi u2) with
 * u = (w + 1/2) 2^-32 for a 32-bit word w, so u is in (0, 1). */
void orc_normals(uint64_t seed, int64_t step, int32_t replica, int32_t atom, double xi[4]) {
  uint32_t w[4];
  philox_words(seed, step, 0u, replica, atom, w);
  const double two_pi = 6.283185307179586476925286766559;
  for (int pair = 0; pair < 2; ++pair) {
    double u1 = ((double)w[2 * pair] + 0.5) * 0x1p-32;
    double u2 = ((double)w[2 * pair + 1] + 0.5) * 0x1p-32;
    double r = sqrt(-2.0 * log(u1));
    xi[2 * pair] = r * cos(two_pi * u2);
    xi[2 * pair + 1] = r * sin(two_pi * u2);
  }
}

uint32_t orc_branch_word(uint64_t seed, int64_t step, int32_t replica) {
  uint32_t w[4];
  philox_words(seed, step, 1u, replica, 0, w);
  return w[0];
}

/* ---------------------------------------------------------------- BAOAB step of Eq. 1
 * B: p += dt/2 F; A: q += dt/2 M^-1 p; O: p = c1 p + sqrt((1 - c1^2) m kT) xi with c1 = exp(-gamma dt)
 * (gamma read as a collision rate); A: q += dt/2 M^-1 p; F = F(q); B: p += dt/2 F. */
/* ---------------------------------------------------------------- bond constraints
 * RATTLE projection of the momenta: Gauss-Seidel sweeps over the constraints, each removing the
 * relative velocity of its two atoms along their bond, until a sweep changes nothing beyond the
 * tolerance |r . v| <= tol d^2 / dt (or the iteration bound). */
static void rattle_momenta(const orc_ctx *c, const double *q, double *p) {
  const orc_system *s = &c->s;
  for (int it = 0; it < s->constraint_max_iter; ++it) {
    int moved = 0;
    for (int k = 0; k < s->n_constraints; ++k) {
      const int i = s->constraint_atoms[2 * k], j = s->constraint_atoms[2 * k + 1];
      const double d = s->constraint_length[k], wi = 1.0 / s->mass[i], wj = 1.0 / s->mass[j];
      double r[3], v[3];
      sub3(q + 3 * i, q + 3 * j, r);
      for (int x = 0; x < 3; ++x) v[x] = p[3 * i + x] * wi - p[3 * j + x] * wj;
      const double rv = dot3(r, v);
      if (fabs(rv) <= s->constraint_tol * d * d / s->dt) continue;
      const double mu = rv / ((wi + wj) * dot3(r, r));
      for (int x = 0; x < 3; ++x) {
        p[3 * i + x] -= mu * r[x];
        p[3 * j + x] += mu * r[x];
      }
      moved = 1;
    }
    if (!moved) return;
  }
  ((orc_ctx *)c)->unconverged++;
}

/* SHAKE after an A step: q holds the unconstrained update of q_old; Gauss-Seidel sweeps move each
 * constrained pair along its bond vector at q_old until | |r|^2 - d^2 | <= tol d^2, adding the
 * matching impulse (the displacement times m / h) to the momenta. */
static void shake_positions(const orc_ctx *c, double *q, const double *q_old, double *p, double h) {
  const orc_system *s = &c->s;
  for (int it = 0; it < s->constraint_max_iter; ++it) {
    int moved = 0;
    for (int k = 0; k < s->n_constraints; ++k) {
      const int i = s->constraint_atoms[2 * k], j = s->constraint_atoms[2 * k + 1];
      const double d = s->constraint_length[k], wi = 1.0 / s->mass[i], wj = 1.0 / s->mass[j];
      double r[3], so[3];
      sub3(q + 3 * i, q + 3 * j, r);
      const double diff = d * d - dot3(r, r);
      if (fabs(diff) <= s->constraint_tol * d * d) continue;
      sub3(q_old + 3 * i, q_old + 3 * j, so);
      const double g = diff / (2.0 * (wi + wj) * dot3(so, r));
      for (int x = 0; x < 3; ++x) {
        q[3 * i + x] += g * wi * so[x];
        q[3 * j + x] -= g * wj * so[x];
        p[3 * i + x] += g / h * so[x];
        p[3 * j + x] -= g / h * so[x];
      }
      moved = 1;
    }
    if (!moved) return;
  }
  ((orc_ctx *)c)->unconverged++;
}

/* BAOAB with constraints: every sub-step of the unconstrained step, in the same order per
 * coordinate, then its projection. */
static void baoab_constrained(const orc_ctx *c, double *q, double *p, double *f, uint64_t seed, int32_t replica,
                              int64_t step) {
  const orc_system *s = &c->s;
  const int n = s->n_atoms, nd = 3 * n;
  const double h = 0.5 * s->dt, c1 = exp(-s->gamma * s->dt);
  double *q_old = (double *)malloc(sizeof(double) * (size_t)nd);
  for (int i = 0; i < nd; ++i) p[i] += h * f[i];                                 /* B */
  rattle_momenta(c, q, p);
  memcpy(q_old, q, sizeof(double) * (size_t)nd);                                /* A */
  for (int i = 0; i < nd; ++i) q[i] += h * p[i] / s->mass[i / 3];
  shake_positions(c, q, q_old, p, h);
  rattle_momenta(c, q, p);
  for (int a = 0; a < n; ++a) {                                                 /* O */
    const double m = s->mass[a], sd = sqrt((1.0 - c1 * c1) * m * s->kT);
    double xi[4];
    orc_normals(seed, step, replica, a, xi);
    for (int x = 0; x < 3; ++x) p[3 * a + x] = c1 * p[3 * a + x] + sd * xi[x];
  }
  rattle_momenta(c, q, p);
  memcpy(q_old, q, sizeof(double) * (size_t)nd);                                /* A */
  for (int i = 0; i < nd; ++i) q[i] += h * p[i] / s->mass[i / 3];
  shake_positions(c, q, q_old, p, h);
  rattle_momenta(c, q, p);
  orc_forces(c, q, f);                                                          /* B */
  for (int i = 0; i < nd; ++i) p[i] += h * f[i];
  rattle_momenta(c, q, p);
  free(q_old);
}

void orc_baoab_step(const orc_ctx *c, double *q, double *p, double *f, uint64_t seed,
                    int32_t replica, int64_t step) {
  const orc_system *s = &c->s;
  if (s->n_constraints > 0) {
    baoab_constrained(c, q, p, f, seed, replica, step);
    return;
  }
  int n = s->n_atoms, dim = s->dim;
  double h = 0.5 * s->dt;
  double c1 = exp(-s->gamma * s->dt);
  for (int a = 0; a < n; ++a) {
    double m = s->mass[a];
    double sd = sqrt((1.0 - c1 * c1) * m * s->kT);
    double xi[4];
    orc_normals(seed, step, replica, a, xi);
    for (int x = 0; x < dim; ++x) {
      int i = dim * a + x;
      p[i] += h * f[i];
      q[i] += h * p[i] / m;
      p[i] = c1 * p[i] + sd * xi[x];
      q[i] += h * p[i] / m;
    }
  }
  orc_forces(c, q, f);
  for (int i = 0; i < n * dim; ++i) p[i] += h * f[i];
}

/* ---------------------------------------------------------------- states (Sections 2.2, 3.3) */
void orc_cv(const orc_ctx *c, const double *q, double cv[4]) {
  const orc_system *s = &c->s;
  cv[0] = cv[1] = cv[2] = cv[3] = 0.0;
  if (s->cv_kind == ORC_CV_DOUBLE_WELL) {
    cv[0] = q[0];
  } else if (s->cv_kind == ORC_CV_DIHEDRAL_RECT) {
    const int *a = s->cv_atoms;
    const double deg = 180.0 / 3.14159265358979323846;
    cv[0] = deg * dihedral_angle(q + 3 * a[0], q + 3 * a[1], q + 3 * a[2], q + 3 * a[3]);
    cv[1] = deg * dihedral_angle(q + 3 * a[1], q + 3 * a[2], q + 3 * a[3], q + 3 * a[4]);
  } else if (s->cv_kind == ORC_CV_COM_DISTANCE) {
    double c0[3], c1[3], d[3];
    group_com(c, 0, q, c0);
    group_com(c, 1, q, c1);
    sub3(c0, c1, d);
    cv[0] = norm3(d);
  } else if (s->cv_kind == ORC_CV_ROTAMERS) {
    const int *a = s->cv_atoms, m = (int)s->cv_params[0];
    const double deg = 180.0 / 3.14159265358979323846;
    for (int t = 0; t < m; ++t)
      cv[t] = deg * dihedral_angle(q + 3 * a[t], q + 3 * a[t + 1], q + 3 * a[t + 2], q + 3 * a[t + 3]);
  }
}

/* Rotamer well of a torsion phi in degrees, (-180, 180]: 0 = gauche+ [0, 120), 1 = trans
 * [120, 180] and (-180, -120), 2 = gauche- [-120, 0). */
static int rotamer_well(double phi) {
  if (phi >= 0.0 && phi < 120.0) return 0;
  if (phi >= -120.0 && phi < 0.0) return 2;
  return 1;
}

/* Angular distance (degrees) from phi to the centre of well w (60, 180, -60). */
static double rotamer_offset(double phi, int w) {
  if (w == 0) return fabs(phi - 60.0);
  if (w == 2) return fabs(phi + 60.0);
  return 180.0 - fabs(phi);
}

/* Rotamers: m = cv_params[0] torsions along the atom path cv_atoms[0..m+2] (torsion t of atoms
 * t..t+3); the configuration is in state sum_t well_t 3^t when every torsion lies within
 * w = cv_params[1] degrees of its well's centre, else in no state; it has left state omega when
 * some torsion's well differs from digit t of omega (the wells tile the circle, the cores do not).
 * Double well: states are the cores x < -w (state 0) and x > w (state 1), w = cv_params[0];
 * the state 0 is left when x >= 0, the state 1 when x < 0.
 * Dihedral rectangle: state 0 = {phi in [p0, p1] and psi in [p2, p3]} (degrees), state 1 = the
 * complement: a two-state partition.
 * Centre-of-mass distance: state 0 = {d < cv_params[0]}, state 1 = the complement. */
int32_t orc_state_of(const orc_ctx *c, const double *q) {
  const orc_system *s = &c->s;
  double cv[4];
  orc_cv(c, q, cv);
  if (s->cv_kind == ORC_CV_DOUBLE_WELL) {
    if (cv[0] < -s->cv_params[0]) return 0;
    if (cv[0] > s->cv_params[0]) return 1;
    return -1;
  }
  if (s->cv_kind == ORC_CV_DIHEDRAL_RECT) {
    int in = cv[0] >= s->cv_params[0] && cv[0] <= s->cv_params[1] && cv[1] >= s->cv_params[2] &&
             cv[1] <= s->cv_params[3];
    return in ? 0 : 1;
  }
  if (s->cv_kind == ORC_CV_ROTAMERS) {
    const int m = (int)s->cv_params[0];
    int label = 0, scale = 1;
    for (int t = 0; t < m; ++t) {
      const int w = rotamer_well(cv[t]);
      if (!(rotamer_offset(cv[t], w) < s->cv_params[1])) return -1;
      label += w * scale;
      scale *= 3;
    }
    return label;
  }
  return cv[0] < s->cv_params[0] ? 0 : 1;
}

int32_t orc_exited(const orc_ctx *c, const double *q, int32_t omega) {
  const orc_system *s = &c->s;
  if (s->cv_kind == ORC_CV_DOUBLE_WELL) {
    double x = q[0];
    return omega == 0 ? (x >= 0.0) : (x < 0.0);
  }
  if (s->cv_kind == ORC_CV_ROTAMERS) {
    double cv[4];
    orc_cv(c, q, cv);
    int rest = omega;
    for (int t = 0; t < (int)s->cv_params[0]; ++t, rest /= 3)
      if (rotamer_well(cv[t]) != rest % 3) return 1;
    return 0;
  }
  return orc_state_of(c, q) != omega;
}

/* ---------------------------------------------------------------- observables (Section 2.4.1) */
double orc_observable(const orc_ctx *c, int32_t j, const double *q, const double *p) {
  const orc_system *s = &c->s;
  const int32_t *arg = s->obs_arg[j];
  int n = s->n_atoms, dim = s->dim;
  switch (s->obs_kind[j]) {
    case ORC_OBS_COORD: return q[dim * arg[0] + arg[1]];
    case ORC_OBS_POTENTIAL: return orc_potential(c, q);
    case ORC_OBS_KINETIC: {
      double k = 0;
      for (int a = 0; a < n; ++a)
        for (int x = 0; x < dim; ++x) k += 0.5 * p[dim * a + x] * p[dim * a + x] / s->mass[a];
      return k;
    }
    case ORC_OBS_DIHEDRAL:
      return dihedral_angle(q + 3 * arg[0], q + 3 * arg[1], q + 3 * arg[2], q + 3 * arg[3]);
    case ORC_OBS_GROUP_DISTANCE: {
      double c0[3], c1[3], d[3];
      group_com(c, arg[0], q, c0);
      group_com(c, arg[1], q, c1);
      sub3(c0, c1, d);
      return norm3(d);
    }
    case ORC_OBS_RMS_VELOCITY: {
      double acc = 0;
      int cnt = 0;
      for (int t = s->group_offsets[arg[0]]; t < s->group_offsets[arg[0] + 1]; ++t) {
        int a = s->group_atoms[t];
        for (int x = 0; x < 3; ++x) {
          double v = p[3 * a + x] / s->mass[a];
          acc += v * v;
        }
        cnt++;
      }
      return sqrt(acc / cnt);
    }
  }
  return 0.0;
}

/* ---------------------------------------------------------------- Gelman-Rubin, Eqs. 2-3
 * Obar^k = mean over the samples of replica k, Obar = mean over k of Obar^k;
 * R = [1/N sum_k 1/n sum_s (O_s^k - Obar)^2] / [1/N sum_k 1/n sum_s (O_s^k - Obar^k)^2]. */
double orc_gelman_rubin(int32_t n_rep, int32_t n_samp, const double *samples) {
  if (n_rep < 1 || n_samp < 1) return INFINITY;
  double *mk = (double *)malloc(sizeof(double) * (size_t)n_rep);
  double grand = 0;
  for (int k = 0; k < n_rep; ++k) {
    double sum = 0;
    for (int t = 0; t < n_samp; ++t) sum += samples[(size_t)k * n_samp + t];
    mk[k] = sum / n_samp;
    grand += mk[k];
  }
  grand /= n_rep;
  double num = 0, den = 0;
  for (int k = 0; k < n_rep; ++k) {
    double a = 0, b = 0;
    for (int t = 0; t < n_samp; ++t) {
      double o = samples[(size_t)k * n_samp + t];
      a += (o - grand) * (o - grand);
      b += (o - mk[k]) * (o - mk[k]);
    }
    num += a / n_samp;
    den += b / n_samp;
  }
  free(mk);
  num /= n_rep;
  den /= n_rep;
  if (!(den > 0)) return INFINITY;
  return num / den;
}

/* ---------------------------------------------------------------- Fleming-Viot branching */
int32_t orc_fv_branch(uint64_t seed, int64_t step, int32_t n_rep, const uint8_t *exited,
                      int32_t *src) {
  int32_t *surv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_rep > 0 ? n_rep : 1));
  int ns = 0, nb = 0;
  for (int r = 1; r < n_rep; ++r)
    if (!exited[r]) surv[ns++] = r;
  src[0] = -1;
  for (int r = 1; r < n_rep; ++r) {
    if (!exited[r]) { src[r] = -1; continue; }
    if (ns == 0) {
      src[r] = 0;
    } else {
      uint32_t w = orc_branch_word(seed, step, r);
      src[r] = surv[((uint64_t)w * (uint64_t)ns) >> 32];
    }
    nb++;
  }
  free(surv);
  return nb;
}

/* ---------------------------------------------------------------- k steps with sampling */
int32_t orc_step_k_from(const orc_ctx *c, int32_t n_rep, int32_t replica0, double *q, double *p, double *f,
                        uint64_t seed, int64_t t0, int64_t tp0, int64_t k, int32_t t_gr,
                        double *samples, int32_t cap) {
  const orc_system *s = &c->s;
  int nd = s->n_atoms * s->dim, no = s->n_obs;
  int ns = 0;
  for (int64_t i = 0; i < k; ++i) {
    for (int r = 0; r < n_rep; ++r)
      orc_baoab_step(c, q + (size_t)r * nd, p + (size_t)r * nd, f + (size_t)r * nd, seed, replica0 + r, t0 + i);
    if (t_gr > 0 && (tp0 + i + 1) % t_gr == 0) {
      if (samples && ns < cap)
        for (int r = 0; r < n_rep; ++r)
          for (int j = 0; j < no; ++j)
            samples[((size_t)r * cap + ns) * no + j] =
                orc_observable(c, j, q + (size_t)r * nd, p + (size_t)r * nd);
      ns++;
    }
  }
  return ns;
}

int32_t orc_step_k(const orc_ctx *c, int32_t n_rep, double *q, double *p, double *f,
                   uint64_t seed, int64_t t0, int64_t tp0, int64_t k, int32_t t_gr,
                   double *samples, int32_t cap) {
  return orc_step_k_from(c, n_rep, 0, q, p, f, seed, t0, tp0, k, t_gr, samples, cap);
}

/* ---------------------------------------------------------------- adjoint of a segment
 * Differentiation through the dynamics (not part of the paper).  Loss
 * L = 1/(R n_s) sum_r sum_{sampled t} g(O_j(q_t^r)) over k BAOAB steps with the noise fixed.
 * Forward: the steps of orc_baoab_step, keeping every configuration.  Backward, one step at a time
 * from the last, on the adjoints (lq, lp) of the state after the step, h = dt/2:
 *   final half kick  p_{t+1} = p'' + h F(q_{t+1}):  lq += h J_F(q_{t+1}) lp;  dL/dtheta += h lp . dF/dtheta;  lp'' = lp
 *   second drift     q_{t+1} = q' + (h/m) p'':       lq' = lq;  lp'' += (h/m) lq
 *   friction, noise  p'' = c1 p' + s xi:             lp' = c1 lp''
 *   first drift      q' = q_t + (h/m) p':            lq_t = lq';  lp' += (h/m) lq'
 *   first half kick  p' = p_t + h F(q_t):            lq_t += h J_F(q_t) lp';  dL/dtheta += h lp' . dF/dtheta;  lp_t = lp'
 * and a loss sample at q_t adds 1/(R n_s) g'(O) dO/dq to lq_t.  J_F = -Hessian of V is symmetric, so
 * J_F^T lp = J_F lp is a central difference of the forces along lp; lp . dF/dtheta =
 * -d/d eps [dV/dtheta (q + eps lp)] is a central difference of orc_param_grad along lp; dO/dq is a
 * central difference of orc_observable per coordinate.  Each difference is Richardson-extrapolated
 * from the steps e and e/2, which leaves an error of order e^4. */
static void fd_forces_dir(const orc_ctx *c, const double *q, const double *v, double *out, double *w1, double *w2) {
  int nd = c->s.n_atoms * c->s.dim;
  double vmax = 0;
  for (int i = 0; i < nd; ++i) vmax = fmax(vmax, fabs(v[i]));
  if (vmax == 0) { memset(out, 0, sizeof(double) * (size_t)nd); return; }
  double e = 1e-4 / vmax;
  double *qq = (double *)malloc(sizeof(double) * (size_t)nd), *d1 = (double *)malloc(sizeof(double) * (size_t)nd);
  for (int pass = 0; pass < 2; ++pass) {
    double ee = pass == 0 ? e : 0.5 * e;
    for (int i = 0; i < nd; ++i) qq[i] = q[i] + ee * v[i];
    orc_forces(c, qq, w1);
    for (int i = 0; i < nd; ++i) qq[i] = q[i] - ee * v[i];
    orc_forces(c, qq, w2);
    for (int i = 0; i < nd; ++i) {
      double d = (w1[i] - w2[i]) / (2.0 * ee);
      if (pass == 0) d1[i] = d;
      else out[i] = (4.0 * d - d1[i]) / 3.0;
    }
  }
  free(qq);
  free(d1);
}

static void fd_param_dir(const orc_ctx *c, const double *q, const double *v, double *out, int nt) {
  int nd = c->s.n_atoms * c->s.dim;
  double vmax = 0;
  for (int i = 0; i < nd; ++i) vmax = fmax(vmax, fabs(v[i]));
  if (vmax == 0) { memset(out, 0, sizeof(double) * (size_t)nt); return; }
  double e = 1e-4 / vmax;
  double *qq = (double *)malloc(sizeof(double) * (size_t)nd);
  double *g1 = (double *)malloc(sizeof(double) * (size_t)nt), *g2 = (double *)malloc(sizeof(double) * (size_t)nt);
  double *d1 = (double *)malloc(sizeof(double) * (size_t)nt);
  for (int pass = 0; pass < 2; ++pass) {
    double ee = pass == 0 ? e : 0.5 * e;
    for (int i = 0; i < nd; ++i) qq[i] = q[i] + ee * v[i];
    orc_param_grad(c, qq, g1);
    for (int i = 0; i < nd; ++i) qq[i] = q[i] - ee * v[i];
    orc_param_grad(c, qq, g2);
    for (int t = 0; t < nt; ++t) {
      double d = (g1[t] - g2[t]) / (2.0 * ee);
      if (pass == 0) d1[t] = d;
      else out[t] = (4.0 * d - d1[t]) / 3.0;
    }
  }
  free(qq); free(g1); free(g2); free(d1);
}

static double loss_g(double x, int32_t transform, double center, double width, double *gp) {
  if (transform == 1) {
    double g = 1.0 / (1.0 + exp(-(x - center) / width));
    *gp = g * (1.0 - g) / width;
    return g;
  }
  *gp = 1.0;
  return x;
}

double orc_adjoint_segment(const orc_ctx *c, int32_t n_rep, int32_t replica0, double *q, double *p, double *f,
                           uint64_t seed, int64_t t0, int64_t tp0, int32_t k, int32_t t_gr, int32_t obs, int32_t transform,
                           double center, double width, double *grad_theta, double *grad_q0, double *grad_p0) {
  const orc_system *s = &c->s;
  int n = s->n_atoms, dim = s->dim, nd = n * dim;
  int nt = 2 * n + s->n_dihedrals;
  double h = 0.5 * s->dt, c1 = exp(-s->gamma * s->dt);
  int64_t n_s = (tp0 + k) / t_gr - tp0 / t_gr;
  double norm = 1.0 / ((double)n_rep * (double)n_s);
  double *Q = (double *)malloc(sizeof(double) * (size_t)(k + 1) * nd);
  double *lq = (double *)malloc(sizeof(double) * (size_t)nd), *lp = (double *)malloc(sizeof(double) * (size_t)nd);
  double *jv = (double *)malloc(sizeof(double) * (size_t)nd), *w1 = (double *)malloc(sizeof(double) * (size_t)nd);
  double *w2 = (double *)malloc(sizeof(double) * (size_t)nd), *qq = (double *)malloc(sizeof(double) * (size_t)nd);
  double *pg = (double *)malloc(sizeof(double) * (size_t)nt);
  double loss = 0.0;
  if (grad_theta) memset(grad_theta, 0, sizeof(double) * (size_t)nt);
  for (int r = 0; r < n_rep; ++r) {
    double *qr = q + (size_t)r * nd, *pr = p + (size_t)r * nd, *fr = f + (size_t)r * nd;
    memcpy(Q, qr, sizeof(double) * (size_t)nd);
    for (int t = 0; t < k; ++t) {
      orc_baoab_step(c, qr, pr, fr, seed, replica0 + r, t0 + t);
      memcpy(Q + (size_t)(t + 1) * nd, qr, sizeof(double) * (size_t)nd);
    }
    memset(lq, 0, sizeof(double) * (size_t)nd);
    memset(lp, 0, sizeof(double) * (size_t)nd);
    for (int t = k; t >= 1; --t) {
      const double *qt = Q + (size_t)t * nd, *qs = Q + (size_t)(t - 1) * nd;
      /* loss sample at q_t */
      if ((tp0 + t) % t_gr == 0) {
        double gp;
        loss += norm * loss_g(orc_observable(c, obs, qt, NULL), transform, center, width, &gp);
        memcpy(qq, qt, sizeof(double) * (size_t)nd);
        for (int i = 0; i < nd; ++i) {
          double e = 1e-5, d1 = 0, d2 = 0;
          for (int pass = 0; pass < 2; ++pass) {
            double ee = pass == 0 ? e : 0.5 * e;
            qq[i] = qt[i] + ee;
            double op = orc_observable(c, obs, qq, NULL);
            qq[i] = qt[i] - ee;
            double om = orc_observable(c, obs, qq, NULL);
            qq[i] = qt[i];
            if (pass == 0) d1 = (op - om) / (2.0 * ee);
            else d2 = (op - om) / (2.0 * ee);
          }
          lq[i] += norm * gp * (4.0 * d2 - d1) / 3.0;
        }
      }
      /* final half kick of step t-1, at q_t */
      fd_forces_dir(c, qt, lp, jv, w1, w2);
      for (int i = 0; i < nd; ++i) lq[i] += h * jv[i];
      if (grad_theta) {
        fd_param_dir(c, qt, lp, pg, nt);
        for (int u = 0; u < nt; ++u) grad_theta[u] -= h * pg[u];
      }
      /* second drift, friction and noise, first drift */
      for (int i = 0; i < nd; ++i) {
        double hm = h / s->mass[i / dim];
        double lpp = lp[i] + hm * lq[i];
        lp[i] = c1 * lpp + hm * lq[i];
      }
      /* first half kick of step t-1, at q_{t-1} */
      fd_forces_dir(c, qs, lp, jv, w1, w2);
      for (int i = 0; i < nd; ++i) lq[i] += h * jv[i];
      if (grad_theta) {
        fd_param_dir(c, qs, lp, pg, nt);
        for (int u = 0; u < nt; ++u) grad_theta[u] -= h * pg[u];
      }
    }
    if (grad_q0) memcpy(grad_q0 + (size_t)r * nd, lq, sizeof(double) * (size_t)nd);
    if (grad_p0) memcpy(grad_p0 + (size_t)r * nd, lp, sizeof(double) * (size_t)nd);
  }
  free(Q); free(lq); free(lp); free(jv); free(w1); free(w2); free(qq); free(pg);
  return loss;
}

/* ---------------------------------------------------------------- parallel dynamics step, Eq. 5 */
int32_t orc_parallel_phase(const orc_ctx *c, int32_t n_rep, double *q, double *p, double *f,
                           uint64_t seed, int64_t t0, int32_t omega, int32_t t_check,
                           int64_t max_checks, orc_exit *out) {
  int nd = c->s.n_atoms * c->s.dim;
  int64_t t = t0;
  for (int64_t M = 1; M <= max_checks; ++M) {
    orc_step_k(c, n_rep, q, p, f, seed, t, 0, t_check, 0, NULL, 0);
    t += t_check;
    for (int r = 0; r < n_rep; ++r) {
      if (orc_exited(c, q + (size_t)r * nd, omega)) {
        out->M = M;
        out->k = r + 1;
        out->label_to = orc_state_of(c, q + (size_t)r * nd);
        out->tau_steps = ((int64_t)n_rep * (M - 1) + (r + 1)) * (int64_t)t_check;
        return 1;
      }
    }
  }
  return 0;
}

/* ---------------------------------------------------------------- the loop of Fig. 1 */
typedef struct {
  double *v;   /* [n_rep][n_obs][cap] */
  int32_t cap, n;
} history;

static void hist_reserve(history *h, int n_rep, int n_obs, int need) {
  if (need <= h->cap) return;
  int ncap = h->cap ? h->cap : 64;
  while (ncap < need) ncap *= 2;
  double *nv = (double *)malloc(sizeof(double) * (size_t)n_rep * n_obs * ncap);
  for (int r = 0; r < n_rep; ++r)
    for (int j = 0; j < n_obs; ++j)
      for (int t = 0; t < h->n; ++t)
        nv[((size_t)r * n_obs + j) * ncap + t] = h->v[((size_t)r * n_obs + j) * h->cap + t];
  free(h->v);
  h->v = nv;
  h->cap = ncap;
}

int32_t orc_run_genparrep(const orc_ctx *c, const orc_run_params *rp, const double *q0,
                          const double *p0, orc_event *events, int32_t max_events,
                          int64_t *t_global_out) {
  const orc_system *s = &c->s;
  int N = rp->n_rep, nd = s->n_atoms * s->dim, no = s->n_obs;
  double *q = (double *)malloc(sizeof(double) * (size_t)N * nd);
  double *p = (double *)malloc(sizeof(double) * (size_t)N * nd);
  double *f = (double *)malloc(sizeof(double) * (size_t)N * nd);
  double *buf = (double *)malloc(sizeof(double) * (size_t)(N > 1 ? N - 1 : 1) * 1);
  uint8_t *ex = (uint8_t *)malloc((size_t)N);
  int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  history h = {NULL, 0, 0};
  memcpy(q, q0, sizeof(double) * nd);
  memcpy(p, p0, sizeof(double) * nd);
  orc_forces(c, q, f);
  int64_t tg = 0, tsim = 0;
  int nev = 0, nexit = 0;
#define LOG_EVENT(KIND, OM, TO, KK, MM, STEPS, NB)                                          \
  do {                                                                                     \
    if (nev < max_events) {                                                                \
      orc_event e_ = {(KIND), (OM), (TO), (KK), (MM), (STEPS), tsim, (NB)};                \
      events[nev] = e_;                                                                    \
    }                                                                                      \
    nev++;                                                                                 \
  } while (0)

  while (nexit < rp->max_exits && tg < rp->max_steps && nev < max_events) {
    /* 1. transient propagation of the reference walker until it is in some state */
    int64_t treach = 0;
    int omega = orc_state_of(c, q);
    while (omega < 0 && tg < rp->max_steps) {
      for (int i = 0; i < rp->t_check; ++i) orc_baoab_step(c, q, p, f, rp->seed, 0, tg++);
      treach += rp->t_check;
      omega = orc_state_of(c, q);
    }
    if (omega < 0) break;
    if (treach > 0) {
      tsim += treach;
      LOG_EVENT(ORC_EV_TRANSIENT, -1, omega, 0, 0, treach, 0);
    }
    /* 2. convergence step: Fleming-Viot process from the broadcast reference, Gelman-Rubin test */
    for (int r = 1; r < N; ++r) {
      memcpy(q + (size_t)r * nd, q, sizeof(double) * nd);
      memcpy(p + (size_t)r * nd, p, sizeof(double) * nd);
      memcpy(f + (size_t)r * nd, f, sizeof(double) * nd);
    }
    h.n = 0;
    int64_t t = 0, nbranch = 0;
    int converged = 0, ref_exit = 0;
    while (tg < rp->max_steps) {
      for (int i = 0; i < rp->t_check; ++i) {
        for (int r = 0; r < N; ++r)
          orc_baoab_step(c, q + (size_t)r * nd, p + (size_t)r * nd, f + (size_t)r * nd, rp->seed, r, tg);
        tg++;
        t++;
        if (t % rp->t_gr == 0) {
          hist_reserve(&h, N, no, h.n + 1);
          for (int r = 0; r < N; ++r)
            for (int j = 0; j < no; ++j)
              h.v[((size_t)r * no + j) * h.cap + h.n] =
                  orc_observable(c, j, q + (size_t)r * nd, p + (size_t)r * nd);
          h.n++;
        }
      }
      /* (a) the reference walker left omega: kill the F-V workers, clock += t_ref */
      if (orc_exited(c, q, omega)) {
        tsim += t;
        LOG_EVENT(ORC_EV_REF_EXIT, omega, orc_state_of(c, q), 0, 0, t, nbranch);
        nexit++;
        ref_exit = 1;
        break;
      }
      /* (b) branching of the exited workers */
      for (int r = 0; r < N; ++r) ex[r] = (uint8_t)(r > 0 && orc_exited(c, q + (size_t)r * nd, omega));
      int nb = orc_fv_branch(rp->seed, tg, N, ex, src);
      if (nb > 0) {
        int all = 1;
        for (int r = 1; r < N; ++r) all &= ex[r];
        if (all) LOG_EVENT(ORC_EV_FV_ALL_EXITED, omega, omega, 0, 0, t, nb);
        for (int r = 1; r < N; ++r) {
          if (src[r] < 0) continue;
          int sr = src[r];
          memcpy(q + (size_t)r * nd, q + (size_t)sr * nd, sizeof(double) * nd);
          memcpy(p + (size_t)r * nd, p + (size_t)sr * nd, sizeof(double) * nd);
          memcpy(f + (size_t)r * nd, f + (size_t)sr * nd, sizeof(double) * nd);
          for (int j = 0; j < no; ++j)
            memcpy(h.v + ((size_t)r * no + j) * h.cap, h.v + ((size_t)sr * no + j) * h.cap,
                   sizeof(double) * (size_t)h.n);
        }
        nbranch += nb;
      }
      /* (c) Gelman-Rubin over the F-V workers, Eq. 4 */
      if (t >= rp->min_fv_steps && N > 1) {
        int all_ok = 1;
        buf = (double *)realloc(buf, sizeof(double) * (size_t)(N - 1) * (h.n > 0 ? h.n : 1));
        for (int j = 0; j < no && all_ok; ++j) {
          for (int r = 1; r < N; ++r)
            for (int u = 0; u < h.n; ++u)
              buf[(size_t)(r - 1) * h.n + u] = h.v[((size_t)r * no + j) * h.cap + u];
          double R = orc_gelman_rubin(N - 1, h.n, buf);
          if (!(R < 1.0 + rp->tol)) all_ok = 0;
        }
        if (all_ok) { converged = 1; break; }
      }
    }
    if (ref_exit) continue;
    if (!converged) break;
    tsim += t;
    LOG_EVENT(ORC_EV_FV_CONVERGED, omega, omega, 0, 0, t, nbranch);
    /* 3. parallel dynamics step, Eqs. 5-6 */
    int64_t M = 0;
    int found = -1;
    while (tg < rp->max_steps) {
      for (int i = 0; i < rp->t_check; ++i) {
        for (int r = 0; r < N; ++r)
          orc_baoab_step(c, q + (size_t)r * nd, p + (size_t)r * nd, f + (size_t)r * nd, rp->seed, r, tg);
        tg++;
      }
      M++;
      for (int r = 0; r < N; ++r)
        if (orc_exited(c, q + (size_t)r * nd, omega)) { found = r; break; }
      if (found >= 0) break;
    }
    if (found < 0) break;
    int64_t tau = ((int64_t)N * (M - 1) + (found + 1)) * (int64_t)rp->t_check;
    tsim += tau;
    LOG_EVENT(ORC_EV_PARALLEL_EXIT, omega, orc_state_of(c, q + (size_t)found * nd), found + 1, M, tau, 0);
    nexit++;
    /* the exit configuration X_tau^k becomes the reference walker */
    memcpy(q, q + (size_t)found * nd, sizeof(double) * nd);
    memcpy(p, p + (size_t)found * nd, sizeof(double) * nd);
    memcpy(f, f + (size_t)found * nd, sizeof(double) * nd);
  }
#undef LOG_EVENT
  if (t_global_out) *t_global_out = tg;
  free(q); free(p); free(f); free(buf); free(ex); free(src); free(h.v);
  return nev < max_events ? nev : max_events;
}

/* ---------------------------------------------------------------- original ParRep (Section 2.4.3)
 * Transient as in Gen. ParRep; decorrelation: the reference walker alone for t_corr steps in its state
 * (checked every t_check); dephasing: each of the N replicas starts from the decorrelated reference and
 * advances until it has stayed t_phase steps in the state since its last (re)start, an exit restarting
 * it from that reference; the dephasing time is not counted in the clock; parallel step: Eq. 5 from
 * the N dephased configurations. */
int32_t orc_run_original(const orc_ctx *c, const orc_original_params *rp, const double *q0,
                         const double *p0, orc_event *events, int32_t max_events, int64_t *t_global_out) {
  const orc_system *s = &c->s;
  int N = rp->n_rep, nd = s->n_atoms * s->dim;
  size_t bytes = sizeof(double) * (size_t)N * nd;
  double *q = (double *)malloc(bytes), *p = (double *)malloc(bytes), *f = (double *)malloc(bytes);
  /* samples of the dephasing: slot r for replica r, slot N the decorrelated reference */
  size_t sbytes = bytes + sizeof(double) * nd;
  double *sq = (double *)malloc(sbytes), *sp = (double *)malloc(sbytes), *sf = (double *)malloc(sbytes);
  int64_t *stay = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  uint8_t *done = (uint8_t *)malloc((size_t)N);
  memcpy(q, q0, sizeof(double) * nd);
  memcpy(p, p0, sizeof(double) * nd);
  orc_forces(c, q, f);
  int64_t tg = 0, tsim = 0;
  int nev = 0, nexit = 0;
#define LOG_EVENT(KIND, OM, TO, KK, MM, STEPS, NB)                                          \
  do {                                                                                     \
    if (nev < max_events) {                                                                \
      orc_event e_ = {(KIND), (OM), (TO), (KK), (MM), (STEPS), tsim, (NB)};                \
      events[nev] = e_;                                                                    \
    }                                                                                      \
    nev++;                                                                                 \
  } while (0)
#define COPY_REPLICA(DQ, DP, DF, DR, SQ, SP, SF, SR)                                       \
  do {                                                                                     \
    memcpy((DQ) + (size_t)(DR) * nd, (SQ) + (size_t)(SR) * nd, sizeof(double) * nd);       \
    memcpy((DP) + (size_t)(DR) * nd, (SP) + (size_t)(SR) * nd, sizeof(double) * nd);       \
    memcpy((DF) + (size_t)(DR) * nd, (SF) + (size_t)(SR) * nd, sizeof(double) * nd);       \
  } while (0)

  while (nexit < rp->max_exits && tg < rp->max_steps && nev < max_events) {
    /* 1. transient propagation of the reference walker */
    int64_t treach = 0;
    int omega = orc_state_of(c, q);
    while (omega < 0 && tg < rp->max_steps) {
      for (int i = 0; i < rp->t_check; ++i) orc_baoab_step(c, q, p, f, rp->seed, 0, tg++);
      treach += rp->t_check;
      omega = orc_state_of(c, q);
    }
    if (omega < 0) break;
    if (treach > 0) {
      tsim += treach;
      LOG_EVENT(ORC_EV_TRANSIENT, -1, omega, 0, 0, treach, 0);
    }
    /* 2. decorrelation: the reference walker must stay t_corr steps in omega */
    int64_t d = 0;
    int ref_exit = 0;
    while (d < rp->t_corr && tg < rp->max_steps) {
      for (int i = 0; i < rp->t_check; ++i) orc_baoab_step(c, q, p, f, rp->seed, 0, tg++);
      d += rp->t_check;
      if (orc_exited(c, q, omega)) {
        tsim += d;
        LOG_EVENT(ORC_EV_REF_EXIT, omega, orc_state_of(c, q), 0, 0, d, 0);
        nexit++;
        ref_exit = 1;
        break;
      }
    }
    if (ref_exit) continue;
    if (d < rp->t_corr) break;
    tsim += d;
    LOG_EVENT(ORC_EV_DECORRELATED, omega, omega, 0, 0, d, 0);
    /* 3. dephasing: replicas restart from the decorrelated reference until each has stayed t_phase */
    COPY_REPLICA(sq, sp, sf, N, q, p, f, 0);
    for (int r = 1; r < N; ++r) COPY_REPLICA(q, p, f, r, q, p, f, 0);
    for (int r = 0; r < N; ++r) { stay[r] = 0; done[r] = 0; }
    int64_t dsteps = 0, restarts = 0;
    int n_done = 0;
    while (n_done < N && tg < rp->max_steps) {
      for (int i = 0; i < rp->t_check; ++i) {
        for (int r = 0; r < N; ++r)
          orc_baoab_step(c, q + (size_t)r * nd, p + (size_t)r * nd, f + (size_t)r * nd, rp->seed, r, tg);
        tg++;
      }
      dsteps += rp->t_check;
      for (int r = 0; r < N; ++r) {
        if (done[r]) continue;
        if (orc_exited(c, q + (size_t)r * nd, omega)) {
          COPY_REPLICA(q, p, f, r, sq, sp, sf, N);
          stay[r] = 0;
          restarts++;
        } else {
          stay[r] += rp->t_check;
          if (stay[r] >= rp->t_phase) {
            COPY_REPLICA(sq, sp, sf, r, q, p, f, r);
            done[r] = 1;
            n_done++;
          }
        }
      }
    }
    if (n_done < N) break;
    LOG_EVENT(ORC_EV_DEPHASED, omega, omega, 0, 0, dsteps, restarts);
    memcpy(q, sq, bytes);
    memcpy(p, sp, bytes);
    memcpy(f, sf, bytes);
    /* 4. parallel dynamics step, Eqs. 5-6 */
    int64_t M = 0;
    int found = -1;
    while (tg < rp->max_steps) {
      for (int i = 0; i < rp->t_check; ++i) {
        for (int r = 0; r < N; ++r)
          orc_baoab_step(c, q + (size_t)r * nd, p + (size_t)r * nd, f + (size_t)r * nd, rp->seed, r, tg);
        tg++;
      }
      M++;
      for (int r = 0; r < N; ++r)
        if (orc_exited(c, q + (size_t)r * nd, omega)) { found = r; break; }
      if (found >= 0) break;
    }
    if (found < 0) break;
    int64_t tau = ((int64_t)N * (M - 1) + (found + 1)) * (int64_t)rp->t_check;
    tsim += tau;
    LOG_EVENT(ORC_EV_PARALLEL_EXIT, omega, orc_state_of(c, q + (size_t)found * nd), found + 1, M, tau, 0);
    nexit++;
    COPY_REPLICA(q, p, f, 0, q, p, f, found);
  }
#undef LOG_EVENT
#undef COPY_REPLICA
  if (t_global_out) *t_global_out = tg;
  free(q); free(p); free(f); free(sq); free(sp); free(sf); free(stay); free(done);
  return nev < max_events ? nev : max_events;
}

/* ---------------------------------------------------------------- brute-force reference dynamics */
int32_t orc_run_bruteforce(const orc_ctx *c, uint64_t seed, int32_t t_check, const double *q0,
                           const double *p0, int64_t max_steps, int64_t *residence,
                           int32_t *from_state, int32_t max_res) {
  int nd = c->s.n_atoms * c->s.dim;
  double *q = (double *)malloc(sizeof(double) * nd);
  double *p = (double *)malloc(sizeof(double) * nd);
  double *f = (double *)malloc(sizeof(double) * nd);
  memcpy(q, q0, sizeof(double) * nd);
  memcpy(p, p0, sizeof(double) * nd);
  orc_forces(c, q, f);
  int64_t t = 0, t_enter = 0;
  int state = orc_state_of(c, q), nres = 0;
  while (t < max_steps && nres < max_res) {
    for (int i = 0; i < t_check; ++i) orc_baoab_step(c, q, p, f, seed, 0, t++);
    if (state >= 0) {
      if (orc_exited(c, q, state)) {
        residence[nres] = t - t_enter;
        from_state[nres] = state;
        nres++;
        state = orc_state_of(c, q);
        t_enter = t;
      }
    } else {
      state = orc_state_of(c, q);
      t_enter = t;
    }
  }
  free(q); free(p); free(f);
  return nres;
}

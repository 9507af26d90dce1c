/*
 * Oracle for Generalized Parallel Replica (Gen. ParRep) dynamics — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64, single-threaded-per-call C implementation of what the method computes:
 * Langevin dynamics (Section 2.1, Eq. 1) discretised by BAOAB, the state functions of Sections 2.2
 * and 3.3, the Fleming-Viot convergence step with the Gelman-Rubin statistic (Section 2.4.1,
 * Eqs. 2-4), the parallel dynamics step and its exit-time formula (Section 2.4.2, Eqs. 5-6) and the
 * three-step loop of Fig. 1.  It shares no code, header, table or constant generator with the CUDA
 * library; only tests, the smoke entry point and the CPU-baseline leg of the benchmark may load it.
 *
 * Layouts: positions and momenta of one replica are [n_atoms][dim] row-major FP64; several
 * replicas are stacked as [n_replicas][n_atoms][dim].  Units are those of the system description.
 *
 * Parity status: every function here is pinned by a CPU test except where "parity unpinned" is
 * written beside it.
 */
#ifndef GRP_ORACLE_H
#define GRP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_POT_DOUBLE_WELL_2D = 0, ORC_POT_FORCE_FIELD = 1 };
enum { ORC_CV_DOUBLE_WELL = 0, ORC_CV_DIHEDRAL_RECT = 1, ORC_CV_COM_DISTANCE = 2, ORC_CV_ROTAMERS = 3 };
enum {
  ORC_OBS_COORD = 0,        /* arg0 = atom, arg1 = axis */
  ORC_OBS_POTENTIAL = 1,    /* V(q) */
  ORC_OBS_KINETIC = 2,      /* K(p) = 1/2 p^T M^-1 p */
  ORC_OBS_DIHEDRAL = 3,     /* arg0..3 = atoms, radians in (-pi, pi] */
  ORC_OBS_GROUP_DISTANCE = 4, /* arg0, arg1 = groups; distance between their centres of mass */
  ORC_OBS_RMS_VELOCITY = 5  /* arg0 = group; sqrt(mean |p_i/m_i|^2) over the group */
};
#define ORC_MAX_OBS 8
#define ORC_MAX_GROUPS 4

typedef struct {
  int32_t n_atoms;
  int32_t dim;        /* 2 for the analytic double well, 3 for a force-field system */
  int32_t potential;  /* ORC_POT_* */
  const double *mass; /* [n_atoms] */
  double dw_a, dw_b;  /* V(x,y) = dw_a (x^2-1)^2 + dw_b y^2 */
  /* nonbonded: Lennard-Jones (Lorentz-Berthelot) + Coulomb (coulomb_mode below) */
  const double *sigma, *epsilon, *charge; /* [n_atoms] */
  int32_t n_excl;
  const int32_t *excl; /* [n_excl][2] excluded nonbonded pairs */
  double cutoff;       /* 0: every pair; else pairs with r < cutoff (plain truncation) */
  double coulomb_k;    /* k_e in energy*length/charge^2 */
  /* bonded */
  int32_t n_bonds;
  const int32_t *bond_atoms; /* [n_bonds][2] */
  const double *bond_k, *bond_r0; /* E = 1/2 k (r - r0)^2 */
  int32_t n_angles;
  const int32_t *angle_atoms; /* [n_angles][3], vertex in the middle */
  const double *angle_k, *angle_theta0; /* E = 1/2 k (theta - theta0)^2, radians */
  int32_t n_dihedrals;  /* one entry per periodic term */
  const int32_t *dihedral_atoms; /* [n_dihedrals][4] */
  const int32_t *dihedral_n;
  const double *dihedral_k, *dihedral_delta; /* E = k (1 + cos(n phi - delta)) */
  /* Langevin parameters */
  double kT, gamma, dt;
  /* state definition (Sections 2.2 and 3.3) */
  int32_t cv_kind;
  int32_t cv_atoms[8];
  double cv_params[8];
  /* atom groups (centres of mass for CVs and observables) */
  int32_t n_groups;
  int32_t group_offsets[ORC_MAX_GROUPS + 1];
  const int32_t *group_atoms;
  /* Gelman-Rubin observables (Section 2.4.1) */
  int32_t n_obs;
  int32_t obs_kind[ORC_MAX_OBS];
  int32_t obs_arg[ORC_MAX_OBS][4];
  int32_t coulomb_mode;   /* 0: dielectric eps = 4r; 1: reaction field (needs cutoff > 0);
                             2: periodic, particle mesh Ewald; 3: periodic, plain Ewald sum */
  double rf_dielectric;   /* eps_rf of the reaction field; 0 = conductor (infinite) */
  /* Generalized Born implicit solvent, OBC model II (the solvent of the paper's protein-ligand setup,
   * Section 4.2); off when gb_radius is NULL.  Per atom: intrinsic radius rho_i (nm) and descreening
   * scale S_i; dielectric constants inside and outside the solute. */
  const double *gb_radius, *gb_scale;
  double gb_solute_dielectric, gb_solvent_dielectric;
  /* Holonomic bond constraints |q_i - q_j| = d (the paper's setups constrain the bonds of hydrogens):
   * [n_constraints][2] atoms, lengths; relative tolerance of the iterations and their bound. */
  int32_t n_constraints;
  const int32_t *constraint_atoms;
  const double *constraint_length;
  double constraint_tol;
  int32_t constraint_max_iter;
  /* Periodic electrostatics (coulomb_mode 2 and 3), the Ewald sums that the particle mesh Ewald
   * method cited among the engine's expected optimisations (Section 3.2) approximates.  Orthorhombic
   * box of edges box[0..2] (nm); splitting parameter beta (nm^-1): each Coulomb pair is split into
   * k_e q_i q_j erfc(beta r)/r, summed over minimum images within the cutoff (at most half the
   * shortest edge), and a smooth remainder summed in reciprocal space.  Mode 2 evaluates the
   * reciprocal sum by smooth particle mesh Ewald (Essmann et al. 1995: B-splines of order pme_order
   * on a pme_grid[0] x pme_grid[1] x pme_grid[2] grid); mode 3 sums it directly over the
   * reciprocal vectors (k_0/L_0, k_1/L_1, k_2/L_2), 0 < max |k_d| <= ewald_kmax.  Lennard-Jones takes
   * the same minimum image and cutoff. */
  double box[3];
  double ewald_beta;
  int32_t pme_grid[3];
  int32_t pme_order;
  int32_t ewald_kmax;
} orc_system;

typedef struct orc_ctx orc_ctx;

orc_ctx *orc_create(const orc_system *sys);
void orc_destroy(orc_ctx *c);

/* Potential and forces (-grad V), Eq. 1. */
double orc_potential(const orc_ctx *c, const double *q);
void orc_forces(const orc_ctx *c, const double *q, double *f);

/* Derivatives of V with respect to the force-field parameters theta (differentiation of the
 * potential, outside the paper): g[0..n) = dV/d sigma_i, g[n..2n) = dV/d epsilon_i (per-atom
 * Lennard-Jones parameters combined by the Lorentz-Berthelot rules), g[2n..2n+n_dihedrals) = dV/dk_t
 * for every dihedral term in the order of the description.  The derivative with respect to
 * epsilon_i does not exist where epsilon_i = 0 (the square root of the combination rule). */
void orc_param_grad(const orc_ctx *c, const double *q, double *g);

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the Philox S-box on a 128-bit
 * counter with a 64-bit key. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Four standard normals for (seed, replica, step, atom): Box-Muller on the four Philox words of
 * stream 0. */
void orc_normals(uint64_t seed, int64_t step, int32_t replica, int32_t atom, double xi[4]);
/* First Philox word of stream 1 for (seed, step, replica): the Fleming-Viot branching draw. */
uint32_t orc_branch_word(uint64_t seed, int64_t step, int32_t replica);

/* One BAOAB step of Eq. 1 for one replica; f holds F(q) on entry and on exit.  With constraints each
 * sub-step is followed by its projection: positions by SHAKE along the bond vectors before the A step,
 * momenta by RATTLE onto the tangent space (relative velocity along each bond zero). */
void orc_baoab_step(const orc_ctx *c, double *q, double *p, double *f, uint64_t seed,
                    int32_t replica, int64_t step);

/* State functions of Section 3.3: (i) index of the state containing q, -1 if none;
 * (ii) whether q is outside the state omega. */
int32_t orc_state_of(const orc_ctx *c, const double *q);
int32_t orc_exited(const orc_ctx *c, const double *q, int32_t omega);
/* Number of SHAKE or RATTLE projections (all steps so far) whose sweeps reached constraint_max_iter
 * without meeting the tolerance; the dynamics carries on from the last sweep. */
int64_t orc_unconverged(const orc_ctx *c);
/* Generalized Born (OBC II) Born radii B[n] and descreening sums I[n] (nm^-1) of configuration q. */
void orc_gb_born(const orc_ctx *c, const double *q, double *born, double *integral);
/* The parts of the periodic Coulomb energy (coulomb_mode 2 or 3) of configuration q: parts[0] the
 * real-space sum over non-excluded pairs, [1] minus the smooth part of the excluded pairs,
 * [2] the self term -k_e beta/sqrt(pi) sum q_i^2, [3] the reciprocal sum, [4] the neutralising
 * background -k_e pi Q^2 / (2 V beta^2) of a net charge Q.  Their sum is the Coulomb part of V. */
void orc_ewald_parts(const orc_ctx *c, const double *q, double parts[5]);

/* Collective variables of the state definition: cv[0..3] (phi/psi in degrees, x, a distance, or
 * the rotamer torsions in degrees; unused entries 0). */
void orc_cv(const orc_ctx *c, const double *q, double cv[4]);
/* Observable j of Section 2.4.1 (iii). */
double orc_observable(const orc_ctx *c, int32_t j, const double *q, const double *p);

/* Gelman-Rubin ratio, Eq. 3, with the time integrals of Eq. 2 replaced by sample means over
 * samples[n_rep][n_samp].  +inf when the denominator is not positive. */
double orc_gelman_rubin(int32_t n_rep, int32_t n_samp, const double *samples);

/* Fleming-Viot branching (Section 2.4.1, task 2): for every exited worker r >= 1, src[r] = a
 * survivor drawn uniformly among the non-exited workers; src[r] = -1 otherwise; src[0] = -1.
 * When no worker survives, every exited worker takes src = 0 (the reference walker).
 * Returns the number of branched workers. */
int32_t orc_fv_branch(uint64_t seed, int64_t step, int32_t n_rep, const uint8_t *exited,
                      int32_t *src);

/* Advance n_rep replicas by k BAOAB steps starting at global step t0 and phase step tp0; after
 * every step where (tp0 + i + 1) % t_gr == 0 (t_gr > 0) the observables of every replica are
 * appended to samples[r][s][j] (s counted from 0; capacity cap per replica).  Returns the number
 * of samples taken per replica. */
int32_t orc_step_k(const orc_ctx *c, int32_t n_rep, double *q, double *p, double *f,
                   uint64_t seed, int64_t t0, int64_t tp0, int64_t k, int32_t t_gr,
                   double *samples, int32_t cap);
/* The same for rows that are the replicas replica0 .. replica0 + n_rep - 1 of a larger set: row r
 * draws the noise of replica replica0 + r (a shard of a run spread over several processes). */
int32_t orc_step_k_from(const orc_ctx *c, int32_t n_rep, int32_t replica0, double *q, double *p, double *f,
                        uint64_t seed, int64_t t0, int64_t tp0, int64_t k, int32_t t_gr,
                        double *samples, int32_t cap);

/* Adjoint of k BAOAB steps with the noise fixed (differentiation through the dynamics, not part of
 * the paper): advances (q, p, f) [n_rep][n][dim] like orc_step_k, row r drawing the noise of replica
 * replica0 + r, and
 * returns L = 1/(n_rep n_s) sum over replicas and over the n_s steps with (tp0 + t) % t_gr == 0 of
 * g(O_obs(q_t)), g(x) = x (transform 0) or 1 / (1 + exp(-(x - center) / width)) (transform 1).
 * grad_theta [2n + n_dihedrals] (theta as for orc_param_grad), grad_q0 and grad_p0 [n_rep][n][dim]
 * (each optional) receive dL/dtheta and dL/d(q, p) of the initial state.  Hessian-vector products
 * and mixed derivatives are central differences with Richardson extrapolation (error ~ e^4). */
double orc_adjoint_segment(const orc_ctx *c, int32_t n_rep, int32_t replica0, double *q, double *p, double *f,
                           uint64_t seed, int64_t t0, int64_t tp0, int32_t k, int32_t t_gr, int32_t obs, int32_t transform,
                           double center, double width, double *grad_theta, double *grad_q0, double *grad_p0);

/* Parallel dynamics step (Section 2.4.2): every replica advances t_check steps at a time until
 * one has exited omega.  M = number of checks, k = lowest 1-based index exited at check M,
 * tau_steps = [N (M-1) + k] t_check (Eq. 5).  Returns 1 on exit, 0 if max_checks passed. */
typedef struct {
  int64_t M;
  int32_t k;
  int32_t label_to;
  int64_t tau_steps;
} orc_exit;
int32_t orc_parallel_phase(const orc_ctx *c, int32_t n_rep, double *q, double *p, double *f,
                           uint64_t seed, int64_t t0, int32_t omega, int32_t t_check,
                           int64_t max_checks, orc_exit *out);

/* Events of the whole loop of Fig. 1. */
enum { ORC_EV_TRANSIENT = 0, ORC_EV_REF_EXIT = 1, ORC_EV_FV_CONVERGED = 2, ORC_EV_PARALLEL_EXIT = 3,
       ORC_EV_FV_ALL_EXITED = 4, ORC_EV_DECORRELATED = 5, ORC_EV_DEPHASED = 6 };
typedef struct {
  int32_t kind;
  int32_t omega;     /* state the event belongs to (-1 for a transient) */
  int32_t label_to;  /* state index after the event (-1: none) */
  int32_t k;         /* parallel exit: 1-based replica index */
  int64_t M;         /* parallel exit: number of checks */
  int64_t steps;     /* t_reach, t_ref, t_FV or tau, in steps */
  int64_t t_sim;     /* simulation clock after the event, in steps */
  int64_t n_branch;  /* F-V: number of branchings during the phase */
} orc_event;

typedef struct {
  int32_t n_rep;
  uint64_t seed;
  int32_t t_gr, t_check;
  double tol;
  int64_t min_fv_steps;
  int64_t max_steps;   /* bound on the global step counter */
  int32_t max_exits;   /* stop after this many parallel exits or reference exits */
} orc_run_params;

/* Whole Gen. ParRep loop of Fig. 1 from the reference configuration (q0, p0).  Writes at most
 * max_events events; returns the number written, and the global step counter in *t_global. */
int32_t orc_run_genparrep(const orc_ctx *c, const orc_run_params *rp, const double *q0,
                          const double *p0, orc_event *events, int32_t max_events,
                          int64_t *t_global);

/* The original ParRep algorithm as Section 2.4.3 contrasts it with Gen. ParRep: decorrelation (the
 * reference walker must stay t_corr steps in its state, tested every t_check steps; leaving earlier is
 * a reference exit, clock += elapsed), then dephasing (each of the N replicas starts from the
 * decorrelated reference and advances until it has stayed t_phase steps in the state since its last
 * start, a replica that leaves restarting from the decorrelated reference; the dephasing time is not
 * counted in the clock), then the parallel step of Eq. 5 from the N dephased replicas.  Events: TRANSIENT, REF_EXIT, DECORRELATED (steps = t_corr reached),
 * DEPHASED (steps = dephasing steps, n_branch = restarts), PARALLEL_EXIT.  All replicas advance in
 * lockstep during dephasing (replica r draws the noise of replica r at the global step). */
typedef struct {
  int32_t n_rep;
  uint64_t seed;
  int32_t t_check;
  int64_t t_corr, t_phase;
  int64_t max_steps;
  int32_t max_exits;
} orc_original_params;
int32_t orc_run_original(const orc_ctx *c, const orc_original_params *rp, const double *q0,
                         const double *p0, orc_event *events, int32_t max_events, int64_t *t_global);

/* Plain Langevin trajectory (replica index 0) checked every t_check steps; residence times (in
 * steps) from the check at which a state is entered to the check at which it is exited.  Returns
 * the number recorded. */
int32_t orc_run_bruteforce(const orc_ctx *c, uint64_t seed, int32_t t_check, const double *q0,
                           const double *p0, int64_t max_steps, int64_t *residence,
                           int32_t *from_state, int32_t max_res);

#ifdef __cplusplus
}
#endif
#endif

/*
 * grp.h — C ABI of libgrp.so: the data-parallel hot path of Generalized Parallel Replica dynamics
 * (Hedin & Lelievre, "gen.parRep: a first implementation of the Generalized Parallel Replica
 * dynamics for the long time simulation of metastable biochemical systems") on one NVIDIA GB300.
 *
 * Conventions for every call:
 *  - Handles (grp_system, grp_replicas) are opaque and owned by the library; destroy them with the
 *    matching grp_destroy_* call.
 *  - Pointer arguments named h_* are host memory, d_* are device memory of the current CUDA device
 *    (for instance the data pointer of a CUDA torch tensor).  The caller owns them; the library
 *    never keeps them after the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are ordered
 *    on that stream; calls that return host values synchronise it before returning.
 *  - Every call returns GRP_OK (0) or a negative grp_status; nothing aborts.  grp_last_error()
 *    returns a thread-local message describing the last failure (library-owned string).  Device-side
 *    faults detected by the kernels (non-finite state, fixed-point overflow) are latched in a sticky
 *    per-replica-set error word and reported by the next synchronising call.
 *  - Replica 0 is the reference walker of Section 2.4.1; indices are 0-based except the exit index
 *    k of Eq. 5, which is 1-based as in the paper.
 *  - State layout on the device and in h_q / h_p: [n_replicas][n_atoms][dim] row-major FP64.
 */
#ifndef GRP_H
#define GRP_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t grp_status;
#define GRP_OK 0
#define GRP_EINVAL (-1)    /* invalid argument (null pointer, bad size, bad index) */
#define GRP_ENOMEM (-2)    /* device or host allocation failed */
#define GRP_ECUDA (-3)     /* a CUDA runtime call failed */
#define GRP_ENAN (-4)      /* a kernel found a non-finite position or momentum */
#define GRP_EOVERFLOW (-5) /* a force or energy term exceeded the fixed-point range (|f| >= 2^22 on
                              the FP64 path, 2^18 on the mixed path) or was not finite */
#define GRP_ETIMEOUT (-6)  /* a bounded loop ran out before its condition was met */
#define GRP_ENOTIMPL (-7)  /* the requested combination is not supported */
#define GRP_NOEXIT 1       /* positive: the parallel phase ended after max_checks without exit */

/* Precision of the compute path. */
enum { GRP_FP64 = 0,  /* FP64 forces, FP64 integration, FP64 noise */
       GRP_MIXED = 1  /* FP32 forces into 64-bit fixed point, double-single integration,
                         FP32 noise; FP64 only for state in memory, CV near boundaries, G-R */ };

enum { GRP_POT_DOUBLE_WELL_2D = 0, GRP_POT_FORCE_FIELD = 1 };
enum { GRP_CV_DOUBLE_WELL = 0, GRP_CV_DIHEDRAL_RECT = 1, GRP_CV_COM_DISTANCE = 2, GRP_CV_ROTAMERS = 3 };
/* Coulomb model: the dielectric eps = 4r, or the reaction field of a cutoff scheme (Section 3.2 names
 * it among the nonbonded methods an engine should offer; the paper's MD setups use a non-periodic
 * cutoff, which the engine it used treats by a reaction field): for r < cutoff,
 * E = k_e q_i q_j (1/r + k_rf r^2 - c_rf), k_rf = (eps_rf - 1) / ((2 eps_rf + 1) r_c^3),
 * c_rf = 1/r_c + k_rf r_c^2 (eps_r = 1); it needs cutoff > 0. */
enum { GRP_COULOMB_EPS4R = 0, GRP_COULOMB_REACTION_FIELD = 1, GRP_COULOMB_PME = 2 };
enum { GRP_OBS_COORD = 0, GRP_OBS_POTENTIAL = 1, GRP_OBS_KINETIC = 2, GRP_OBS_DIHEDRAL = 3,
       GRP_OBS_GROUP_DISTANCE = 4, GRP_OBS_RMS_VELOCITY = 5 };
#define GRP_MAX_OBS 8
#define GRP_MAX_GROUPS 4

/* Molecular system and Langevin parameters (Section 2.1, Eq. 1; Sections 2.2, 3.3 for the states;
 * Section 2.4.1 for the observables).  All pointers are host memory, copied by grp_create_system.
 *   potential GRP_POT_DOUBLE_WELL_2D: one particle, dim = 2, V = dw_a (x^2 - 1)^2 + dw_b y^2.
 *   potential GRP_POT_FORCE_FIELD: dim = 3, V = sum of
 *     bonds 1/2 k (r - r0)^2, angles 1/2 k (theta - theta0)^2 (radians), dihedral terms
 *     k (1 + cos(n phi - delta)), Lennard-Jones 4 eps_ij ((s_ij/r)^12 - (s_ij/r)^6) with
 *     s_ij = (s_i + s_j)/2, eps_ij = sqrt(eps_i eps_j), and Coulomb k_e q_i q_j / (4 r^2)
 *     (dielectric 4r; or the reaction field, coulomb_mode), over every pair not in excl, truncated at
 *     `cutoff` when cutoff > 0.
 *   States: GRP_CV_DOUBLE_WELL: state 0 = {x < -w}, state 1 = {x > w} (w = cv_params[0]);
 *     state 0 is left when x >= 0, state 1 when x < 0.  GRP_CV_DIHEDRAL_RECT: phi = dihedral of
 *     cv_atoms[0..3], psi of cv_atoms[1..4] (degrees, IUPAC sign); state 0 = phi in
 *     [cv_params[0], cv_params[1]] and psi in [cv_params[2], cv_params[3]], state 1 = complement.
 *     GRP_CV_COM_DISTANCE: d = |COM(group 0) - COM(group 1)|; state 0 = {d < cv_params[0]},
 *     state 1 = complement.  GRP_CV_ROTAMERS (many disjoint states, not a partition: Section 2.4.1's
 *     transient case): m = cv_params[0] (1..4) torsions phi_t of cv_atoms[t..t+3]; the wells of a
 *     torsion are gauche+ [0, 120), trans [120, 180] and (-180, -120), gauche- [-120, 0) degrees
 *     (digits 0, 1, 2); the configuration is in state sum_t well_t 3^t when every torsion lies
 *     within w = cv_params[1] degrees (0 < w <= 60) of its well's centre (60, 180, -60), else in no
 *     state; state omega is left when some torsion's well differs from digit t of omega.
 *   Observables: GRP_OBS_COORD (atom, axis), POTENTIAL, KINETIC, DIHEDRAL (4 atoms, radians),
 *     GROUP_DISTANCE (group a, group b), RMS_VELOCITY (group). */
typedef struct {
  int32_t n_atoms;
  int32_t dim;
  int32_t potential;
  int32_t precision;
  const double *mass;
  double dw_a, dw_b;
  const double *sigma, *epsilon, *charge;
  int32_t n_excl;
  const int32_t *excl;          /* [n_excl][2] */
  double cutoff;
  double coulomb_k;
  int32_t n_bonds;
  const int32_t *bond_atoms;    /* [n_bonds][2] */
  const double *bond_k, *bond_r0;
  int32_t n_angles;
  const int32_t *angle_atoms;   /* [n_angles][3], vertex in the middle */
  const double *angle_k, *angle_theta0;
  int32_t n_dihedrals;          /* one entry per periodic term */
  const int32_t *dihedral_atoms; /* [n_dihedrals][4] */
  const int32_t *dihedral_n;
  const double *dihedral_k, *dihedral_delta;
  double kT, gamma, dt;         /* gamma is a collision rate: c1 = exp(-gamma dt) */
  int32_t cv_kind;
  int32_t cv_atoms[8];
  double cv_params[8];
  int32_t n_groups;
  int32_t group_offsets[GRP_MAX_GROUPS + 1];
  const int32_t *group_atoms;
  int32_t n_obs;
  int32_t obs_kind[GRP_MAX_OBS];
  int32_t obs_arg[GRP_MAX_OBS][4];
  int32_t coulomb_mode;         /* GRP_COULOMB_EPS4R, GRP_COULOMB_REACTION_FIELD or GRP_COULOMB_PME */
  double rf_dielectric;         /* eps_rf of the reaction field (>= 1; 0 = infinity, a conductor) */
  /* Generalized Born implicit solvent, OBC model II (the solvent of the paper's protein-ligand setup,
   * Section 4.2), added to V when gb_radius is not NULL: per-atom intrinsic radii rho_i (nm, > 0.009)
   * and descreening scales S_i (copied), solute and solvent dielectric constants.  With offset radii
   * a_i = rho_i - 0.009 nm, pairwise descreening integrals give I_i, psi_i = a_i I_i, Born radii
   * 1/B_i = 1/a_i - tanh(psi - 0.8 psi^2 + 4.85 psi^3)/rho_i, and
   * E = -(1/2) k_e (1/eps_in - 1/eps_out) sum_i sum_j q_i q_j / sqrt(r^2 + B_i B_j exp(-r^2/(4 B_i B_j)))
   * over all pairs and each atom with itself.  Systems of 64 atoms or more with a cutoff (Verlet lists)
   * truncate the descreening sums and the pair terms at the cutoff (each atom with itself kept).
   * GRP_ENOTIMPL for 64 atoms or more without a cutoff, below 64 atoms with a cutoff, with the reaction
   * field or particle mesh Ewald, in a batch, and for grp_adjoint_segment. */
  const double *gb_radius, *gb_scale;
  double gb_solute_dielectric, gb_solvent_dielectric;
  /* Bond constraints |q_i - q_j| = d (the paper's MD setups hold the bonds of hydrogens fixed): each
   * sub-step of BAOAB is followed by its projection, positions by SHAKE along the bond vectors, momenta
   * by RATTLE (no relative velocity along any bond), Gauss-Seidel sweeps until |r^2 - d^2| <= tol d^2
   * and |r . v| <= tol d^2 / dt; GRP_ETIMEOUT (latched) when constraint_max_iter sweeps do not reach
   * that.  A constrained pair should be excluded from the nonbonded terms and carry no bond term.
   * Below 64 atoms without implicit solvent, or with a cutoff (Verlet lists, with or without implicit
   * solvent); GRP_ENOTIMPL otherwise, with the reaction field or particle mesh Ewald, for groups of
   * coupled constraints larger than 16 constraints or atoms, in a batch, and for grp_adjoint_segment.  On the mixed path a group of one constraint is integrated in double-single
   * arithmetic, a larger group in FP64; both meet the same tolerances. */
  int32_t n_constraints;
  const int32_t *constraint_atoms;  /* [n_constraints][2] */
  const double *constraint_length;  /* [n_constraints] */
  double constraint_tol;            /* relative, e.g. 1e-10 */
  int32_t constraint_max_iter;
  /* Periodic electrostatics, coulomb_mode GRP_COULOMB_PME (particle mesh Ewald, one of the nonbonded
   * methods Section 3.2 expects of an engine): an orthorhombic box of edges box[0..2] (nm), plain
   * Coulomb (eps = 1) summed over all periodic images by Ewald's splitting with parameter ewald_beta
   * (nm^-1).  Real space: k_e q_i q_j erfc(beta r)/r over the minimum images of non-excluded pairs
   * within `cutoff` (required, at most half the shortest edge); excluded pairs: -k_e q_i q_j erf(beta r)/r;
   * self: -k_e beta/sqrt(pi) sum q_i^2; background of a net charge Q: -k_e pi Q^2 / (2 V beta^2);
   * reciprocal space by smooth particle mesh Ewald (Essmann et al. 1995) with cardinal B-splines of
   * order pme_order on a pme_grid[0] x pme_grid[1] x pme_grid[2] grid.  Lennard-Jones takes the same
   * minimum images and cutoff; bonded terms use the positions as they are (molecules are never
   * wrapped).  Positions may leave the box.  Systems of 64 atoms or more keep Verlet lists over nearest
   * images, so there cutoff + skin (7/6 of the cutoff) must be at most half the shortest edge.
   * GRP_EINVAL for a non-positive edge or beta, a missing or too long cutoff; GRP_ENOTIMPL for grid
   * sizes other than 8 or 16, an order other than 4, with implicit solvent or constraints, in a batch,
   * and for grp_adjoint_segment. */
  double box[3];
  double ewald_beta;
  int32_t pme_grid[3];
  int32_t pme_order;
} grp_system_desc;

typedef struct grp_system grp_system;
typedef struct grp_replicas grp_replicas;

/* Step counters of a replica set.  t_global keys the noise (Philox counter), t_phase counts steps
 * since the last broadcast (the F-V time t of Eqs. 2-4, sampled every t_GR). */
typedef struct {
  int64_t t_global;
  int64_t t_phase;
} grp_counters;

/* Result of the parallel dynamics step (Section 2.4.2). */
typedef struct {
  int64_t M;          /* number of checks performed, the exit being seen at check M */
  int32_t k;          /* 1-based index of the lowest replica exited at check M */
  int32_t label_to;   /* state of X_tau^k (-1: in no state) */
  int64_t tau_steps;  /* [N (M - 1) + k] t_check, Eq. 5 */
} grp_exit;

/* Device pointers of a replica set, for zero-copy access (valid until grp_destroy_replicas). */
typedef struct {
  double *q, *p, *f;  /* [R][n][dim] positions, momenta, forces F(q) */
  double *acc;        /* [R][n_obs][4]: shift c, sum (O - c), sum (O - c)^2, sample count */
  int8_t *labels;     /* [R] state index from the last check (-1: none) */
  uint8_t *exited;    /* [R] 1 when the replica was outside omega at the last check */
} grp_device_view;

/* Parameters of the whole loop of Fig. 1. */
typedef struct {
  int32_t t_gr;          /* observable sampling period, steps (Section 3.4) */
  int32_t t_check;       /* exit-test period, steps */
  double tol;            /* Gelman-Rubin tolerance: converged when every R < 1 + tol (Eq. 4) */
  int64_t min_fv_steps;  /* no convergence before this many F-V steps */
  int64_t max_steps;     /* bound on the global step counter */
  int32_t max_exits;     /* stop after this many reference or parallel exits */
} grp_run_params;

/* Parameters of the original ParRep loop (Section 2.4.3): the decorrelation and dephasing times
 * replace the Fleming-Viot convergence test. */
typedef struct {
  int32_t t_check;       /* exit-test period, steps */
  int32_t max_exits;     /* stop after this many reference or parallel exits */
  int64_t t_corr;        /* decorrelation time: the reference walker stays this long before the parallel step */
  int64_t t_phase;       /* dephasing time: each replica's stay since its last restart */
  int64_t max_steps;     /* bound on the global step counter */
} grp_original_params;

enum { GRP_EV_TRANSIENT = 0, GRP_EV_REF_EXIT = 1, GRP_EV_FV_CONVERGED = 2, GRP_EV_PARALLEL_EXIT = 3,
       GRP_EV_FV_ALL_EXITED = 4, GRP_EV_DECORRELATED = 5, GRP_EV_DEPHASED = 6 };
typedef struct {
  int32_t kind;
  int32_t omega;      /* state of the visit (-1 for a transient) */
  int32_t label_to;   /* state after the event (-1: none) */
  int32_t k;          /* parallel exit: 1-based replica index */
  int64_t M;          /* parallel exit: number of checks */
  int64_t steps;      /* t_reach, t_ref, t_FV or tau, in steps */
  int64_t t_sim;      /* simulation clock after the event, in steps */
  int64_t n_branch;   /* F-V: branchings during the phase */
} grp_event;

/* Thread-local description of the last error (library-owned, valid until the next call). */
const char *grp_last_error(void);

/* Build a system on the current device from a host description (copied).  Validates every index
 * and size (GRP_EINVAL).  Section 2.1 (Eq. 1) and Section 3.2 (the engine's requirements). */
grp_status grp_create_system(const grp_system_desc *d, grp_system **out);
void grp_destroy_system(grp_system *s);

/* Allocate n_replicas >= 1 replicas of s on the device; every replica starts at (h_q0, h_p0), a
 * host [n][dim] configuration (per_replica = 0) or host [n_replicas][n][dim] (per_replica = 1);
 * forces are evaluated at q0, counters and accumulators are zero.  `seed` keys the Philox4x32-10
 * noise: counter (t_global, stream, replica, atom).  Section 2.4.1 (replicas, reference walker). */
grp_status grp_init_replicas(grp_system *s, int32_t n_replicas, uint64_t seed, const double *h_q0,
                             const double *h_p0, int32_t per_replica, void *stream,
                             grp_replicas **out);
void grp_destroy_replicas(grp_replicas *r);

/* Advance replicas [0, n_active) by k BAOAB steps of Eq. 1 (n_active = 0: all).  After each step
 * that brings t_phase to a multiple of t_gr (t_gr > 0) every observable of the active replicas is
 * accumulated (Eq. 2 with the time integral replaced by samples every t_GR, Section 2.4.1).
 * Increments t_global and t_phase by k.  Section 3.2: "one code block realising discretisation
 * steps".  Systems with a cutoff keep a Verlet list per replica, of capacity twice the pairs within
 * cutoff + skin of the first configuration (over nearest images in a periodic box), at least 65,536
 * entries or every pair; a list that outgrows it is cut and GRP_ENOMEM is reported by the next call
 * that reads the replicas' error flags (grp_get_state, the check and loop calls). */
grp_status grp_step_k(grp_replicas *r, int64_t k, int32_t t_gr, int32_t n_active, void *stream);

/* State functions of Section 3.3 for every replica: d_labels[r] = state containing replica r
 * (-1: none), d_exited[r] = 1 when replica r is outside omega.  Either pointer may be NULL; the
 * results are also kept in the replica set (grp_device_view). */
grp_status grp_check_states(grp_replicas *r, int32_t omega, int8_t *d_labels, uint8_t *d_exited,
                            void *stream);

/* Fleming-Viot branching (Section 2.4.1, task 2): every worker r >= 1 with d_exited[r] = 1 is
 * overwritten by a copy of a surviving worker drawn uniformly (Philox stream 1, counter
 * (t_global, replica r)): positions, momenta, forces and its observable history (Section 3.1).
 * When no worker survives, exited workers copy the reference walker.  d_exited NULL = the mask of
 * the last grp_check_states.  d_src (device [R], optional) receives the source index or -1;
 * h_n_branched (optional) the number of copies.  The reference walker (replica 0) is never
 * branched. */
grp_status grp_fv_branch(grp_replicas *r, const uint8_t *d_exited, int32_t *d_src,
                         int32_t *h_n_branched, void *stream);

/* Gelman-Rubin ratios of Eq. 3 over the F-V workers (replicas 1..R-1) for every observable, from
 * the accumulated samples; h_rhat[n_obs] receives R_j (+inf when undefined) and h_converged
 * whether every R_j < 1 + tol (Eq. 4).  Either pointer may be NULL. */
grp_status grp_gelman_rubin(grp_replicas *r, double tol, double *h_rhat, int32_t *h_converged,
                            void *stream);

/* Parallel dynamics step (Section 2.4.2): all replicas advance t_check steps at a time until one
 * is outside omega, at most max_checks times.  Returns GRP_OK with h_out = (M, k, label_to, tau)
 * of Eq. 5, or GRP_NOEXIT.  Replica k-1 then holds X_tau^k. */
grp_status grp_run_parallel_phase(grp_replicas *r, int32_t omega, int32_t t_check, int64_t max_checks,
                                  grp_exit *h_out, void *stream);

/* Copy replica src to every replica, clear the accumulators and set t_phase = 0 (the broadcast of
 * the reference configuration before a convergence step, Section 3.1). */
grp_status grp_broadcast(grp_replicas *r, int32_t src, void *stream);

/* Status of one exit test of the convergence step. */
typedef struct {
  int32_t ref_exited;   /* the reference walker left omega at this check */
  int32_t label0;       /* state of the reference walker (-1: none) */
  int32_t n_branched;   /* F-V workers overwritten at this check */
  int32_t converged;    /* Gelman-Rubin criterion met (only when evaluated) */
  int32_t gr_evaluated; /* t_phase >= min_fv_steps, so the ratios were computed */
  int32_t pad;
  int64_t t_phase;      /* F-V time after the check, steps */
  double rhat[GRP_MAX_OBS];
} grp_fv_status;

/* One exit test of the convergence step (Section 2.4.1): every replica advances t_check BAOAB steps
 * sampling observables every t_gr, the exit test runs on every replica, exited workers are branched,
 * and when t_phase >= min_fv_steps the Gelman-Rubin ratios are evaluated; one small readback fills
 * h_out.  When the reference walker exited, the caller abandons the phase (the branching done on the
 * workers is then irrelevant). */
grp_status grp_fv_check(grp_replicas *r, int32_t omega, int32_t t_check, int32_t t_gr, double tol,
                        int64_t min_fv_steps, grp_fv_status *h_out, void *stream);

/* ---- Runs sharded over several processes, one GPU each.  Section 3.1 distributes the replicas of a
 * run over processes and names the exchanges (the F-V copies between processes, the Gelman-Rubin sums,
 * the first exit of the parallel step); Section 5 names GPUs as the next target.  A shard is a replica
 * set holding the global replicas [first, first + R) of a run of n_global replicas; the shard with
 * first = 0 holds the reference walker.  The caller moves the small per-check data between processes
 * with its own communicator (exit flags, sources, the sums below, packed rows); these calls do each
 * shard's part on its GPU.  grp_fv_branch, grp_gelman_rubin, grp_fv_check, grp_run_parallel_phase,
 * grp_run, grp_run_original and grp_batch_create treat a set as a whole run and refuse a shard
 * (GRP_EINVAL). */

/* Make r the shard [first, first + R) of a run of n_global replicas (GRP_EINVAL unless 0 <= first and
 * first + R <= n_global).  The noise of local replica i is that of global replica first + i, so the
 * shards of a run draw exactly the noise of one unsharded set of n_global replicas. */
grp_status grp_set_shard(grp_replicas *r, int32_t first, int32_t n_global);

/* Fleming-Viot sources (Section 2.4.1, task 2) of the shard's replicas from the exit flags of all
 * n_global replicas (d_exited_global: device u8 [n_global]; the flag of the reference walker is not
 * read): d_src[i] (device int32 [R]) = the global index of the survivor that global replica
 * g = first + i copies, drawn as grp_fv_branch draws it (Philox stream 1, counter (t_global, g), the
 * survivors being the workers 1..n_global-1 not exited, or the reference walker when none survives),
 * or -1 when g is the reference walker or did not exit.  Changes no state. */
grp_status grp_fv_plan(grp_replicas *r, const uint8_t *d_exited_global, int32_t *d_src, void *stream);

/* Rows for copies between shards (Section 3.1: a branched replica receives positions, momenta and the
 * observable history of its source): row i = q, p, F of local replica d_idx[i] (3 n dim doubles each,
 * layout as the state) followed by its 4 n_obs accumulator words.  grp_pack_rows writes the rows to
 * d_buf (device [n][3 n dim + 4 n_obs] FP64); grp_unpack_rows writes them into the replicas.  d_idx:
 * device int32 [n]; an index outside [0, R) is skipped and reported (GRP_EINVAL) by the next
 * synchronising call. */
grp_status grp_pack_rows(grp_replicas *r, int32_t n, const int32_t *d_idx, double *d_buf, void *stream);
grp_status grp_unpack_rows(grp_replicas *r, int32_t n, const int32_t *d_idx, const double *d_buf, void *stream);

/* Gelman-Rubin sums of Eq. 3 over the shard's F-V workers (global index >= 1), from the accumulators.
 * pass 1: h_out[3 j + 0..2] = (sum over workers of the sample mean O^k_j, workers with samples, workers
 * without samples).  pass 2, with h_sums1 = the pass-1 sums added over every shard: h_out[2 j + 0..1] =
 * (sum of (O^k_j - O_j)^2 with O_j the mean over all workers, sum of the within-worker variances).
 * Synchronises `stream`. */
grp_status grp_gr_partials(grp_replicas *r, int32_t pass, const double *h_sums1, double *h_out, void *stream);

/* Ratios of Eq. 3 from the pass-1 and pass-2 sums added over every shard: R_j = 1 + B_j / W_j with B_j
 * and W_j the sums of pass 2 divided by the number of workers (+inf when a worker has no sample, there
 * is none or W_j <= 0), as grp_gelman_rubin gives on one unsharded set; h_converged = every R_j < 1 +
 * tol (Eq. 4).  Host arithmetic only; either output may be NULL. */
grp_status grp_gr_combine(int32_t n_obs, const double *h_sums1, const double *h_sums2, double tol, double *h_rhat,
                          int32_t *h_converged);

/* Batched runs: several independent Gen. ParRep runs (replica sets, of the same or of different
 * systems, all of one precision) advanced by one persistent kernel that takes (run, replica) units
 * from a queue sorted by decreasing system size; branching, Gelman-Rubin and the status readback are
 * one launch each for the whole batch.  The batch refers to the replica sets (it does not own them;
 * destroy it before them).  Each run keeps its own seed and counters. */
typedef struct grp_batch grp_batch;
grp_status grp_batch_create(grp_replicas *const *runs, int32_t n_runs, grp_batch **out);
void grp_batch_destroy(grp_batch *b);
/* k BAOAB steps of every replica of every run, sampling every t_gr (grp_step_k for all runs). */
grp_status grp_batch_step_k(grp_batch *b, int64_t k, int32_t t_gr, void *stream);
/* One exit test of the convergence step for every run (grp_fv_check for all runs); h_omega[n_runs]
 * gives each run's state, h_out[n_runs] receives each run's status. */
grp_status grp_batch_fv_check(grp_batch *b, const int32_t *h_omega, int32_t t_check, int32_t t_gr, double tol,
                              int64_t min_fv_steps, grp_fv_status *h_out, void *stream);
/* The whole loop of Fig. 1 for every run of the batch at once, each run in its own phase
 * (transient, convergence, parallel step) and its own visits of its states: per tick one batched
 * segment of t_check steps (replica 0 alone for a run in its transient, every replica otherwise),
 * batched branching and Gelman-Rubin ratios for the runs in their convergence step, one readback.
 * After the first tick the tick's launches and copies are replayed as one captured CUDA graph.
 * Each run's decisions and events are those of grp_run on that run alone (same parameters p, its
 * own seed and state).  h_events is [n_runs][max_events] (run i's log at h_events + i max_events),
 * h_n_events[n_runs] and h_t_sim[n_runs] (optional) receive each run's event count and clock.
 * GRP_EINVAL for t_gr < 1, t_check outside [1, 20000] or tol <= 0. */
grp_status grp_batch_run(grp_batch *b, const grp_run_params *p, grp_event *h_events, int32_t max_events,
                         int32_t *h_n_events, int64_t *h_t_sim, void *stream);
/* Ticks of the last grp_batch_run, and how many of them were replayed as a captured CUDA graph (all
 * but the first, unless the capture was unavailable and every tick was launched node by node). */
grp_status grp_batch_stats(const grp_batch *b, int64_t *h_ticks, int64_t *h_graph_ticks);
/* Pick the block size of the batched kernel by timing candidate sizes on a short segment (the
 * replicas' state and counters are restored afterwards); h_threads (optional) gets the choice. */
grp_status grp_batch_autotune(grp_batch *b, int32_t t_gr, void *stream, int32_t *h_threads);

/* Whole loop of Fig. 1 from the current state of replica 0: transient, convergence (F-V with
 * Gelman-Rubin), parallel step, clock updates (Section 2.4.1, Eq. 6).  Writes at most max_events
 * events to h_events, their count to h_n_events, and the final clock to h_t_sim (optional). */
grp_status grp_run(grp_replicas *r, const grp_run_params *p, grp_event *h_events, int32_t max_events,
                   int32_t *h_n_events, int64_t *h_t_sim, void *stream);

/* The original ParRep loop (Section 2.4.3) from the current state of replica 0.  Per visit of a
 * state omega: transient as in grp_run; decorrelation, replica 0 alone checked every t_check until it
 * has stayed t_corr steps (GRP_EV_DECORRELATED, counted in the clock) or left omega
 * (GRP_EV_REF_EXIT, t_ref counted); dephasing, each of the R replicas starts from the decorrelated
 * configuration, all advance in lockstep, a replica that leaves omega restarts from that
 * configuration and one that has stayed t_phase steps since its last start keeps that state as its
 * sample (GRP_EV_DEPHASED: steps = the dephasing time, n_branch = the restarts; not counted in the
 * clock); parallel step, Eq. 5 from the R samples, the exit configuration becoming replica 0.
 * Events and the clock as for grp_run.  The dephasing keeps the samples and the reference beside
 * the replicas (3 (R + 1) n dim doubles of device memory, allocated per call; GRP_ENOMEM when that
 * fails).  GRP_EINVAL for t_check < 1, t_corr < 0 or t_phase < 0; t_corr and t_phase
 * are rounded up to whole checks. */
grp_status grp_run_original(grp_replicas *r, const grp_original_params *p, grp_event *h_events,
                            int32_t max_events, int32_t *h_n_events, int64_t *h_t_sim, void *stream);

/* Checkpoint and resume: copy positions, momenta, accumulators (each optional) and counters
 * between the replica set and host memory.  grp_set_state re-evaluates the forces. */
grp_status grp_get_state(grp_replicas *r, double *h_q, double *h_p, double *h_acc, grp_counters *h_ctr,
                         void *stream);
grp_status grp_set_state(grp_replicas *r, const double *h_q, const double *h_p, const double *h_acc,
                         const grp_counters *h_ctr, void *stream);

/* Device pointers of the replica set. */
grp_status grp_get_device_view(grp_replicas *r, grp_device_view *out);

/* Potential energy and forces of B configurations (device [B][n][dim] FP64) with the system's
 * precision: d_energy[B] (optional) and d_forces [B][n][dim] (optional). */
grp_status grp_energy_forces(grp_system *s, int32_t n_conf, const double *d_q, double *d_energy,
                             double *d_forces, void *stream);

/* Differentiation of V (Eq. 1) with respect to positions and force-field parameters (not in the
 * paper; for fitting the force field that drives the dynamics).  The parameters theta of a
 * GRP_POT_FORCE_FIELD system are, in this order: sigma_i (n values), epsilon_i (n values) and k of
 * every dihedral term in the order of grp_system_desc (n_dihedrals values); n_theta = 2 n +
 * n_dihedrals (0 for the double well).  Lennard-Jones pairs combine them by the Lorentz-Berthelot
 * rules, so dV/d epsilon_i does not exist where epsilon_i = 0 (GRP_EOVERFLOW is then returned). */
grp_status grp_param_count(const grp_system *s, int32_t *h_n_theta);
/* d_theta (device [n_theta] FP64) receives the current parameters. */
grp_status grp_get_params(const grp_system *s, double *d_theta, void *stream);
/* Replace the parameters by d_theta (device [n_theta] FP64, copied); later calls on every replica
 * set of s (dynamics included) use them.  GRP_EINVAL, with nothing changed, unless every sigma_i > 0,
 * every epsilon_i >= 0 and every value is finite.  Synchronises `stream`.  Not to be called while a
 * kernel of a replica set of s runs on another stream.  Replica sets keep the forces stored with
 * their state until grp_set_state (or grp_adjoint_segment) re-evaluates them. */
grp_status grp_set_params(grp_system *s, const double *d_theta, void *stream);
/* For B configurations d_q (device [B][n][dim] FP64) and weights d_w (device [B], NULL = all 1):
 *   d_energy     (optional, device [B])        V(q_b), unweighted;
 *   d_grad_q     (optional, device [B][n][dim]) w_b dV/dq (q_b) = -w_b F(q_b);
 *   d_grad_theta (optional, device [n_theta])   sum_b w_b dV/d theta (q_b), summed in order of b.
 * This is the vector-Jacobian product of the map q -> (V(q_b))_b for the cotangent w, as reverse-
 * mode differentiation needs it.  Computed in the system's precision (the mixed path: FP32 terms,
 * fixed-point sums).  Synchronises `stream`. */
grp_status grp_energy_grad(grp_system *s, int32_t n_conf, const double *d_q, const double *d_w,
                           double *d_energy, double *d_grad_q, double *d_grad_theta, void *stream);

/* Loss of a dynamics segment: L = 1/(R n_s) sum over replicas and over the n_s sampling steps of
 * g(O(q_t)), with O the system's observable `obs` (GRP_OBS_COORD, GRP_OBS_GROUP_DISTANCE or
 * GRP_OBS_DIHEDRAL, radians) and g the identity (GRP_LOSS_IDENTITY) or the logistic function
 * g(x) = 1 / (1 + exp(-(x - center) / width)) (GRP_LOSS_LOGISTIC: a smoothed occupancy of x > center). */
enum { GRP_LOSS_IDENTITY = 0, GRP_LOSS_LOGISTIC = 1 };
typedef struct {
  int32_t obs;
  int32_t transform;
  double center, width;
} grp_loss;

/* Adjoint (reverse-mode) differentiation through k BAOAB steps of Eq. 1 with the noise held fixed
 * (the same Philox stream: common random numbers; not in the paper).  Re-evaluates the forces of the
 * current state with the system's current parameters, then advances every replica k steps exactly as
 * grp_step_k(r, k, 0, 0) does (observable accumulators untouched),
 * sampling O after every step that brings t_phase to a multiple of t_gr (at least one sample is
 * required), and returns
 *   h_loss       (optional, host)              L of the segment;
 *   d_grad_theta (optional, device [n_theta])   dL/d theta, theta as for grp_energy_grad;
 *   d_grad_q0, d_grad_p0 (optional, device [R][n][dim]) dL/dq and dL/dp of the state before the segment.
 * The reverse sweep recomputes states from checkpoints saved every `checkpoint` steps and applies the
 * transposed BAOAB step, whose Hessian-vector products and mixed parameter derivatives come from a
 * dual-number pass of the force field.  The recomputation runs the system's own precision path, so it
 * reproduces the forward trajectory; on a GRP_MIXED system the dual numbers are FP32 and their
 * tangents are summed in the mixed path's fixed point (the adjoint vectors and dL/d theta stay FP64).
 * Needs a force-field system below 64 atoms in vacuum (else GRP_ENOTIMPL) and (checkpoint + 1) n dim 8
 * bytes of shared memory for the recomputed states (at most
 * about 180 KB; else GRP_EINVAL).  Allocates R ceil(k / checkpoint) 3 n dim 8 bytes of device memory
 * for the checkpoints.  Synchronises `stream`. */
grp_status grp_adjoint_segment(grp_replicas *r, int32_t k, int32_t t_gr, int32_t checkpoint,
                               const grp_loss *loss, double *h_loss, double *d_grad_theta, double *d_grad_q0,
                               double *d_grad_p0, void *stream);

/* Fleming-Viot branching, as grp_fv_branch, on replica arrays the caller owns, allocating nothing.
 * (No counterpart in the paper: this serves callers that cannot allocate device memory while they
 * run, because their memory belongs to another allocator with a fixed budget or because the
 * implicit synchronisation of cudaMalloc/cudaFree is not acceptable in their loop.)
 *   d_q, d_p, d_f: device [n_rep][n][dim] FP64, updated in place; d_acc: device [n_rep][n_obs][4]
 *   (may be NULL when the system has no observables); d_exited: device [n_rep] u8 exit flags;
 *   seed and t_global key the branching draw exactly as in grp_fv_branch; h_n_branched (host)
 *   receives the number of copies.  Synchronises `stream` before returning.
 * Scratch: one source index per replica plus a counter in a static device array that every GPU which
 * loads the library holds until exit (256 KB); n_rep above 65,536 is rejected with GRP_EINVAL.  The
 * kernel stores the count itself, so nothing needs clearing between calls; calls that overlap on the
 * GPU share the array and race.  The device that was current when `s` was created must be current
 * (else GRP_EINVAL, before anything is launched).  The first call on each device looks the array's
 * address up (cudaGetSymbolAddress) with that device current. */
grp_status grp_fv_branch_noalloc(const grp_system *s, int32_t n_rep, double *d_q, double *d_p, double *d_f,
                                 double *d_acc, const uint8_t *d_exited, uint64_t seed, int64_t t_global,
                                 int32_t *h_n_branched, void *stream);

#ifdef __cplusplus
}
#endif
#endif

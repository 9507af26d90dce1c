// Internal launch interface between the C-ABI layer (api.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace grp {

// Arguments of one segment launch: k BAOAB steps of every active replica with observable sampling
// and an optional state check at the end.
struct SegArgs {
  SysDev S;
  double *q, *p, *f;         // [R][n][dim] state in HBM
  double *acc;               // [R][n_obs][4]
  int8_t *labels;            // [R]
  uint8_t *exited;           // [R]
  unsigned long long *exit_key;  // packed (check << 32 | replica), ~0 = none
  int *err;                  // sticky error bits
  uint64_t seed;
  long long t_global0, t_phase0;
  int k, t_gr;
  int n_active;
  int rep0;                  // global index of replica 0 of the set (noise stream of a shard)
  int do_check, omega;
  long long M;               // check index written into the exit key
  int skip_if_exit;          // return at once when *exit_key holds an exit of a check before M
  int pairs_in_smem;
  int noise_batch;           // steps of noise generated together (0: drawn inline per atom)
  int lean;                  // atom parameters read from the global table (large systems)
  uint32_t *nbl;             // [R][nbl_cap] Verlet lists (systems with use_list), else null
  float4 *qref;              // [R][n] positions at the last list build
  int nbl_cap;
  double *gb_glob;           // [R][2n] Born radii and chain-rule weights (solvent with Verlet lists)
  void *gb_gr;               // [R][gb_gr_stride] pass-3 force factor of each candidate pair (path precision)
  int gb_gr_stride;          // nbl_cap + the excluded pairs: list entries first, then excluded pairs
  double h, c1;              // dt/2 and exp(-gamma dt)
};

// Launch configuration chosen per system (threads per replica block).
struct SegConfig {
  int threads;
  size_t smem;
  int pairs_in_smem;
  int noise_batch;
  int lean;
};

// Largest dynamic shared memory of one block on sm_103a.
constexpr size_t kMaxSmem = 227 * 1024;

SegConfig segment_config(const SysDev &S, int threads_hint);
// The noise amplitude of every atom in FP64 and FP32 (the system's tables for lean replica states).
cudaError_t launch_noise_sd(const SysDev &S, double c1, double *sd_d, float *sd_f, cudaStream_t st);
cudaError_t launch_segment(const SegArgs &a, const SegConfig &cfg, cudaStream_t st);

// State functions at the current state (FP64), writing labels/exited; exit key as above.
cudaError_t launch_check(const SysDev &S, const double *q, int n_rep, int omega, int8_t *labels,
                         uint8_t *exited, unsigned long long *exit_key, long long M, cudaStream_t st);

// Fleming-Viot branching of exited workers; n_branched (device int) receives the number branched; err
// (optional) the sticky error word (kErrTimeout when a bulk copy did not complete in time).
cudaError_t launch_fv_branch(const SysDev &S, int n_rep, double *q, double *p, double *f, double *acc,
                             const uint8_t *exited, int32_t *src, int *n_branched, uint64_t seed,
                             long long t_global, cudaStream_t st, int *err = nullptr);

// Gelman-Rubin ratio per observable over workers 1..R-1; rhat[n_obs], converged flag.
cudaError_t launch_gelman_rubin(const SysDev &S, int n_rep, const double *acc, double tol, double *rhat,
                                int *converged, cudaStream_t st);

// Copy replica src to every other replica (or only to dst >= 0); clear accumulators when asked.
cudaError_t launch_copy_replica(const SysDev &S, int n_rep, double *q, double *p, double *f, double *acc,
                                int src, int dst, int clear_acc, cudaStream_t st);

// Dephasing step of the original ParRep after one check: restart exited replicas from slot R of
// (sq, sp, sf) [R + 1][nd], store those that have stayed t_phase steps as their sample (slot r).
cudaError_t launch_dephase(const SysDev &S, int n_rep, double *q, double *p, double *f, double *sq, double *sp,
                           double *sf, const uint8_t *exited, long long *stay, uint8_t *done, int t_check,
                           long long t_phase, int *counters, cudaStream_t st);

// ---- runs sharded over several processes (the shard holds global replicas [first, first + n_local))
// Fleming-Viot source (global index, -1 = kept) of each local replica from the global exit flags.
cudaError_t launch_fv_plan(int n_local, int first, int n_global, const uint8_t *exited_global, int32_t *src,
                           uint64_t seed, long long t_global, cudaStream_t st);
// Rows (q, p, F, accumulators) of replicas idx[0..n) to (unpack = 0) or from (unpack = 1) buf.
cudaError_t launch_pack_rows(const SysDev &S, int n_rep, double *q, double *p, double *f, double *acc, int n,
                             const int32_t *idx, double *buf, int unpack, int *err, cudaStream_t st);
// Gelman-Rubin sums of the shard's workers: pass 1 [n_obs][3], pass 2 [n_obs][2] (see fvgr.cu).
struct GrGrand {
  double v[kMaxObs];
};
cudaError_t launch_gr_partials(const SysDev &S, int n_local, int first, const double *acc, int pass,
                               const GrGrand &grand, double *out, cudaStream_t st);

// ---- batched runs (many replica sets, possibly of different systems, in one launch)
// Device arrays of one run for the batched branching / Gelman-Rubin / status kernels.
struct RunArrays {
  double *q, *p, *f, *acc;
  uint8_t *exited;
  int8_t *labels;
  int32_t *src;
  int *n_branched;
  double *rhat;
  int *err;
  int nd, nacc, n_rep, n_obs;
  uint64_t seed;
  long long t_global;
  unsigned long long *exit_key;
  int branch;  // the run is in its convergence step: branch its exited workers
  int gr;      // evaluate its Gelman-Rubin ratios
};
struct BatchStatus {
  int n_branched;
  int label0;
  int exited0;
  int err;
  double rhat[kMaxObs];
  unsigned long long exit_key;  // (M << 32 | replica) of the first exit of a parallel step, or ~0
  int label_k;                  // state of that replica (-1 when none)
  int pad;
};
static_assert(sizeof(SegArgs) % sizeof(int) == 0, "SegArgs is copied word by word");

// Persistent batched segment kernel over (run, replica) units; returns the number of blocks used.
cudaError_t launch_segment_batch(const SegArgs *d_runs, const uint2 *d_units, int n_units, int *d_counter,
                                 int precision, int threads, size_t smem, cudaStream_t st, int *blocks_used);
cudaError_t launch_fv_branch_batch(const RunArrays *d_runs, const uint2 *d_units, int n_units, cudaStream_t st);
cudaError_t launch_gelman_rubin_batch(const RunArrays *d_runs, const uint2 *d_units, int n_units, cudaStream_t st);
cudaError_t launch_collect_status(const RunArrays *d_runs, int n_runs, BatchStatus *d_out, cudaStream_t st);

// Energies and forces of B configurations.
cudaError_t launch_energy_forces(const SysDev &S, int n_conf, const double *q, double *energy,
                                 double *forces, int *err, cudaStream_t st);

// ---- differentiation with respect to the force-field parameters theta = (sigma_i, eps_i, k_t)
// Rewrite the parameter tables of S from theta [2n + n_terms] (device); *bad = 1 (and the tables
// unchanged) when some sigma_i <= 0 or eps_i < 0 or a value is not finite.
cudaError_t launch_set_params(const SysDev &S, int n_terms, const double *theta, int *bad, cudaStream_t st);
// partial[b][t] = w_b dV/d theta_t at configuration b (w = NULL: 1); grad_q[b] (optional) holds the
// forces on entry and w_b grad_q V = -w_b F on exit.
cudaError_t launch_param_grad(const SysDev &S, int n_terms, int n_conf, const double *q, const double *w,
                              double *grad_q, double *partial, int *err, cudaStream_t st);
// x[b][i] *= alpha w_b (w = NULL: 1).
cudaError_t launch_scale_rows(double *x, int rows, int cols, const double *w, double alpha, cudaStream_t st);
// Adjoint of a k-step FP64 BAOAB segment (one block per replica), for the loss
// L = 1/(R n_s) sum_r sum_samples g(O(q_t)) with the noise fixed: dL/d theta per replica, the loss
// per replica and optionally dL/dq_0, dL/dp_0.
struct AdjArgs {
  SysDev S;
  const double *ckpt;          // [R][n_ck][3][nd]: q, p, f at steps 0, ck, 2 ck, ...
  int n_ck, ck, k;
  uint64_t seed;
  long long t_global0, t_phase0;
  int t_gr;
  int obs_kind, obs_arg[4];    // observable O
  int transform;               // 0: g(x) = x; 1: g(x) = 1 / (1 + exp(-(x - center) / width))
  double center, width;
  double inv_norm;             // 1 / (R n_s)
  double h, c1;
  int n_terms;
  double *partial;             // [R][n_theta]
  double *loss;                // [R]
  double *grad_q0, *grad_p0;   // [R][nd] or null
  int *err;
};
size_t adjoint_smem_bytes(const SysDev &S, int n_terms, int ck);
cudaError_t launch_adjoint(const AdjArgs &a, int n_rep, cudaStream_t st);
// out[t] = sum_b partial[b][t] in order of b.
cudaError_t launch_column_sum(const double *partial, int rows, int cols, double *out, cudaStream_t st);

}  // namespace grp

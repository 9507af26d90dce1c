// Fleming-Viot branching (Section 2.4.1, task 2; copies of Section 3.1), Gelman-Rubin reduction
// (Eqs. 2-4) and replica broadcast/copy kernels.  All of them are HBM- or latency-bound copies and
// reductions over replicas; none needs the tensor cores.
#include "kernels.h"

namespace grp {

// One block per replica r.  An exited worker r >= 1 draws u from Philox stream 1 at counter
// (t_global, replica r), picks survivor number floor(u * |S| / 2^32) in ascending index order among
// the non-exited workers S (the reference walker when S is empty) and copies q, p, F and the
// observable accumulators from it.  Sources are never destinations, so the copies do not race.
__device__ __forceinline__ void fv_branch_one(int r, int n_rep, int nd, int nacc, double *q, double *p, double *f,
                                              double *acc, const uint8_t *exited, int32_t *src, int *n_branched,
                                              uint64_t seed, long long t_global) {
  __shared__ int s_src;
  __shared__ int s_cnt[8];
  if (r == 0 || !exited[r]) {
    if (threadIdx.x == 0 && src) src[r] = -1;
    return;
  }
  int cnt = 0;
  for (int w = 1 + threadIdx.x; w < n_rep; w += blockDim.x) cnt += exited[w] ? 0 : 1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int ns = lane < (int)(blockDim.x >> 5) ? s_cnt[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ns += __shfl_xor_sync(0xffffffffu, ns, o);
    int found = 0;  // no surviving worker: copy the reference walker
    if (ns > 0) {
      const uint32_t u = philox_stream(seed, t_global, 1u, r, 0).v[0];
      int remaining = (int)(((unsigned long long)u * (unsigned long long)ns) >> 32);
      found = -1;
      for (int base = 1; base < n_rep && found < 0; base += 32) {
        const int w = base + lane;
        const unsigned m = __ballot_sync(0xffffffffu, w < n_rep && !exited[w]);
        const int c = __popc(m);
        if (remaining < c) {
          unsigned mm = m;
          for (int i = 0; i < remaining; ++i) mm &= mm - 1;
          found = base + __ffs(mm) - 1;
        } else {
          remaining -= c;
        }
      }
    }
    if (lane == 0) s_src = found;
  }
  __syncthreads();
  const int s = s_src;
  if (s < 0) return;  // unreachable: ns counts the same survivors the scan walks
  const size_t a = (size_t)s * nd, b = (size_t)r * nd;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) {
    q[b + i] = q[a + i];
    p[b + i] = p[a + i];
    f[b + i] = f[a + i];
  }
  for (int i = threadIdx.x; i < nacc; i += blockDim.x) acc[(size_t)r * nacc + i] = acc[(size_t)s * nacc + i];
  if (threadIdx.x == 0) {
    if (src) src[r] = s;
    atomicAdd(n_branched, 1);
  }
}

__global__ void __launch_bounds__(256) fv_branch_kernel(int n_rep, int nd, int nacc, double *q, double *p,
                                                        double *f, double *acc, const uint8_t *exited,
                                                        int32_t *src, int *n_branched, uint64_t seed,
                                                        long long t_global) {
  fv_branch_one(blockIdx.x, n_rep, nd, nacc, q, p, f, acc, exited, src, n_branched, seed, t_global);
}

cudaError_t launch_fv_branch(const SysDev &S, int n_rep, double *q, double *p, double *f, double *acc,
                             const uint8_t *exited, int32_t *src, int *n_branched, uint64_t seed,
                             long long t_global, cudaStream_t st) {
  fv_branch_kernel<<<n_rep, 256, 0, st>>>(n_rep, S.nd, S.n_obs * 4, q, p, f, acc, exited, src, n_branched,
                                          seed, t_global);
  return cudaGetLastError();
}

// Batched branching: one block per (run, replica) unit.
__global__ void __launch_bounds__(256) fv_branch_batch_kernel(const RunArrays *runs, const uint2 *units) {
  const uint2 u = units[blockIdx.x];
  const RunArrays &a = runs[u.x];
  if (!a.branch) return;
  fv_branch_one((int)u.y, a.n_rep, a.nd, a.nacc, a.q, a.p, a.f, a.acc, a.exited, a.src, a.n_branched, a.seed,
                a.t_global);
}

cudaError_t launch_fv_branch_batch(const RunArrays *d_runs, const uint2 *d_units, int n_units, cudaStream_t st) {
  if (n_units <= 0) return cudaSuccess;
  fv_branch_batch_kernel<<<n_units, 256, 0, st>>>(d_runs, d_units);
  return cudaGetLastError();
}

// Deterministic block sum of doubles (fixed tree), result broadcast to every thread.
__device__ __forceinline__ double block_sum_d(double v, double *scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < (int)(blockDim.x >> 5) ? scratch[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) scratch[32] = t;
  }
  __syncthreads();
  const double r = scratch[32];
  __syncthreads();
  return r;
}

// One block per observable j.  With per-worker accumulators (c, S1, S2, n): Obar^k = c + S1/n and
// the within variance var_k = S2/n - (S1/n)^2; the numerator of Eq. 3 equals W + B with
// W = mean_k var_k and B = mean_k (Obar^k - Obar)^2, its denominator is W, so R = 1 + B / W.
__device__ __forceinline__ void gelman_rubin_one(int j, int n_rep, int n_obs, const double *acc, double *rhat) {
  __shared__ double scratch[33];
  const int nw = n_rep - 1;
  double sm = 0, bad = 0;
  for (int r = 1 + threadIdx.x; r < n_rep; r += blockDim.x) {
    const double *a = acc + ((size_t)r * n_obs + j) * 4;
    if (a[3] < 1.0) bad += 1.0;
    else sm += a[0] + a[1] / a[3];
  }
  const double nbad = block_sum_d(bad, scratch);
  const double grand = block_sum_d(sm, scratch) / nw;
  double sb = 0, sw = 0;
  for (int r = 1 + threadIdx.x; r < n_rep; r += blockDim.x) {
    const double *a = acc + ((size_t)r * n_obs + j) * 4;
    if (a[3] < 1.0) continue;
    const double m1 = a[1] / a[3];
    const double mk = a[0] + m1;
    sb += (mk - grand) * (mk - grand);
    sw += a[2] / a[3] - m1 * m1;
  }
  const double B = block_sum_d(sb, scratch) / nw;
  const double W = block_sum_d(sw, scratch) / nw;
  if (threadIdx.x == 0) rhat[j] = (nw < 1 || nbad > 0 || !(W > 0)) ? __longlong_as_double(0x7FF0000000000000LL)
                                                                    : 1.0 + B / W;
}

__global__ void __launch_bounds__(256) gelman_rubin_kernel(int n_rep, int n_obs, const double *acc, double *rhat) {
  gelman_rubin_one(blockIdx.x, n_rep, n_obs, acc, rhat);
}

// Batched Gelman-Rubin: one block per (run, observable) unit.
__global__ void __launch_bounds__(256) gelman_rubin_batch_kernel(const RunArrays *runs, const uint2 *units) {
  const uint2 u = units[blockIdx.x];
  const RunArrays &a = runs[u.x];
  if (!a.gr) return;
  gelman_rubin_one((int)u.y, a.n_rep, a.n_obs, a.acc, a.rhat);
}

cudaError_t launch_gelman_rubin_batch(const RunArrays *d_runs, const uint2 *d_units, int n_units, cudaStream_t st) {
  if (n_units <= 0) return cudaSuccess;
  gelman_rubin_batch_kernel<<<n_units, 256, 0, st>>>(d_runs, d_units);
  return cudaGetLastError();
}

// Per-run status of one batched exit test, gathered for a single readback.
__global__ void collect_status_kernel(const RunArrays *runs, int n_runs, BatchStatus *out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_runs) return;
  const RunArrays &a = runs[r];
  BatchStatus s;
  s.n_branched = *a.n_branched;
  s.label0 = a.labels[0];
  s.exited0 = a.exited[0];
  s.err = *a.err;
  for (int j = 0; j < kMaxObs; ++j) s.rhat[j] = j < a.n_obs ? a.rhat[j] : 0.0;
  s.exit_key = a.exit_key ? *a.exit_key : ~0ull;
  s.label_k = s.exit_key != ~0ull ? a.labels[(int)(s.exit_key & 0xffffffffu)] : -1;
  s.pad = 0;
  out[r] = s;
}

cudaError_t launch_collect_status(const RunArrays *d_runs, int n_runs, BatchStatus *d_out, cudaStream_t st) {
  if (n_runs <= 0) return cudaSuccess;
  collect_status_kernel<<<(n_runs + 63) / 64, 64, 0, st>>>(d_runs, n_runs, d_out);
  return cudaGetLastError();
}

cudaError_t launch_gelman_rubin(const SysDev &S, int n_rep, const double *acc, double tol, double *rhat,
                                int *converged, cudaStream_t st) {
  (void)tol;
  (void)converged;
  if (S.n_obs == 0) return cudaSuccess;
  gelman_rubin_kernel<<<S.n_obs, 256, 0, st>>>(n_rep, S.n_obs, acc, rhat);
  return cudaGetLastError();
}

// Copy replica src to every other replica (dst < 0) or to dst only; optionally clear every
// replica's accumulators.
__global__ void __launch_bounds__(256) copy_replica_kernel(int n_rep, int nd, int nacc, double *q, double *p,
                                                           double *f, double *acc, int src, int dst, int clear_acc) {
  const int r = blockIdx.x;
  if (clear_acc)
    for (int i = threadIdx.x; i < nacc; i += blockDim.x) acc[(size_t)r * nacc + i] = 0.0;
  if (r == src || (dst >= 0 && r != dst)) return;
  const size_t a = (size_t)src * nd, b = (size_t)r * nd;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) {
    q[b + i] = q[a + i];
    p[b + i] = p[a + i];
    f[b + i] = f[a + i];
  }
}

cudaError_t launch_copy_replica(const SysDev &S, int n_rep, double *q, double *p, double *f, double *acc,
                                int src, int dst, int clear_acc, cudaStream_t st) {
  copy_replica_kernel<<<n_rep, 256, 0, st>>>(n_rep, S.nd, S.n_obs * 4, q, p, f, acc, src, dst, clear_acc);
  return cudaGetLastError();
}

// Dephasing of the original ParRep (Section 2.4.3), after each check: one block per replica r not yet
// dephased.  A replica outside omega restarts from the decorrelated reference (slot n_rep of the
// sample arrays); otherwise its stay grows by t_check and, once it reaches t_phase, its state becomes
// sample r.  counters[0] counts the replicas dephased, counters[1] the restarts.
__global__ void __launch_bounds__(256) dephase_kernel(int n_rep, int nd, double *q, double *p, double *f,
                                                      double *sq, double *sp, double *sf,
                                                      const uint8_t *exited, long long *stay, uint8_t *done,
                                                      int t_check, long long t_phase, int *counters) {
  const int r = blockIdx.x;
  if (done[r]) return;
  const bool out = exited[r] != 0;
  const long long s = out ? 0 : stay[r] + t_check;
  __syncthreads();  // every thread has read stay[r] before thread 0 rewrites it
  const size_t b = (size_t)r * nd, ref = (size_t)n_rep * nd;
  if (out) {
    for (int i = threadIdx.x; i < nd; i += blockDim.x) {
      q[b + i] = sq[ref + i];
      p[b + i] = sp[ref + i];
      f[b + i] = sf[ref + i];
    }
  } else if (s >= t_phase) {
    for (int i = threadIdx.x; i < nd; i += blockDim.x) {
      sq[b + i] = q[b + i];
      sp[b + i] = p[b + i];
      sf[b + i] = f[b + i];
    }
  }
  if (threadIdx.x == 0) {
    stay[r] = s;
    if (out) {
      atomicAdd(counters + 1, 1);
    } else if (s >= t_phase) {
      done[r] = 1;
      atomicAdd(counters, 1);
    }
  }
}

cudaError_t launch_dephase(const SysDev &S, int n_rep, double *q, double *p, double *f, double *sq, double *sp,
                           double *sf, const uint8_t *exited, long long *stay, uint8_t *done, int t_check,
                           long long t_phase, int *counters, cudaStream_t st) {
  dephase_kernel<<<n_rep, 256, 0, st>>>(n_rep, S.nd, q, p, f, sq, sp, sf, exited, stay, done, t_check, t_phase,
                                        counters);
  return cudaGetLastError();
}

}  // namespace grp

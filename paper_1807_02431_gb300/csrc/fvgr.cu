// Fleming-Viot branching (Section 2.4.1, task 2; copies of Section 3.1), Gelman-Rubin reduction
// (Eqs. 2-4) and replica broadcast/copy kernels.  All of them are HBM- or latency-bound copies and
// reductions over replicas; none needs the tensor cores.
#include <algorithm>

#include "kernels.h"

namespace grp {

// Copy of part `part` of `parts` equal slices of one replica's q, p and F rows (nd doubles each) by
// the whole block.  When every row starts on a 16-byte boundary (nd even on the library's own
// 256-byte-aligned arrays; caller-owned arrays are checked) the copy moves double2 words, issuing
// up to four loads per thread and array (twelve 16-byte loads in flight) before the stores: enough
// bytes in flight to approach the HBM bandwidth (measured: 8-byte loads one at a time reached 36 %
// of it).  Source and destination rows never overlap, and no thread writes a source row while the
// kernel runs.
__device__ __forceinline__ void copy_row3(double *__restrict__ qd, double *__restrict__ pd, double *__restrict__ fd,
                                          const double *__restrict__ qs, const double *__restrict__ ps,
                                          const double *__restrict__ fs, int nd, int part = 0, int parts = 1) {
  const int bd = (int)blockDim.x;
  const uintptr_t any = (uintptr_t)qd | (uintptr_t)pd | (uintptr_t)fd | (uintptr_t)qs | (uintptr_t)ps | (uintptr_t)fs;
  if ((nd & 1) == 0 && (any & 15) == 0) {
    const int n2 = nd >> 1, per = (n2 + parts - 1) / parts;
    const int lo = part * per, hi = min(n2, lo + per);
    const double2 *q2 = reinterpret_cast<const double2 *>(qs), *p2 = reinterpret_cast<const double2 *>(ps),
                  *f2 = reinterpret_cast<const double2 *>(fs);
    double2 *qo = reinterpret_cast<double2 *>(qd), *po = reinterpret_cast<double2 *>(pd),
            *fo = reinterpret_cast<double2 *>(fd);
    for (int base = lo + (int)threadIdx.x; base < hi; base += 4 * bd) {
      double2 a[4], b[4], c[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = base + u * bd;
        if (i < hi) {
          a[u] = __ldg(q2 + i);
          b[u] = __ldg(p2 + i);
          c[u] = __ldg(f2 + i);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = base + u * bd;
        if (i < hi) {
          qo[i] = a[u];
          po[i] = b[u];
          fo[i] = c[u];
        }
      }
    }
    return;
  }
  const int per = (nd + parts - 1) / parts;
  const int lo = part * per, hi = min(nd, lo + per);
  for (int i = lo + (int)threadIdx.x; i < hi; i += bd) {
    qd[i] = qs[i];
    pd[i] = ps[i];
    fd[i] = fs[i];
  }
}

// The survivor that exited worker r copies (Section 2.4.1, task 2), called by the whole block:
// survivors S = the workers 1..n_rep-1 not exited, in ascending order; u from Philox stream 1 at
// counter (t_global, replica r) picks survivor number floor(u |S| / 2^32); with no survivor, the
// reference walker (0).  Each thread counts the survivors of its contiguous chunk of the mask; a
// block-wide scan of the counts gives |S| and the rank of each chunk's first survivor; the thread whose
// chunk holds rank m walks it to that survivor.  (Three dependent rounds of loads, where a warp scanning
// the mask 32 workers at a time took n_rep/32 dependent rounds.)  Blocks of at most 256 threads.
__device__ __forceinline__ int draw_survivor(int r, int n_rep, const uint8_t *exited, uint64_t seed,
                                             long long t_global) {
  __shared__ int s_src;
  __shared__ int s_cnt[8];
  const int nt = (int)blockDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int chunk = (n_rep - 1 + nt - 1) / nt;
  const int lo = 1 + threadIdx.x * chunk, hi = min(n_rep, lo + chunk);
  int cnt = 0;
  for (int w = lo; w < hi; ++w) cnt += exited[w] ? 0 : 1;
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_cnt[warp] = incl;
  if (threadIdx.x == 0) s_src = 0;  // no surviving worker: copy the reference walker
  __syncthreads();
  int ns = 0, first = incl - cnt;
  for (int w = 0; w < (nt >> 5); ++w) {
    const int c = s_cnt[w];
    ns += c;
    if (w < warp) first += c;
  }
  if (ns > 0) {
    const uint32_t u = philox_stream(seed, t_global, 1u, r, 0).v[0];
    const int m = (int)(((unsigned long long)u * (unsigned long long)ns) >> 32);
    if (m >= first && m < first + cnt) {
      int rem = m - first;
      for (int w = lo; w < hi; ++w) {
        if (exited[w]) continue;
        if (rem == 0) { s_src = w; break; }
        --rem;
      }
    }
  }
  __syncthreads();
  const int s = s_src;
  __syncthreads();  // every thread has read s_src before a later call rewrites it
  return s;
}

// One block per replica r.  An exited worker r >= 1 draws u from Philox stream 1 at counter
// (t_global, replica r), picks survivor number floor(u * |S| / 2^32) in ascending index order among
// the non-exited workers S (the reference walker when S is empty) and copies q, p, F and the
// observable accumulators from it.  Sources are never destinations, so the copies do not race.
// Every exited worker is branched, so the block of the reference walker (r = 0, never branched)
// stores their number in *n_branched: no counter to clear before the launch, no atomics.  Large
// replicas are copied by `parts` blocks, each drawing the same survivor and copying one slice of the
// rows (slice 0 also copies the accumulators and records the source), so that the copies of a few
// hundred branched workers spread evenly over the SMs.
__device__ __forceinline__ void fv_branch_one(int r, int n_rep, int nd, int nacc, double *q, double *p, double *f,
                                              double *acc, const uint8_t *exited, int32_t *src, int *n_branched,
                                              uint64_t seed, long long t_global, int part = 0, int parts = 1) {
  __shared__ int s_cnt[8];
  if (r == 0) {
    if (part != 0) return;
    int ne = 0;
    for (int w = 1 + threadIdx.x; w < n_rep; w += blockDim.x) ne += exited[w] ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ne += __shfl_down_sync(0xffffffffu, ne, o);
    if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = ne;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_cnt[w];
      *n_branched = tot;
      if (src) src[0] = -1;
    }
    return;
  }
  if (!exited[r]) {
    if (threadIdx.x == 0 && src && part == 0) src[r] = -1;
    return;
  }
  const int s = draw_survivor(r, n_rep, exited, seed, t_global);
  const size_t a = (size_t)s * nd, b = (size_t)r * nd;
  copy_row3(q + b, p + b, f + b, q + a, p + a, f + a, nd, part, parts);
  if (part != 0) return;
  for (int i = threadIdx.x; i < nacc; i += blockDim.x) acc[(size_t)r * nacc + i] = acc[(size_t)s * nacc + i];
  if (threadIdx.x == 0 && src) src[r] = s;
}

__global__ void __launch_bounds__(256) fv_branch_kernel(int n_rep, int nd, int nacc, double *q, double *p,
                                                        double *f, double *acc, const uint8_t *exited,
                                                        int32_t *src, int *n_branched, uint64_t seed,
                                                        long long t_global) {
  fv_branch_one(blockIdx.x, n_rep, nd, nacc, q, p, f, acc, exited, src, n_branched, seed, t_global, blockIdx.y,
                gridDim.y);
}

// ---- the same branching with the copies done by the bulk-copy (TMA) engine
// One elected thread moves a row through shared memory in chunks: cp.async.bulk loads (global -> shared,
// completion counted in bytes on an mbarrier) kBulkStages chunks ahead, cp.async.bulk stores (shared ->
// global) as each chunk lands; a buffer is reloaded once the store that read it has finished reading.  The
// bulk copies need 16-byte aligned addresses and sizes: rows of an even number of doubles on 16-byte
// aligned arrays (checked on the host).  Every wait on an mbarrier is bounded by ~1 s of SM clock, after
// which the block records kErrTimeout, waits for its issued stores and stops.
constexpr int kBulkStages = 4;
constexpr uint32_t kBulkChunk = 12288;  // bytes; 4 stages = 48 KB of shared memory, four blocks per SM

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst_smem)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void bulk_store(void *dst, const void *src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src_smem)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all_but_one() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Bounded wait for phase `parity` of an mbarrier: false after ~2^31 SM cycles (about one second).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}

// Grid (worker r, row part): part 0, 1, 2 copies the q, p or F row of an exited worker; the survivor is
// drawn as in fv_branch_one; part 0 also copies the accumulators and records the source.  The reference
// walker's block (r = 0) stores the branch count.
__global__ void __launch_bounds__(128) fv_branch_bulk_kernel(int n_rep, int nd, int nacc, double *q, double *p,
                                                             double *f, double *acc, const uint8_t *exited,
                                                             int32_t *src, int *n_branched, uint64_t seed,
                                                             long long t_global, int *err) {
  extern __shared__ __align__(128) unsigned char stage[];  // kBulkStages x kBulkChunk
  __shared__ __align__(8) uint64_t bar[kBulkStages];
  const int r = blockIdx.x, part = blockIdx.y;
  if (r == 0 || !exited[r]) {  // the count, or a kept worker: no copy
    fv_branch_one(r, n_rep, nd, nacc, q, p, f, acc, exited, src, n_branched, seed, t_global, part, gridDim.y);
    return;
  }
  const int s = draw_survivor(r, n_rep, exited, seed, t_global);
  if (part == 0) {
    for (int i = threadIdx.x; i < nacc; i += blockDim.x) acc[(size_t)r * nacc + i] = acc[(size_t)s * nacc + i];
    if (threadIdx.x == 0 && src) src[r] = s;
  }
  if (threadIdx.x == 0) {
    double *arr = part == 0 ? q : (part == 1 ? p : f);
    const char *from = reinterpret_cast<const char *>(arr + (size_t)s * nd);
    char *to = reinterpret_cast<char *>(arr + (size_t)r * nd);
    const uint32_t row = (uint32_t)nd * 8u;
    const int nc = (int)((row + kBulkChunk - 1) / kBulkChunk);
    auto bytes_of = [&](int c) { return min(kBulkChunk, row - (uint32_t)c * kBulkChunk); };
    for (int b = 0; b < kBulkStages; ++b) mbar_init(&bar[b], 1);
    mbar_init_fence();
    for (int c = 0; c < nc && c < kBulkStages; ++c) {
      mbar_expect_tx(&bar[c], bytes_of(c));
      bulk_load(stage + (size_t)c * kBulkChunk, from + (size_t)c * kBulkChunk, bytes_of(c), &bar[c]);
    }
    bool ok = true;
    for (int c = 0; c < nc; ++c) {
      const int b = c % kBulkStages;
      if (!mbar_wait_bounded(&bar[b], (uint32_t)(c / kBulkStages) & 1u)) {
        ok = false;
        break;
      }
      bulk_store(to + (size_t)c * kBulkChunk, stage + (size_t)b * kBulkChunk, bytes_of(c));
      bulk_commit();
      // refill the buffer of chunk c - 1 with chunk c - 1 + kBulkStages once its store has read it
      const int nxt = c - 1 + kBulkStages;
      if (c >= 1 && nxt < nc) {
        bulk_wait_read_all_but_one();
        const int bb = (c - 1) % kBulkStages;
        mbar_expect_tx(&bar[bb], bytes_of(nxt));
        bulk_load(stage + (size_t)bb * kBulkChunk, from + (size_t)nxt * kBulkChunk, bytes_of(nxt), &bar[bb]);
      }
    }
    if (!ok && err) atomicOr(err, (int)kErrTimeout);
    bulk_wait_all();  // the stores issued have completed (and read the shared memory)
  }
  __syncthreads();  // the block's shared memory outlives thread 0's copies
}

static bool aligned16(const void *x) { return ((uintptr_t)x & 15u) == 0; }

cudaError_t launch_fv_branch(const SysDev &S, int n_rep, double *q, double *p, double *f, double *acc,
                             const uint8_t *exited, int32_t *src, int *n_branched, uint64_t seed,
                             long long t_global, cudaStream_t st, int *err) {
  // large rows on 16-byte aligned arrays: the bulk-copy kernel, one block per worker and row
  if (S.nd % 2 == 0 && S.nd * 8 >= 8192 && aligned16(q) && aligned16(p) && aligned16(f)) {
    const int smem = kBulkStages * (int)kBulkChunk;
    cudaError_t e = cudaFuncSetAttribute(fv_branch_bulk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    fv_branch_bulk_kernel<<<dim3(n_rep, 3), 128, smem, st>>>(n_rep, S.nd, S.n_obs * 4, q, p, f, acc, exited, src,
                                                             n_branched, seed, t_global, err);
    return cudaGetLastError();
  }
  // slices of about 48 KB (256 threads x twelve 16-byte loads) per block
  const long long row_bytes = 3ll * S.nd * 8;
  const int parts = (int)std::min<long long>(16, std::max<long long>(1, (row_bytes + 49151) / 49152));
  fv_branch_kernel<<<dim3(n_rep, parts), 256, 0, st>>>(n_rep, S.nd, S.n_obs * 4, q, p, f, acc, exited, src,
                                                      n_branched, seed, t_global);
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

// ---- runs sharded over several processes: the shard holds the global replicas [first, first + n_local)
// Fleming-Viot sources of the shard's replicas from the exit flags of all n_global replicas: one block per
// local replica, the survivor drawn exactly as fv_branch_one draws it, with global indices.
__global__ void __launch_bounds__(256) fv_plan_kernel(int n_local, int first, int n_global,
                                                      const uint8_t *exited_global, int32_t *src, uint64_t seed,
                                                      long long t_global) {
  const int g = first + (int)blockIdx.x;
  if (g == 0 || !exited_global[g]) {
    if (threadIdx.x == 0) src[blockIdx.x] = -1;
    return;
  }
  const int s = draw_survivor(g, n_global, exited_global, seed, t_global);
  if (threadIdx.x == 0) src[blockIdx.x] = s;
}

cudaError_t launch_fv_plan(int n_local, int first, int n_global, const uint8_t *exited_global, int32_t *src,
                           uint64_t seed, long long t_global, cudaStream_t st) {
  if (n_local <= 0) return cudaSuccess;
  fv_plan_kernel<<<n_local, 256, 0, st>>>(n_local, first, n_global, exited_global, src, seed, t_global);
  return cudaGetLastError();
}

// Rows of replicas idx[i] (q, p, F, accumulators) to or from a packed buffer [n][3 nd + nacc]: one
// block per row.  An index outside [0, n_rep) is skipped and flagged.
__global__ void __launch_bounds__(256) pack_rows_kernel(int n_rep, int nd, int nacc, double *q, double *p,
                                                        double *f, double *acc, const int32_t *idx, double *buf,
                                                        int unpack, int *err) {
  const int r = idx[blockIdx.x];
  if (r < 0 || r >= n_rep) {
    if (threadIdx.x == 0) atomicOr(err, (int)kErrIndex);
    return;
  }
  double *b = buf + (size_t)blockIdx.x * (3 * (size_t)nd + nacc);
  double *rows[3] = {q + (size_t)r * nd, p + (size_t)r * nd, f + (size_t)r * nd};
  for (int c = 0; c < 3; ++c)
    for (int t = threadIdx.x; t < nd; t += blockDim.x) {
      if (unpack) rows[c][t] = b[(size_t)c * nd + t];
      else b[(size_t)c * nd + t] = rows[c][t];
    }
  double *a = acc + (size_t)r * nacc, *ba = b + 3 * (size_t)nd;
  for (int t = threadIdx.x; t < nacc; t += blockDim.x) {
    if (unpack) a[t] = ba[t];
    else ba[t] = a[t];
  }
}

cudaError_t launch_pack_rows(const SysDev &S, int n_rep, double *q, double *p, double *f, double *acc, int n,
                             const int32_t *idx, double *buf, int unpack, int *err, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  pack_rows_kernel<<<n, 256, 0, st>>>(n_rep, S.nd, S.n_obs * 4, q, p, f, acc, idx, buf, unpack, err);
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

// Gelman-Rubin sums of a shard's workers (global index >= 1), one block per observable j, from the
// shifted accumulators (c, S1, S2, n) as in gelman_rubin_one.  Pass 1: out[3 j ..] = (sum of the worker
// means O^k, workers with samples, workers without); pass 2, grand = the global mean of the worker
// means: out[2 j ..] = (sum of (O^k - grand)^2, sum of within-worker variances S2/n - (S1/n)^2).
__global__ void __launch_bounds__(256) gr_partials_kernel(int n_local, int first, int n_obs, const double *acc,
                                                          int pass, GrGrand grand, double *out) {
  __shared__ double scratch[33];
  const int j = blockIdx.x;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int i = threadIdx.x; i < n_local; i += blockDim.x) {
    if (first + i == 0) continue;  // the reference walker is not a Fleming-Viot worker
    const double *a = acc + ((size_t)i * n_obs + j) * 4;
    if (pass == 1) {
      if (a[3] < 1.0) {
        a2 += 1.0;
      } else {
        a0 += a[0] + a[1] / a[3];
        a1 += 1.0;
      }
    } else if (a[3] >= 1.0) {
      const double m1 = a[1] / a[3];
      const double mk = a[0] + m1;
      a0 += (mk - grand.v[j]) * (mk - grand.v[j]);
      a1 += a[2] / a[3] - m1 * m1;
    }
  }
  a0 = block_sum_d(a0, scratch);
  a1 = block_sum_d(a1, scratch);
  a2 = block_sum_d(a2, scratch);
  if (threadIdx.x == 0) {
    if (pass == 1) {
      out[3 * j] = a0; out[3 * j + 1] = a1; out[3 * j + 2] = a2;
    } else {
      out[2 * j] = a0; out[2 * j + 1] = a1;
    }
  }
}

cudaError_t launch_gr_partials(const SysDev &S, int n_local, int first, const double *acc, int pass,
                               const GrGrand &grand, double *out, cudaStream_t st) {
  if (S.n_obs == 0) return cudaSuccess;
  gr_partials_kernel<<<S.n_obs, 256, 0, st>>>(n_local, first, S.n_obs, acc, pass, grand, out);
  return cudaGetLastError();
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
  copy_row3(q + b, p + b, f + b, q + a, p + a, f + a, nd);
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
  if (out) copy_row3(q + b, p + b, f + b, sq + ref, sp + ref, sf + ref, nd);
  else if (s >= t_phase) copy_row3(sq + b, sp + b, sf + b, q + b, p + b, f + b, nd);
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

// Fleming-Viot branching on caller-owned replica arrays without any allocation.
//
// Some callers cannot call cudaMalloc while they run: their device memory is owned by another
// allocator (a framework's caching pool whose budget is fixed when it starts), or they cannot accept
// the implicit device-wide synchronisation that cudaMalloc/cudaFree may add inside a timed loop.
// grp_fv_branch_noalloc serves them: its only scratch (one source index per replica and a branch
// counter) lives in a file-scope device array of fixed size that every GPU loading the library keeps
// until the process exits.  It launches the same branching kernel as grp_fv_branch.
#include <atomic>
#include <cstdio>
#include <string>

#include "kernels.h"

namespace {

constexpr int kNoAllocMaxReplicas = 65536;
constexpr int kMaxDevices = 64;

// [0, kNoAllocMaxReplicas): source index per replica; [kNoAllocMaxReplicas]: branch counter.
static __device__ __align__(256) int g_fv_scratch[kNoAllocMaxReplicas + 64];

// Device address of g_fv_scratch, looked up once per device.  In host code the symbol is only a
// host-side stand-in, so kernels must be given the address cudaGetSymbolAddress returns.  Two host
// threads making their first call on one device at once both look it up and store the same value;
// the atomics make that well defined.
std::atomic<int *> g_scratch_ptr[kMaxDevices];
}  // namespace

// Implemented in api.cu.
grp::SysDev grp_system_device_view(const grp_system *s);
int grp_system_device_index(const grp_system *s);
void grp_set_last_error(const char *msg);

// Host-only part of the entry point's device check: the system's parameter tables live on the
// device that was current when it was created, and the scratch address is per device, so a call
// made with another device current is refused before anything is launched.  Returns GRP_OK or
// GRP_EINVAL (with the message set).  Exported without a header declaration so that the tests can
// check it on a machine without a GPU.
extern "C" grp_status grp_noalloc_check_device(int32_t system_device, int32_t current_device) {
  if (system_device == current_device) return GRP_OK;
  char msg[200];
  snprintf(msg, sizeof msg,
           "grp_fv_branch_noalloc: the current device is %d but the system was created on device %d; "
           "make that device current before the call",
           (int)current_device, (int)system_device);
  grp_set_last_error(msg);
  return GRP_EINVAL;
}

extern "C" grp_status grp_fv_branch_noalloc(const grp_system *s, int32_t n_rep, double *d_q, double *d_p,
                                            double *d_f, double *d_acc, const uint8_t *d_exited, uint64_t seed,
                                            int64_t t_global, int32_t *h_n_branched, void *stream) {
  char msg[256];
  if (!s || !d_q || !d_p || !d_f || !d_exited || !h_n_branched) {
    grp_set_last_error("grp_fv_branch_noalloc: null argument");
    return GRP_EINVAL;
  }
  const grp::SysDev D = grp_system_device_view(s);
  if ((D.n_obs > 0 && !d_acc) || n_rep < 1) {
    grp_set_last_error("grp_fv_branch_noalloc: need n_rep >= 1 and d_acc when the system has observables");
    return GRP_EINVAL;
  }
  if (n_rep > kNoAllocMaxReplicas) {
    snprintf(msg, sizeof msg, "grp_fv_branch_noalloc: n_rep = %d exceeds the static scratch maximum of %d replicas",
             n_rep, kNoAllocMaxReplicas);
    grp_set_last_error(msg);
    return GRP_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    grp_set_last_error("grp_fv_branch_noalloc: no usable current device");
    return GRP_ECUDA;
  }
  if (grp_noalloc_check_device(grp_system_device_index(s), dev) != GRP_OK) return GRP_EINVAL;
  int *src = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!src) {  // first call on this device: look the scratch address up
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fv_scratch);
    if (e != cudaSuccess) {
      snprintf(msg, sizeof msg, "grp_fv_branch_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      grp_set_last_error(msg);
      return GRP_ECUDA;
    }
    src = (int *)p;
    g_scratch_ptr[dev].store(src, std::memory_order_release);
  }
  int *counter = src + kNoAllocMaxReplicas;
  cudaStream_t st = (cudaStream_t)stream;
  // the kernel stores the count (the block of replica 0 writes it), so the scratch needs no clearing
  e = grp::launch_fv_branch(D, n_rep, d_q, d_p, d_f, d_acc, d_exited, src, counter, seed, (long long)t_global, st);
  int nb = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nb, counter, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "grp_fv_branch_noalloc: %s", cudaGetErrorString(e));
    grp_set_last_error(msg);
    return GRP_ECUDA;
  }
  *h_n_branched = nb;
  return GRP_OK;
}

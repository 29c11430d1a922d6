// sim_log_contacts_noalloc: the contact-impulse log gather without any device
// allocation.
//
// Who needs it: code that must not allocate device memory while it runs --
// a training loop whose framework allocator has already claimed the GPU's
// memory budget, or a real-time control loop that cannot afford the implicit
// device synchronisation a cudaMalloc/cudaFree may cause.  sim_log_contacts
// keeps its per-environment prefix sums in a handle-owned staging buffer that
// it may (re)allocate on first use; this variant keeps them in a fixed array
// of this file instead.  Both launch the same kernels (enqueue_contact_log).
//
// The scratch is a file-scope __device__ array of SIM_NOALLOC_MAX_ENVS + 1
// ints (256 KB + 4 B).  Every GPU that loads this library holds it until the
// process exits.  Host code cannot pass the array's name to a kernel -- on the
// host that name is only a stand-in, not a device address -- so its address on
// each device is looked up with cudaGetSymbolAddress, with that device current,
// when a handle is created there (sim_create, which is never inside a stream
// capture because it allocates), and cached per device; a handle created after
// a device reset therefore refreshes it.  All calls share the one array and it
// keeps the last call's contents: each call rewrites every entry it reads
// (count and prefix of every env, and the total) before reading it, so nothing
// has to start at zero, but calls whose work overlaps on the GPU (two streams,
// or two handles on one device) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/sim.h"
#include "sim_internal.cuh"

namespace gb {
// defined in sim_api.cu
int handle_internals(SimHandle* h, const Dev** d, cudaStream_t* s, int* device);
int report_error(int code, const std::string& msg);
int enqueue_contact_log(const Dev& d, cudaStream_t s, int* prefix, float* feats, float* lams, int cap, bool preds);
void note_handle_error(SimHandle* h);
}  // namespace gb

static __device__ __align__(256) int g_log_scratch[SIM_NOALLOC_MAX_ENVS + 1];

static std::mutex g_scratch_mu;
static int* g_scratch_ptr[256];  // per device ordinal

// Looks the scratch's address up on the current device and caches it.
static int lookup_scratch(int dev, int** out) {
  int* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&p, g_log_scratch);
  if (e != cudaSuccess || !p)
    return gb::report_error(SIM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  g_scratch_ptr[dev] = p;
  *out = p;
  return SIM_OK;
}

static int current_device(int* dev) {
  cudaError_t e = cudaGetDevice(dev);
  if (e != cudaSuccess) return gb::report_error(SIM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (*dev < 0 || *dev >= 256) return gb::report_error(SIM_ERR_CUDA, "device ordinal out of range");
  return SIM_OK;
}

namespace gb {
// Called by sim_create on the new handle's device.
int noalloc_scratch_refresh() {
  int dev = 0, r;
  if ((r = current_device(&dev))) return r;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  int* p = nullptr;
  return lookup_scratch(dev, &p);
}
}  // namespace gb

static int scratch_on_current_device(int** out) {
  int dev = 0, r;
  if ((r = current_device(&dev))) return r;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_ptr[dev]) {
    *out = g_scratch_ptr[dev];
    return SIM_OK;
  }
  return lookup_scratch(dev, out);
}

static int log_contacts_noalloc(SimHandle* h, float* feats, float* lams, int cap, int* n_out);

extern "C" int sim_log_contacts_noalloc(SimHandle* h, float* feats, float* lams, int cap, int* n_out) {
  const int r = log_contacts_noalloc(h, feats, lams, cap, n_out);
  if (r) gb::note_handle_error(h);  // the handle's last error, as for every call on a handle
  return r;
}

static int log_contacts_noalloc(SimHandle* h, float* feats, float* lams, int cap, int* n_out) {
  if (!h || !n_out) return gb::report_error(SIM_ERR_INVALID_ARG, "sim_log_contacts_noalloc: NULL argument");
  const gb::Dev* d = nullptr;
  cudaStream_t st = nullptr;
  int device = 0;
  int r = gb::handle_internals(h, &d, &st, &device);
  if (r) return r;
  // the checks in the order of sim_log_contacts, so that both report the same error
  if (!d->feat) return gb::report_error(SIM_ERR_STATE, "sim_log_contacts_noalloc: log_features was not enabled");
  if (cap < 0 || (cap > 0 && (!feats || !lams)))
    return gb::report_error(SIM_ERR_INVALID_ARG, "sim_log_contacts_noalloc: bad output buffers");
  if (d->E > SIM_NOALLOC_MAX_ENVS)
    return gb::report_error(SIM_ERR_INVALID_ARG, "sim_log_contacts_noalloc: " + std::to_string(d->E) +
                                                     " environments exceed its fixed scratch of SIM_NOALLOC_MAX_ENVS = " +
                                                     std::to_string(SIM_NOALLOC_MAX_ENVS));
  // the handle's device for this call, the caller's current device again afterwards
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != device && cudaSetDevice(device) != cudaSuccess)
    return gb::report_error(SIM_ERR_CUDA, "sim_log_contacts_noalloc: cannot select the handle's device");
  int* prefix = nullptr;
  r = scratch_on_current_device(&prefix);
  cudaError_t e = cudaSuccess;
  if (!r) r = gb::enqueue_contact_log(*d, st, prefix, feats, lams, cap, false);
  if (!r) {
    e = cudaMemcpyAsync(n_out, prefix + d->E, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (r) return r;
  if (e != cudaSuccess) return gb::report_error(SIM_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e));
  return SIM_OK;
}

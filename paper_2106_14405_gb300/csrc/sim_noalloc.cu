// sim_log_contacts_noalloc: the contact-impulse log gather without any device
// allocation.
//
// Who needs it: code that must not allocate device memory while it runs --
// a training loop whose framework allocator has already claimed the GPU's
// memory budget, a real-time control loop that cannot afford the implicit
// device synchronisation a cudaMalloc/cudaFree may cause, or code that
// enqueues work while a stream capture is in progress.  sim_log_contacts
// keeps its per-environment prefix sums in a handle-owned staging buffer that
// it may (re)allocate on first use; this variant keeps them in a fixed array
// of this file instead.
//
// The scratch is a file-scope __device__ array of SIM_NOALLOC_MAX_ENVS + 1
// ints (256 KB + 4 B).  Every GPU that loads this library holds it until the
// process exits.  Host code cannot pass the array's name to a kernel -- on the
// host that name is only a stand-in, not a device address -- so the first call
// on each device (with that device current) looks the address up with
// cudaGetSymbolAddress and caches it; make that first call before any stream
// capture.  All calls share the one array and it keeps the last call's
// contents: each call rewrites every entry it reads (prefix of every env and
// the total) before reading it, so nothing has to start at zero, but calls
// whose work overlaps on the GPU (two streams, or two handles on one device)
// race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/sim.h"
#include "sim_internal.cuh"

namespace gb {
// defined in sim_api.cu
int handle_internals(SimHandle* h, const Dev** d, cudaStream_t* s);
int report_error(int code, const std::string& msg);
}  // namespace gb

static __device__ __align__(256) int g_log_scratch[SIM_NOALLOC_MAX_ENVS + 1];

static std::mutex g_scratch_mu;
static int* g_scratch_ptr[256];  // per device ordinal

static int scratch_on_current_device(int** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gb::report_error(SIM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 256) return gb::report_error(SIM_ERR_CUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    int* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_log_scratch);
    if (e != cudaSuccess || !p)
      return gb::report_error(SIM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return SIM_OK;
}

// prefix[e] = contacts of envs before e, prefix[E] = total (one thread, as in the allocating path)
__global__ void k_scan_counts_fixed(const int* n, int E, int* prefix) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int acc = 0;
  for (int e = 0; e < E; ++e) {
    prefix[e] = acc;
    acc += n[e];
  }
  prefix[E] = acc;
}

__global__ void k_log_gather_fixed(const float* feat, const float4* c_lam, const float4* r_meff, const int* n_contacts,
                                   const int* prefix, int E, int C, float scale, float* feats, float* lams, int cap) {
  int e = blockIdx.x;
  if (e >= E) return;
  int n = n_contacts[e], base = prefix[e];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int o = base + i;
    if (o >= cap) break;
    size_t g = (size_t)e * C + i;
    for (int k = 0; k < gb::NFEAT; ++k) feats[(size_t)o * gb::NFEAT + k] = feat[g * gb::NFEAT + k];
    float sc = r_meff[g].x * scale;
    float4 l = c_lam[g];
    const float* prior = feat + g * gb::NFEAT + 23;  // prior-frame impulses (features 23..25)
    lams[3 * (size_t)o] = (l.x - prior[0]) / sc;
    lams[3 * (size_t)o + 1] = (l.y - prior[1]) / sc;
    lams[3 * (size_t)o + 2] = (l.z - prior[2]) / sc;
  }
}

extern "C" int sim_log_contacts_noalloc(SimHandle* h, float* feats, float* lams, int cap, int* n_out) {
  if (!h || !n_out) return gb::report_error(SIM_ERR_INVALID_ARG, "sim_log_contacts_noalloc: NULL argument");
  if (cap < 0 || (cap > 0 && (!feats || !lams)))
    return gb::report_error(SIM_ERR_INVALID_ARG, "sim_log_contacts_noalloc: bad output buffers");
  const gb::Dev* d = nullptr;
  cudaStream_t st = nullptr;
  int r = gb::handle_internals(h, &d, &st);
  if (r) return r;
  if (!d->feat) return gb::report_error(SIM_ERR_STATE, "sim_log_contacts_noalloc: log_features was not enabled");
  if (d->E > SIM_NOALLOC_MAX_ENVS)
    return gb::report_error(SIM_ERR_INVALID_ARG, "sim_log_contacts_noalloc: " + std::to_string(d->E) +
                                                     " environments exceed its fixed scratch of SIM_NOALLOC_MAX_ENVS = " +
                                                     std::to_string(SIM_NOALLOC_MAX_ENVS));
  int* prefix = nullptr;
  if ((r = scratch_on_current_device(&prefix))) return r;
  k_scan_counts_fixed<<<1, 1, 0, st>>>(d->n_contacts, d->E, prefix);
  float scale = sqrtf(d->gx * d->gx + d->gy * d->gy + d->gz * d->gz) * d->dt;
  if (cap > 0 && d->E)
    k_log_gather_fixed<<<d->E, 64, 0, st>>>(d->feat, d->c_lam, d->r_meff, d->n_contacts, prefix, d->E, d->C, scale,
                                             feats, lams, cap);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gb::report_error(SIM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  e = cudaMemcpyAsync(n_out, prefix + d->E, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return gb::report_error(SIM_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e));
  return SIM_OK;
}

// FP32 FMA throughput of the device: the denominator of the solver kernels' ALU
// roofline.  Every thread runs NCHAIN independent fused multiply-add chains on
// registers (enough independent work per warp to cover the FMA pipe's latency), the
// grid fills every SM to its resident-thread limit, and the chains' results are
// stored so that none can be removed.  Work per launch: 2 flops x NCHAIN x iters x
// threads.  Timed with CUDA events on the given stream; the best of `reps` launches
// after one warm-up launch.
#include <cuda_runtime.h>

#include <string>

#include "../../include/sim.h"

namespace gb {
int report_error(int code, const std::string& msg);
}

namespace {
constexpr int NCHAIN = 8;
constexpr int THREADS = 256;

__global__ void __launch_bounds__(THREADS) k_fma_chains(float* out, int iters, float a, float b) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  float x[NCHAIN];
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) x[k] = 1e-3f * (float)(tid + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < NCHAIN; ++k) x[k] = __fmaf_rn(x[k], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) s += x[k];
  out[tid] = s;
}
}  // namespace

extern "C" int sim_fp32_fma_peak(void* cuda_stream, int iters, int reps, double* tflops, double* ms_best) {
  if (!tflops || iters < 1 || reps < 1) return gb::report_error(SIM_ERR_INVALID_ARG, "sim_fp32_fma_peak: bad argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0, per_sm = 0;
  auto ck = [](cudaError_t e, const char* what) {
    return e == cudaSuccess ? SIM_OK : gb::report_error(SIM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  int r;
  if ((r = ck(cudaGetDevice(&dev), "cudaGetDevice"))) return r;
  if ((r = ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attribute"))) return r;
  if ((r = ck(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains, THREADS, 0), "occupancy"))) return r;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  const long threads = (long)blocks * THREADS;
  float* out = nullptr;
  if ((r = ck(cudaMalloc((void**)&out, sizeof(float) * threads), "cudaMalloc"))) return r;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 0.f;
  cudaError_t err = cudaSuccess;
  for (int k = 0; k <= reps && err == cudaSuccess; ++k) {
    cudaEventRecord(e0, s);
    k_fma_chains<<<blocks, THREADS, 0, s>>>(out, iters, 0.999999f, 1e-7f);
    cudaEventRecord(e1, s);
    err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (k > 0 && (best == 0.f || ms < best)) best = ms;  // launch 0 is the warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if ((r = ck(err, "sim_fp32_fma_peak"))) return r;
  const double flops = 2.0 * NCHAIN * 16.0 * (double)iters * (double)threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms_best) *ms_best = best;
  return SIM_OK;
}

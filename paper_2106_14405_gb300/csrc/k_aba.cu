// Articulated-body kernels: one warp per multi-joint articulation (aba_multi),
// one thread per single-joint articulation (aba_single); the device code is in
// aba.cuh.
#include "aba.cuh"

namespace gb {

__global__ void __launch_bounds__(128) k_aba(Dev d) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int slot = blockIdx.x * (blockDim.x >> 5) + wib;
  if (slot >= d.n_art_multi) return;
  aba_multi(d, d.art_multi[slot], lane, reinterpret_cast<AbaSh*>(sm_raw)[wib]);
}

__global__ void __launch_bounds__(256) k_aba1(Dev d) {
  int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= d.n_art_single) return;
  aba_single(d, d.art_single[slot]);
}

void configure_aba() {
  cudaFuncSetAttribute(k_aba, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(AbaSh) * 4));
}

void launch_aba(const Dev& d, cudaStream_t st) {
  const int warps = 4;
  if (d.n_art_multi > 0) k_aba<<<(d.n_art_multi + warps - 1) / warps, 32 * warps, sizeof(AbaSh) * warps, st>>>(d);
  if (d.n_art_single > 0) k_aba1<<<(d.n_art_single + 255) / 256, 256, 0, st>>>(d);
}

}  // namespace gb

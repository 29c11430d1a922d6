// Collision kernel: one warp per environment (collide_env in collide.cuh).
#include "collide.cuh"

namespace gb {

__global__ void __launch_bounds__(256, 3) k_collide(Dev d, int NC, WorkQueue q) {
  extern __shared__ float smc[];
  const int lane = threadIdx.x & 31;
  float* base = smc + (size_t)(threadIdx.x >> 5) * CollLayout{NC}.floats();
  for (int s = wq_first(q, lane); s < d.E; s = wq_next(q, lane)) {
    collide_env(d, NC, base, wq_env(q, s), lane);
    __syncwarp();
  }
  wq_done(q, lane);
}

static size_t collide_smem_warp(int max_coll) {
  int NC = (max_coll + 3) & ~3;
  return sizeof(float) * CollLayout{NC}.floats();
}

static int max_optin_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

void configure_collide(int max_coll) {
  size_t w = collide_smem_warp(max_coll);
  int warps = MAX_WARPS_PER_CTA;
  while (warps > 1 && w * warps > (size_t)max_optin_smem()) warps >>= 1;
  cudaFuncSetAttribute(k_collide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(w * warps));
}

int occupancy_collide(int max_coll, int warps) {
  size_t smem = collide_smem_warp(max_coll) * warps;
  if (smem > (size_t)max_optin_smem()) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_collide, 32 * warps, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

void launch_collide(const Dev& d, cudaStream_t st, int max_coll, KShape k) {
  if (d.E == 0) return;
  int NC = (max_coll + 3) & ~3;
  int blocks = (d.E + k.warps - 1) / k.warps;
  if (k.persistent) blocks = min(blocks, k.grid_cap);
  WorkQueue q{d.wq + 0, nullptr, k.persistent};
  k_collide<<<blocks, 32 * k.warps, collide_smem_warp(max_coll) * k.warps, st>>>(d, NC, q);
}

}  // namespace gb
